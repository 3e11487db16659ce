"""Sample sharding over two gloo ranks on CPU: the gathered per-sample values
equal a single-process run over the same global samples bit for bit, so the
merged statistics are the single run's (replicas; no data-path exchange)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import estimator, krylov, multigrid  # noqa: E402
from paper_1909_12234_gb300 import parallel, synth  # noqa: E402

DIMS, M0, SEED, BATCH, STEPS = (2, 2, 2, 2), -0.3, 5, 3, 2


def _samples(idx):
    U = synth.random_su3_links(DIMS, 0.3, 1)
    lev = multigrid.fine_level(U, M0, DIMS)
    t, _, _ = estimator.hutchinson(lev.matvec, lev.n, SEED, idx, 1e-12)
    return t


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    idx = parallel.sample_indices(rank, world, BATCH, STEPS)
    t = _samples(idx)
    gi, gt = parallel.gather_samples(t, idx)
    if rank == 0:
        np.save(out, np.stack([gi.astype(np.complex128), gt]))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_sample_offsets_partition_the_samples():
    world, batch, steps = 3, 4, 5
    allidx = np.concatenate([parallel.sample_indices(r, world, batch, steps) for r in range(world)])
    assert np.array_equal(np.sort(allidx), np.arange(world * batch * steps))
    with pytest.raises(ValueError):
        parallel.sample_offset(3, 3, 4, 0)


def test_two_rank_gather_equals_single_run(tmp_path):
    out = str(tmp_path / "gathered.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    gi, gt = np.load(out)
    n = 2 * BATCH * STEPS
    assert np.array_equal(gi.real.astype(int), np.arange(n))
    single = _samples(np.arange(n))
    assert np.array_equal(gt, single)
    a, b = estimator.statistics(gt), estimator.statistics(single)
    assert a == b
