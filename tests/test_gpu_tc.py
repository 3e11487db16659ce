"""The coarsest solve of the FP32 V-cycle on tcgen05 tensor cores (BF16
operands, FP32 accumulate) against the FP64 direct solve: relative error at
BF16 level (the inputs carry 8 mantissa bits), for several right-hand-side
counts including a ragged 16-column tail and a chunked batch."""
import numpy as np
import pytest

from paper_1909_12234_gb300 import synth

from gpu_util import dev, host, need_gpu, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qd():
    need_gpu()
    from paper_1909_12234_gb300 import qdtrace
    qdtrace.load()
    return qdtrace


@pytest.fixture(scope="module")
def ctx(qd):
    return qd.Context(0)


def _coarse_pair(qd, mg, level, n, s, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((n, s)) + 1j * rng.standard_normal((n, s))
    y64 = torch.empty((n * s,), dtype=torch.complex128, device="cuda:0")
    qd.coarse_solve(mg, level, s, dev(x), y64)
    x32 = torch.from_numpy(np.ascontiguousarray(x.astype(np.complex64))).to("cuda:0")
    y32 = torch.empty((n, s), dtype=torch.complex64, device="cuda:0")
    qd.coarse_solve_f32(mg, level, s, x32, y32)
    return host(y32).astype(np.complex128), host(y64).reshape(n, s)


@pytest.mark.parametrize("dims,m0,nv,svals", [((4, 4, 4, 4), -0.4, 6, [3, 64]),
                                              ((8, 8, 8, 8), -0.8, 12, [64, 5, 130])])
def test_tensor_core_coarsest_solve(qd, ctx, dims, m0, nv, svals):
    g = qd.Gauge(ctx, dims, synth.random_su3_links(dims, 0.3, 2))
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [nv], null_maxit=30))
    n = (np.prod(dims) // 16) * 2 * nv
    for i, s in enumerate(svals):
        got, ref = _coarse_pair(qd, mg, 1, n, s, i)
        err = rel_err(got, ref)
        assert err < 3e-2, (s, err)
        # column-wise relative error as well (each right-hand side separately)
        colerr = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert colerr.max() < 3e-2, (s, colerr.max())


def test_fp32_cuda_core_coarsest_solve(qd, ctx):
    dims = (4, 4, 4, 4)
    g = qd.Gauge(ctx, dims, synth.random_su3_links(dims, 0.3, 2))
    mg = qd.Multigrid(ctx, g, -0.4, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [6], null_maxit=30, coarsest_bf16=0))
    got, ref = _coarse_pair(qd, mg, 1, 16 * 12, 7, 3)
    assert rel_err(got, ref) < 1e-5
