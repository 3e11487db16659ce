"""The uneven batch (qd_hutchinson_batch): several estimators of different
lattice size, mass, depth, precision and sample count solved concurrently
give per-sample values bit-identical to lone calls on the same inputs, and
each meets its FP64 true residual."""
import numpy as np
import pytest

from paper_1909_12234_gb300 import synth

from gpu_util import need_gpu

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


def _problem(qd, ctx, dims, eps, seed, m0, blocks, nvs, k, s, precision, mg_kw):
    U = synth.random_su3_links(dims, eps, seed)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(len(blocks), blocks, nvs, **mg_kw))
    d = qd.Deflation(ctx, g, mg, m0, 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, k, guard=16, eig_tol=1e-6,
                                                         solve_tol=1e-10, maxit=60))
    return dict(gauge=g, mg=mg, defl=d, m0=m0, tau=0.0, seed=100 + seed, sample_offset=3, nsamples=s, tol=1e-8,
                maxit=500, restart=16, precision=precision, inner_tol=1e-5, max_refine=10)


def test_batch_matches_lone_calls(qd, ctx):
    fixed = {"coarse_tol": 0.0, "coarse_maxit": 6}
    probs = [
        _problem(qd, ctx, (8, 8, 8, 8), 0.2, 4, -0.6, [(2, 2, 2, 2)], [12], 16, 16, qd.QD_PREC_MIXED, {}),
        _problem(qd, ctx, (12, 12, 12, 12), 0.2, 5, -0.75, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16], 24, 48,
                 qd.QD_PREC_MIXED, fixed),
        _problem(qd, ctx, (8, 8, 8, 8), 0.2, 6, -0.8, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16], 24, 24,
                 qd.QD_PREC_F64, {}),
    ]
    keys = ("gauge", "mg", "defl", "m0", "tau", "seed", "sample_offset", "nsamples", "tol")
    lone = []
    for p in probs:
        kw = {k: v for k, v in p.items() if k not in keys}
        lone.append(qd.hutchinson_trace(ctx, p["gauge"], p["mg"], p["defl"], p["m0"], 0.0, p["seed"],
                                        p["sample_offset"], p["nsamples"], p["tol"], **kw))
    for nstreams in (3, 2, 1):
        got = qd.hutchinson_batch(ctx, probs, nstreams=nstreams)
        for a, b in zip(got, lone):
            assert a["status"] == qd.QD_OK
            assert np.array_equal(a["t"], b["t"])
            assert a["estimate"] == b["estimate"] and a["var"] == b["var"]
            assert a["max_true_rel_residual"] <= 1e-8


def test_batch_rejects_shared_handles(qd, ctx):
    p = _problem(qd, ctx, (4, 4, 4, 4), 0.3, 1, -0.4, [(2, 2, 2, 2)], [6], 8, 4, qd.QD_PREC_F64, {})
    with pytest.raises(qd.QDError) as e:
        qd.hutchinson_batch(ctx, [p, dict(p)], nstreams=2)
    assert e.value.code == qd.QD_ERR_INVALID
    assert qd.hutchinson_batch(ctx, [], nstreams=2) == []
