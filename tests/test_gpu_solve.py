"""GPU solves (Sec. 1 inexact solves, Sec. 2 multigrid): the true residual
meets the tolerance when checked by the oracle's operator, the error obeys
the kappa * xi bound against a dense solve, and failures are reported."""
import numpy as np
import pytest

from oracle import dense, multigrid as omg
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


def test_unpreconditioned_solve_small(qd, ctx):
    dims, m0 = (4, 4, 2, 2), -0.4
    U = synth.random_su3_links(dims, 0.3, 8)
    g = qd.Gauge(ctx, dims, U)
    A = dense.dirac_matrix(U, m0, dims)
    b = synth.random_field(dims, 5, 1)
    bd = qd.to_qd(ctx, g, b)
    xd = torch.empty_like(bd)
    rc, its, it_col, rel = qd.solve(ctx, g, None, m0, 0.0, 5, bd, xd, 1e-10, maxit=5000, restart=16)
    x = qd.from_qd(ctx, g, xd).reshape(-1, 5)
    B = b.reshape(-1, 5)
    true_rel = np.linalg.norm(B - A @ x, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(true_rel <= 1e-10)
    assert np.allclose(true_rel, rel, rtol=1e-3)
    x_lu = np.linalg.solve(A, B)
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= np.linalg.cond(A) * 1e-10


def test_mg_solve_8x4(qd, ctx):
    dims, m0, s = (8, 8, 8, 8), -0.8, 8
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [12]))
    b = synth.random_field(dims, s, 4)
    bd = qd.to_qd(ctx, g, b)
    xd = torch.empty_like(bd)
    rc, its, it_col, rel = qd.solve(ctx, g, mg, m0, 0.0, s, bd, xd, 1e-8, maxit=500, restart=16)
    x = qd.from_qd(ctx, g, xd).reshape(-1, s)
    A = omg.fine_level(U, m0, dims).matrix
    B = b.reshape(-1, s)
    true_rel = np.linalg.norm(B - A @ x, axis=0) / np.linalg.norm(B, axis=0)
    assert np.all(true_rel <= 1e-8), true_rel
    assert its < 100, its  # multigrid preconditioning works


def test_not_converged_is_reported(qd, ctx):
    dims, m0 = (4, 4, 4, 4), -0.4
    g = qd.Gauge(ctx, dims, synth.random_su3_links(dims, 0.3, 1))
    bd = qd.to_qd(ctx, g, synth.random_field(dims, 2, 1))
    xd = torch.empty_like(bd)
    rc, its, it_col, rel = qd.solve(ctx, g, None, m0, 0.0, 2, bd, xd, 1e-12, maxit=1, restart=4,
                                    allow_not_converged=True)
    assert rc == qd.QD_ERR_NOT_CONVERGED and its == 1 and all(r > 1e-12 for r in rel)


def test_nonfinite_input_is_reported(qd, ctx):
    dims, m0 = (4, 4, 4, 4), -0.4
    g = qd.Gauge(ctx, dims, synth.random_su3_links(dims, 0.3, 1))
    b = synth.random_field(dims, 2, 1)
    b[3, 1, 2, 1] = np.nan
    bd = qd.to_qd(ctx, g, b)
    xd = torch.empty_like(bd)
    with pytest.raises(qd.QDError) as e:
        qd.solve(ctx, g, None, m0, 0.0, 2, bd, xd, 1e-8, maxit=10)
    assert e.value.code == qd.QD_ERR_NONFINITE


def test_zero_rhs_column(qd, ctx):
    dims, m0 = (4, 4, 4, 4), -0.4
    g = qd.Gauge(ctx, dims, synth.random_su3_links(dims, 0.3, 1))
    b = synth.random_field(dims, 3, 1)
    b[..., 1] = 0.0
    bd = qd.to_qd(ctx, g, b)
    xd = torch.empty_like(bd)
    rc, its, it_col, rel = qd.solve(ctx, g, None, m0, 0.0, 3, bd, xd, 1e-9, maxit=3000)
    x = qd.from_qd(ctx, g, xd)
    assert np.all(x[..., 1] == 0) and rel[1] == 0.0 and rel[0] <= 1e-9


@pytest.mark.parametrize("dims,m0,seed,blocks,nvs", [((4, 4, 4, 4), -0.4, 1, [(2, 2, 2, 2)], [6]),
                                                     ((8, 8, 8, 8), -0.8, 2, [(2, 2, 2, 2)], [12]),
                                                     ((8, 8, 8, 8), -0.8, 2, [(2, 2, 2, 2), (2, 2, 2, 2)],
                                                      [12, 16])])
def test_mixed_precision_refinement(qd, ctx, dims, m0, seed, blocks, nvs):
    # FP32 V-cycle + FP32 GCR inside FP64 refinement: the FP64 true residual
    # (checked here with the oracle's operator) meets 1e-8 and 1e-10
    s = 6
    U = synth.random_su3_links(dims, 0.3, seed)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(len(blocks), blocks, nvs))
    A = omg.fine_level(U, m0, dims).matrix
    b = synth.random_field(dims, s, 7)
    bd = qd.to_qd(ctx, g, b)
    for tol in (1e-8, 1e-10):
        xd = torch.empty_like(bd)
        rc, its, it_col, rel = qd.solve(ctx, g, mg, m0, 0.0, s, bd, xd, tol, maxit=200, restart=16,
                                        precision=qd.QD_PREC_MIXED, inner_tol=1e-5, max_refine=10)
        x = qd.from_qd(ctx, g, xd).reshape(-1, s)
        B = b.reshape(-1, s)
        true_rel = np.linalg.norm(B - A @ x, axis=0) / np.linalg.norm(B, axis=0)
        assert np.all(true_rel <= tol), true_rel
        assert np.allclose(true_rel, rel, rtol=1e-3, atol=1e-3 * tol)


@pytest.mark.parametrize("blocks,nvs,kw", [([(2, 2, 2, 2)], [12], {}),
                                           ([(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16],
                                            {"coarse_tol": 0.0, "coarse_maxit": 6})])
def test_vcycle_graph_replay_matches_eager(qd, ctx, blocks, nvs, kw):
    # the captured V-cycle (CUDA graph) replays exactly the eager launches:
    # bit-identical solutions, mixed and FP64, two and three levels (the
    # three-level case with a fixed-iteration level-1 GCR, which needs no
    # host synchronisation); the solution meets the FP64 true residual
    dims, m0, s = (8, 8, 8, 8), -0.8, 8
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    b = synth.random_field(dims, s, 11)
    bd = qd.to_qd(ctx, g, b)
    A = omg.fine_level(U, m0, dims).matrix
    for prec in (qd.QD_PREC_MIXED, qd.QD_PREC_F64):
        xs = []
        for graphs in (0, 1):
            mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(len(blocks), blocks, nvs, use_graphs=graphs, **kw))
            for rep in range(3):  # eager warm-up, capture, replay
                xd = torch.empty_like(bd)
                rc, its, _, rel = qd.solve(ctx, g, mg, m0, 0.0, s, bd, xd, 1e-10, maxit=300, restart=16,
                                           precision=prec, inner_tol=1e-5, max_refine=10)
                xs.append(xd.clone())
            mg.close()
        for x in xs[1:]:
            assert torch.equal(x, xs[0])
        x = qd.from_qd(ctx, g, xs[-1]).reshape(-1, s)
        B = b.reshape(-1, s)
        assert np.all(np.linalg.norm(B - A @ x, axis=0) / np.linalg.norm(B, axis=0) <= 1e-10)
