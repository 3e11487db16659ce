"""GPU parity for the even-odd (Schur complement) fine solves (Sec. 4: the
paper's multigrid solves are even-odd preconditioned): the odd-site Schur
complement S = A_oo - A_oe A_ee^{-1} A_eo against the oracle's sparse S, and
solves through S (FP64 and mixed precision) against the oracle's operator."""
import numpy as np
import pytest

from oracle import lattice, wilson
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


@pytest.mark.parametrize("dims,tau", [((8, 4, 4, 4), 0.0), ((4, 4, 4, 8), 0.25), ((4, 2, 6, 2), 0.1)])
def test_schur_operator_against_oracle(qd, ctx, dims, tau):
    # the odd half of the qd layout holds the odd sites in lexicographic
    # order (one odd site per pair of lexicographic indices 2j, 2j + 1), so
    # a half field is the oracle's odd-site vector as it stands.  FP64 to
    # 1e-12; FP32: the stencil's two hops, each ~40 products per output, plus
    # the rounding of links and input, below 1e-5 relative
    m0 = -0.6
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    S, od = wilson.schur_odd_sparse(U, m0, dims, tau)
    assert np.array_equal(od // 2, np.arange(len(od)))
    rng = np.random.default_rng(4)
    for s in (1, 3, 64, 130):
        x = rng.standard_normal((len(od) * 12, s)) + 1j * rng.standard_normal((len(od) * 12, s))
        ref = S @ x
        xd = dev(x)
        y = torch.empty_like(xd)
        qd.dirac_schur_apply(ctx, g, m0, tau, s, xd, y)
        assert rel_err(host(y), ref) < 1e-12, s
        x32 = xd.to(torch.complex64)
        y32 = torch.empty_like(x32)
        qd.dirac_schur_apply_f32(ctx, g, m0, tau, s, x32, y32)
        assert rel_err(host(y32).astype(np.complex128), ref) < 1e-5, s
        # the launch shapes of the parity-restricted hops: whole, chunks of 64
        # and 32 columns (the same bits), projection on load, the operands
        # staged by bulk copies (4-6, nrhs a multiple of 64) or by cp.async
        # one hop ahead (7-8) (rounding)
        try:
            outs = []
            for cand in range(9):
                qd.autotune_force(cand)
                o = torch.full_like(x32, float("nan"))
                qd.dirac_schur_apply_f32(ctx, g, m0, tau, s, x32, o)
                outs.append(o)
            assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2]), s
            for cand in (3, 4, 5, 6, 7, 8):
                assert rel_err(host(outs[cand]), host(outs[0])) < 1e-6, (s, cand)
        finally:
            qd.autotune_force(-1)
    g.close()


def test_schur_staged_hops_at_8x4(qd, ctx):
    # the staged parity-restricted hops on 8^4 at 128 rhs: bulk-staged (4-6;
    # each warp takes several sites, 4096 units of 64 columns, the last
    # round ragged) and cp.async-staged (7-8), against the oracle's S
    # (sampled columns, FP32 tolerance as above)
    dims, m0, tau, s = (8, 8, 8, 8), -0.6, 0.1, 128
    U = synth.random_su3_links(dims, 0.3, 6)
    g = qd.Gauge(ctx, dims, U)
    S, od = wilson.schur_odd_sparse(U, m0, dims, tau)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((len(od) * 12, s)) + 1j * rng.standard_normal((len(od) * 12, s))
    x32 = dev(x).to(torch.complex64)
    cols = [0, 63, 64, 127]
    ref = S @ host(x32).astype(np.complex128)[:, cols]
    try:
        for cand in (4, 5, 6, 7, 8):
            qd.autotune_force(cand)
            o = torch.full_like(x32, float("nan"))
            qd.dirac_schur_apply_f32(ctx, g, m0, tau, s, x32, o)
            got = host(o).astype(np.complex128)
            assert np.isfinite(got).all(), cand
            assert rel_err(got[:, cols], ref) < 1e-5, cand
    finally:
        qd.autotune_force(-1)
    g.close()


@pytest.mark.parametrize("precision", ["f64", "mixed"])
def test_schur_solve_residual_against_oracle(qd, ctx, precision):
    # A x = b through the Schur complement, preconditioned by the odd block
    # of the three-level V-cycle: the true residual, recomputed with the
    # oracle's operator, meets the tolerance per column, and the solution
    # agrees with the full-lattice solve to the conditioning of A
    dims, m0, tol, s = (8, 8, 8, 8), -0.8, 1e-8, 6
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(2, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16], coarse_tol=0.0,
                                                     coarse_maxit=6))
    rng = np.random.default_rng(9)
    b = rng.standard_normal((g.V, 12, s)) + 1j * rng.standard_normal((g.V, 12, s))
    bd = dev(b)
    prec = qd.QD_PREC_MIXED if precision == "mixed" else qd.QD_PREC_F64
    x_eo = torch.empty_like(bd)
    x_full = torch.empty_like(bd)
    _, its_eo, _, rel_eo = qd.solve(ctx, g, mg, m0, 0.0, s, bd, x_eo, tol, maxit=500, precision=prec, schur=1)
    _, its_full, _, rel_full = qd.solve(ctx, g, mg, m0, 0.0, s, bd, x_full, tol, maxit=500, precision=prec)
    assert max(rel_eo) <= tol
    A = wilson.dirac_sparse(U, m0, dims)
    eo = lattice.eo_index(dims)
    xl = host(x_eo)[eo].reshape(-1, s)
    bl = b[eo].reshape(-1, s)
    res = np.linalg.norm(bl - A @ xl, axis=0) / np.linalg.norm(bl, axis=0)
    assert res.max() <= 1.05 * tol, res
    # both solutions within kappa * tol of each other (kappa of A at this
    # mass is below 100 on this lattice; the bound is generous)
    assert rel_err(host(x_eo), host(x_full)) < 100 * 2 * tol
    print(precision, "iterations: even-odd", its_eo, "full", its_full)
    mg.close()
    g.close()


def test_schur_trace_matches_full_solve(qd, ctx):
    # the estimator's per-sample values with the even-odd solves agree with
    # the full-lattice solves to the solve tolerance
    dims, m0 = (8, 8, 8, 8), -0.8
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [12]))
    d = qd.Deflation(ctx, g, mg, m0, 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, 24))
    out = {}
    for schur in (0, 1):
        out[schur] = qd.hutchinson_trace(ctx, g, mg, d, m0, 0.0, seed=7, sample_offset=0, nsamples=16, tol=1e-9,
                                         precision=qd.QD_PREC_MIXED, schur=schur)
    t0, t1 = np.asarray(out[0]["t"]), np.asarray(out[1]["t"])
    assert np.abs(t0 - t1).max() < 1e-6 * np.abs(t0).max()
    for o in (d, mg, g):
        o.close()
