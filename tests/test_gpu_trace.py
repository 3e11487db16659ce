"""GPU parity for the deflated Hutchinson estimator (Eq. 1, Algorithms 1 and
2): per-sample values against the oracle within the solver tolerance, the
device statistics against the oracle's statistics to rounding, the estimate
against the dense trace, and full-size properties of the estimator workload."""
import math

import numpy as np
import pytest

from oracle import deflation as odefl
from oracle import dense, estimator, philox
from oracle import multigrid as omg
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


def _check_stats(res):
    ref = estimator.statistics(res["t"], res["t0"])
    assert abs(res["mean"] - ref["mean"]) <= 1e-13 * abs(ref["mean"]) + 1e-13
    for key in ("var", "var_re", "stderr", "var_jackknife_err"):
        assert math.isclose(res[key], ref[key], rel_tol=1e-11), (key, res[key], ref[key])


def test_config1_alg1_against_oracle_and_dense_trace(qd, ctx):
    # 4^4, eps 0.3, m0 -0.4, s = 32, xi = 1e-10, 24 smallest eigvecs of A gamma5
    dims, m0, s, xi, k = (4, 4, 4, 4), -0.4, 32, 1e-10, 24
    U = synth.random_su3_links(dims, 0.3, 1)
    g = qd.Gauge(ctx, dims, U)
    A = dense.dirac_matrix(U, m0, dims)
    Ainv = dense.inverse(A)
    G5 = dense.gamma5_matrix(256)
    mu, Ue = odefl.fine_eigvecs_dense(A, G5, k)
    d = qd.Deflation(ctx, g, None, m0, 0.0, qd.defl_params(qd.QD_DEFL_EIG_ORTHO, k, solve_tol=xi),
                     injected_basis=qd.to_qd(ctx, g, Ue.reshape(256, 4, 3, k)))
    res = qd.hutchinson_trace(ctx, g, None, d, m0, 0.0, seed=101, sample_offset=0, nsamples=s, tol=xi,
                              maxit=20000, restart=32)
    assert res["max_true_rel_residual"] <= xi
    Z = philox.rademacher(3072, 101, range(s))
    B = Z - Ue @ (Ue.conj().T @ Z)
    t_exact = np.einsum("ij,ij->j", Z, Ainv @ B)
    kappa = np.linalg.cond(A)
    bound = kappa * xi * np.linalg.norm(Z, axis=0) * np.linalg.norm(B, axis=0)
    assert np.all(np.abs(res["t"] - t_exact) <= bound)
    _check_stats(res)
    tr = np.trace(Ainv)
    exact_t0 = np.sum(np.einsum("ni,nn,ni->i", Ue.conj(), G5, Ue) / mu)
    assert abs(res["t0"] - exact_t0) < 1e-6 * abs(exact_t0)
    var_exact = dense.exact_variance_real_rademacher(Ainv @ (np.eye(3072) - Ue @ Ue.conj().T))
    assert abs(res["estimate"].real - tr.real) < 4.0 * math.sqrt(var_exact / s)


def test_config1_gpu_eigensolver_end_to_end(qd, ctx):
    dims, m0, s, xi, k = (4, 4, 4, 4), -0.4, 32, 1e-10, 24
    U = synth.random_su3_links(dims, 0.3, 1)
    g = qd.Gauge(ctx, dims, U)
    A = dense.dirac_matrix(U, m0, dims)
    d = qd.Deflation(ctx, g, None, m0, 0.0, qd.defl_params(qd.QD_DEFL_EIG_ORTHO, k, guard=16, eig_tol=1e-8,
                                                           solve_tol=xi, maxit=60))
    mu_ref, _ = odefl.fine_eigvecs_dense(A, dense.gamma5_matrix(256), k)
    mu, _, _ = d.info()
    sep = np.abs(mu_ref) < 0.5 * np.abs(mu_ref[-1])   # the 12 isolated small modes
    assert sep.sum() >= 8
    assert np.allclose(np.abs(mu[sep]), np.abs(mu_ref[sep]), rtol=1e-7)
    assert np.allclose(np.abs(mu), np.abs(mu_ref), rtol=1e-2)
    res = qd.hutchinson_trace(ctx, g, None, d, m0, 0.0, seed=101, sample_offset=0, nsamples=s, tol=xi,
                              maxit=20000, restart=32)
    tr = np.trace(dense.inverse(A)).real
    assert abs(res["estimate"].real - tr) < 5.0 * res["stderr"] + 1e-6 * abs(tr)


def test_alg2_trace_matches_oracle_per_sample(qd, ctx):
    dims, m0, s, xi, k = (4, 4, 4, 4), -0.4, 16, 1e-10, 12
    U = synth.random_su3_links(dims, 0.3, 1)
    g = qd.Gauge(ctx, dims, U)
    p = qd.mg_params(1, [(2, 2, 2, 2)], [6], null_maxit=0, seed=3)
    mg = qd.Multigrid(ctx, g, m0, 0.0, p)
    H = omg.setup(U, m0, dims, [(2, 2, 2, 2)], [6], seed=3, null_maxit=0)
    alg = odefl.Alg2(H.transfers[0], H.matrices[0], k)
    d = qd.Deflation(ctx, g, mg, m0, 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, k), injected_basis=dev(alg.Ubar))
    res = qd.hutchinson_trace(ctx, g, mg, d, m0, 0.0, seed=7, sample_offset=5, nsamples=s, tol=xi,
                              want_coeffs=True)
    A = H.levels[0].matrix.toarray()
    Z = philox.rademacher(3072, 7, range(5, 5 + s))
    B = alg.project(H.levels[0].matvec, Z.astype(complex))
    t_exact = np.einsum("ij,ij->j", Z, np.linalg.solve(A, B))
    bound = np.linalg.cond(A) * xi * np.linalg.norm(Z, axis=0) * np.linalg.norm(B, axis=0)
    assert np.all(np.abs(res["t"] - t_exact) <= bound)
    _check_stats(res)
    rZhV, rUhKZ = alg.coeffs(Z.astype(complex))
    assert rel_err(res["ZhV"], rZhV) < 1e-11 and rel_err(res["UhKZ"], rUhKZ) < 1e-11
    # trace split: t0 + E[t1] = tr A^{-1} (one-SE check against the dense trace)
    tr = np.trace(np.linalg.inv(A)).real
    Bfull = np.linalg.inv(A) @ alg.project(H.levels[0].matvec, np.eye(3072, dtype=complex))
    var_exact = dense.exact_variance_real_rademacher(Bfull)
    assert abs(res["estimate"].real - tr) < 4.0 * math.sqrt(var_exact / s)


def test_estimator_workload_8x4_properties(qd, ctx):
    # the estimator workload at full size: 8^4, eps 0.3, m0 -0.8, two-level
    # MG (2^4, nv 12), Algorithm 2 with k = 24, s = 64, xi = 1e-8
    dims, m0, s, xi, k = (8, 8, 8, 8), -0.8, 64, 1e-8, 24
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [12]))
    d = qd.Deflation(ctx, g, mg, m0, 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, k, guard=16, eig_tol=1e-6,
                                                         solve_tol=1e-10, maxit=60))
    res = qd.hutchinson_trace(ctx, g, mg, d, m0, 0.0, seed=102, sample_offset=0, nsamples=s, tol=xi,
                              maxit=500, restart=16)
    assert res["status"] == qd.QD_OK and res["max_true_rel_residual"] <= xi
    _check_stats(res)
    # (I - P) is a projector and U^H g5 W^H (I - P) z = 0 (any size)
    z = torch.empty((g.V, 12, 4), dtype=torch.complex128, device="cuda:0")
    qd.rademacher(ctx, g, 102, 0, 4, z)
    pz = torch.empty_like(z)
    ppz = torch.empty_like(z)
    d.project(4, z, pz)
    d.project(4, pz, ppz)
    assert rel_err(host(ppz), host(pz)) < 1e-9
    _, uhkz = d.coeffs(4, pz)
    _, uhkz0 = d.coeffs(4, z)
    assert np.abs(uhkz).max() < 1e-9 * np.abs(uhkz0).max()
    # true residual of the GPU solve checked with the oracle's operator on two samples
    A = omg.fine_level(U, m0, dims).matrix
    b = host(pz)[..., :2]
    bd = dev(b)
    xd = torch.empty_like(bd)
    qd.solve(ctx, g, mg, m0, 0.0, 2, bd, xd, xi, maxit=500)
    eo = __import__("oracle.lattice", fromlist=["x"]).eo_index(dims)
    x_lex = host(xd)[eo].reshape(-1, 2)
    b_lex = b[eo].reshape(-1, 2)
    rel = np.linalg.norm(b_lex - A @ x_lex, axis=0) / np.linalg.norm(b_lex, axis=0)
    assert np.all(rel <= xi)
    # deflation reduces the sample variance against the undeflated estimator
    res0 = qd.hutchinson_trace(ctx, g, mg, None, m0, 0.0, seed=102, sample_offset=0, nsamples=s, tol=xi,
                               maxit=500, restart=16)
    assert res["var"] < res0["var"]


def test_trace_stats_entry_point_matches_oracle(qd, ctx):
    rng = np.random.default_rng(9)
    for s in (1, 2, 3, 17, 256):
        t = rng.standard_normal(s) * 3 + 1j * rng.standard_normal(s)
        got = qd.trace_stats(ctx, t, 2.5 - 0.5j)
        ref = estimator.statistics(t, 2.5 - 0.5j)
        assert abs(got["estimate"] - ref["estimate"]) <= 1e-13 * abs(ref["estimate"])
        for key in ("var", "var_re", "stderr", "var_jackknife_err"):
            assert math.isclose(got[key], ref[key], rel_tol=1e-11, abs_tol=1e-300), (s, key)


@pytest.mark.slow
def test_config3_three_level_mixed_precision(qd, ctx):
    # config 3 at full lattice size: 16^3 x 32, eps 0.2, m0 -0.8, three-level
    # MG (2^4, 2^4; nv 12, 16), Algorithm 2 (k = 24), mixed precision to a
    # true FP64 residual 1e-8; 16 samples keep the test short
    dims, m0, s, xi = (16, 16, 16, 32), -0.8, 16, 1e-8
    U = synth.random_su3_links(dims, 0.2, 3)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(2, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16]))
    assert mg.level_info(2)[1:3] == (32, 512)  # coarsest: 512 sites x 32 dofs (direct inverse)
    d = qd.Deflation(ctx, g, mg, m0, 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, 24, guard=16, eig_tol=1e-5,
                                                         solve_tol=1e-9, maxit=40))
    res = qd.hutchinson_trace(ctx, g, mg, d, m0, 0.0, seed=103, sample_offset=0, nsamples=s, tol=xi,
                              maxit=400, restart=16, precision=qd.QD_PREC_MIXED, inner_tol=1e-5, max_refine=10)
    assert res["status"] == qd.QD_OK and res["max_true_rel_residual"] <= xi
    _check_stats(res)
    # the FP64 residual of two samples recomputed with the oracle's operator
    z = torch.empty((g.V, 12, 2), dtype=torch.complex128, device="cuda:0")
    qd.rademacher(ctx, g, 103, 0, 2, z)
    b = torch.empty_like(z)
    d.project(2, z, b)
    x = torch.empty_like(b)
    qd.solve(ctx, g, mg, m0, 0.0, 2, b, x, xi, maxit=400, precision=qd.QD_PREC_MIXED, inner_tol=1e-5,
             max_refine=10)
    # (the oracle's matrix-free operator: its sparse matrix would be ~4 GB here)
    from oracle import wilson
    eo = __import__("oracle.lattice", fromlist=["x"]).eo_index(dims)
    bl = host(b)[eo].reshape(-1, 4, 3, 2)
    xl = host(x)[eo].reshape(-1, 4, 3, 2)
    r = bl - wilson.dirac_apply(U, xl, m0, dims)
    rel = np.linalg.norm(r.reshape(-1, 2), axis=0) / np.linalg.norm(bl.reshape(-1, 2), axis=0)
    assert np.all(rel <= xi), rel
    # t_j = z_j^H x_j for those samples
    zl = host(z)[eo].reshape(-1, 2)
    assert np.allclose(np.einsum("ij,ij->j", zl.conj(), xl.reshape(-1, 2)), res["t"][:2], rtol=1e-5)


def test_bench_path_8x4_against_oracle(qd, ctx):
    # The estimator workload's exact GPU path at 8^4 (eps 0.3, m0 -0.8,
    # two-level MG 2^4 / nv 12, Algorithm 2 with k = 24, xi = 1e-8): mixed
    # precision (FP32 GCR + FP32 V-cycle inside FP64 refinement), the learned
    # smoother with one MR step, captured V-cycle graphs, tensor-core coarsest
    # solve; compared per sample with the oracle on the same noise.  Both sides
    # use the oracle's null vectors (minimal residual to 1e-2 / 200 steps) and
    # its Algorithm 2 basis, so W, C and P are the same; the learned smoother
    # and the precisions only change how the solves get to xi.
    #
    # Bound: t_gpu - t_exact = z^H (x - A^{-1} b) = -(A^{-H} z)^H r with r the
    # GPU's final residual, so |t_gpu - t_exact| <= ||A^{-H} z|| ||r||.  The
    # oracle solves A y = gamma5 z to 1e-11: gamma5 A gamma5 = A^H gives
    # ||A^{-H} z|| = ||y|| and z^H A^{-1} z = y^H gamma5 z, and the deflated
    # t_exact = z^H A^{-1} z - (W^H z)^H U Lambda^{-1} U^H gamma5^W (W^H z)
    # (the scalar form of Algorithm 2, exact for any z).
    from oracle import krylov
    dims, m0, k, s, xi = (8, 8, 8, 8), -0.8, 24, 6, 1e-8
    U = synth.random_su3_links(dims, 0.3, 2)
    lev0 = omg.fine_level(U, m0, dims)
    Y, _ = omg.null_vectors(lev0, 12, 7, 1e-2, 200)
    H = omg.setup(U, m0, dims, [(2, 2, 2, 2)], [12], seed=7, injected_null=[Y])
    alg = odefl.Alg2(H.transfers[0], H.matrices[0], k)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [12], seed=7),
                      injected_null=qd.to_qd(ctx, g, Y.reshape(g.V, 4, 3, 12)))
    qd.smoother_train(mg, nsamples=4, solve_tol=1e-3, mr_steps=1)
    qd.smoother_enable(mg, True, 1)
    d = qd.Deflation(ctx, g, mg, m0, 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, k),
                     injected_basis=torch.from_numpy(np.ascontiguousarray(alg.Ubar)).to("cuda:0"))
    kw = dict(seed=102, sample_offset=0, nsamples=s, tol=xi, maxit=500, restart=16,
              precision=qd.QD_PREC_MIXED, inner_tol=1e-5, max_refine=10)
    runs = [qd.hutchinson_trace(ctx, g, mg, d, m0, 0.0, **kw) for _ in range(3)]  # eager, capture, replay
    res0 = qd.hutchinson_trace(ctx, g, mg, None, m0, 0.0, **kw)
    for r in runs + [res0]:
        assert r["status"] == qd.QD_OK and r["max_true_rel_residual"] <= xi
    assert abs(runs[-1]["t0"] - alg.t0) <= 1e-9 * abs(alg.t0)
    # oracle, per sample
    Z = philox.rademacher(lev0.n, 102, range(s)).astype(complex)
    g5 = np.tile(np.repeat([1.0, -1.0], 6), g.V)
    ZhV, UhKZ = alg.coeffs(Z)
    corr = alg.correction(ZhV, UhKZ, k)
    B = alg.project(lev0.matvec, Z)
    t_u, t_d, bound_u, bound_d = [], [], [], []
    for j in range(s):
        y, _, rel = krylov.gcr(lev0.matvec, g5 * Z[:, j], 1e-11, restart=16, precond=lambda v: H.vcycle(0, v))
        assert rel <= 1e-11
        tu = np.vdot(y, g5 * Z[:, j])
        t_u.append(tu)
        t_d.append(tu - corr[j])
        ny, nz = np.linalg.norm(y), np.linalg.norm(Z[:, j])
        slack = 1e-10 * ny * nz  # the oracle's own 1e-11 solve
        bound_u.append(ny * xi * nz + slack)
        bound_d.append(ny * xi * np.linalg.norm(B[:, j]) + slack)
    t_u, t_d = np.array(t_u), np.array(t_d)
    for r in runs:
        assert np.all(np.abs(r["t"] - t_d) <= bound_d), (np.abs(r["t"] - t_d) / bound_d).max()
    assert np.all(np.abs(res0["t"] - t_u) <= bound_u), (np.abs(res0["t"] - t_u) / bound_u).max()
    # the oracle's statistics of the same samples, and the variance reduction
    ref_d = estimator.statistics(t_d, alg.t0)
    ref_u = estimator.statistics(t_u)
    assert abs(runs[-1]["estimate"] - ref_d["estimate"]) <= max(bound_d) + 1e-9 * abs(alg.t0)
    ratio_gpu = res0["var"] / runs[-1]["var"]
    ratio_orc = ref_u["var"] / ref_d["var"]
    assert abs(ratio_gpu - ratio_orc) <= 1e-3 * ratio_orc, (ratio_gpu, ratio_orc)
    for o in (d, mg, g):
        o.close()
