"""GPU parity for the deflation spaces (Algorithm 1 and Algorithm 2): with an
injected basis the projector, t0, Lambda and the Sec. 2.2 coefficients match
the oracle to rounding; the GPU eigensolver finds the oracle's eigenvalues."""
import numpy as np
import pytest

from oracle import deflation as odefl
from oracle import dense
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


@pytest.fixture(scope="module")
def two_level(qd, ctx):
    dims, m0 = (4, 4, 4, 4), -0.4
    U = synth.random_su3_links(dims, 0.3, 1)
    g = qd.Gauge(ctx, dims, U)
    p = qd.mg_params(1, [(2, 2, 2, 2)], [6], null_maxit=0, seed=3)
    mg = qd.Multigrid(ctx, g, m0, 0.0, p)
    H = omg.setup(U, m0, dims, [(2, 2, 2, 2)], [6], seed=3, null_maxit=0)
    return dict(dims=dims, m0=m0, U=U, g=g, mg=mg, H=H)


def _check_spectrum(mu, mu_ref):
    """Eigenvalues well separated from the cut (|mu| < |mu_k| / 2) to 1e-7;
    the rest, which may sit in a dense cluster, to 1e-2."""
    mu, mu_ref = np.abs(mu), np.abs(mu_ref)
    sep = mu_ref < 0.5 * mu_ref[-1]
    assert np.allclose(mu[sep], mu_ref[sep], rtol=1e-7)
    assert np.allclose(mu, mu_ref, rtol=1e-2)


def test_alg2_injected_basis(qd, ctx, two_level):
    t = two_level
    k = 10
    alg = odefl.Alg2(t["H"].transfers[0], t["H"].matrices[0], k)
    d = qd.Deflation(ctx, t["g"], t["mg"], t["m0"], 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, k),
                     injected_basis=dev(alg.Ubar))
    t0 = d.set_rank(k)
    assert abs(t0 - alg.t0) < 1e-10 * abs(alg.t0)
    _, lam, _ = d.info()
    assert rel_err(np.sort(lam), np.sort(alg.lam)) < 1e-11
    # (I - P) z for Rademacher-like and complex z
    s = 3
    z = synth.random_field(t["dims"], s, 4)
    zd = qd.to_qd(ctx, t["g"], z)
    out = torch.empty_like(zd)
    d.project(s, zd, out)
    got = qd.from_qd(ctx, t["g"], out).reshape(-1, s)
    ref = alg.project(t["H"].levels[0].matvec, z.reshape(-1, s))
    assert rel_err(got, ref) < 1e-10
    # Sec. 2.2 coefficients
    ZhV, UhKZ = d.coeffs(s, zd)
    rZhV, rUhKZ = alg.coeffs(z.reshape(-1, s))
    assert rel_err(ZhV, rZhV) < 1e-11 and rel_err(UhKZ, rUhKZ) < 1e-11
    # a-posteriori rank sweep: set_rank(r) equals the oracle at rank r
    for r in (4, 7):
        t0r = d.set_rank(r)
        assert abs(t0r - alg.t0_rank(r)) < 1e-9 * abs(alg.t0_rank(r))
        alg.set_rank(r)
        d.project(s, zd, out)
        ref = alg.project(t["H"].levels[0].matvec, z.reshape(-1, s))
        assert rel_err(qd.from_qd(ctx, t["g"], out).reshape(-1, s), ref) < 1e-10
    alg.set_rank(k)


def test_alg2_eigensolver(qd, ctx):
    # real null vectors (oracle MR iteration, injected) give a coarse operator
    # whose C gamma5^W has isolated small eigenvalues; k = 8 sits at a gap
    dims, m0, nv, k = (4, 4, 4, 4), -0.4, 6, 8
    U = synth.random_su3_links(dims, 0.3, 1)
    g = qd.Gauge(ctx, dims, U)
    lev = omg.fine_level(U, m0, dims)
    Y, _ = omg.null_vectors(lev, nv, 3, 1e-2, 200)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [nv], seed=3),
                      injected_null=qd.to_qd(ctx, g, Y.reshape(g.V, 4, 3, nv)))
    T = omg.build_transfer(lev, (2, 2, 2, 2), Y)
    C = omg.coarse_matrix(lev, T)
    g5 = np.tile(np.repeat([1.0, -1.0], nv), C.shape[0] // (2 * nv))
    Hm = C.toarray() * g5[None, :]
    mu_all = np.linalg.eigvalsh(0.5 * (Hm + Hm.conj().T))
    mu_ref = mu_all[np.argsort(np.abs(mu_all))[:k]]
    d = qd.Deflation(ctx, g, mg, m0, 0.0,
                     qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, k, guard=8, eig_tol=1e-9, solve_tol=1e-12, maxit=60))
    mu, lam, its = d.info()
    assert its < 60
    assert np.allclose(np.sort(np.abs(mu)), np.sort(np.abs(mu_ref)), rtol=1e-8)
    # the converged k-space is unique, so t0 and the projector agree with the
    # oracle's Algorithm 2 built on the exact eigenvectors
    alg = odefl.Alg2(T, C, k)
    assert abs(d.set_rank(k) - alg.t0) < 1e-7 * abs(alg.t0)
    s = 2
    z = synth.random_field(dims, s, 4)
    zd = qd.to_qd(ctx, g, z)
    out = torch.empty_like(zd)
    d.project(s, zd, out)
    ref = alg.project(lev.matvec, z.reshape(-1, s))
    assert rel_err(qd.from_qd(ctx, g, out).reshape(-1, s), ref) < 1e-7


def test_alg1_injected_and_eigensolver(qd, ctx):
    dims, m0 = (4, 4, 2, 2), -0.4
    U = synth.random_su3_links(dims, 0.3, 8)
    g = qd.Gauge(ctx, dims, U)
    A = dense.dirac_matrix(U, m0, dims)
    G5 = dense.gamma5_matrix(64)
    k = 12
    mu_ref, Ue = odefl.fine_eigvecs_dense(A, G5, k)
    Ud = qd.to_qd(ctx, g, Ue.reshape(64, 4, 3, k))
    d = qd.Deflation(ctx, g, None, m0, 0.0, qd.defl_params(qd.QD_DEFL_EIG_ORTHO, k, solve_tol=1e-11),
                     injected_basis=Ud)
    t0 = d.set_rank(k)
    direct = np.sum(np.einsum("ni,nn,ni->i", Ue.conj(), G5, Ue) / mu_ref)
    assert abs(t0 - direct) < 1e-7 * abs(direct)
    s = 2
    z = synth.random_field(dims, s, 3)
    zd = qd.to_qd(ctx, g, z)
    out = torch.empty_like(zd)
    d.project(s, zd, out)
    Z = z.reshape(-1, s)
    assert rel_err(qd.from_qd(ctx, g, out).reshape(-1, s), Z - Ue @ (Ue.conj().T @ Z)) < 1e-12
    # eigensolver on the fine operator (unpreconditioned inner solves)
    d2 = qd.Deflation(ctx, g, None, m0, 0.0, qd.defl_params(qd.QD_DEFL_EIG_ORTHO, k, guard=12, eig_tol=1e-8,
                                                             solve_tol=1e-12, maxit=60))
    mu, _, its = d2.info()
    _check_spectrum(mu, mu_ref)


def test_alg2_three_level_composite(qd, ctx):
    # two coarse levels: the deflation space lives on the coarsest level
    # (4 sites x 8 dofs here) and W is the composite prolongator W_0 W_1
    dims, m0, k, blocks, nvs = (4, 4, 4, 4), -0.4, 10, [(2, 2, 2, 2), (2, 2, 1, 1)], [6, 4]
    U = synth.random_su3_links(dims, 0.3, 1)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(2, blocks, nvs, null_maxit=0, seed=3))
    H = omg.setup(U, m0, dims, blocks, nvs, seed=3, null_maxit=0)
    alg = odefl.Alg2(odefl.Composite(H.transfers), H.matrices[-1], k)
    d = qd.Deflation(ctx, g, mg, m0, 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, k),
                     injected_basis=dev(alg.Ubar))
    t0 = d.set_rank(k)
    assert abs(t0 - alg.t0) < 1e-10 * abs(alg.t0)
    _, lam, _ = d.info()
    assert rel_err(np.sort(lam), np.sort(alg.lam)) < 1e-11
    s = 3
    z = synth.random_field(dims, s, 4)
    zd = qd.to_qd(ctx, g, z)
    out = torch.empty_like(zd)
    d.project(s, zd, out)
    ref = alg.project(H.levels[0].matvec, z.reshape(-1, s))
    assert rel_err(qd.from_qd(ctx, g, out).reshape(-1, s), ref) < 1e-10
    ZhV, UhKZ = d.coeffs(s, zd)
    rZhV, rUhKZ = alg.coeffs(z.reshape(-1, s))
    assert rel_err(ZhV, rZhV) < 1e-11 and rel_err(UhKZ, rUhKZ) < 1e-11
    # the GPU eigensolver on the coarsest operator (direct inverse) finds the
    # oracle's eigenvalues of C gamma5^W, and the estimator's trace split holds
    d2 = qd.Deflation(ctx, g, mg, m0, 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, k, guard=8, eig_tol=1e-10,
                                                          maxit=60))
    mu, _, _ = d2.info()
    _check_spectrum(mu, alg.mu)
    A = H.levels[0].matrix.toarray()
    res = qd.hutchinson_trace(ctx, g, mg, d2, m0, 0.0, seed=7, sample_offset=0, nsamples=16, tol=1e-10)
    Ainv = np.linalg.inv(A)
    assert abs(res["estimate"].real - np.trace(Ainv).real) < 5.0 * res["stderr"] + 1e-8
