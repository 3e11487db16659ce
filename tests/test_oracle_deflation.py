"""Pins for oracle.deflation against dense matrices (Algorithms 1 and 2)."""
import numpy as np
import pytest

from oracle import deflation, dense, multigrid
from paper_1909_12234_gb300 import synth


@pytest.fixture(scope="module")
def setup():
    dims = (4, 4, 2, 2)
    U = synth.random_su3_links(dims, 0.3, 8)  # kappa(A) ~ 160: restarted GCR converges
    m0 = -0.4
    H = multigrid.setup(U, m0, dims, [(2, 2, 2, 2)], [6], seed=3, null_maxit=50)
    A = H.levels[0].matrix.toarray()
    Ainv = dense.inverse(A)
    G5 = dense.gamma5_matrix(64)
    return dict(H=H, A=A, Ainv=Ainv, G5=G5)


def _dense_P(alg, setup):
    W = alg.T.matrix().toarray()
    g5c = np.diag(alg.g5)
    return setup["A"] @ W @ alg.U @ np.diag(1.0 / alg.lam) @ alg.U.conj().T @ g5c @ W.conj().T


def test_alg2_projector_identities(setup):
    H = setup["H"]
    alg = deflation.Alg2(H.transfers[0], H.matrices[0], 10)
    P = _dense_P(alg, setup)
    assert np.abs(P @ P - P).max() < 1e-10 * np.abs(P).max()
    B = setup["Ainv"] @ (np.eye(P.shape[0]) - P)
    G5 = setup["G5"]
    assert np.abs(G5 @ B @ G5 - B.conj().T).max() < 1e-10 * np.abs(B).max()
    # trace split of Sec. 2.1: t0 + tr(A^{-1}(I - P)) = tr A^{-1}
    assert abs(alg.t0 + np.trace(B) - np.trace(setup["Ainv"])) < 1e-9 * abs(np.trace(setup["Ainv"]))
    # t0 equals tr(A^{-1} P) computed densely
    assert abs(alg.t0 - np.trace(setup["Ainv"] @ P)) < 1e-9 * abs(alg.t0)


def test_alg2_vector_and_scalar_forms(setup):
    H = setup["H"]
    alg = deflation.Alg2(H.transfers[0], H.matrices[0], 10)
    rng = np.random.default_rng(4)
    Z = np.sign(rng.standard_normal((setup["A"].shape[0], 3))) + 0j
    Ainv = setup["Ainv"]
    vec = np.einsum("ij,ij->j", Z.conj(), Ainv @ alg.project(H.levels[0].matvec, Z))
    ZhV, UhKZ = alg.coeffs(Z)
    scal = np.einsum("ij,ij->j", Z.conj(), Ainv @ Z) - alg.correction(ZhV, UhKZ, alg.k)
    assert np.allclose(vec, scal, rtol=1e-10)
    # rank sweep from the stored k x s matrices equals rebuilding at that rank
    for r in (3, 7):
        t0r = alg.t0_rank(r)
        corr = alg.correction(ZhV, UhKZ, r)
        alg.set_rank(r)
        assert abs(t0r - alg.t0) < 1e-10 * abs(alg.t0)
        v = np.einsum("ij,ij->j", Z.conj(), Ainv @ alg.project(H.levels[0].matvec, Z))
        s = np.einsum("ij,ij->j", Z.conj(), Ainv @ Z) - corr
        assert np.allclose(v, s, rtol=1e-10)
    alg.set_rank(alg.k)


def test_alg2_smallest_eigvecs(setup):
    H = setup["H"]
    alg = deflation.Alg2(H.transfers[0], H.matrices[0], 10)
    Hd = H.matrices[0].toarray() * alg.g5[None, :]
    mu_all = np.linalg.eigvalsh(0.5 * (Hd + Hd.conj().T))
    want = np.sort(np.abs(mu_all))[:10]
    assert np.allclose(np.abs(alg.mu), want, rtol=1e-10)
    assert np.allclose(alg.Ubar.conj().T @ alg.Ubar, np.eye(10), atol=1e-12)


def test_alg1_identities(setup):
    A, Ainv, G5 = setup["A"], setup["Ainv"], setup["G5"]
    mu, Ue = deflation.fine_eigvecs_dense(A, G5, 12)
    # exact eigenvectors: u^H A^{-1} u = u^H gamma5 u / mu
    direct = np.sum(np.einsum("ni,nn,ni->i", Ue.conj(), G5, Ue) / mu)
    xi = 1e-11
    a1 = deflation.Alg1(Ue, setup["H"].levels[0].matvec, xi)
    # each solve is within kappa * xi of the exact one (k = 12 solves)
    bound = 12 * np.linalg.cond(A) * xi * np.max(np.abs(1.0 / mu))
    assert abs(a1.t0 - direct) < 10 * bound
    Pp = np.eye(A.shape[0]) - Ue @ Ue.conj().T
    assert abs(a1.t0 + np.trace(Ainv @ Pp) - np.trace(Ainv)) < 10 * bound
    # deflating the smallest |mu| lowers the exact variance
    v0 = dense.exact_variance_real_rademacher(Ainv)
    v1 = dense.exact_variance_real_rademacher(Ainv @ Pp)
    assert v1 < v0


def test_alg2_three_level_composite(setup):
    # two coarse levels (2^4 then 2^4): the deflation space lives on the
    # coarsest level and W is the composite prolongator
    dims = (4, 4, 4, 4)
    U = synth.random_su3_links(dims, 0.3, 1)
    H = multigrid.setup(U, -0.4, dims, [(2, 2, 2, 2), (2, 2, 2, 2)], [6, 8], seed=3, null_maxit=30)
    A = H.levels[0].matrix.toarray()
    W = deflation.Composite(H.transfers)
    Wd = W.matrix().toarray()
    C2 = H.matrices[1].toarray()
    assert Wd.shape == (3072, 16) and C2.shape == (16, 16)
    # composite Galerkin identity and chirality of the composite
    assert np.abs(Wd.conj().T @ A @ Wd - C2).max() < 1e-12 * np.abs(C2).max()
    G5 = dense.gamma5_matrix(256)
    g5c = np.repeat([1.0, -1.0], 8)
    assert np.abs(G5 @ Wd - Wd * g5c[None, :]).max() < 1e-13
    assert np.abs(Wd.conj().T @ Wd - np.eye(16)).max() < 1e-12
    rng = np.random.default_rng(2)
    x = rng.standard_normal((16, 2)) + 1j * rng.standard_normal((16, 2))
    assert np.allclose(W.prolong(x), Wd @ x, atol=1e-13)
    f = rng.standard_normal((3072, 2)) + 1j * rng.standard_normal((3072, 2))
    assert np.allclose(W.restrict(f), Wd.conj().T @ f, atol=1e-12)
    alg = deflation.Alg2(W, H.matrices[1], 12)
    Ainv = dense.inverse(A)
    P = A @ Wd @ alg.U @ np.diag(1.0 / alg.lam) @ alg.U.conj().T @ np.diag(alg.g5) @ Wd.conj().T
    assert np.abs(P @ P - P).max() < 1e-10 * np.abs(P).max()
    B = Ainv @ (np.eye(3072) - P)
    assert abs(alg.t0 + np.trace(B) - np.trace(Ainv)) < 1e-9 * abs(np.trace(Ainv))
    Z = np.sign(rng.standard_normal((3072, 3))) + 0j
    assert np.allclose(alg.project(H.levels[0].matvec, Z), Z - P @ Z, atol=1e-10)


def test_alg1_rank_sweep_coefficients(setup):
    # z^H A^{-1}(I - U_r U_r^H) z from the stored s x k and k x s matrices
    # equals the vector form for every r, and t0 at rank r is the partial sum
    A, Ainv, G5 = setup["A"], setup["Ainv"], setup["G5"]
    _, Ue = deflation.fine_eigvecs_dense(A, G5, 12)
    lev = setup["H"].levels[0]
    a1 = deflation.Alg1(Ue, lev.matvec, 1e-12)
    rng = np.random.default_rng(5)
    Z = np.sign(rng.standard_normal((A.shape[0], 4))) + 0j
    ZhAU, UhZ = a1.coeffs(Z)
    t_und = np.einsum("ij,ij->j", Z.conj(), Ainv @ Z)
    for r in (1, 5, 12):
        Ur = Ue[:, :r]
        vec = np.einsum("ij,ij->j", Z.conj(), Ainv @ (Z - Ur @ (Ur.conj().T @ Z)))
        assert np.allclose(t_und - a1.correction(ZhAU, UhZ, r), vec, rtol=1e-9)
        assert abs(a1.t0_rank(r) - np.trace(Ur.conj().T @ Ainv @ Ur)) < 1e-9 * abs(a1.t0_rank(r))


def test_subspace_sines(setup):
    # columns of W: angle 0; vectors orthogonal to range(W): sin 1; random:
    # the dense projector's value
    T = setup["H"].transfers[0]
    W = T.matrix().toarray()
    s0 = deflation.subspace_sines(T, W[:, :5])
    assert np.all(s0 < 1e-12)
    rng = np.random.default_rng(6)
    V = rng.standard_normal((W.shape[0], 3)) + 1j * rng.standard_normal((W.shape[0], 3))
    Vperp = V - W @ (W.conj().T @ V)
    assert np.allclose(deflation.subspace_sines(T, Vperp), 1.0, atol=1e-12)
    ref = np.linalg.norm(V - W @ (W.conj().T @ V), axis=0) / np.linalg.norm(V, axis=0)
    assert np.allclose(deflation.subspace_sines(T, V), ref, rtol=1e-12)
    # and for the composite prolongator of a three-level hierarchy
    dims = (4, 4, 4, 4)
    U = synth.random_su3_links(dims, 0.3, 1)
    H3 = multigrid.setup(U, -0.4, dims, [(2, 2, 2, 2), (2, 2, 1, 1)], [6, 4], seed=11, null_maxit=10)
    Cp = deflation.Composite(H3.transfers)
    Wc = Cp.matrix().toarray()
    V = rng.standard_normal((Wc.shape[0], 2)) + 0j
    ref = np.linalg.norm(V - Wc @ (Wc.conj().T @ V), axis=0) / np.linalg.norm(V, axis=0)
    assert np.allclose(deflation.subspace_sines(Cp, V), ref, rtol=1e-12)
