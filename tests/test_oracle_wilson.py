"""Pins for oracle.wilson: Clifford algebra, gamma5-Hermiticity, free field,
gauge covariance, and agreement of the two written forms of A."""
import numpy as np
import pytest

from oracle import dense, wilson
from paper_1909_12234_gb300 import synth


def test_clifford_algebra_and_gamma5():
    g = wilson.gammas()
    for a in range(4):
        assert np.allclose(g[a], g[a].conj().T)  # Hermitian
        for b in range(4):
            assert np.allclose(g[a] @ g[b] + g[b] @ g[a], 2.0 * (a == b) * np.eye(4))
    assert np.allclose(wilson.gamma5(), np.diag([1, 1, -1, -1]))


def _ops(dims, eps, seed, m0, tau=0.0):
    U = synth.random_su3_links(dims, eps, seed)
    return U, dense.dirac_matrix(U, m0, dims, tau=tau)


def test_gamma5_hermiticity_dense():
    dims = (4, 4, 2, 2)
    U, A = _ops(dims, 0.3, 3, -0.4)
    G5 = dense.gamma5_matrix(64)
    assert np.abs(G5 @ A @ G5 - A.conj().T).max() < 1e-14


def test_adjoint_identity_with_shift():
    dims = (4, 2, 2, 4)
    U = synth.random_su3_links(dims, 0.5, 4)
    x = synth.random_field(dims, 2, 1)
    y = synth.random_field(dims, 2, 2)
    for tau in (0.0, 0.37):
        Ax = wilson.dirac_apply(U, x, -0.3, dims, tau=tau)
        Ahy = wilson.dirac_apply(U, y, -0.3, dims, tau=tau, dagger=True)
        lhs = np.einsum("vsar,vsar->r", y.conj(), Ax)
        rhs = np.einsum("vsar,vsar->r", Ahy.conj(), x)
        assert np.allclose(lhs, rhs, rtol=1e-13, atol=1e-10)


def test_sparse_and_apply_forms_agree():
    # lattice extent 2 in two directions: +mu and -mu neighbours coincide
    dims = (4, 2, 2, 4)
    U = synth.random_su3_links(dims, 0.3, 5)
    x = synth.random_field(dims, 3, 3)
    for tau in (0.0, 0.2):
        A = wilson.dirac_sparse(U, -0.5, dims, tau=tau)
        y1 = (A @ x.reshape(-1, 3)).reshape(x.shape)
        y2 = wilson.dirac_apply(U, x, -0.5, dims, tau=tau)
        assert np.abs(y1 - y2).max() < 1e-13


def _match_multisets(a, b):
    a = sorted(a, key=lambda z: (round(z.real, 9), round(z.imag, 9)))
    b = sorted(b, key=lambda z: (round(z.real, 9), round(z.imag, 9)))
    return np.max(np.abs(np.asarray(a) - np.asarray(b)))


@pytest.mark.parametrize("dims", [(4, 4, 2, 2), (2, 4, 2, 4)])
def test_free_field_spectrum(dims):
    U = synth.random_su3_links(dims, 0.0, 0, unit=True)
    A = dense.dirac_matrix(U, -0.4, dims)
    ev = np.linalg.eigvals(A)
    assert _match_multisets(ev, wilson.free_field_eigenvalues(dims, -0.4)) < 1e-10


def test_free_field_plane_wave_is_eigenvector():
    dims = (4, 4, 4, 4)
    U = synth.random_su3_links(dims, 0.0, 0, unit=True)
    from oracle import lattice
    c = lattice.coords(dims)
    p = 2 * np.pi * np.array([1, 0, 3, 2]) / np.array(dims)
    phase = np.exp(1j * (c @ p))
    g = wilson.gammas()
    M = -0.4 + np.sum(1 - np.cos(p))
    Dp = M * np.eye(4) + 1j * sum(g[m] * np.sin(p[m]) for m in range(4))
    lam, vec = np.linalg.eig(Dp)
    for i in range(4):
        x = phase[:, None, None] * vec[:, i][None, :, None] * np.array([1, 0.3, -0.2])[None, None, :]
        y = wilson.dirac_apply(U, x, -0.4, dims)
        assert np.abs(y - lam[i] * x).max() < 1e-12
    S = np.sqrt(np.sum(np.sin(p) ** 2))
    assert np.allclose(sorted(lam, key=lambda z: z.imag), [M - 1j * S] * 2 + [M + 1j * S] * 2)


def test_free_field_trace_inverse_dense():
    dims = (4, 4, 4, 4)
    U = synth.random_su3_links(dims, 0.0, 0, unit=True)
    A = wilson.dirac_sparse(U, -0.4, dims).toarray()
    tr = np.trace(np.linalg.inv(A))
    assert abs(tr - wilson.free_field_trace_inverse(dims, -0.4)) < 1e-10 * abs(tr)


@pytest.mark.parametrize("dims,m0", [((4, 2, 2, 2), -0.4), ((2, 4, 2, 4), -0.8), ((4, 4, 2, 2), 0.3)])
def test_free_field_variance_closed_form_against_dense(dims, m0):
    # the closed form against the dense exact variance of the same A^{-1}
    # (itself pinned by enumeration of all sign vectors)
    from oracle import dense
    U = synth.random_su3_links(dims, 0.0, 0, unit=True)
    B = np.linalg.inv(wilson.dirac_sparse(U, m0, dims).toarray())
    ref = dense.exact_variance_real_rademacher(B)
    got = wilson.free_field_variance_real_rademacher(dims, m0)
    assert abs(got - ref) < 1e-10 * ref
    # a wrong basis reading (gamma_2 instead of gamma_3 antisymmetric) fails
    ks = np.meshgrid(*[2 * np.pi * np.arange(L) / L for L in dims], indexing="ij")
    M = m0 + sum(1 - np.cos(k) for k in ks)
    sn = [np.sin(k) for k in ks]
    den = M * M + sum(x ** 2 for x in sn)
    V = int(np.prod(dims))
    bad = 2 * np.sum(12.0 * (M * M + sn[0] ** 2 + sn[1] ** 2) / den ** 2) - 24 * V * (np.sum(M / den) / V) ** 2
    if not np.allclose(sn[1] ** 2, sn[2] ** 2):
        assert abs(bad - ref) > 1e-6 * ref


def test_gauge_covariance():
    dims = (4, 4, 2, 2)
    U = synth.random_su3_links(dims, 0.3, 6)
    Ug, g = synth.gauge_transform(U, dims, 9)
    x = synth.random_field(dims, 2, 4)
    gx = np.einsum("vab,vsbr->vsar", g, x)
    lhs = wilson.dirac_apply(Ug, gx, -0.4, dims, tau=0.1)
    rhs = np.einsum("vab,vsbr->vsar", g, wilson.dirac_apply(U, x, -0.4, dims, tau=0.1))
    assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("dims,tau", [((4, 4, 2, 2), 0.0), ((4, 2, 2, 4), 0.3)])
def test_schur_complement_eliminates_even_sites(dims, tau):
    # through the matrix-free operator: with x_e = -A_ee^{-1} A_eo x_o (A_ee
    # = (4 + m0) + i tau gamma5 written out here), the full field X = (x_e,
    # x_o) has (A X)_e = 0 and (A X)_o = S x_o
    from oracle import lattice
    m0 = -0.4
    U = synth.random_su3_links(dims, 0.4, 3)
    S, od = wilson.schur_odd_sparse(U, m0, dims, tau)
    V = int(np.prod(dims))
    par = lattice.parity(dims)
    rng = np.random.default_rng(2)
    X = np.zeros((V, 4, 3), dtype=np.complex128)
    X[par == 1] = rng.standard_normal((len(od), 4, 3)) + 1j * rng.standard_normal((len(od), 4, 3))
    Ax = wilson.dirac_apply(U, X[..., None], m0, dims, tau=tau)[..., 0]  # (A_eo x_o) on even sites
    m = 4.0 + m0
    g5 = np.array([1.0, 1.0, -1.0, -1.0])[None, :, None]
    inv_diag = (m - 1j * tau * g5) / (m * m + tau * tau)
    X[par == 0] = -(inv_diag * Ax)[par == 0]
    AX = wilson.dirac_apply(U, X[..., None], m0, dims, tau=tau)[..., 0]
    assert np.abs(AX[par == 0]).max() < 1e-12
    Sx = (S @ X[par == 1].reshape(-1)).reshape(-1, 4, 3)
    assert np.abs(AX[par == 1] - Sx).max() < 1e-12


def test_schur_complement_is_inverse_of_odd_block():
    # (A^{-1})_oo = S^{-1} (block inverse), dense on a 4 x 2 x 2 x 2 lattice
    from oracle import lattice
    dims, m0, tau = (4, 2, 2, 2), -0.3, 0.2
    U = synth.random_su3_links(dims, 0.5, 4)
    A = wilson.dirac_sparse(U, m0, dims, tau).toarray()
    S, od = wilson.schur_odd_sparse(U, m0, dims, tau)
    O = (12 * od[:, None] + np.arange(12)[None, :]).ravel()
    Ainv = np.linalg.inv(A)
    assert np.abs(Ainv[np.ix_(O, O)] @ S.toarray() - np.eye(len(O))).max() < 1e-10
    assert len(od) == lattice.volume(dims) // 2
