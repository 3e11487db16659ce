"""Gamma matrices and the Wilson-Dirac operator A.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper works with the Wilson(-clover) Dirac operator and its
gamma5-Hermiticity (Sec. 2.1, Sec. 3 opening paragraph) but never writes the
operator out.  This library's reading is the textbook Wilson operator with
Wilson parameter r = 1 and no clover term:

    (A x)(n) = (4 + m0) x(n)
               - 1/2 sum_mu [ (1 - gamma_mu) U_mu(n) x(n + mu)
                              + (1 + gamma_mu) U_mu(n - mu)^H x(n - mu) ]
               + i tau gamma5 x(n),

periodic in all four directions.  The i*tau*gamma5 term is the shift of
Sec. 3.2 ("shifting the operator by the diagonal i gamma5"); tau = 0 unless a
caller asks for it.  Gamma matrices are in the chiral basis
gamma_k = [[0, -i sigma_k], [i sigma_k, 0]], gamma_4 = [[0, 1], [1, 0]],
so gamma5 = gamma1 gamma2 gamma3 gamma4 = diag(1, 1, -1, -1).

Pinned by: the Clifford algebra and gamma5 (test), gamma5 A gamma5 = A^H,
the adjoint identity <y, A x> = <A^H y, x>, the free-field plane-wave
spectrum M(p) +- i sqrt(sum sin^2 p) and gauge covariance
(``tests/test_oracle_wilson.py``).  The odd-site Schur complement is pinned
by eliminating the even sites through the matrix-free operator and by the
block-inverse identity (A^{-1})_oo = S^{-1}.
"""

import numpy as np
import scipy.sparse as sp

from . import lattice

_S1 = np.array([[0, 1], [1, 0]], dtype=np.complex128)
_S2 = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
_S3 = np.array([[1, 0], [0, -1]], dtype=np.complex128)
_I2 = np.eye(2, dtype=np.complex128)
_Z2 = np.zeros((2, 2), dtype=np.complex128)


def gammas():
    """(gamma_1, gamma_2, gamma_3, gamma_4) in the chiral basis, each 4x4."""
    gs = [np.block([[_Z2, -1j * s], [1j * s, _Z2]]) for s in (_S1, _S2, _S3)]
    gs.append(np.block([[_Z2, _I2], [_I2, _Z2]]))
    return gs


def gamma5():
    g = gammas()
    return g[0] @ g[1] @ g[2] @ g[3]


def apply_gamma5(x):
    """gamma5 acting on the spin index (axis 1) of a (V, 4, 3[, s]) field."""
    return np.einsum("ab,vb...->va...", gamma5(), x)


def _colour_mul(M, f):
    """sum_b M[v, a, b] f[v, s, b, ...] for links M (V, 3, 3), field f (V, 4, 3, ...)."""
    V = f.shape[0]
    tail = f.shape[3:]
    g = np.moveaxis(f, 2, 1).reshape(V, 3, -1)        # (V, 3, 4 * prod(tail))
    h = np.matmul(M, g).reshape((V, 3, 4) + tail)
    return np.moveaxis(h, 1, 2)


def _spin_mul(P, f):
    """sum_t P[s, t] f[v, t, ...] for a 4x4 spin matrix P."""
    return np.moveaxis(np.tensordot(P, f, axes=([1], [1])), 0, 1)


def dirac_apply(U, x, m0, dims, tau=0.0, dagger=False):
    """A x (or A^H x) for a field x of shape (V, 4, 3) or (V, 4, 3, s).

    Straight from the formula in the module docstring: for every direction
    the full 4x4 spin matrices (1 -+ gamma_mu) multiply the colour-rotated
    neighbour.  A^H swaps (1 - gamma_mu) and (1 + gamma_mu) and negates tau.
    """
    x = np.asarray(x, dtype=np.complex128)
    nb = lattice.neighbours(dims)
    g = gammas()
    one = np.eye(4, dtype=np.complex128)
    sgn = -1.0 if dagger else 1.0
    y = (4.0 + m0) * x
    if tau != 0.0:
        y = y + sgn * 1j * tau * apply_gamma5(x)
    for mu in range(4):
        p_fwd = one - sgn * g[mu]  # multiplies U_mu(n) x(n + mu)
        p_bwd = one + sgn * g[mu]  # multiplies U_mu(n - mu)^H x(n - mu)
        fwd = _colour_mul(U[mu], x[nb[0, mu]])
        Ubh = np.conj(np.swapaxes(U[mu][nb[1, mu]], -1, -2))
        bwd = _colour_mul(Ubh, x[nb[1, mu]])
        y = y - 0.5 * (_spin_mul(p_fwd, fwd) + _spin_mul(p_bwd, bwd))
    return y


def dirac_sparse(U, m0, dims, tau=0.0):
    """A as a sparse N x N matrix (N = 12 V, dof 12*lex + 3*spin + colour).

    The same formula as :func:`dirac_apply`, written as 12 x 12 blocks: the
    diagonal block (4 + m0) 1 + i tau gamma5, the block (n, n + mu) equal to
    -1/2 (1 - gamma_mu) (x) U_mu(n) and the block (n, n - mu) equal to
    -1/2 (1 + gamma_mu) (x) U_mu(n - mu)^H (Kronecker product of spin and
    colour).  Blocks that land on the same pair of sites (lattice extent 2)
    are summed.
    """
    V = lattice.volume(dims)
    nb = lattice.neighbours(dims)
    g = gammas()
    one = np.eye(4, dtype=np.complex128)
    diag = (4.0 + m0) * np.eye(12, dtype=np.complex128) + 1j * tau * np.kron(gamma5(), np.eye(3))
    rows, cols, vals = [], [], []
    site = np.arange(V)
    ii, jj = np.meshgrid(np.arange(12), np.arange(12), indexing="ij")

    def add(r_sites, c_sites, blocks):
        rows.append((12 * r_sites[:, None, None] + ii[None]).ravel())
        cols.append((12 * c_sites[:, None, None] + jj[None]).ravel())
        vals.append(blocks.ravel())

    add(site, site, np.broadcast_to(diag, (V, 12, 12)))
    for mu in range(4):
        Pm, Pp = one - g[mu], one + g[mu]
        fwd = np.einsum("st,vab->vsatb", Pm, U[mu]).reshape(V, 12, 12)
        Ubh = np.conj(np.swapaxes(U[mu][nb[1, mu]], -1, -2))
        bwd = np.einsum("st,vab->vsatb", Pp, Ubh).reshape(V, 12, 12)
        add(site, nb[0, mu], -0.5 * fwd)
        add(site, nb[1, mu], -0.5 * bwd)
    N = 12 * V
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    return A.tocsr()  # duplicate entries are summed


def schur_odd_sparse(U, m0, dims, tau=0.0):
    """The Schur complement of A on the odd sites (even-odd solves, Sec. 4).

    With the dofs split by site parity (sum of coordinates even / odd),
    S = A_oo - A_oe A_ee^{-1} A_eo.  Every hop joins sites of opposite
    parity, so A_ee is block diagonal (one 12 x 12 block per even site,
    (4 + m0) 1 + i tau gamma5) and is inverted block by block.  Rows and
    columns of S run over the odd sites in lexicographic order, dof
    12 k + 3 spin + colour for the k-th odd site.  Returns (S, odd_sites).
    """
    A = dirac_sparse(U, m0, dims, tau)
    par = lattice.parity(dims)
    ev, od = np.flatnonzero(par == 0), np.flatnonzero(par == 1)
    E = (12 * ev[:, None] + np.arange(12)[None, :]).ravel()
    O = (12 * od[:, None] + np.arange(12)[None, :]).ravel()
    Aee = A[E][:, E].tocsr()
    blocks = [np.linalg.inv(Aee[12 * k:12 * k + 12, 12 * k:12 * k + 12].toarray()) for k in range(len(ev))]
    Aee_inv = sp.block_diag(blocks, format="csr")
    S = A[O][:, O] - A[O][:, E] @ Aee_inv @ A[E][:, O]
    return S.tocsr(), od


def free_field_eigenvalues(dims, m0):
    """Closed-form spectrum of A with unit links (free field).

    A plane wave exp(i p.n) chi gives A(p) = M(p) + i sum_mu gamma_mu sin p_mu
    with M(p) = m0 + sum_mu (1 - cos p_mu), p_mu = 2 pi k_mu / L_mu; since
    (sum gamma_mu s_mu)^2 = sum s_mu^2, the eigenvalues are
    M(p) +- i sqrt(sum sin^2 p_mu), each 6-fold (2 spins x 3 colours).
    Returns an array of all 12 V eigenvalues.
    """
    ks = np.meshgrid(*[2 * np.pi * np.arange(L) / L for L in dims], indexing="ij")
    M = m0 + sum(1 - np.cos(k) for k in ks)
    S = np.sqrt(sum(np.sin(k) ** 2 for k in ks))
    lam = np.concatenate([(M + 1j * S).ravel(), (M - 1j * S).ravel()])
    return np.repeat(lam, 6)


def free_field_trace_inverse(dims, m0):
    """tr A^{-1} for unit links: sum_p 12 M(p) / (M(p)^2 + sum sin^2 p_mu).

    A(p)^{-1} = (M - i sum gamma s) / (M^2 + S^2) and the gammas are
    traceless, so each momentum contributes 3 colours x 4 spins x M/(M^2+S^2).
    """
    ks = np.meshgrid(*[2 * np.pi * np.arange(L) / L for L in dims], indexing="ij")
    M = m0 + sum(1 - np.cos(k) for k in ks)
    S2 = sum(np.sin(k) ** 2 for k in ks)
    return float(np.sum(12.0 * M / (M * M + S2)))


def free_field_variance_real_rademacher(dims, m0):
    """E|t - tr A^{-1}|^2 of one real Rademacher sample t = z^T A^{-1} z, unit links.

    The variance is 2||S||_F^2 - 2 sum_i |S_ii|^2 with S = (B + B^T)/2,
    B = A^{-1} (see ``dense.exact_variance_real_rademacher``).  With unit links
    B is translation invariant, B(x, y) = G(x - y), and Parseval turns
    ||S||_F^2 into sum_p ||F(p)||_F^2 with F(p) = (A(p)^{-1} + A(-p)^{-T}) / 2,
    A(p)^{-1} = (M - i sum_mu s_mu gamma_mu) / (M^2 + S^2) (s_mu = sin p_mu,
    S^2 = sum s_mu^2), times the colour identity.  In the chiral basis gamma_1
    and gamma_3 are antisymmetric and gamma_2, gamma_4 symmetric, so
    F(p) = (M - i (s_1 gamma_1 + s_3 gamma_3)) / (M^2 + S^2) and
    ||F(p)||_F^2 = 12 (M^2 + s_1^2 + s_3^2) / (M^2 + S^2)^2.  The diagonal of
    S is that of G(0), 12 V entries g0 = (1/V) sum_p M / (M^2 + S^2) (the
    gammas have zero diagonal).
    """
    ks = np.meshgrid(*[2 * np.pi * np.arange(L) / L for L in dims], indexing="ij")
    M = m0 + sum(1 - np.cos(k) for k in ks)
    s = [np.sin(k) for k in ks]
    S2 = sum(x ** 2 for x in s)
    den = M * M + S2
    V = int(np.prod(dims))
    frob = np.sum(12.0 * (M * M + s[0] ** 2 + s[2] ** 2) / den ** 2)
    g0 = np.sum(M / den) / V
    return float(2.0 * frob - 2.0 * 12 * V * g0 * g0)

