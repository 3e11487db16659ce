"""Deflation spaces and projectors: Algorithm 1 and Algorithm 2.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Algorithm 1 (orthogonal projector, approximate singular vectors of A):
  U = eigenvectors of gamma5 (A + i tau gamma5)^{-1} of largest magnitude,
  i.e. eigenvectors of the Hermitian A gamma5 (tau = 0) with the k smallest
  |eigenvalue|;  t0 = sum_i u_i^H A^{-1}_xi u_i;
  t1 = t(A^{-1}_xi (I - U U^H)).

Algorithm 2 (oblique projector from the coarse operator C = W^H A W):
  U_bar = eigenvectors of gamma5^W (C + i tau gamma5^W)^{-1} of largest
  magnitude; at tau = 0 that operator is (C gamma5^W)^{-1}, so U_bar holds the
  eigenvectors of the Hermitian C gamma5^W with the k smallest |mu|;
  factorise U_hat Lambda U_hat^H = U_bar^H gamma5^W C U_bar, U = U_bar U_hat;
  t0 = sum_i u_i^H gamma5^W u_i / lambda_i;
  t1 = t(A^{-1}_xi (I - P)), P = A W U Lambda^{-1} U^H gamma5^W W^H.

Reading of Algorithm 2, step 5: the printed projector A W gamma5 U ... is
taken as the K = gamma5 projector of Sec. 2.1,
I - A V (V^H K A V)^{-1} V^H K with V = W U, which is
I - A W U Lambda^{-1} U^H gamma5^W W^H (gamma5 W = W gamma5^W).  Step 4's
gamma5 acts on the coarse vector u_i, so it is gamma5^W.

The a-posteriori analysis of Sec. 2.2 needs only Z^H W U_bar and
U_bar^H gamma5^W W^H Z: the rank-r correction to z^H A^{-1} z is
(z^H W U_bar_r) G_r^{-1} (U_bar_r^H gamma5^W W^H z), G_r the leading r x r
block of U_bar^H gamma5^W C U_bar.

Hierarchies with more than one coarse level: Table 2 sizes the eigenproblem
of Algorithm 2 by the coarsest level ("dimension of coarsest"), so W is the
composite prolongator W_0 W_1 ... W_{L-1} from the coarsest level to the fine
one and C = W^H A W is the coarsest Galerkin operator (each level's operator
is the Galerkin product of the one above it).  Every W_l maps chirality to
chirality, so gamma5 W = W gamma5^W holds for the composite as well.

Pins: projector identities P^2 = P, gamma5-Hermiticity of A^{-1}(I - P),
t0 + tr(A^{-1}(I - P)) = tr A^{-1}; for three levels also C_2 = W^H A W and
gamma5 W = W gamma5^W with the composite W (dense,
tests/test_oracle_deflation.py).
The eigensolver (scipy ARPACK shift-invert, or dense eigh for small sizes)
is a library routine; which eigenvectors it returns inside a degenerate
cluster is not unique, so only projector-invariant results are compared.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import krylov


def smallest_abs_eigh(H, k, dense_limit=4096):
    """k eigenpairs of a Hermitian matrix with smallest |eigenvalue|, ascending |mu|."""
    n = H.shape[0]
    if n <= dense_limit:
        Hd = H.toarray() if sp.issparse(H) else np.asarray(H)
        mu, X = np.linalg.eigh(0.5 * (Hd + Hd.conj().T))
    else:
        mu, X = spla.eigsh(H, k=k, sigma=0.0, which="LM", tol=1e-13)
    order = np.argsort(np.abs(mu), kind="stable")[:k]
    return mu[order], X[:, order]


class Composite:
    """W = W_0 W_1 ... W_{L-1} for transfers listed fine to coarse."""

    def __init__(self, transfers):
        self.transfers = list(transfers)
        self.nv = self.transfers[-1].nv

    def restrict(self, f):
        for T in self.transfers:
            f = T.restrict(f)
        return f

    def prolong(self, c):
        for T in reversed(self.transfers):
            c = T.prolong(c)
        return c

    def matrix(self):
        W = self.transfers[0].matrix()
        for T in self.transfers[1:]:
            W = W @ T.matrix()
        return W


class Alg2:
    """Algorithm 2 deflation built from a transfer T (fine level -> the level
    of C; a ``Composite`` for more than one coarse level) and C = W^H A W."""

    def __init__(self, T, C, k, Ubar=None):
        self.T = T
        self.C = C
        self.nv = T.nv
        n = C.shape[0]
        self.g5 = np.tile(np.repeat([1.0, -1.0], T.nv), n // (2 * T.nv))
        if Ubar is None:
            H = C @ sp.diags(self.g5)  # C gamma5^W, Hermitian
            self.mu, Ubar = smallest_abs_eigh(H, k)
        self.Ubar = np.asarray(Ubar, dtype=np.complex128)
        self.k = self.Ubar.shape[1]
        # G = U_bar^H gamma5^W C U_bar (Hermitian because gamma5^W C is)
        self.G = self.Ubar.conj().T @ (self.g5[:, None] * (C @ self.Ubar))
        self.set_rank(self.k)

    def set_rank(self, r):
        """Step 3 of Algorithm 2 on the leading r columns of U_bar."""
        Gr = self.G[:r, :r]
        lam, Uhat = np.linalg.eigh(0.5 * (Gr + Gr.conj().T))
        self.rank = r
        self.lam = lam
        self.U = self.Ubar[:, :r] @ Uhat
        # step 4: t0 = sum_i u_i^H gamma5^W u_i / lambda_i
        self.t0 = complex(np.sum(np.einsum("ci,c,ci->i", self.U.conj(), self.g5, self.U) / lam))
        return self

    def project(self, A_matvec, z):
        """(I - P) z = z - A W U Lambda^{-1} U^H gamma5^W W^H z."""
        c = self.T.restrict(z)
        coef = self.U.conj().T @ (self.g5.reshape((-1,) + (1,) * (c.ndim - 1)) * c)
        coef = coef / self.lam.reshape((-1,) + (1,) * (coef.ndim - 1))
        return z - A_matvec(self.T.prolong(self.U @ coef))

    def coeffs(self, z):
        """(Z^H W U_bar (s x k), U_bar^H gamma5^W W^H Z (k x s)) of Sec. 2.2."""
        c = self.T.restrict(z)
        ZhV = (self.Ubar.conj().T @ c).conj().T
        UhKZ = self.Ubar.conj().T @ (self.g5[:, None] * c)
        return ZhV, UhKZ

    def correction(self, ZhV, UhKZ, r):
        """Per-sample rank-r correction (z^H W U_bar_r) G_r^{-1} (U_bar_r^H g5 W^H z)."""
        Gr = self.G[:r, :r]
        X = np.linalg.solve(Gr, UhKZ[:r])
        return np.einsum("ji,ij->j", ZhV[:, :r], X)

    def t0_rank(self, r):
        """t0 at rank r: tr(U_bar_r^H gamma5^W U_bar_r G_r^{-1})."""
        Ur = self.Ubar[:, :r]
        M = Ur.conj().T @ (self.g5[:, None] * Ur)
        return complex(np.trace(M @ np.linalg.inv(self.G[:r, :r])))


class Alg1:
    """Algorithm 1 deflation with fine vectors U (n x k), orthonormal."""

    def __init__(self, U, A_matvec, xi, restart=16, precond=None, maxit=100000):
        self.U = np.asarray(U, dtype=np.complex128)
        self.k = self.U.shape[1]
        # step 2: t0 = sum_i u_i^H A^{-1}_xi u_i, keeping Y = A^{-1}_xi U
        self.Y = np.empty_like(self.U)
        for i in range(self.k):
            self.Y[:, i], _, _ = krylov.gcr(A_matvec, self.U[:, i], xi, maxit=maxit,
                                            restart=restart, precond=precond)
        self.d = np.einsum("ni,ni->i", self.U.conj(), self.Y)
        self.t0 = complex(np.sum(self.d))

    def project(self, z):
        """(I - U U^H) z."""
        return z - self.U @ (self.U.conj().T @ z)

    def coeffs(self, z):
        """(z_j^H A^{-1}_xi u_i (s x k), u_i^H z_j (k x s)): with them the
        deflated value of a rank-r space is, for every sample,
        z^H A^{-1}(I - U_r U_r^H) z = z^H A^{-1} z - sum_{i<r} (z^H A^{-1} u_i)(u_i^H z)."""
        return (z.conj().T @ self.Y), (self.U.conj().T @ z)

    def correction(self, ZhAU, UhZ, r):
        return np.einsum("ji,ij->j", ZhAU[:, :r], UhZ[:r])

    def t0_rank(self, r):
        return complex(np.sum(self.d[:r]))


def subspace_sines(T, V):
    """sin of the angle between each column v of V and the range of the
    (orthonormal) prolongator W of T (a Transfer or a Composite):
    ||v - W W^H v|| / ||v|| (Sec. 4.1, Fig. 3 right)."""
    V = np.asarray(V, dtype=np.complex128)
    R = V - T.prolong(T.restrict(V))
    return np.linalg.norm(R, axis=0) / np.linalg.norm(V, axis=0)


def fine_eigvecs_dense(A, g5, k):
    """Algorithm 1, step 1 by dense eigh of A gamma5 (small lattices only)."""
    H = A @ g5
    return smallest_abs_eigh(H, k, dense_limit=1 << 30)
