"""Adaptive multigrid: null vectors, blocking, prolongator W, W^H A W, V-cycle.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Follows Sec. 2 of the paper:

1. adaptive setup: approximate solutions of A y = 0 from n random initial
   guesses; Sec. 3 (paragraph after Algorithm 2) stops them at relative
   residual 1e-2 or after 200 iterations.  Here: minimal-residual iterations
   from the Philox starts of ``philox.random_starts`` ("relative" = relative
   to the starting residual ||A y0||);
2. chirality split: Algorithm 2 asks for gamma5 W = W gamma5^W, so every null
   vector y is split into (1 + gamma5)/2 y and (1 - gamma5)/2 y;
3. blocking onto disjoint subdomains D_j (2^4 blocks, Table 2) and an
   orthonormal basis of each block: classical Gram-Schmidt applied twice
   (CGS2), in null-vector order;
4. the coarse operator C = W^H A W, formed as the sparse product of W^H,
   the sparse A and W (and, for small sizes, column by column
   W e_c -> A -> W^H); either way aliasing of neighbours on coarse lattices of
   extent 1 or 2 is handled by construction;
5. the two-grid iteration of Sec. 2: coarse-grid correction
   x = W C^{-1} W^H r, then smoothing x += M^{-1}(r - A x) with M^{-1} a few
   minimal-residual steps; a deeper level replaces C^{-1} by GCR on C
   preconditioned with the next level (no recursion on the coarsest level).

Coarse dof order inside a coarse site: d = chirality * nv + j, chirality 0
for gamma5 = +1, so gamma5^W = diag(+1 x nv, -1 x nv) per coarse site.
A coarse vector is indexed lex_coarse_site * 2 nv + d.

Pins (tests/test_oracle_multigrid.py): W^H W = I, gamma5 W = W gamma5^W,
gamma5^W C Hermitian, the coarse dimension arithmetic of Table 2, Galerkin
identity W^H A W e = W^H (A (W e)) against dense matrices; the V-cycle equals
the dense coarse-grid correction W C^{-1} W^H r without smoothing (and kills
the restricted residual), equals A^{-1} r when W spans the whole space, moves
along the corrected residual with the minimal-residual optimality when it
smooths (two and three levels), and planted mistakes (smoothing r instead of
r - A x, a wrong transfer order) fail these pins.  The quality of the setup
(how well W captures low modes) is parity unpinned.
"""

import numpy as np
import scipy.sparse as sp

from . import krylov, lattice, philox, wilson


class Level:
    """One level of the hierarchy: a lattice, dofs per site and its operator
    as a sparse matrix (flat dof index lex_site * dof + d)."""

    def __init__(self, dims, dof, chirality_of_dof, matrix):
        self.dims = tuple(dims)
        self.dof = dof
        self.chir = np.asarray(chirality_of_dof)  # (dof,) 0 or 1
        self.V = lattice.volume(dims)
        self.n = self.V * dof
        self.matrix = matrix

    def matvec(self, x):
        """A x for a flat vector (n,) or a block (n, s)."""
        return self.matrix @ x

    def gamma5(self, x):
        sign = np.where(np.tile(self.chir, self.V) == 0, 1.0, -1.0)
        return sign.reshape((-1,) + (1,) * (x.ndim - 1)) * x


def fine_level(U, m0, dims, tau=0.0):
    return Level(dims, 12, np.repeat([0, 0, 1, 1], 3), wilson.dirac_sparse(U, m0, dims, tau))


class Transfer:
    """Prolongator W between a level and the next coarser one."""

    def __init__(self, level, block, nv, W_blocks, rows):
        self.level = level
        self.block = tuple(block)
        self.nv = nv
        self.cdims = lattice.coarse_dims(level.dims, block)
        self.Vc = lattice.volume(self.cdims)
        self.W = W_blocks  # (Vc, 2, nrow, nv)
        self.rows = rows   # (Vc, 2, nrow) flat fine dof indices
        self.nc = self.Vc * 2 * nv

    def prolong(self, c):
        """W c for a coarse vector (nc,) or (nc, s)."""
        tail = c.shape[1:]
        cb = c.reshape((self.Vc, 2, self.nv) + tail)
        f = np.zeros((self.level.n,) + tail, dtype=np.complex128)
        vals = np.einsum("acrj,acj...->acr...", self.W, cb)
        f[self.rows.reshape(-1)] = vals.reshape((-1,) + tail)
        return f

    def matrix(self):
        """W as a sparse (n, nc) matrix."""
        Vc, _, nrow, nv = self.W.shape
        cidx = (np.arange(Vc)[:, None, None, None] * 2 * nv
                + np.arange(2)[None, :, None, None] * nv
                + np.arange(nv)[None, None, None, :])
        rows = np.broadcast_to(self.rows[..., None], self.W.shape)
        cols = np.broadcast_to(cidx, self.W.shape)
        return sp.csr_matrix((self.W.ravel(), (rows.ravel(), cols.ravel())),
                             shape=(self.level.n, self.nc))

    def restrict(self, f):
        """W^H f for a fine vector (n,) or (n, s)."""
        tail = f.shape[1:]
        g = f[self.rows.reshape(-1)].reshape(self.rows.shape + tail)
        c = np.einsum("acrj,acr...->acj...", self.W.conj(), g)
        return c.reshape((self.nc,) + tail)


def block_rows(level, block):
    """Flat dof indices of each (aggregate, chirality) block, (Vc, 2, nrow)."""
    members = lattice.aggregate_members(level.dims, block)  # (Vc, b)
    rows = []
    for c in (0, 1):
        dofs = np.nonzero(level.chir == c)[0]
        r = (members[:, :, None] * level.dof + dofs[None, None, :]).reshape(len(members), -1)
        rows.append(r)
    return np.stack(rows, axis=1)


def null_vectors(level, nv, seed, tol=1e-2, maxit=200):
    """Approximate solutions of A y = 0 from nv random starts (Sec. 2, Sec. 3).

    Each column runs its own minimal-residual iteration (see
    ``krylov.minres_columns``).  Returns (Y (n, nv), iterations per vector)."""
    Y0 = philox.random_starts(level.n, seed, nv)
    zero = np.zeros_like(Y0)
    Y, its = krylov.minres_columns(level.matvec, zero, maxit, X0=Y0, tol=tol)
    return Y, its


def cgs2(Y):
    """Orthonormal basis of the columns of Y, classical Gram-Schmidt twice."""
    Q = np.zeros_like(Y)
    for v in range(Y.shape[1]):
        w = Y[:, v].copy()
        for _ in range(2):
            w = w - Q[:, :v] @ (Q[:, :v].conj().T @ w)
        nrm = np.linalg.norm(w)
        if nrm == 0.0:
            raise np.linalg.LinAlgError("null vectors are linearly dependent on a block")
        Q[:, v] = w / nrm
    return Q


def build_transfer(level, block, Y):
    """Chirality split + blocking + per-block CGS2 of null vectors Y (n, nv)."""
    nv = Y.shape[1]
    rows = block_rows(level, block)
    Vc = rows.shape[0]
    W = np.empty((Vc, 2, rows.shape[2], nv), dtype=np.complex128)
    for a in range(Vc):
        for c in (0, 1):
            # D_a (1 +- gamma5)/2 y keeps exactly the rows of this block
            W[a, c] = cgs2(Y[rows[a, c], :])
    return Transfer(level, block, nv, W, rows)


def coarse_matrix(level, T):
    """C = W^H A W (Galerkin coarse operator) as a sparse matrix product."""
    W = T.matrix()
    return (W.conj().T @ (level.matrix @ W)).tocsr()


def coarse_matrix_by_columns(level, T, batch=128):
    """C = W^H A W column by column (W e_c -> A -> W^H), dense; small sizes."""
    C = np.empty((T.nc, T.nc), dtype=np.complex128)
    for c0 in range(0, T.nc, batch):
        nb = min(batch, T.nc - c0)
        E = np.zeros((T.nc, nb), dtype=np.complex128)
        E[c0 + np.arange(nb), np.arange(nb)] = 1.0
        C[:, c0:c0 + nb] = T.restrict(level.matvec(T.prolong(E)))
    return C


def coarse_level(T, C):
    chir = np.repeat([0, 1], T.nv)
    return Level(T.cdims, 2 * T.nv, chir, C)


class Hierarchy:
    """Levels 0..L-1, transfers 0..L-2 and coarse matrices 1..L-1."""

    def __init__(self, levels, transfers, matrices, smoother_steps=4,
                 coarse_tol=0.1, coarse_maxit=256, restart=16, coarse_smoother_steps=None):
        self.levels = levels
        self.transfers = transfers
        self.matrices = matrices
        self.nu = smoother_steps
        # smoothing steps of the V-cycles on coarse levels (default: the same)
        self.nu_coarse = smoother_steps if coarse_smoother_steps is None else coarse_smoother_steps
        self.coarse_tol = coarse_tol
        self.coarse_maxit = coarse_maxit
        self.restart = restart

    def vcycle(self, lvl, r):
        """One application of the level-lvl preconditioner to residual r (flat)."""
        T = self.transfers[lvl]
        A = self.levels[lvl]
        rc = T.restrict(r)
        nxt = lvl + 1
        pre = (lambda v: self.vcycle(nxt, v)) if nxt < len(self.transfers) else None
        ec, _, _ = krylov.gcr(self.levels[nxt].matvec, rc, self.coarse_tol,
                              maxit=self.coarse_maxit, restart=self.restart, precond=pre)
        x = T.prolong(ec)
        nu = self.nu if lvl == 0 else self.nu_coarse
        e, _, _ = krylov.minres_steps(A.matvec, r - A.matvec(x), nu)
        return x + e


def setup(U, m0, dims, blocks, nvs, seed, null_tol=1e-2, null_maxit=200, tau=0.0,
          injected_null=None, **vcycle_kw):
    """Full adaptive setup (Sec. 2).  ``injected_null[l]`` (n_l, nv_l) replaces
    the null-vector iteration on level l (used to compare implementations)."""
    levels = [fine_level(U, m0, dims, tau)]
    transfers, mats = [], []
    for l, (blk, nv) in enumerate(zip(blocks, nvs)):
        lev = levels[-1]
        if injected_null is not None and injected_null[l] is not None:
            Y = np.asarray(injected_null[l], dtype=np.complex128)
        else:
            Y, _ = null_vectors(lev, nv, seed + l, null_tol, null_maxit)
        T = build_transfer(lev, blk, Y)
        C = coarse_matrix(lev, T)
        transfers.append(T)
        mats.append(C)
        levels.append(coarse_level(T, C))
    return Hierarchy(levels, transfers, mats, **vcycle_kw)
