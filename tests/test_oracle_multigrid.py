"""Pins for oracle.multigrid: orthonormality, chirality, Galerkin operator,
Table 2 dimension arithmetic."""
import os

import numpy as np
import pytest

from oracle import lattice, multigrid
from paper_1909_12234_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden", "table2_dims.txt")


@pytest.fixture(scope="module")
def hier():
    dims = (4, 4, 4, 4)
    U = synth.random_su3_links(dims, 0.3, 1)
    return multigrid.setup(U, -0.4, dims, [(2, 2, 2, 2), (2, 2, 1, 1)], [6, 4], seed=11,
                           null_maxit=30)


def test_transfer_is_orthonormal_and_chiral(hier):
    for l, T in enumerate(hier.transfers):
        W = T.matrix().toarray()
        assert np.abs(W.conj().T @ W - np.eye(T.nc)).max() < 1e-13
        lev = hier.levels[l]
        g5W = lev.gamma5(W)
        coarse_g5 = np.tile(np.repeat([1.0, -1.0], T.nv), T.Vc)
        assert np.abs(g5W - W * coarse_g5[None, :]).max() < 1e-15
        # W has support on its own aggregate only
        agg = lattice.aggregate_of(lev.dims, T.block)
        site = np.arange(lev.n) // lev.dof
        for c in range(T.nc):
            nz = np.nonzero(W[:, c])[0]
            assert np.all(agg[site[nz]] == c // (2 * T.nv))


def test_galerkin_operator(hier):
    for l, T in enumerate(hier.transfers):
        lev = hier.levels[l]
        C = hier.matrices[l].toarray()
        C_cols = multigrid.coarse_matrix_by_columns(lev, T)
        assert np.abs(C - C_cols).max() < 1e-13
        # gamma5^W C is Hermitian (gamma5-Hermiticity survives W^H A W)
        g5 = np.tile(np.repeat([1.0, -1.0], T.nv), T.Vc)
        G = g5[:, None] * C
        assert np.abs(G - G.conj().T).max() < 1e-13


def test_prolong_restrict_are_adjoint(hier):
    T = hier.transfers[0]
    rng = np.random.default_rng(3)
    c = rng.standard_normal((T.nc, 2)) + 1j * rng.standard_normal((T.nc, 2))
    f = rng.standard_normal((T.level.n, 2)) + 1j * rng.standard_normal((T.level.n, 2))
    lhs = np.sum(f.conj() * T.prolong(c), axis=0)
    rhs = np.sum(T.restrict(f).conj() * c, axis=0)
    assert np.allclose(lhs, rhs, rtol=1e-13)
    assert np.abs(T.restrict(T.prolong(c)) - c).max() < 1e-13


def test_vcycle_preconditioner_reduces_iterations(hier):
    from oracle import krylov
    lev = hier.levels[0]
    b = np.ones(lev.n, dtype=complex)
    _, its_plain, _ = krylov.gcr(lev.matvec, b, 1e-8)
    _, its_mg, rel = krylov.gcr(lev.matvec, b, 1e-8, precond=lambda r: hier.vcycle(0, r))
    assert rel <= 1e-8 and its_mg < its_plain


def _table2_rows():
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        f = [p.strip() for p in line.split("|")]
        dims = tuple(int(v) for v in f[0].split())
        N = int(f[1])
        blocks = [tuple(int(v) for v in b.split(",")) for b in f[2].split(";")]
        nvs = [int(v) for v in f[3].split(",")]
        yield dims, N, blocks, nvs, int(f[4])


def test_table2_dimension_arithmetic():
    rows = list(_table2_rows())
    assert len(rows) == 6
    for dims, N, blocks, nvs, coarsest in rows:
        assert 12 * lattice.volume(dims) == N
        d = dims
        for b in blocks:
            d = lattice.coarse_dims(d, b)
        assert lattice.volume(d) * 2 * nvs[-1] == coarsest


# --- the V-cycle (Sec. 2 two-grid iteration) ----------------------------------
# With an exact coarse solve and no smoothing the V-cycle is the coarse-grid
# correction W C^{-1} W^H r; with W spanning the whole space it is A^{-1} r;
# one minimal-residual post-smoothing step moves along the residual of the
# coarse-grid correction and leaves a residual orthogonal to A times it.

EXACT = dict(coarse_tol=1e-14, coarse_maxit=20000, restart=64)


@pytest.fixture(scope="module")
def two_level_exact():
    dims = (4, 4, 4, 4)
    U = synth.random_su3_links(dims, 0.3, 1)
    H0 = multigrid.setup(U, -0.4, dims, [(2, 2, 2, 2)], [6], seed=11, null_maxit=30, smoother_steps=0, **EXACT)
    H1 = multigrid.Hierarchy(H0.levels, H0.transfers, H0.matrices, smoother_steps=1, **EXACT)
    return H0, H1


def _dense_cgc(H, r):
    T = H.transfers[0]
    W = T.matrix().toarray()
    C = H.matrices[0].toarray()
    return W @ np.linalg.solve(C, W.conj().T @ r), W


def _rhs(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def test_vcycle_without_smoothing_is_the_coarse_grid_correction(two_level_exact):
    H0, _ = two_level_exact
    A = H0.levels[0].matrix
    r = _rhs(H0.levels[0].n, 7)
    z = H0.vcycle(0, r)
    xc, W = _dense_cgc(H0, r)
    assert np.linalg.norm(z - xc) <= 1e-11 * np.linalg.norm(xc)
    # the coarse-grid correction annihilates the restricted residual
    assert np.linalg.norm(W.conj().T @ (r - A @ z)) <= 1e-11 * np.linalg.norm(r)


def _smoothing_step_holds(A, r, z, xc):
    """z - xc is a multiple of res = r - A xc and r - A z is orthogonal to A res."""
    res = r - A @ xc
    e = z - xc
    a = np.vdot(res, e) / np.vdot(res, res)
    if np.linalg.norm(e - a * res) > 1e-9 * np.linalg.norm(e):
        return False
    q = A @ res
    return abs(np.vdot(q, r - A @ z)) <= 1e-9 * np.linalg.norm(q) * np.linalg.norm(res)


def test_vcycle_post_smoothing_acts_on_the_corrected_residual(two_level_exact):
    _, H1 = two_level_exact
    A = H1.levels[0].matrix
    r = _rhs(H1.levels[0].n, 8)
    xc, _ = _dense_cgc(H1, r)
    z = H1.vcycle(0, r)
    assert _smoothing_step_holds(A, r, z, xc)
    # and it reduces the residual of the coarse-grid correction
    assert np.linalg.norm(r - A @ z) < np.linalg.norm(r - A @ xc)


class _SmoothsWrongResidual(multigrid.Hierarchy):
    """A planted mistake: smoothing r instead of r - A x."""

    def vcycle(self, lvl, r):
        T = self.transfers[lvl]
        A = self.levels[lvl]
        from oracle import krylov
        ec, _, _ = krylov.gcr(self.levels[lvl + 1].matvec, T.restrict(r), self.coarse_tol,
                              maxit=self.coarse_maxit, restart=self.restart)
        x = T.prolong(ec)
        e, _, _ = krylov.minres_steps(A.matvec, r, self.nu)
        return x + e


class _ProlongsTwice(multigrid.Hierarchy):
    """A planted mistake: the coarse-grid correction without the restriction
    (W C^{-1} applied to the restriction's transpose order)."""

    def vcycle(self, lvl, r):
        T = self.transfers[lvl]
        from oracle import krylov
        rc = T.restrict(self.levels[lvl].matvec(r))
        ec, _, _ = krylov.gcr(self.levels[lvl + 1].matvec, rc, self.coarse_tol,
                              maxit=self.coarse_maxit, restart=self.restart)
        return T.prolong(ec)


def test_vcycle_pins_catch_planted_mistakes(two_level_exact):
    H0, H1 = two_level_exact
    A = H1.levels[0].matrix
    r = _rhs(H1.levels[0].n, 9)
    xc, W = _dense_cgc(H1, r)
    bad = _SmoothsWrongResidual(H1.levels, H1.transfers, H1.matrices, smoother_steps=1, **EXACT)
    assert not _smoothing_step_holds(A, r, bad.vcycle(0, r), xc)
    bad0 = _ProlongsTwice(H0.levels, H0.transfers, H0.matrices, smoother_steps=0, **EXACT)
    zb = bad0.vcycle(0, r)
    assert np.linalg.norm(zb - xc) > 1e-3 * np.linalg.norm(xc)


def test_vcycle_with_full_space_prolongator_is_the_inverse():
    # 1^4 aggregates with nv = 6 per chirality: W is unitary block by block,
    # so W C^{-1} W^H = A^{-1}, and the smoother then sees a zero residual
    dims = (4, 4, 2, 2)
    U = synth.random_su3_links(dims, 0.3, 4)
    for nu in (0, 2):
        H = multigrid.setup(U, -0.4, dims, [(1, 1, 1, 1)], [6], seed=5, null_maxit=5, smoother_steps=nu, **EXACT)
        A = H.levels[0].matrix.toarray()
        W = H.transfers[0].matrix().toarray()
        assert np.abs(W.conj().T @ W - np.eye(W.shape[0])).max() < 1e-13
        r = _rhs(H.levels[0].n, 10 + nu)
        z = H.vcycle(0, r)
        x = np.linalg.solve(A, r)
        assert np.linalg.norm(z - x) <= 1e-10 * np.linalg.norm(x)


def test_three_level_vcycle_with_exact_level1_solve():
    # the level-1 solve is GCR on C_1 preconditioned by the level-1 V-cycle
    # (which needs smoothing: without it that V-cycle has the rank of W_1 and
    # GCR cannot converge with it); solved exactly, the three-level V-cycle is
    # the coarse-grid correction W_0 C_1^{-1} W_0^H r followed by one smoothing
    # step, and the level-1 V-cycle is the same with W_1 and C_2
    dims = (4, 4, 4, 4)
    U = synth.random_su3_links(dims, 0.3, 1)
    H = multigrid.setup(U, -0.4, dims, [(2, 2, 2, 2), (2, 2, 1, 1)], [6, 4], seed=11, null_maxit=30,
                        smoother_steps=1, **EXACT)
    A = H.levels[0].matrix
    r = _rhs(H.levels[0].n, 12)
    W0 = H.transfers[0].matrix().toarray()
    C1 = H.matrices[0].toarray()
    xc = W0 @ np.linalg.solve(C1, W0.conj().T @ r)
    assert _smoothing_step_holds(A, r, H.vcycle(0, r), xc)
    rc = W0.conj().T @ r
    W1 = H.transfers[1].matrix().toarray()
    C2 = H.matrices[1].toarray()
    xc1 = W1 @ np.linalg.solve(C2, W1.conj().T @ rc)
    assert _smoothing_step_holds(H.matrices[0], rc, H.vcycle(1, rc), xc1)
