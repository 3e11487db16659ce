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
