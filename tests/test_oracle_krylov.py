"""Pins for oracle.krylov: the true-residual stopping rule against dense solves."""
import numpy as np

from oracle import dense, krylov, multigrid
from paper_1909_12234_gb300 import synth


def _system():
    dims = (4, 4, 2, 2)
    U = synth.random_su3_links(dims, 0.3, 1)
    lev = multigrid.fine_level(U, -0.4, dims)
    return lev, lev.matrix.toarray()


def test_gcr_true_residual_and_error_bound():
    lev, A = _system()
    rng = np.random.default_rng(0)
    b = rng.standard_normal(lev.n) + 1j * rng.standard_normal(lev.n)
    x_lu = np.linalg.solve(A, b)
    kappa = np.linalg.cond(A)
    for tol in (1e-4, 1e-8, 1e-11):
        x, its, rel = krylov.gcr(lev.matvec, b, tol, restart=8)
        true_rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert true_rel <= tol and abs(true_rel - rel) <= 1e-3 * tol
        assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= kappa * tol


def test_gcr_with_exact_preconditioner_converges_in_one_step():
    lev, A = _system()
    Ainv = np.linalg.inv(A)
    b = np.ones(lev.n, dtype=complex)
    x, its, rel = krylov.gcr(lev.matvec, b, 1e-10, precond=lambda r: Ainv @ r)
    assert its == 1 and rel <= 1e-10


def test_minres_columns_matches_single_column_runs():
    lev, A = _system()
    rng = np.random.default_rng(2)
    B = rng.standard_normal((lev.n, 3)) + 0j
    X, steps = krylov.minres_columns(lev.matvec, B, 40, tol=0.3)
    for v in range(3):
        x, k, rel = krylov.minres_steps(lev.matvec, B[:, v], 40, tol=0.3)
        assert k == steps[v]
        assert np.abs(x - X[:, v]).max() < 1e-12
        assert rel <= 0.3 or k == 40
