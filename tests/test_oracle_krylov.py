"""Pins for oracle.krylov: the true-residual stopping rule against dense
solves, and the minimal-residual iteration against what the mathematics fixes
(the hand-computed first step, the orthogonality of each new residual to the
direction it minimised over, monotone residuals, convergence)."""
import numpy as np
import pytest

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


# --- minimal residual -------------------------------------------------------

def test_minres_first_step_by_hand():
    # A = diag(i, 2), b = (1, 1), x0 = 0: r0 = b, q = A r0 = (i, 2),
    # <q, r0> = conj(i) + 2 = 2 - i, <q, q> = 5, so a = (2 - i) / 5 and
    # x1 = a b.  A transposed conjugation (<r0, q>) would give (2 + i) / 5.
    A = np.diag([1j, 2.0])
    b = np.array([1.0, 1.0], dtype=complex)
    x, k, rel = krylov.minres_steps(lambda v: A @ v, b, 1)
    assert k == 1
    assert np.allclose(x, [(2 - 1j) / 5, (2 - 1j) / 5], rtol=0, atol=1e-15)
    # residual after the step: b - a A b = (1 - a i, 1 - 2a)
    a = (2 - 1j) / 5
    r1 = np.array([1 - a * 1j, 1 - 2 * a])
    assert abs(rel - np.linalg.norm(r1) / np.sqrt(2)) < 1e-15
    # the column form takes the same step
    X, steps = krylov.minres_columns(lambda V: A @ V, b[:, None], 1)
    assert steps[0] == 1 and np.allclose(X[:, 0], x, atol=1e-15)


def test_minres_real_scalar_operator_converges_in_one_step():
    # A = c I: q = c r, a = 1 / c, so one step solves exactly
    c = 3.0 - 2.0j
    b = np.array([1.0, -2.0, 0.5j])
    x, k, rel = krylov.minres_steps(lambda v: c * v, b, 5)
    assert k == 1 and rel < 1e-15
    assert np.allclose(x, b / c, atol=1e-15)


def _residual_history(op, b, nsteps):
    return [b - op(krylov.minres_steps(op, b, k)[0]) for k in range(nsteps + 1)]


def test_minres_residual_orthogonal_to_its_direction_and_monotone():
    # each step minimises ||r - a A r|| over a: the new residual is
    # orthogonal to A r_k, and ||r|| never grows
    lev, A = _system()
    rng = np.random.default_rng(4)
    b = rng.standard_normal(lev.n) + 1j * rng.standard_normal(lev.n)
    R = _residual_history(lev.matvec, b, 12)
    for k in range(12):
        q = A @ R[k]
        assert abs(np.vdot(q, R[k + 1])) <= 1e-12 * np.linalg.norm(q) * np.linalg.norm(R[k])
        assert np.linalg.norm(R[k + 1]) <= np.linalg.norm(R[k]) * (1 + 1e-14)
        # and it is the optimum: perturbing a in either direction is worse
        a = np.vdot(q, R[k]) / np.vdot(q, q)
        best = np.linalg.norm(R[k] - a * q)
        assert abs(best - np.linalg.norm(R[k + 1])) <= 1e-12 * np.linalg.norm(R[k])
        for da in (1e-3, -1e-3, 1e-3j):
            assert np.linalg.norm(R[k] - (a + da) * q) > best


def test_minres_stopping_rule_and_convergence():
    lev, A = _system()
    rng = np.random.default_rng(2)
    b = rng.standard_normal(lev.n) + 0j
    x, k, rel = krylov.minres_steps(lev.matvec, b, 400, tol=0.3)
    assert rel <= 0.3 and k < 400, "minimal residual must reach 0.3 on this operator"
    # it stops at the first step that meets the rule
    _, _, rel_prev = krylov.minres_steps(lev.matvec, b, k - 1)
    assert rel_prev > 0.3
    assert abs(np.linalg.norm(b - A @ x) / np.linalg.norm(b) - rel) < 1e-13
    # with an initial guess the rule is relative to ||b - A x0||
    x0 = 0.5 * x
    x2, k2, rel2 = krylov.minres_steps(lev.matvec, b, 400, x0=x0, tol=0.5)
    assert np.linalg.norm(b - A @ x2) <= 0.5 * np.linalg.norm(b - A @ x0) * (1 + 1e-13)


def test_minres_columns_matches_single_column_runs():
    lev, A = _system()
    rng = np.random.default_rng(2)
    B = rng.standard_normal((lev.n, 3)) + 0j
    B[:, 2] *= 1e-3
    X, steps = krylov.minres_columns(lev.matvec, B, 400, tol=0.3)
    for v in range(3):
        x, k, rel = krylov.minres_steps(lev.matvec, B[:, v], 400, tol=0.3)
        assert k == steps[v] and k < 400
        assert np.abs(x - X[:, v]).max() < 1e-12 * np.abs(x).max()
        assert rel <= 0.3
    # a zero column takes no step and stays zero
    B[:, 1] = 0.0
    X, steps = krylov.minres_columns(lev.matvec, B, 40, tol=0.3)
    assert steps[1] == 0 and not np.any(X[:, 1])


def test_minres_columns_null_vector_form():
    # the adaptive setup runs A y = 0 from y0: the residual is -A y, the rule
    # relative to ||A y0||; every column must end at or below it
    lev, A = _system()
    rng = np.random.default_rng(5)
    Y0 = rng.standard_normal((lev.n, 4)) + 1j * rng.standard_normal((lev.n, 4))
    Y, steps = krylov.minres_columns(lev.matvec, np.zeros_like(Y0), 200, X0=Y0, tol=0.1)
    assert np.all(steps < 200)
    for v in range(4):
        assert np.linalg.norm(A @ Y[:, v]) <= 0.1 * np.linalg.norm(A @ Y0[:, v]) * (1 + 1e-12)


@pytest.mark.parametrize("planted", ["conj", "sign"])
def test_minres_pins_catch_planted_mistakes(planted):
    # a wrong conjugation or sign in the step length must fail the pins above
    A = np.diag([1j, 2.0])
    b = np.array([1.0, 1.0], dtype=complex)
    r = b.copy()
    q = A @ r
    if planted == "conj":
        a = np.vdot(r, q) / np.vdot(q, q)
    else:
        a = -np.vdot(q, r) / np.vdot(q, q)
    x_bad = a * b
    assert not np.allclose(x_bad, [(2 - 1j) / 5, (2 - 1j) / 5], atol=1e-12)
    assert abs(np.vdot(q, r - a * q)) > 1e-3
