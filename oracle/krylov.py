"""Krylov solvers: restarted (flexible) GCR and minimal residual.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Sec. 1: A^{-1}_xi(x) is computed by an iterative solver that stops once
  ||A A^{-1}_xi(x) - x|| <= xi ||x||.  ``gcr`` stops on the TRUE residual
  b - A x, recomputed at every restart and before returning.
* Sec. 2: the smoother M^{-1} is "a few iterations of a linear system solver,
  e.g. GCR"; Sec. 3 (paragraph after Algorithm 2) uses GCR at the coarse
  levels.  ``gcr`` accepts a right preconditioner (possibly variable, i.e.
  flexible GCR), which is how the multigrid V-cycle is used.
* ``minres_steps`` is the minimal-residual iteration x += a r,
  a = <A r, r> / <A r, A r>, used for the adaptive null vectors (Sec. 2) and
  as the smoother.

Vectors are flat complex128 arrays; ``op`` maps one vector to one vector.
Each right-hand side is solved independently (no block Krylov).

Pinned by (tests/test_oracle_krylov.py): the true-residual stopping rule and
the kappa * xi error bound against dense solves; for the minimal-residual
iteration a first step computed by hand on diag(i, 2) (which fixes the
conjugation in a), one-step convergence on c I, the orthogonality of every new
residual to A r_k with ||r|| non-increasing and a the exact minimiser, the
stopping rule, and the column form against single-column runs.
"""

import numpy as np


def dot(a, b):
    """<a, b> = a^H b."""
    return np.vdot(a, b)


def gcr(op, b, tol, maxit=10000, restart=16, precond=None, x0=None):
    """Right-preconditioned restarted GCR to ||b - A x|| <= tol ||b||.

    Returns (x, iterations, true relative residual).  With ``precond`` the
    search direction is p = M^{-1} r (flexible: M may change every call).
    """
    b = np.asarray(b, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    r = b - op(x)
    its = 0
    while True:
        rel = np.linalg.norm(r) / bnorm
        if rel <= tol or its >= maxit:
            return x, its, rel
        P, Q = [], []  # directions p_i and q_i = A p_i with ||q_i|| = 1
        for _ in range(restart):
            p = r.copy() if precond is None else precond(r)
            q = op(p)
            for pi, qi in zip(P, Q):  # modified Gram-Schmidt on A p
                beta = dot(qi, q)
                q = q - beta * qi
                p = p - beta * pi
            nq = np.linalg.norm(q)
            if nq == 0.0:
                break
            q, p = q / nq, p / nq
            alpha = dot(q, r)
            x = x + alpha * p
            r = r - alpha * q
            P.append(p)
            Q.append(q)
            its += 1
            if np.linalg.norm(r) <= tol * bnorm or its >= maxit:
                break
        r = b - op(x)  # true residual at every restart


def minres_steps(op, b, nsteps, x0=None, tol=0.0):
    """``nsteps`` minimal-residual steps on A x = b; stops early once
    ||b - A x|| <= tol ||b - A x0||.  Returns (x, steps taken, rel. residual)."""
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - op(x)
    r0 = np.linalg.norm(r)
    if r0 == 0.0:
        return x, 0, 0.0
    k = 0
    for k in range(1, nsteps + 1):
        q = op(r)
        qq = dot(q, q).real
        if qq == 0.0:
            break
        a = dot(q, r) / qq
        x = x + a * r
        r = r - a * q
        if np.linalg.norm(r) <= tol * r0:
            break
    return x, k, np.linalg.norm(r) / r0


def minres_columns(op, B, nsteps, X0=None, tol=0.0):
    """``minres_steps`` run on every column of B (n, s) independently.

    Column v stops once ||b_v - A x_v|| <= tol ||b_v - A x0_v|| (it is then
    left unchanged).  ``op`` maps an (n, s) block to an (n, s) block; frozen
    columns are still multiplied but never updated.  Returns (X, steps per
    column)."""
    X = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.complex128)
    R = B - op(X)
    r0 = np.linalg.norm(R, axis=0)
    active = r0 > 0.0
    steps = np.zeros(B.shape[1], dtype=np.int64)
    for _ in range(nsteps):
        if not active.any():
            break
        Q = op(R)
        qq = np.sum(np.abs(Q) ** 2, axis=0)
        qr = np.sum(Q.conj() * R, axis=0)
        a = np.where(active & (qq > 0.0), qr / np.where(qq > 0.0, qq, 1.0), 0.0)
        X = X + a * R
        R = R - a * Q
        steps += active
        active = active & (np.linalg.norm(R, axis=0) > tol * r0)
    return X, steps
