"""Dense references for small lattices: A as a matrix, tr A^{-1}, variances.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Eq. 1 (Sec. 1): t = (1/s) sum_j x_j^H A^{-1} x_j.  The printed left-hand
  side E[x^H A x] is read as E[x^H A^{-1} x], the quantity the sum estimates.
* Eq. 2 (Sec. 1): Var[t] = (2/s)||A^{-1}||_F^2 - (2/s) sum_i |(A^{-1})_ii|^2.
  For real Rademacher noise and a matrix B that is not symmetric, the exact
  variance is that of the symmetrised matrix S = (B + B^T)/2 (Sec. 2.1 says
  symmetrisation keeps the trace and never raises the variance).  Both the
  literal Eq. 2 and the exact value are provided; the exact one is what
  sample variances are compared with.

Pinned by brute-force enumeration of all sign vectors on small matrices and
by the free-field closed form of tr A^{-1} (tests/test_oracle_dense.py).
"""

import itertools

import numpy as np

from . import wilson


def dirac_matrix(U, m0, dims, tau=0.0):
    """Dense N x N matrix of A, N = 12 V, dof index 12*lex + 3*spin + colour."""
    V = int(np.prod(dims))
    N = 12 * V
    E = np.eye(N, dtype=np.complex128).reshape(V, 4, 3, N)
    return wilson.dirac_apply(U, E, m0, dims, tau=tau).reshape(N, N)


def gamma5_matrix(V):
    """gamma5 on the 12 V dof space: +1 on spins 0, 1 and -1 on spins 2, 3."""
    d = np.tile(np.repeat([1.0, 1.0, -1.0, -1.0], 3), V)
    return np.diag(d).astype(np.complex128)


def inverse(A):
    """A^{-1} by LU with partial pivoting (numpy/LAPACK getrf + getrs)."""
    return np.linalg.solve(A, np.eye(A.shape[0], dtype=A.dtype))


def eq2_variance(B, s=1):
    """Eq. 2 as printed, for a matrix B standing for A^{-1} (or its deflated part)."""
    return (2.0 / s) * (np.sum(np.abs(B) ** 2) - np.sum(np.abs(np.diag(B)) ** 2))


def exact_variance_real_rademacher(B, s=1):
    """E|t - tr B|^2 for t = (1/s) sum_j z_j^T B z_j, z_j real +-1 i.i.d.

    z^T B z - tr B = sum_{i<j} z_i z_j (B_ij + B_ji) and the products z_i z_j
    (i < j) are uncorrelated with unit variance, so the variance is
    sum_{i<j} |B_ij + B_ji|^2 = 2||S||_F^2 - 2 sum_i |S_ii|^2, S = (B + B^T)/2.
    """
    S = 0.5 * (B + B.T)
    return (2.0 / s) * (np.sum(np.abs(S) ** 2) - np.sum(np.abs(np.diag(S)) ** 2))


def exact_variance_real_part(B, s=1):
    """Var(Re t) for real Rademacher noise: sum_{i<j} (Re(B_ij + B_ji))^2 / s."""
    R = (B + B.T).real
    iu = np.triu_indices(B.shape[0], 1)
    return float(np.sum(R[iu] ** 2)) / s


def brute_force_variances(B):
    """Enumerate all 2^n sign vectors: (mean, E|t-mean|^2, Var Re t) for s = 1."""
    n = B.shape[0]
    ts = []
    for signs in itertools.product((1.0, -1.0), repeat=n):
        z = np.asarray(signs)
        ts.append(z @ B @ z)
    ts = np.asarray(ts)
    mean = ts.mean()
    return mean, float(np.mean(np.abs(ts - mean) ** 2)), float(np.var(ts.real))


def exact_variance_real_rademacher_diluted(B, classes, s=1):
    """E|t - tr B|^2 of the diluted estimator t = sum_h z_h^T B z_h, where z is
    real +-1 noise and z_h keeps the entries of class h (spin-colour
    dilution: class = dof mod 12).  Only products z_i z_j of one class
    survive, so the variance is sum_{i<j, same class} |B_ij + B_ji|^2."""
    c = np.asarray(classes)
    M = c[:, None] == c[None, :]
    S = 0.5 * (B + B.T)
    return (2.0 / s) * (np.sum(np.abs(S[M]) ** 2) - np.sum(np.abs(np.diag(S)) ** 2))


def brute_force_diluted_variance(B, classes):
    """Enumerate all sign vectors: E|t - mean|^2 of t = sum_h z_h^T B z_h."""
    n = B.shape[0]
    c = np.asarray(classes)
    ts = []
    for signs in itertools.product((1.0, -1.0), repeat=n):
        z = np.asarray(signs)
        t = 0.0
        for h in np.unique(c):
            zh = np.where(c == h, z, 0.0)
            t = t + zh @ B @ zh
        ts.append(t)
    ts = np.asarray(ts)
    return float(np.mean(np.abs(ts - ts.mean()) ** 2))

