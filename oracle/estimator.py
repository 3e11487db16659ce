"""The deflated Hutchinson estimator and its statistics.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Eq. 1 (Sec. 1): t = (1/s) sum_j x_j^H A^{-1} x_j with Rademacher x_j.
* Algorithms 1 and 2 (Sec. 4): estimate = t0 + t1, t1 the Hutchinson
  estimate of tr(A^{-1}_xi (I - P)), H = identity (no probing).
* Sec. 4.1 reports variances with jackknife errors.

Per-sample values t_j = z_j^H A^{-1}_xi (I - P) z_j ("vector form": solve
with the deflated right-hand side).  Statistics, for complex samples t_j:

* mean = (1/s) sum t_j; the estimate of tr A^{-1} is t0 + mean;
* var = (1/(s-1)) sum |t_j - mean|^2 (the |.|^2 of Eq. 2), and var_re the
  same for Re t_j;
* stderr = sqrt(var / s);
* jackknife error of var: delete-one variances v_(i) over s - 1 samples,
  err = sqrt((s-1)/s * sum (v_(i) - mean v)^2).

A sample variance needs s >= 2 and its jackknife s >= 3; below that the
value is undefined and reported as 0 (this library's convention).

Sums use ``math.fsum`` (correctly rounded), so the result does not depend on
summation order.  Pinned by hand-computed examples and the identity that the
jackknife error of a mean equals its standard error
(tests/test_oracle_estimator.py).
"""

import math

import numpy as np

from . import krylov, philox


def _fsum_c(v):
    v = np.asarray(v, dtype=np.complex128)
    return complex(math.fsum(v.real), math.fsum(v.imag))


def sample_variance(t):
    t = np.asarray(t, dtype=np.complex128)
    s = t.size
    if s < 2:
        return 0.0
    m = _fsum_c(t) / s
    return math.fsum(np.abs(t - m) ** 2) / (s - 1)


def statistics(t, t0=0.0):
    """Mean, variances, stderr and jackknife error of the per-sample t_j."""
    t = np.asarray(t, dtype=np.complex128)
    s = t.size
    mean = _fsum_c(t) / s
    var = sample_variance(t)
    var_re = sample_variance(t.real)
    if s >= 3:
        loo = np.array([sample_variance(np.delete(t, i)) for i in range(s)])
        loo_mean = math.fsum(loo) / s
        jk = math.sqrt((s - 1) / s * math.fsum((loo - loo_mean) ** 2))
    else:
        jk = 0.0
    return {
        "t0": complex(t0),
        "mean": mean,
        "estimate": complex(t0) + mean,
        "var": var,
        "var_re": var_re,
        "stderr": math.sqrt(var / s),
        "var_jackknife_err": jk,
        "s": s,
    }


def dilute(z, nclass=12):
    """Spin-colour dilution (the probing basis H of Algorithms 1 and 2 with
    its 12 spin-colour vectors): z_h keeps the entries of z whose dof
    (12 lex + 3 spin + colour) is h modulo 12.  Returns (n, nclass)."""
    z = np.asarray(z)
    cls = np.arange(z.shape[0]) % nclass
    return np.stack([np.where(cls == h, z, 0) for h in range(nclass)], axis=1)


def hutchinson(A_matvec, ndof, seed, samples, xi, project=None, t0=0.0,
               precond=None, restart=16, maxit=100000, dilution=False):
    """Per-sample t_j = z_j^H A^{-1}_xi (project(z_j)) and their statistics.

    ``project`` is (I - P) of Algorithm 1 or 2, or None (plain Eq. 1).  With
    ``dilution`` every sample is t_j = sum_h z_jh^H A^{-1}_xi project(z_jh)
    over the 12 spin-colour parts z_jh of z_j (t(... odot H H^H) of
    Algorithms 1 and 2 with H the spin-colour basis).
    Returns (t (s,), stats dict, per-sample (iterations, true rel residual)).
    """
    Z = philox.rademacher(ndof, seed, samples)
    ts, info = [], []
    for j in range(Z.shape[1]):
        z = Z[:, j].astype(np.complex128)
        parts = dilute(z).T if dilution else [z]
        tj, its_j, rel_j = 0j, 0, 0.0
        for zh in parts:
            b = zh if project is None else project(zh)
            x, its, rel = krylov.gcr(A_matvec, b, xi, maxit=maxit, restart=restart,
                                     precond=precond)
            tj += np.vdot(zh, x)
            its_j, rel_j = max(its_j, its), max(rel_j, rel)
        ts.append(tj)
        info.append((its_j, rel_j))
    t = np.asarray(ts)
    return t, statistics(t, t0), info
