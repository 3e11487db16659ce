"""Pins for oracle.estimator: hand-computed statistics, the jackknife-of-mean
identity, and the estimator against the exact trace and variance."""
import math

import numpy as np
import pytest

from oracle import deflation, dense, estimator, multigrid
from paper_1909_12234_gb300 import synth


def test_statistics_hand_example():
    st = estimator.statistics([1.0, 2.0, 3.0, 4.0], t0=10.0)
    assert st["mean"] == 2.5 and st["estimate"] == 12.5
    assert math.isclose(st["var"], 5.0 / 3.0)
    assert math.isclose(st["stderr"], math.sqrt(5.0 / 12.0))
    # delete-one variances: 1, 7/3, 7/3, 1 -> jackknife error sqrt(4/3)
    assert math.isclose(st["var_jackknife_err"], math.sqrt(4.0 / 3.0))


def test_statistics_degenerate_sample_counts():
    st = estimator.statistics([3.0 + 1j])
    assert st["mean"] == 3.0 + 1j and st["var"] == 0.0 and st["var_jackknife_err"] == 0.0
    st = estimator.statistics([1.0, 3.0])
    assert st["var"] == 2.0 and st["var_jackknife_err"] == 0.0


def test_statistics_complex_and_real_part():
    t = np.array([1 + 1j, 1 - 1j, 3 + 1j, 3 - 1j])
    st = estimator.statistics(t)
    assert st["mean"] == 2.0
    assert math.isclose(st["var"], (4 * 2.0) / 3.0)  # |t - 2|^2 = 2 each
    assert math.isclose(st["var_re"], 4.0 / 3.0)


def test_jackknife_of_mean_equals_stderr():
    rng = np.random.default_rng(1)
    t = rng.standard_normal(25)
    s = t.size
    loo = np.array([np.delete(t, i).mean() for i in range(s)])
    jk_mean = math.sqrt((s - 1) / s * np.sum((loo - loo.mean()) ** 2))
    assert math.isclose(jk_mean, estimator.statistics(t)["stderr"], rel_tol=1e-12)


@pytest.fixture(scope="module")
def small():
    dims = (4, 4, 2, 2)
    U = synth.random_su3_links(dims, 0.3, 8)
    m0 = -0.4
    lev = multigrid.fine_level(U, m0, dims)
    A = lev.matrix.toarray()
    return lev, A, dense.inverse(A)


def test_undeflated_estimator_unbiased(small):
    lev, A, Ainv = small
    s = 48
    t, st, info = estimator.hutchinson(lev.matvec, lev.n, 5, range(s), 1e-11)
    assert all(rel <= 1e-11 for _, rel in info)
    exact = np.trace(Ainv)
    # per-sample values equal z^T A^{-1} z from the dense inverse
    from oracle import philox
    Z = philox.rademacher(lev.n, 5, range(s))
    assert np.allclose(t, np.einsum("ij,ij->j", Z, Ainv @ Z), rtol=1e-8)
    var_exact = dense.exact_variance_real_rademacher(Ainv)
    assert abs(st["estimate"] - exact) < 4.0 * math.sqrt(var_exact / s)
    assert abs(st["var"] - var_exact) < 5.0 * st["var_jackknife_err"] + 0.2 * var_exact


def test_deflated_estimator_alg1(small):
    lev, A, Ainv = small
    G5 = dense.gamma5_matrix(64)
    mu, Ue = deflation.fine_eigvecs_dense(A, G5, 16)
    a1 = deflation.Alg1(Ue, lev.matvec, 1e-11)
    s = 32
    t, st, _ = estimator.hutchinson(lev.matvec, lev.n, 6, range(s), 1e-11,
                                    project=a1.project, t0=a1.t0)
    B = Ainv @ (np.eye(lev.n) - Ue @ Ue.conj().T)
    var_exact = dense.exact_variance_real_rademacher(B)
    assert var_exact < dense.exact_variance_real_rademacher(Ainv)
    assert abs(st["estimate"] - np.trace(Ainv)) < 4.0 * math.sqrt(var_exact / s)


def test_diluted_variance_formula_by_enumeration():
    # t = sum_h z_h^T B z_h over classes of the dofs: the formula against all
    # 2^n sign vectors, and dilution never raises the variance
    rng = np.random.default_rng(11)
    n = 10
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    cls = np.arange(n) % 3
    ref = dense.brute_force_diluted_variance(B, cls)
    got = dense.exact_variance_real_rademacher_diluted(B, cls)
    assert abs(got - ref) < 1e-10 * ref
    assert got <= dense.exact_variance_real_rademacher(B) + 1e-12
    # one class per dof: no variance at all; one class for all: no dilution
    assert abs(dense.exact_variance_real_rademacher_diluted(B, np.arange(n))) < 1e-12
    assert abs(dense.exact_variance_real_rademacher_diluted(B, np.zeros(n)) -
               dense.exact_variance_real_rademacher(B)) < 1e-12


def test_dilute_parts_sum_to_the_vector():
    z = np.sign(np.random.default_rng(2).standard_normal(48))
    P = estimator.dilute(z)
    assert P.shape == (48, 12)
    assert np.array_equal(P.sum(axis=1), z)
    assert np.count_nonzero(P) == 48
    assert all(np.all(np.nonzero(P[:, h])[0] % 12 == h) for h in range(12))


def test_diluted_estimator_against_dense_trace_and_variance():
    # t_j = sum_h z_jh^H A^{-1} z_jh: per sample against the dense inverse,
    # mean within 4 SE of tr A^{-1}, sample variance within 4 jackknife
    # errors of the exact diluted variance (a 4 x 2 x 2 x 2 lattice keeps
    # the 12 solves per sample cheap)
    from oracle import philox
    dims = (4, 2, 2, 2)
    U = synth.random_su3_links(dims, 0.3, 8)
    lev = multigrid.fine_level(U, -0.4, dims)
    Ainv = dense.inverse(lev.matrix.toarray())
    s = 32
    t, st, _ = estimator.hutchinson(lev.matvec, lev.n, 5, range(s), 1e-10, dilution=True)
    Z = philox.rademacher(lev.n, 5, range(s))
    for j in (0, 7):
        Zh = estimator.dilute(Z[:, j].astype(complex))
        assert abs(t[j] - np.einsum("ih,ih->", Zh.conj(), Ainv @ Zh)) < 1e-8 * abs(t[j])
    var = dense.exact_variance_real_rademacher_diluted(Ainv, np.arange(lev.n) % 12)
    assert var < dense.exact_variance_real_rademacher(Ainv)
    assert abs(st["mean"].real - np.trace(Ainv).real) < 4 * math.sqrt(var / s)
    assert abs(st["var"] - var) < 4 * st["var_jackknife_err"] + 1e-9
