"""Pins for oracle.dense: variance formulas against brute-force enumeration."""
import numpy as np

from oracle import dense, wilson
from paper_1909_12234_gb300 import synth


def _rand(n, seed, sym=False):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return 0.5 * (B + B.T) if sym else B


def test_exact_variance_matches_enumeration():
    for n, seed in [(6, 1), (9, 2), (11, 3)]:
        B = _rand(n, seed)
        mean, var, var_re = dense.brute_force_variances(B)
        assert abs(mean - np.trace(B)) < 1e-10
        assert abs(var - dense.exact_variance_real_rademacher(B)) < 1e-9 * var
        assert abs(var_re - dense.exact_variance_real_part(B)) < 1e-9 * var_re


def test_eq2_is_exact_only_for_symmetric_matrices():
    S = _rand(8, 4, sym=True)
    _, var, _ = dense.brute_force_variances(S)
    assert abs(dense.eq2_variance(S) - var) < 1e-9 * var
    B = _rand(8, 5)
    _, var, _ = dense.brute_force_variances(B)
    assert abs(dense.eq2_variance(B) - var) > 1e-3 * var  # Eq. 2 misses the symmetrisation


def test_variance_scales_with_samples():
    B = _rand(7, 6)
    assert np.isclose(dense.exact_variance_real_rademacher(B, s=4),
                      dense.exact_variance_real_rademacher(B) / 4)


def test_dense_inverse_trace_free_field():
    dims = (4, 4, 2, 2)
    U = synth.random_su3_links(dims, 0.0, 0, unit=True)
    A = dense.dirac_matrix(U, -0.3, dims)
    assert np.allclose(A @ dense.inverse(A), np.eye(A.shape[0]), atol=1e-12)
    assert abs(np.trace(dense.inverse(A)) - wilson.free_field_trace_inverse(dims, -0.3)) < 1e-10
