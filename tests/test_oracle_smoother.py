"""Pins for oracle.smoother (the learned gauge-covariant smoother)."""
import numpy as np

from oracle import smoother, wilson
from paper_1909_12234_gb300 import synth


def test_wilson_weights_reproduce_the_operator():
    dims = (4, 4, 2, 6)
    U = synth.random_su3_links(dims, 0.4, 3)
    r = synth.random_field(dims, 3, 1)
    got = smoother.apply(U, smoother.wilson_weights(-0.7), r, dims)
    assert np.abs(got - wilson.dirac_apply(U, r, -0.7, dims)).max() < 1e-13


def test_identity_weights():
    dims = (2, 4, 2, 2)
    U = synth.random_su3_links(dims, 0.5, 1)
    r = synth.random_field(dims, 2, 2)
    w = np.zeros((9, 4, 4), complex)
    w[0] = np.eye(4)
    assert np.array_equal(smoother.apply(U, w, r, dims), r)


def test_fit_recovers_planted_weights():
    dims = (4, 2, 4, 2)
    U = synth.random_su3_links(dims, 0.3, 5)
    rng = np.random.default_rng(3)
    w0 = rng.standard_normal((9, 4, 4)) + 1j * rng.standard_normal((9, 4, 4))
    R = synth.random_field(dims, 4, 6)
    E = smoother.apply(U, w0, R, dims)
    w = smoother.fit(U, E, R, dims)
    assert np.abs(w - w0).max() < 1e-10 * np.abs(w0).max()


def test_gauge_covariance():
    dims = (4, 4, 2, 2)
    U = synth.random_su3_links(dims, 0.3, 7)
    rng = np.random.default_rng(1)
    w = rng.standard_normal((9, 4, 4)) + 1j * rng.standard_normal((9, 4, 4))
    r = synth.random_field(dims, 2, 8)
    Ug, g = synth.gauge_transform(U, dims, 9)
    rg = np.einsum("vab,vsbj->vsaj", g, r)
    lhs = smoother.apply(Ug, w, rg, dims)
    rhs = np.einsum("vab,vsbj->vsaj", g, smoother.apply(U, w, r, dims))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()
