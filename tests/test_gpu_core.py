"""GPU parity: reorder, Rademacher noise (bit-exact) and the FP64 Wilson
stencil (1e-12 relative) against the oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import lattice, philox, wilson
from paper_1909_12234_gb300 import synth

from gpu_util import dev, host, need_gpu, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qd():
    need_gpu()
    from paper_1909_12234_gb300 import qdtrace
    qdtrace.load()
    return qdtrace


@pytest.fixture(scope="module")
def ctx(qd):
    return qd.Context(0)


DIMS = [(4, 4, 4, 4), (2, 2, 2, 2), (8, 4, 6, 2), (4, 2, 2, 6), (6, 6, 6, 6)]


@pytest.mark.parametrize("dims", DIMS)
def test_reorder_places_sites_by_even_odd_index(qd, ctx, dims):
    U = synth.random_su3_links(dims, 0.3, 1)
    g = qd.Gauge(ctx, dims, U)
    V = g.V
    s = 3
    x = synth.random_field(dims, s, 2)
    y = qd.to_qd(ctx, g, x)
    eo = lattice.eo_index(dims)
    want = np.empty((V, 12, s), dtype=complex)
    want[eo] = x.reshape(V, 12, s)
    assert np.array_equal(host(y), want)
    assert np.array_equal(qd.from_qd(ctx, g, y), x)


@pytest.mark.parametrize("dims,seed,offset,s", [((4, 4, 4, 4), 101, 0, 32), ((8, 4, 6, 2), 7, 5, 3),
                                                ((2, 2, 2, 2), 2**40 + 3, 1000, 1), ((6, 6, 6, 6), 9, 0, 70)])
def test_rademacher_bit_exact(qd, ctx, dims, seed, offset, s):
    U = synth.random_su3_links(dims, 0.0, 0, unit=True)
    g = qd.Gauge(ctx, dims, U)
    out = torch.empty((g.V, 12, s), dtype=torch.complex128, device="cuda:0")
    qd.rademacher(ctx, g, seed, offset, s, out)
    got = qd.from_qd(ctx, g, out).reshape(12 * g.V, s)
    want = philox.rademacher(12 * g.V, seed, range(offset, offset + s))
    assert np.array_equal(got.real, want) and np.all(got.imag == 0)


def _apply(qd, ctx, g, m0, tau, dag, x):
    xin = qd.to_qd(ctx, g, x)
    out = torch.empty_like(xin)
    qd.dirac_apply(ctx, g, m0, tau, dag, x.shape[3], xin, out)
    return qd.from_qd(ctx, g, out)


@pytest.mark.parametrize("dims,s", [((4, 4, 4, 4), 1), ((4, 4, 4, 4), 32), ((8, 4, 6, 2), 3),
                                    ((4, 2, 2, 6), 70), ((2, 2, 2, 2), 5), ((6, 6, 6, 6), 33)])
@pytest.mark.parametrize("tau,dag", [(0.0, False), (0.25, False), (0.25, True)])
def test_wilson_fp64_matches_oracle(qd, ctx, dims, s, tau, dag):
    U = synth.random_su3_links(dims, 0.3, 4)
    g = qd.Gauge(ctx, dims, U)
    x = synth.random_field(dims, s, 3)
    got = _apply(qd, ctx, g, -0.4, tau, dag, x)
    ref = wilson.dirac_apply(U, x, -0.4, dims, tau=tau, dagger=dag)
    assert rel_err(got, ref) < 1e-12


def test_wilson_full_size_8x4_64rhs(qd, ctx):
    # the estimator workload's size: 8^4 lattice, 64 right-hand sides
    dims = (8, 8, 8, 8)
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    x = synth.random_field(dims, 64, 9)
    got = _apply(qd, ctx, g, -0.8, 0.0, False, x)
    cols = [0, 17, 63]
    ref = wilson.dirac_apply(U, x[..., cols], -0.8, dims)
    assert rel_err(got[..., cols], ref) < 1e-12


@pytest.mark.parametrize("dims,s", [((4, 4, 4, 4), 32), ((8, 4, 6, 2), 3), ((4, 2, 2, 6), 70),
                                    ((16, 16, 16, 32), 4)])
@pytest.mark.parametrize("tau,dag", [(0.0, False), (0.25, True)])
def test_wilson_fp32_matches_oracle(qd, ctx, dims, s, tau, dag):
    # FP32 inputs, links and arithmetic: each output is a sum of about 60
    # products of O(1) terms, so |error| <= ~60 u max|y| (u = 2^-24), taken
    # as 1e-5 relative to max|y|
    U = synth.random_su3_links(dims, 0.2, 4)
    g = qd.Gauge(ctx, dims, U)
    x = synth.random_field(dims, s, 3)
    xin = qd.to_qd(ctx, g, x).to(torch.complex64)
    out = torch.empty_like(xin)
    qd.dirac_apply_f32(ctx, g, -0.8, tau, dag, s, xin, out)
    got = qd.from_qd(ctx, g, out.to(torch.complex128))
    cols = list(range(min(s, 3)))
    ref = wilson.dirac_apply(U, x[..., cols], -0.8, dims, tau=tau, dagger=dag)
    assert rel_err(got[..., cols], ref) < 1e-5


@pytest.mark.parametrize("dims,s", [((4, 4, 4, 4), 64), ((8, 8, 8, 8), 64), ((8, 4, 6, 2), 128),
                                    ((6, 6, 6, 6), 128)])
@pytest.mark.parametrize("tau,dag", [(0.0, False), (0.25, True)])
def test_wilson_fp32_staged_matches_oracle(qd, ctx, dims, s, tau, dag):
    # the stencil with its operands staged in shared memory: by bulk copies
    # (launch shapes 10-12: rings of 8 warps x 4 slots, 4 x 8 and 6 x 5; one
    # to seven sites per warp here, the last round of sites ragged) and by
    # cp.async one hop ahead (13-14: columns whole or in chunks of 64), as
    # A x and as the residual b - A x, against the oracle (tolerance as
    # above); every output element written (NaN-filled outputs) and equal to
    # the register-only form to FP32 rounding
    U = synth.random_su3_links(dims, 0.2, 4)
    g = qd.Gauge(ctx, dims, U)
    x = synth.random_field(dims, s, 3)
    b = synth.random_field(dims, s, 5)
    xin = qd.to_qd(ctx, g, x).to(torch.complex64)
    bin_ = qd.to_qd(ctx, g, b).to(torch.complex64)
    cols = [0, s // 2 + 1, s - 1]
    ref = wilson.dirac_apply(U, x[..., cols], -0.8, dims, tau=tau, dagger=dag)
    refr = b[..., cols] - ref
    try:
        qd.autotune_force(0)
        y0 = torch.empty_like(xin)
        qd.dirac_apply_f32(ctx, g, -0.8, tau, dag, s, xin, y0)
        r0 = torch.empty_like(xin)
        qd.dirac_residual_f32(ctx, g, -0.8, tau, dag, s, bin_, xin, r0)
        for cand in (10, 11, 12, 13, 14):
            qd.autotune_force(cand)
            y = torch.full_like(xin, float("nan"))
            qd.dirac_apply_f32(ctx, g, -0.8, tau, dag, s, xin, y)
            got = qd.from_qd(ctx, g, y.to(torch.complex128))
            assert rel_err(got[..., cols], ref) < 1e-5, cand
            assert rel_err(host(y), host(y0)) < 1e-6, cand
            r = torch.full_like(xin, float("nan"))
            qd.dirac_residual_f32(ctx, g, -0.8, tau, dag, s, bin_, xin, r)
            gotr = qd.from_qd(ctx, g, r.to(torch.complex128))
            assert rel_err(gotr[..., cols], refr) < 1e-5, cand
            assert rel_err(host(r), host(r0)) < 1e-6, cand
    finally:
        qd.autotune_force(-1)
    g.close()


def test_gamma5_hermiticity_on_gpu(qd, ctx):
    dims = (4, 4, 4, 4)
    U = synth.random_su3_links(dims, 0.3, 6)
    g = qd.Gauge(ctx, dims, U)
    x = synth.random_field(dims, 2, 1)
    y = synth.random_field(dims, 2, 2)
    Ax = _apply(qd, ctx, g, -0.4, 0.0, False, x)
    g5 = np.array([1, 1, -1, -1])[None, :, None, None]
    g5Ag5y = g5 * _apply(qd, ctx, g, -0.4, 0.0, False, g5 * y)
    lhs = np.einsum("vsar,vsar->r", y.conj(), Ax)
    rhs = np.einsum("vsar,vsar->r", g5Ag5y.conj(), x)
    assert np.allclose(lhs, rhs, rtol=1e-12)


def test_free_field_plane_wave_on_gpu(qd, ctx):
    dims = (4, 4, 4, 4)
    U = synth.random_su3_links(dims, 0.0, 0, unit=True)
    g = qd.Gauge(ctx, dims, U)
    c = lattice.coords(dims)
    p = 2 * np.pi * np.array([1, 2, 0, 3]) / np.array(dims)
    gm = wilson.gammas()
    M = -0.4 + np.sum(1 - np.cos(p))
    Dp = M * np.eye(4) + 1j * sum(gm[m] * np.sin(p[m]) for m in range(4))
    lam, vec = np.linalg.eig(Dp)
    x = (np.exp(1j * (c @ p))[:, None, None] * vec[:, 0][None, :, None] * np.array([1.0, -0.5, 0.25])[None, None, :])
    y = _apply(qd, ctx, g, -0.4, 0.0, False, x[..., None])[..., 0]
    assert np.abs(y - lam[0] * x).max() < 1e-12


def test_invalid_arguments_are_rejected(qd, ctx):
    dims = (4, 4, 4, 4)
    g = qd.Gauge(ctx, dims, synth.random_su3_links(dims, 0.0, 0, unit=True))
    t = torch.zeros((g.V, 12, 1), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(qd.QDError) as e:
        qd.dirac_apply(ctx, g, -0.4, 0.0, False, 1, t, t)  # in == out
    assert e.value.code == qd.QD_ERR_INVALID
    with pytest.raises(qd.QDError):
        qd.Gauge(ctx, (3, 4, 4, 4), np.zeros((4, 48, 3, 3), complex))  # odd Lx
    with pytest.raises(qd.QDError):
        qd.rademacher(ctx, g, 1, 2**32 - 1, 2, torch.zeros((g.V, 12, 2), dtype=torch.complex128, device="cuda:0"))
