"""GPU parity for the multigrid pieces (Sec. 2): prolongation, restriction
and the Galerkin coarse operator against the oracle to 1e-12, with
null_maxit = 0 so that both sides block the same Philox random starts."""
import numpy as np
import pytest

from oracle import multigrid as omg
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


CASES = [
    # dims, m0, blocks, nvs  (coarse extents 2 and 1 on the deeper levels)
    ((4, 4, 4, 4), -0.4, [(2, 2, 2, 2)], [6]),
    ((4, 4, 4, 4), -0.4, [(2, 2, 2, 2), (2, 2, 1, 1)], [6, 4]),
    ((8, 4, 4, 4), -0.6, [(2, 2, 2, 2), (2, 1, 2, 1)], [5, 3]),
    ((8, 8, 8, 8), -0.8, [(2, 2, 2, 2)], [12]),
]


def _build(qd, ctx, dims, m0, blocks, nvs, null_maxit=0, tau=0.0):
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    p = qd.mg_params(len(blocks), blocks, nvs, null_maxit=null_maxit, seed=5)
    mg = qd.Multigrid(ctx, g, m0, tau, p)
    H = omg.setup(U, m0, dims, blocks, nvs, seed=5, null_maxit=null_maxit, tau=tau)
    return U, g, mg, H


@pytest.mark.parametrize("dims,m0,blocks,nvs", CASES)
def test_transfer_and_coarse_operator(qd, ctx, dims, m0, blocks, nvs):
    U, g, mg, H = _build(qd, ctx, dims, m0, blocks, nvs)
    rng = np.random.default_rng(1)
    for l, T in enumerate(H.transfers):
        s = 3
        c = rng.standard_normal((T.nc, s)) + 1j * rng.standard_normal((T.nc, s))
        f = rng.standard_normal((T.level.n, s)) + 1j * rng.standard_normal((T.level.n, s))
        cd = dev(c)
        fine = torch.empty((T.level.n * s,), dtype=torch.complex128, device="cuda:0")
        qd.prolongate(mg, l, s, cd, fine)
        if l == 0:
            got_f = qd.from_qd(ctx, g, fine.reshape(g.V, 12, s)).reshape(T.level.n, s)
            fd = qd.to_qd(ctx, g, f.reshape(g.V, 4, 3, s))
        else:
            got_f = host(fine).reshape(T.level.n, s)
            fd = dev(f)
        assert rel_err(got_f, T.prolong(c)) < 1e-12
        coarse = torch.empty((T.nc * s,), dtype=torch.complex128, device="cuda:0")
        qd.restrict(mg, l, s, fd, coarse)
        assert rel_err(host(coarse).reshape(T.nc, s), T.restrict(f)) < 1e-12
        # coarse operator of level l + 1
        out = torch.empty_like(coarse)
        qd.coarse_apply(mg, l + 1, s, cd, out)
        assert rel_err(host(out).reshape(T.nc, s), H.matrices[l] @ c) < 1e-12
        dims_c, dof, ns, _ = mg.level_info(l + 1)
        assert tuple(dims_c) == T.cdims and dof == 2 * T.nv and ns == T.Vc


@pytest.mark.parametrize("dims,m0,blocks,nvs", CASES + [((8, 8, 8, 8), -0.8, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16])])
def test_coarse_stencil_fp64_fp32_rhs_counts(qd, ctx, dims, m0, blocks, nvs):
    # the register-blocked coarse stencil for every level, with right-hand
    # side counts that leave ragged chunks (odd counts take the scalar FP32
    # loads); FP64 to 1e-12, FP32 within its rounding bound: at most 9 D
    # products per output (D <= 32), error <= ~300 u sum|c||x| with
    # u = 2^-24, and sum|c||x| <= 3 max|y| here, taken as 5e-5
    U, g, mg, H = _build(qd, ctx, dims, m0, blocks, nvs)
    rng = np.random.default_rng(5)
    for l in range(len(blocks)):
        nc = H.transfers[l].nc
        for s in (1, 2, 3, 64, 130, 300):
            c = rng.standard_normal((nc, s)) + 1j * rng.standard_normal((nc, s))
            ref = H.matrices[l] @ c
            cd = dev(c)
            out = torch.empty_like(cd)
            qd.coarse_apply(mg, l + 1, s, cd, out)
            assert rel_err(host(out).reshape(nc, s), ref) < 1e-12, (l, s)
            c32 = cd.to(torch.complex64)
            o32 = torch.empty_like(c32)
            qd.coarse_apply_f32(mg, l + 1, s, c32, o32)
            assert rel_err(host(o32).astype(np.complex128).reshape(nc, s), ref) < 5e-5, (l, s)


@pytest.mark.parametrize("dims,m0,blocks,nvs", CASES + [((8, 8, 8, 8), -0.8, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16]),
                                                        ((4, 4, 4, 8), -0.6, [(2, 2, 2, 2), (1, 1, 2, 2)], [8, 8])])
def test_prolongation_fp32(qd, ctx, dims, m0, blocks, nvs):
    # the FP32 prolongation of the V-cycle (register-blocked two-column form
    # for even counts, scalar form for odd ones) against the oracle's W c:
    # nv FP32 complex products per output plus the rounding of W and c, so
    # |error| <= 4 (nv + 2) 2^-24 (|W| |c|) elementwise
    U, g, mg, H = _build(qd, ctx, dims, m0, blocks, nvs)
    rng = np.random.default_rng(11)
    for l, T in enumerate(H.transfers):
        Wabs = T.matrix().copy()
        Wabs.data = np.abs(Wabs.data)
        for s in (1, 2, 3, 64, 130):
            c = rng.standard_normal((T.nc, s)) + 1j * rng.standard_normal((T.nc, s))
            c32 = dev(c).to(torch.complex64)
            c_r = host(c32).astype(np.complex128)  # the rounded input both sides use
            ref = T.prolong(c_r)
            fine = torch.empty((T.level.n * s,), dtype=torch.complex64, device="cuda:0")
            qd.prolongate_f32(mg, l, s, c32, fine)
            got = host(fine).astype(np.complex128)
            if l == 0:
                got = qd.from_qd(ctx, g, torch.from_numpy(got).to("cuda:0").reshape(g.V, 12, s))
            got = np.asarray(got).reshape(T.level.n, s)
            bound = 4 * (T.nv + 2) * 2.0 ** -24 * (Wabs @ np.abs(c_r)) + 1e-30
            assert np.all(np.abs(got - ref) <= bound), (l, s, np.max(np.abs(got - ref) / bound))


def test_null_vector_iteration(qd, ctx):
    # the full adaptive setup (MR on A y = 0 to 1e-2 / 200 steps): the same
    # step counts per vector as the oracle, an orthonormal chiral W, and a
    # gamma5^W-Hermitian coarse operator
    dims, m0 = (4, 4, 4, 4), -0.4
    U, g, mg, H = _build(qd, ctx, dims, m0, [(2, 2, 2, 2)], [6], null_maxit=200)
    _, _, _, steps = mg.level_info(0)
    from oracle import multigrid as om
    _, its = om.null_vectors(H.levels[0], 6, 5, 1e-2, 200)
    assert list(steps) == list(its)
    T = H.transfers[0]
    rng = np.random.default_rng(3)
    s = 2
    c = rng.standard_normal((T.nc, s)) + 1j * rng.standard_normal((T.nc, s))
    fine = torch.empty((T.level.n * s,), dtype=torch.complex128, device="cuda:0")
    qd.prolongate(mg, 0, s, dev(c), fine)
    back = torch.empty((T.nc * s,), dtype=torch.complex128, device="cuda:0")
    qd.restrict(mg, 0, s, fine, back)
    assert rel_err(host(back).reshape(T.nc, s), c) < 1e-12  # W^H W = I
    g5 = np.tile(np.repeat([1.0, -1.0], T.nv), T.Vc)[:, None]
    y = rng.standard_normal((T.nc, s)) + 1j * rng.standard_normal((T.nc, s))
    Cc = torch.empty_like(back)
    qd.coarse_apply(mg, 1, s, dev(c), Cc)
    Cy = torch.empty_like(back)
    qd.coarse_apply(mg, 1, s, dev(g5 * y), Cy)
    lhs = np.sum((g5 * y).conj() * host(Cc).reshape(T.nc, s), axis=0)   # <g5 y, C c>
    rhs = np.sum((host(Cy).reshape(T.nc, s)).conj() * c, axis=0)          # <C g5 y, c>... via g5 C hermitian
    G = g5 * H.matrices[0].toarray()
    assert np.abs(G - G.conj().T).max() < 1e-12
    assert np.allclose(lhs, np.sum((g5 * y).conj() * (H.matrices[0] @ c), axis=0), rtol=1e-9)


def test_injected_null_vectors(qd, ctx):
    dims, m0 = (4, 4, 4, 4), -0.4
    U = synth.random_su3_links(dims, 0.3, 7)
    g = qd.Gauge(ctx, dims, U)
    rng = np.random.default_rng(8)
    Y = rng.standard_normal((12 * g.V, 4)) + 1j * rng.standard_normal((12 * g.V, 4))
    Yd = qd.to_qd(ctx, g, Y.reshape(g.V, 4, 3, 4))
    p = qd.mg_params(1, [(2, 2, 2, 2)], [4], seed=1)
    mg = qd.Multigrid(ctx, g, m0, 0.0, p, injected_null=Yd)
    lev = omg.fine_level(U, m0, dims)
    T = omg.build_transfer(lev, (2, 2, 2, 2), Y)
    C = omg.coarse_matrix(lev, T)
    c = rng.standard_normal((T.nc, 2)) + 0j
    out = torch.empty((T.nc * 2,), dtype=torch.complex128, device="cuda:0")
    qd.coarse_apply(mg, 1, 2, dev(c), out)
    assert rel_err(host(out).reshape(T.nc, 2), C @ c) < 1e-12


@pytest.mark.parametrize("dims,m0,blocks,nvs", [((4, 4, 4, 4), -0.4, [(2, 2, 2, 2)], [6]),
                                                ((8, 8, 8, 8), -0.8, [(2, 2, 2, 2)], [12]),
                                                ((4, 4, 4, 4), -0.4, [(2, 2, 2, 2), (2, 2, 1, 1)], [6, 4])])
def test_direct_coarsest_solve(qd, ctx, dims, m0, blocks, nvs):
    # the coarsest operator's dense Gauss-Jordan inverse: C (C^{-1} x) = x, and
    # C^{-1} x equals the oracle's sparse LU solve
    U, g, mg, H = _build(qd, ctx, dims, m0, blocks, nvs, null_maxit=50)
    L = len(blocks)
    T = H.transfers[-1]
    rng = np.random.default_rng(5)
    s = 4
    x = rng.standard_normal((T.nc, s)) + 1j * rng.standard_normal((T.nc, s))
    y = torch.empty((T.nc * s,), dtype=torch.complex128, device="cuda:0")
    qd.coarse_solve(mg, L, s, dev(x), y)
    back = torch.empty_like(y)
    qd.coarse_apply(mg, L, s, y, back)
    assert rel_err(host(back).reshape(T.nc, s), x) < 1e-10
    import scipy.sparse.linalg as spla
    ref = spla.splu(H.matrices[-1].tocsc()).solve(x)
    assert rel_err(host(y).reshape(T.nc, s), ref) < 1e-9


def test_null_vectors_in_fp32(qd, ctx):
    # null_f32: the same minimal-residual iteration in FP32 (the vectors need
    # only the 1e-2 null_tol); step counts within one or two of the FP64
    # iteration's, an orthonormal W, and a solve that reaches the FP64
    # tolerance with the resulting hierarchy
    dims, m0 = (8, 8, 8, 8), -0.8
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    steps = {}
    for f32 in (0, 1):
        mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(2, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16], null_f32=f32,
                                                         coarse_tol=0.0, coarse_maxit=6))
        steps[f32] = [mg.level_info(l)[3] for l in (0, 1)]
        if f32:
            T_nc = mg.level_info(1)[2] * mg.level_info(1)[1]
            c = np.random.default_rng(1).standard_normal((T_nc, 2)) + 0j
            fine = torch.empty((g.V * 12 * 2,), dtype=torch.complex128, device="cuda:0")
            qd.prolongate(mg, 0, 2, dev(c), fine)
            back = torch.empty((T_nc * 2,), dtype=torch.complex128, device="cuda:0")
            qd.restrict(mg, 0, 2, fine, back)
            assert rel_err(host(back).reshape(T_nc, 2), c) < 1e-12  # W^H W = I
            b = dev(np.random.default_rng(2).standard_normal((g.V, 12, 4)) + 0j)
            x = torch.empty_like(b)
            _, its, _, rel = qd.solve(ctx, g, mg, m0, 0.0, 4, b, x, 1e-8, maxit=500, precision=qd.QD_PREC_MIXED)
            assert max(rel) <= 1e-8
        mg.close()
    for l in (0, 1):
        assert all(abs(int(a) - int(b)) <= 2 for a, b in zip(steps[0][l], steps[1][l])), (l, steps)
    g.close()
