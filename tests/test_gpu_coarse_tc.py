"""GPU parity for the coarse-operator stencil on tcgen05 tensor cores against
the oracle's C = W^H A W (Sec. 2), with null_maxit = 0 so that both sides
block the same Philox starts.

The kernel splits every operand v into two BF16 terms, hi = bf16(v) and
lo = bf16(v - hi) (8 significant bits each, unit roundoff u = 2^-8), and
forms a_hi b_hi + a_hi b_lo + a_lo b_hi with FP32 accumulation.  Per real
product, with a = a_hi + a_lo + e_a, |e_a| <= u^2 |a| (likewise b):
ab - computed = e_a b + a e_b - e_a e_b + a_lo b_lo, at most
(3u^2 + 3u^3)|a||b|; the FP64 entries of C pass through FP32 first (2^-24).
Each of the 2 x 9 x (2D/16) MMA steps adds its products to the FP32
accumulator with an error below 2^-22 of the magnitudes summed so far, and
the epilogue adds two columns (2^-24).  So, for the real and the imaginary
part alike, |y - y_ref| <= (3u^2 + 3u^3 + 2^-23 + (18 (2D/16) + 1) 2^-22) S
with S = sum_dir P(C_dir) P(x), P(z) = |Re z| + |Im z| elementwise, over the
nine direction blocks the kernel rounds separately.  The oracle forms each
C_dir as W^H A_dir W, with A_dir the entries of the level's operator A whose
hop (site s -> site t) crosses the face dir of s's aggregate (dir 0: the
site term and hops inside the aggregate); the level's own extents are >= 3,
so a site pair fixes its hop.  On coarse lattices of extent 1 or 2 the +mu
and -mu blocks share entries of C (and may cancel there), which is why the
blocks are kept apart."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import lattice
from oracle import multigrid as omg
from paper_1909_12234_gb300 import synth

from gpu_util import dev, host, need_gpu, torch

pytestmark = pytest.mark.gpu

U_BF16 = 2.0 ** -8
N_TC_CANDIDATES = 11  # launch shapes of the tensor-core stencil


@pytest.fixture(scope="module")
def qd():
    need_gpu()
    from paper_1909_12234_gb300 import qdtrace
    qdtrace.load()
    return qdtrace


@pytest.fixture(scope="module")
def ctx(qd):
    return qd.Context(0)


def _abs_parts(M):
    return abs(M.real) + abs(M.imag)


def _check(got, ref, S, D):
    u = U_BF16
    tol = (3 * u ** 2 + 3 * u ** 3 + 2.0 ** -23 + (18 * (2 * D // 16) + 1) * 2.0 ** -22) * S
    err_re = np.abs(got.real - ref.real)
    err_im = np.abs(got.imag - ref.imag)
    assert np.all(err_re <= tol) and np.all(err_im <= tol), float(max((err_re / tol).max(), (err_im / tol).max()))
    # and the result is not far off in plain terms either
    assert np.abs(got - ref).max() < 1e-4 * np.abs(ref).max()


def _direction_blocks(H, l):
    """P(C_dir) for the nine coarse directions of level l + 1 (sparse)."""
    lev, T = H.levels[l], H.transfers[l]
    dims, dof = lev.dims, lev.dof
    assert min(dims) >= 3, "site pairs must fix the hop"
    A = lev.matrix.tocoo()
    cs, ct = lattice.coords(dims)[A.row // dof], lattice.coords(dims)[A.col // dof]
    L = np.asarray(dims)
    diff = (ct - cs) % L  # +1 forward, L-1 backward in the one direction that moves
    cd = np.zeros(A.nnz, dtype=np.int64)
    for mu in range(4):
        rem = cs[:, mu] % T.block[mu]
        fwd = diff[:, mu] == 1
        bwd = diff[:, mu] == L[mu] - 1
        cd[fwd & (rem == T.block[mu] - 1)] = 1 + mu
        cd[bwd & (rem == 0)] = 5 + mu
    W = T.matrix()
    out = []
    for d in range(9):
        m = cd == d
        Ad = sp.csr_matrix((A.data[m], (A.row[m], A.col[m])), shape=A.shape)
        out.append(sp.csr_matrix(_abs_parts((W.conj().T @ Ad @ W).tocsr())))
    # the blocks add up to the oracle's C
    Csum = sum((W.conj().T @ sp.csr_matrix((A.data[cd == d], (A.row[cd == d], A.col[cd == d])), shape=A.shape) @ W)
               for d in range(9))
    assert abs(Csum - H.matrices[l]).max() < 1e-12
    return out


CASES = [
    # dims, m0, blocks, nvs -> coarse dof 2 nv on each level
    ((8, 8, 8, 8), -0.8, [(2, 2, 2, 2)], [12]),                    # D = 24 on 4^4
    ((8, 8, 8, 8), -0.8, [(2, 2, 2, 2)], [4]),                     # D = 8 on 4^4
    ((8, 8, 8, 8), -0.8, [(2, 2, 2, 2), (2, 2, 2, 2)], [8, 16]),   # D = 16 on 4^4, D = 32 on 2^4
    ((4, 4, 4, 4), -0.4, [(2, 2, 2, 2)], [4]),                     # D = 8 on 2^4
    ((4, 4, 4, 4), -0.4, [(4, 4, 2, 2)], [8]),                     # D = 16 on 1 x 1 x 2 x 2
]


@pytest.mark.parametrize("dims,m0,blocks,nvs", CASES)
def test_tensor_core_coarse_stencil(qd, ctx, dims, m0, blocks, nvs):
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(len(blocks), blocks, nvs, null_maxit=0, seed=5))
    H = omg.setup(U, m0, dims, blocks, nvs, seed=5, null_maxit=0)
    rng = np.random.default_rng(7)
    for l in range(len(blocks)):
        nc = H.transfers[l].nc
        D = 2 * nvs[l]
        C = H.matrices[l]
        blocks_abs = _direction_blocks(H, l)
        for s in (1, 2, 3, 64, 127, 128, 130, 300):
            x = (rng.standard_normal((nc, s)) + 1j * rng.standard_normal((nc, s))).astype(np.complex64)
            xd = torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")
            out = torch.full_like(xd, float("nan"))
            qd.coarse_apply_tc(mg, l + 1, s, xd, out)
            got = host(out).astype(np.complex128)
            x64 = x.astype(np.complex128)
            px = _abs_parts(x64)
            _check(got, C @ x64, sum(b @ px for b in blocks_abs), D)
            # deterministic: a second call gives the same bits
            out2 = torch.empty_like(xd)
            qd.coarse_apply_tc(mg, l + 1, s, xd, out2)
            assert torch.equal(out, out2)
            # every launch shape (input split into operand tiles first, or
            # converted inside the kernel; operand/staging ring depths) forms
            # the same operands and MMAs: the same bits
            # the residual form subtracts in the epilogue: the same bits as
            # b - (C x) in FP32
            bd = torch.from_numpy(np.ascontiguousarray(
                (rng.standard_normal((nc, s)) + 1j * rng.standard_normal((nc, s))).astype(np.complex64))).to("cuda:0")
            want = bd - out
            try:
                for cand in range(N_TC_CANDIDATES):
                    qd.autotune_force(cand)
                    out3 = torch.full_like(xd, float("nan"))
                    qd.coarse_apply_tc(mg, l + 1, s, xd, out3)
                    assert torch.equal(out, out3), (l, s, cand)
                    res = torch.full_like(xd, float("nan"))
                    qd.coarse_residual_tc(mg, l + 1, s, bd, xd, res)
                    assert torch.equal(res, want), (l, s, cand)
            finally:
                qd.autotune_force(-1)
    for o in (mg, g):
        o.close()


def test_tensor_core_coarse_stencil_rejects_unsupported(qd, ctx):
    dims = (4, 4, 4, 4)
    g = qd.Gauge(ctx, dims, synth.random_su3_links(dims, 0.3, 2))
    mg = qd.Multigrid(ctx, g, -0.4, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [6], null_maxit=0, seed=5))  # D = 12
    x = torch.zeros((16 * 12, 4), dtype=torch.complex64, device="cuda:0")
    with pytest.raises(qd.QDError) as ei:
        qd.coarse_apply_tc(mg, 1, 4, x, torch.empty_like(x))
    assert ei.value.code == qd.QD_ERR_INVALID
    mg2 = qd.Multigrid(ctx, g, -0.4, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [4], null_maxit=0, seed=5))  # D = 8
    x = torch.zeros((16 * 8, 131), dtype=torch.complex64, device="cuda:0")  # odd and above 128
    with pytest.raises(qd.QDError) as ei:
        qd.coarse_apply_tc(mg2, 1, 131, x, torch.empty_like(x))
    assert ei.value.code == qd.QD_ERR_INVALID
    for o in (mg2, mg, g):
        o.close()


def test_mixed_solve_with_tensor_core_coarse_stencil(qd, ctx):
    # three-level mixed-precision solve with the level-1 stencil on tensor
    # cores reaches the FP64 true residual, like the CUDA-core form
    dims, m0, s, xi = (8, 8, 8, 8), -0.8, 16, 1e-8
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    out = {}
    for tc in (0, 1):
        mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(2, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16],
                                                       coarse_tol=0.0, coarse_maxit=6, coarse_tc=tc))
        rng = np.random.default_rng(3)
        b = rng.standard_normal((g.V, 12, s)) + 0j
        bd = dev(b)
        x = torch.empty_like(bd)
        st, its, _, rel = qd.solve(ctx, g, mg, m0, 0.0, s, bd, x, xi, maxit=500, precision=qd.QD_PREC_MIXED,
                                   inner_tol=1e-5, max_refine=10)
        assert max(rel) <= xi
        out[tc] = its
        mg.close()
    # the split-BF16 stencil is a slightly perturbed preconditioner:
    # comparable iteration counts
    assert out[1] <= 1.2 * out[0] + 2, out
    g.close()


@pytest.mark.parametrize("dims,m0,blocks,nvs", CASES)
def test_tensor_core_restriction(qd, ctx, dims, m0, blocks, nvs):
    # coarse = W^H fine with split-BF16 operands against the oracle's
    # restriction; bound as above with S = P(W)^T P(fine) (the sum of
    # magnitudes of the products of one output) and 2 x (sites per
    # aggregate) x (2 Df / 16) MMA steps
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(len(blocks), blocks, nvs, null_maxit=0, seed=5))
    H = omg.setup(U, m0, dims, blocks, nvs, seed=5, null_maxit=0)
    rng = np.random.default_rng(8)
    u = U_BF16
    for l, T in enumerate(H.transfers):
        Df, Dc, n, nc = T.level.dof, 2 * T.nv, T.level.n, T.nc
        supported = Df in (12, 16, 24, 32) and Dc in (16, 24, 32)
        PW = sp.csr_matrix(_abs_parts(T.matrix()))
        steps = 2 * int(np.prod(T.block)) * ((2 * Df + 15) // 16)
        for s in (1, 3, 64, 128, 130):
            f = (rng.standard_normal((n, s)) + 1j * rng.standard_normal((n, s))).astype(np.complex64)
            if l == 0:
                fd = qd.to_qd(ctx, g, f.astype(np.complex128).reshape(g.V, 4, 3, s)).to(torch.complex64)
            else:
                fd = torch.from_numpy(np.ascontiguousarray(f)).to("cuda:0")
            out = torch.full((nc, s), float("nan"), dtype=torch.complex64, device="cuda:0")
            if not supported:
                with pytest.raises(qd.QDError) as ei:
                    qd.restrict_tc(mg, l, s, fd, out)
                assert ei.value.code == qd.QD_ERR_INVALID
                break
            qd.restrict_tc(mg, l, s, fd, out)
            got = host(out).astype(np.complex128)
            f64 = f.astype(np.complex128)
            ref = T.restrict(f64)
            S = PW.T @ _abs_parts(f64)
            tol = (3 * u ** 2 + 3 * u ** 3 + 2.0 ** -23 + (steps + 1) * 2.0 ** -22) * S
            err_re, err_im = np.abs(got.real - ref.real), np.abs(got.imag - ref.imag)
            assert np.all(err_re <= tol) and np.all(err_im <= tol), (l, s, float(max((err_re / tol).max(),
                                                                                   (err_im / tol).max())))
            out2 = torch.empty_like(out)
            qd.restrict_tc(mg, l, s, fd, out2)
            assert torch.equal(out, out2)
    for o in (mg, g):
        o.close()
