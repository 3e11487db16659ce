"""qd_deflate_project_static: out = (I - U U^H) z for an orthonormal
eigenvector space, for callers that cannot let the library allocate device
memory during a call (an application that gave all device memory to its own
pool, or a loop that must not pay cudaMalloc / cudaFree).  It keeps its
scratch in a fixed device array.  Its output must equal qd_deflate_project's
on consecutive calls, and no call may allocate (qd_alloc_count stays put),
whether this file runs alone or after the others."""
import numpy as np
import pytest

from paper_1909_12234_gb300 import synth

from gpu_util import need_gpu, rel_err, torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qd():
    need_gpu()
    from paper_1909_12234_gb300 import qdtrace
    qdtrace.load()
    return qdtrace


def _orthonormal(n, k, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, k)) + 1j * rng.standard_normal((n, k)))
    return Q


def test_static_scratch_projection_matches_allocating_one(qd):
    ctx = qd.Context(0)
    dims, m0, k = (4, 4, 4, 4), -0.4, 16
    g = qd.Gauge(ctx, dims, synth.random_su3_links(dims, 0.3, 1))
    U = _orthonormal(12 * g.V, k, 3)
    d = qd.Deflation(ctx, g, None, m0, 0.0, qd.defl_params(qd.QD_DEFL_EIG_ORTHO, k, solve_tol=1e-10),
                     injected_basis=qd.to_qd(ctx, g, U.reshape(g.V, 4, 3, k)))
    for call, (s, seed) in enumerate([(5, 11), (32, 12)]):  # two calls in a row, different sizes
        z = qd.to_qd(ctx, g, synth.random_field(dims, s, seed))
        ref = torch.empty_like(z)
        out = torch.full_like(z, complex("nan"))
        d.project(s, z, ref)
        torch.cuda.synchronize()
        n_alloc = qd.alloc_count()
        d.project_static(s, z, out)
        torch.cuda.synchronize()
        assert qd.alloc_count() == n_alloc, "the static projection allocated device memory"
        assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) < 1e-12, call
    # a smaller active rank reuses the same array
    d.set_rank(7)
    z = qd.to_qd(ctx, g, synth.random_field(dims, 3, 13))
    ref, out = torch.empty_like(z), torch.empty_like(z)
    d.project(3, z, ref)
    d.project_static(3, z, out)
    torch.cuda.synchronize()
    assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) < 1e-12
    for o in (d, g, ctx):
        o.close()


def test_static_scratch_rejects_oversize_and_oblique(qd):
    ctx = qd.Context(0)
    dims = (4, 4, 4, 4)
    g = qd.Gauge(ctx, dims, synth.random_su3_links(dims, 0.3, 1))
    k = 64
    U = _orthonormal(12 * g.V, k, 4)
    d = qd.Deflation(ctx, g, None, -0.4, 0.0, qd.defl_params(qd.QD_DEFL_EIG_ORTHO, k, solve_tol=1e-6),
                     injected_basis=qd.to_qd(ctx, g, U.reshape(g.V, 4, 3, k)))
    s = 4097  # 64 x 4097 > 262144 coefficients: beyond the 8 MiB array
    z = torch.zeros((g.V, 12, s), dtype=torch.complex128, device="cuda:0")
    out = torch.empty_like(z)
    with pytest.raises(qd.QDError) as e:
        d.project_static(s, z, out)
    assert e.value.code == qd.QD_ERR_INVALID
    mg = qd.Multigrid(ctx, g, -0.4, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [4], null_maxit=0))
    lev_n = 16 * 8
    rng = np.random.default_rng(2)
    Ub = np.linalg.qr(rng.standard_normal((lev_n, 4)) + 0j)[0]
    d2 = qd.Deflation(ctx, g, mg, -0.4, 0.0, qd.defl_params(qd.QD_DEFL_MG_OBLIQUE, 4),
                      injected_basis=torch.from_numpy(np.ascontiguousarray(Ub)).to("cuda:0"))
    z1 = torch.zeros((g.V, 12, 1), dtype=torch.complex128, device="cuda:0")
    with pytest.raises(qd.QDError) as e:
        d2.project_static(1, z1, torch.empty_like(z1))
    assert e.value.code == qd.QD_ERR_INVALID
    # partially overlapping input and output ranges are rejected, not corrupted
    buf = torch.zeros((2 * g.V * 12 * 2,), dtype=torch.complex128, device="cuda:0")
    zz, oo = buf[: g.V * 12 * 2], buf[g.V * 12: g.V * 12 * 3]
    for fn in (d.project_static, d.project):
        with pytest.raises(qd.QDError) as e:
            fn(2, zz, oo)
        assert e.value.code == qd.QD_ERR_INVALID
    for o in (d2, mg, d, g, ctx):
        o.close()
