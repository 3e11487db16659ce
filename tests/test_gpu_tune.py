"""The launch-shape autotuner: tuned coarse-stencil shapes give results
bit-identical to the defaults; the tuned FP32 Wilson shape agrees with the
default to FP32 rounding; the table records one choice per problem shape."""
import numpy as np
import pytest

from paper_1909_12234_gb300 import synth

from gpu_util import host, need_gpu, rel_err, torch

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


def test_autotuned_shapes_match_defaults(qd, ctx):
    dims = (8, 8, 8, 8)
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, -0.8, 0.0, qd.mg_params(2, [(2, 2, 2, 2), (2, 2, 2, 2)], [12, 16], null_maxit=20))
    try:
        for s in (64, 130, 7):
            outs = {}
            for mode in (0, 1):
                qd.autotune_clear()
                qd.autotune_set(mode)
                for level in (1, 2):
                    n = mg.level_info(level)[2] * mg.level_info(level)[1]
                    x = torch.randn((n * s,), dtype=torch.complex64, device="cuda:0",
                                    generator=torch.Generator("cuda:0").manual_seed(level))
                    y = torch.empty_like(x)
                    qd.coarse_apply_f32(mg, level, s, x, y)
                    outs[(mode, level)] = host(y)
                xf = torch.randn((g.V, 12, s), dtype=torch.complex64, device="cuda:0",
                                 generator=torch.Generator("cuda:0").manual_seed(3))
                yf = torch.empty_like(xf)
                qd.dirac_apply_f32(ctx, g, -0.8, 0.0, False, s, xf, yf)
                outs[(mode, "w")] = host(yf)
                rep = qd.autotune_report()
                if mode == 0:
                    assert rep == {}
                else:
                    keys = [k for k in rep if k.startswith("coarse_stencil") and k.endswith(f"rhs{s}")]
                    assert len(keys) == 2
                    for k in keys:
                        choice, ms = rep[k]
                        assert len(ms) == 11 and ms[choice] > 0 and ms[choice] == min(m for m in ms if m > 0)
            for level in (1, 2):
                assert np.array_equal(outs[(0, level)], outs[(1, level)])
            assert rel_err(outs[(1, "w")], outs[(0, "w")]) < 1e-6
    finally:
        qd.autotune_set(1)


def test_wilson_f32_launch_shapes(qd, ctx):
    # the FP32 Wilson stencil's shapes: two columns per thread swept whole
    # (0) or in chunks of 64, 32 or 16 columns with blocks of 128-512
    # threads (2-7) -- the same arithmetic per element, so the same bits --
    # the neighbours projected as they load (8-9) and one column per thread
    # (1) and the operands staged in shared memory by bulk copies (10-12) or
    # by cp.async one hop ahead (13-14), which agree to FP32 rounding; A and
    # A^H
    dims = (8, 8, 8, 8)
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    try:
        for s in (128, 96, 64, 130, 6):
            xf = torch.randn((g.V, 12, s), dtype=torch.complex64, device="cuda:0",
                             generator=torch.Generator("cuda:0").manual_seed(s))
            for dag in (False, True):
                outs = {}
                for cand in range(15):
                    qd.autotune_force(cand)
                    yf = torch.full_like(xf, float("nan"))
                    qd.dirac_apply_f32(ctx, g, -0.8, 0.1, dag, s, xf, yf)
                    outs[cand] = yf
                for cand in (2, 3, 4, 5, 6, 7):
                    assert torch.equal(outs[0], outs[cand]), (s, dag, cand)
                for cand in (8, 9):  # projection on load: the same sums, possibly contracted differently
                    assert rel_err(host(outs[cand]), host(outs[0])) < 1e-6, (s, dag, cand)
                assert rel_err(host(outs[1]), host(outs[0])) < 1e-6, (s, dag)
                # operands staged by bulk copies (10-12, nrhs a multiple of 64) or
                # by cp.async one hop ahead (13-14)
                for cand in (10, 11, 12, 13, 14):
                    assert rel_err(host(outs[cand]), host(outs[0])) < 1e-6, (s, dag, cand)
    finally:
        qd.autotune_force(-1)
    g.close()
