"""GPU parity for the learned gauge-covariant smoother: S r and the
least-squares fit against the oracle, and solves that use S inside the
V-cycle reach the FP64 true residual (mixed and FP64), replaying the
captured V-cycle bit-identically."""
import numpy as np
import pytest

from oracle import multigrid as omg
from oracle import smoother as osm
from paper_1909_12234_gb300 import synth

from gpu_util import need_gpu, rel_err, torch

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


def test_apply_and_fit_match_oracle(qd, ctx):
    dims = (8, 4, 4, 6)
    U = synth.random_su3_links(dims, 0.3, 3)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, -0.5, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [4], null_maxit=0))
    rng = np.random.default_rng(5)
    w0 = rng.standard_normal((9, 4, 4)) + 1j * rng.standard_normal((9, 4, 4))
    qd.smoother_set_weights(mg, w0)
    assert np.array_equal(qd.smoother_get_weights(mg), w0)
    for s in (1, 5):
        r = synth.random_field(dims, s, 10 + s)
        out = torch.empty((g.V, 12, s), dtype=torch.complex128, device="cuda:0")
        qd.smoother_apply(mg, s, qd.to_qd(ctx, g, r), out)
        assert rel_err(qd.from_qd(ctx, g, out), osm.apply(U, w0, r, dims)) < 1e-12
    # the Wilson weights give the Wilson operator
    qd.smoother_set_weights(mg, osm.wilson_weights(-0.5))
    r = synth.random_field(dims, 3, 1)
    out = torch.empty((g.V, 12, 3), dtype=torch.complex128, device="cuda:0")
    ref = torch.empty_like(out)
    qd.smoother_apply(mg, 3, qd.to_qd(ctx, g, r), out)
    qd.dirac_apply(ctx, g, -0.5, 0.0, False, 3, qd.to_qd(ctx, g, r), ref)
    assert rel_err(out.cpu().numpy(), ref.cpu().numpy()) < 1e-13
    # fit: exact recovery of planted weights, and the oracle's least squares
    # on noisy pairs
    R = synth.random_field(dims, 4, 2)
    E = osm.apply(U, w0, R, dims)
    qd.smoother_fit(mg, 4, qd.to_qd(ctx, g, E), qd.to_qd(ctx, g, R))
    assert rel_err(qd.smoother_get_weights(mg), w0) < 1e-10
    En = E + 0.3 * synth.random_field(dims, 4, 3)
    qd.smoother_fit(mg, 4, qd.to_qd(ctx, g, En), qd.to_qd(ctx, g, R))
    assert rel_err(qd.smoother_get_weights(mg), osm.fit(U, En, R, dims)) < 1e-9


def test_fp32_apply_matches_oracle_with_fp16_weights(qd, ctx):
    # the FP32 form (two RHS per thread for even counts, one otherwise)
    # against the oracle applied with the same FP16-rounded weights; FP32
    # rounding of ~160 products per output bounds the error by ~1e-5 of max|y|
    dims = (8, 4, 4, 6)
    U = synth.random_su3_links(dims, 0.3, 4)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, -0.5, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [4], null_maxit=0))
    rng = np.random.default_rng(8)
    w0 = rng.standard_normal((9, 4, 4)) + 1j * rng.standard_normal((9, 4, 4))
    qd.smoother_set_weights(mg, w0)
    w16 = (w0.real.astype(np.float32).astype(np.float16).astype(np.float64)
           + 1j * w0.imag.astype(np.float32).astype(np.float16).astype(np.float64))
    for s in (2, 3, 64):
        r = synth.random_field(dims, s, 20 + s)
        x32 = qd.to_qd(ctx, g, r).to(torch.complex64)
        out = torch.empty_like(x32)
        qd.smoother_apply_f32(mg, s, x32, out)
        got = qd.from_qd(ctx, g, out.to(torch.complex128))
        assert rel_err(got, osm.apply(U, w16, r, dims)) < 1e-5, s


def test_solves_with_the_learned_smoother(qd, ctx):
    dims, m0, s = (8, 8, 8, 8), -0.8, 8
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, m0, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [12]))
    info = qd.smoother_train(mg, nsamples=8, solve_tol=1e-6, mr_steps=2)
    assert 0.0 < info["err_learned"] < 1.0 and 0.0 < info["err_plain"] < 1.0
    assert info["enabled"] == (info["err_learned"] < info["err_plain"])
    qd.smoother_enable(mg, True, 2)  # exercise the learned path whatever the judge said
    A = omg.fine_level(U, m0, dims).matrix
    b = synth.random_field(dims, s, 7)
    bd = qd.to_qd(ctx, g, b)
    for prec in (qd.QD_PREC_MIXED, qd.QD_PREC_F64):
        xs = []
        for rep in range(3):  # eager, capture, replay
            xd = torch.empty_like(bd)
            qd.solve(ctx, g, mg, m0, 0.0, s, bd, xd, 1e-10, maxit=400, restart=16, precision=prec,
                     inner_tol=1e-5, max_refine=10)
            xs.append(xd.clone())
        assert torch.equal(xs[1], xs[0]) and torch.equal(xs[2], xs[0])
        x = qd.from_qd(ctx, g, xs[0]).reshape(-1, s)
        B = b.reshape(-1, s)
        assert np.all(np.linalg.norm(B - A @ x, axis=0) / np.linalg.norm(B, axis=0) <= 1e-10)
    qd.smoother_enable(mg, False, 2)


def test_layered_smoother_against_oracle(qd, ctx):
    # S = S_3 S_2 S_1 (each layer the one-hop form): FP64 against the
    # oracle's composition, FP32 (FP16-rounded weights) within its rounding;
    # greedy training: each layer fits e ~ S_l (S_{l-1} ... S_1 r) by least
    # squares with the layers below fixed, checked against the oracle's fit
    # of the same pairs
    dims = (8, 4, 4, 6)
    U = synth.random_su3_links(dims, 0.3, 3)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, -0.5, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [4], null_maxit=0))
    rng = np.random.default_rng(8)
    W = 0.3 * (rng.standard_normal((3, 9, 4, 4)) + 1j * rng.standard_normal((3, 9, 4, 4)))
    qd.smoother_set_layer_weights(mg, W)
    assert qd.smoother_layers(mg) == 3
    assert np.array_equal(qd.smoother_get_layer_weights(mg), W)
    assert np.array_equal(qd.smoother_get_weights(mg), W[0])
    for s in (1, 4):
        r = synth.random_field(dims, s, 20 + s)
        ref = r
        for l in range(3):
            ref = osm.apply(U, W[l], ref, dims)
        out = torch.empty((g.V, 12, s), dtype=torch.complex128, device="cuda:0")
        qd.smoother_apply(mg, s, qd.to_qd(ctx, g, r), out)
        assert rel_err(qd.from_qd(ctx, g, out), ref) < 1e-12
        x32 = qd.to_qd(ctx, g, r).to(torch.complex64)
        o32 = torch.empty_like(x32)
        qd.smoother_apply_f32(mg, s, x32, o32)
        # FP16 weights (u = 2^-11) in each of three layers
        assert rel_err(qd.from_qd(ctx, g, o32.to(torch.complex128)), ref) < 3e-2
    # one layer again: the single-layer entry points still apply
    qd.smoother_set_weights(mg, W[1])
    assert qd.smoother_layers(mg) == 1
    mg.close()
    g.close()


def test_layered_training_builds_on_the_one_layer_fit(qd, ctx):
    # greedy training: the first layer of a layered fit is the one-layer fit
    # of the same pairs, and the depth is what was asked for (each added
    # layer's family holds the identity, so its least-squares error on the
    # training pairs cannot exceed the stack below it; the held-out judge
    # still decides whether the V-cycle uses S)
    dims = (8, 8, 8, 8)
    U = synth.random_su3_links(dims, 0.3, 2)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, -0.8, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [12]))
    # the training pairs come from solves preconditioned by the V-cycle, so
    # the smoother is switched off before each training to give every call
    # the same pairs
    infos = []
    for layers in (1, 2, 3):
        if qd.smoother_layers(mg):
            qd.smoother_enable(mg, False, 1)
        info = qd.smoother_train(mg, nsamples=8, solve_tol=1e-6, mr_steps=1, layers=layers)
        assert qd.smoother_layers(mg) == layers
        infos.append(info)
    # the first layer of the layered fit is the one-layer fit (same pairs)
    w_all = qd.smoother_get_layer_weights(mg)
    qd.smoother_enable(mg, False, 1)
    qd.smoother_train(mg, nsamples=8, solve_tol=1e-6, mr_steps=1, layers=1)
    assert rel_err(w_all[0], qd.smoother_get_weights(mg)) < 1e-10
    print("held-out errors (learned, plain) by depth:", [(i["err_learned"], i["err_plain"]) for i in infos])
    mg.close()
    g.close()


def test_fp32_smoother_launch_shapes_are_bit_identical(qd, ctx):
    # the FP32 smoother's launch shapes: index order, the stencil visiting
    # order with the columns whole or in chunks of 64 / 32, and packed
    # multiply-adds (fma.rn.f32x2: lane by lane the same multiply-adds in the
    # same order): the same bits, for one and two layers
    dims = (8, 8, 4, 4)
    U = synth.random_su3_links(dims, 0.3, 4)
    g = qd.Gauge(ctx, dims, U)
    mg = qd.Multigrid(ctx, g, -0.5, 0.0, qd.mg_params(1, [(2, 2, 2, 2)], [4], null_maxit=0))
    rng = np.random.default_rng(12)
    W = rng.standard_normal((2, 9, 4, 4)) + 1j * rng.standard_normal((2, 9, 4, 4))
    try:
        for layers in (1, 2):
            qd.smoother_set_layer_weights(mg, W[:layers])
            for s in (2, 64, 130):
                x = torch.randn((g.V, 12, s), dtype=torch.complex64, device="cuda:0",
                                generator=torch.Generator("cuda:0").manual_seed(s))
                outs = []
                for cand in range(5):
                    qd.autotune_force(cand)
                    o = torch.full_like(x, float("nan"))
                    qd.smoother_apply_f32(mg, s, x, o)
                    outs.append(o)
                for cand in range(1, 5):
                    assert torch.equal(outs[0], outs[cand]), (layers, s, cand)
    finally:
        qd.autotune_force(-1)
    mg.close()
    g.close()
