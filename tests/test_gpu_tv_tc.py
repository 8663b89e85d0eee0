"""TV recovery on the tensor cores (k_tv_tc: 16 x 16 blocks, M <= 128) against
the FP64 oracle's TV augmented-Lagrangian decode and against the plain FP32
kernel: several tiles with a ragged last one, cropped edge blocks, M from one
16-row step to the 128-row maximum, iteration counts 0 .. 3 (the deferred
multiplier step starts reading its state at the third), other penalties, the
engine rules and the bounded-wait failure path."""
import time

import numpy as np
import pytest

from oracle import cs_oracle as O
from paper_1311_1419_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1311_1419_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def ctx(B):
    c = B.cs_ctx_create(0)
    yield c
    B.cs_ctx_destroy(c)


def _decode(B, ctx, frames, gop, n_gops, m, iters, engine, beta=0.125, mu=1.0, seed=3):
    h, w = frames.shape[1:]
    plan = B.cs_make_phi(ctx, 256, m, seed)
    try:
        p = B.make_params(h, w, gop, 16, m, iters=iters, n_gops=n_gops, engine=engine)
        nblk = (-(-h // 16)) * (-(-w // 16))
        s = torch.cuda.current_stream()
        y = torch.empty((n_gops * (gop - 1), nblk, m), dtype=torch.float32, device="cuda")
        B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, s)
        keys = torch.from_numpy(np.ascontiguousarray(frames[::gop])).cuda()
        out = torch.full((y.shape[0], h, w), float("nan"), dtype=torch.float32, device="cuda")
        u8 = torch.zeros((y.shape[0], h, w), dtype=torch.uint8, device="cuda")
        B.cs_decode_gop_tv(plan, p, keys, y, out, u8, s, beta=beta, mu=mu)
        B.cs_ctx_status(ctx)
        return out.cpu().numpy().astype(np.float64), u8.cpu().numpy()
    finally:
        B.cs_plan_destroy(plan)


@pytest.mark.parametrize("h,w,gop,n_gops,m,iters,beta,mu", [
    (144, 176, 4, 1, 64, 100, 0.125, 1.0),    # QCIF: 297 blocks, 3 tiles (last 41)
    (136, 168, 3, 2, 128, 60, 0.125, 1.0),    # cropped edges, two GOPs, M = 128, 4 tiles
    (64, 96, 3, 1, 13, 80, 0.125, 1.0),       # M16 = 16, one partial tile
    (80, 112, 3, 1, 100, 3, 0.125, 1.0),      # third iteration reads the stored lambda
    (80, 112, 3, 1, 100, 1, 0.125, 1.0),      # a single step
    (96, 128, 3, 1, 72, 80, 0.3, 2.5),        # other penalties (P scaled for mu > 1)
])
def test_tv_tensor_cores_match_the_oracle(B, ctx, h, w, gop, n_gops, m, iters, beta, mu):
    frames = scenes.surveillance_video(gop * n_gops, h, w, seed=3)
    got, u8 = _decode(B, ctx, frames, gop, n_gops, m, iters, B.CS_ENGINE_TC, beta, mu)
    oplan = O.Plan(256, m, 3)
    ref = O.decode_tv(oplan, frames[::gop], O.encode(oplan, frames, gop), gop, gop * n_gops, iters,
                      beta, mu)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    cs = frames[[t for t in range(frames.shape[0]) if t % gop]]
    dpsnr = O.psnr(cs, got) - O.psnr(cs, ref)
    keys = np.repeat(frames[::gop].astype(np.float64), gop - 1, axis=0)
    res_err = np.linalg.norm((got - keys) - (ref - keys)) / max(np.linalg.norm(ref - keys), 1e-30)
    print("TV tc M=%d K=%d: frame rel-l2 %.3g residual rel-l2 %.3g dPSNR %.3g dB" % (m, iters, err, res_err, dpsnr))
    assert err <= 1e-4 and abs(dpsnr) <= 0.01
    assert res_err <= 1e-3
    assert np.array_equal(u8, np.clip(np.rint(got), 0, 255).astype(np.uint8))


def test_tv_tensor_cores_agree_with_the_plain_kernel(B, ctx):
    frames = scenes.surveillance_video(6, 144, 176, seed=11)
    tc, _ = _decode(B, ctx, frames, 3, 2, 96, 150, B.CS_ENGINE_TC, seed=11)
    plain, _ = _decode(B, ctx, frames, 3, 2, 96, 150, B.CS_ENGINE_PLAIN, seed=11)
    auto, _ = _decode(B, ctx, frames, 3, 2, 96, 150, B.CS_ENGINE_AUTO, seed=11)
    keys = np.repeat(frames[::3].astype(np.float64), 2, axis=0)
    rel = np.linalg.norm(tc - plain) / np.linalg.norm(plain - keys)
    print("TV tc vs plain: residual rel-l2 %.3g" % rel)
    assert rel <= 1e-4
    assert np.array_equal(auto, tc)          # AUTO takes the tensor cores for this shape


def test_tv_tensor_cores_zero_iterations_return_the_key(B, ctx):
    frames = scenes.surveillance_video(3, 48, 80, seed=2)
    got, u8 = _decode(B, ctx, frames, 3, 1, 32, 0, B.CS_ENGINE_TC)
    assert np.array_equal(got, np.repeat(frames[:1].astype(np.float64), 2, axis=0))
    assert np.array_equal(u8, np.repeat(frames[:1], 2, axis=0))


def test_tv_engine_rules(B, ctx):
    s = torch.cuda.current_stream()
    # the on-chip kernel takes 16 x 16 blocks with M <= 128 only; the streaming one
    # N = 64, 256, 1024 only
    for b, m, engine in [(8, 24, B.CS_ENGINE_TC), (16, 200, B.CS_ENGINE_TC), (4, 8, B.CS_ENGINE_TC_STREAM)]:
        plan = B.cs_make_phi(ctx, b * b, m, 1)
        try:
            p = B.make_params(64, 64, 2, b, m, iters=5, engine=engine)
            nblk = (64 // b) ** 2
            y = torch.zeros((1, nblk, m), dtype=torch.float32, device="cuda")
            keys = torch.zeros((1, 64, 64), dtype=torch.uint8, device="cuda")
            out = torch.empty((1, 64, 64), dtype=torch.float32, device="cuda")
            with pytest.raises(B.CsError) as ei:
                B.cs_decode_gop_tv(plan, p, keys, y, out, None, s)
            assert ei.value.status == B.CS_EINVAL
        finally:
            B.cs_plan_destroy(plan)


def test_tv_tensor_cores_withheld_arrival_times_out_and_recovers(B):
    c = B.cs_ctx_create(0)
    plan = B.cs_make_phi(c, 256, 48, 5)
    try:
        h, w = 64, 128
        frames = scenes.surveillance_video(2, h, w, seed=5)
        p = B.make_params(h, w, 2, 16, 48, iters=20, engine=B.CS_ENGINE_TC)
        s = torch.cuda.current_stream()
        f = torch.from_numpy(frames).cuda()
        y = torch.empty((1, 32, 48), dtype=torch.float32, device="cuda")
        B.cs_encode_gop(plan, p, f, y, s)
        ref = torch.empty((1, h, w), dtype=torch.float32, device="cuda")
        B.cs_decode_gop_tv(plan, p, f[:1], y, ref, None, s)
        B.cs_ctx_status(c)

        B.cs_ctx_set_debug(c, B.CS_DEBUG_DROP_ARRIVAL)
        out = torch.full((1, h, w), -1.0, dtype=torch.float32, device="cuda")
        t0 = time.time()
        B.cs_decode_gop_tv(plan, p, f[:1], y, out, None, s)
        with pytest.raises(B.CsError) as ei:
            B.cs_ctx_status(c)
        assert ei.value.status == B.CS_ETIMEDOUT
        assert time.time() - t0 < 30
        B.cs_ctx_status(c)

        again = torch.empty((1, h, w), dtype=torch.float32, device="cuda")
        B.cs_decode_gop_tv(plan, p, f[:1], y, again, None, s)
        B.cs_ctx_status(c)
        assert np.array_equal(again.cpu().numpy(), ref.cpu().numpy())
    finally:
        B.cs_plan_destroy(plan)
        B.cs_ctx_destroy(c)
