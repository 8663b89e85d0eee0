"""TV recovery on the tensor cores with streamed operands (k_tv_tcs: 8x8, 16x16
with M > 128, 32x32; M <= 512) against the FP64 oracle's TV augmented-Lagrangian
decode and against the plain FP32 kernel: ragged last tiles, more tiles than
SMs, cropped edge blocks, a GEMM1 in two column chunks
(M16 > 256), iteration counts 0 .. 3, other penalties, CS_ENGINE_TC_STREAM equal
to the automatic choice, and the bounded-wait failure path."""
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


def _decode(B, ctx, frames, gop, n_gops, b, m, iters, engine, beta=0.125, mu=1.0, seed=4):
    h, w = frames.shape[1:]
    plan = B.cs_make_phi(ctx, b * b, m, seed)
    try:
        p = B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops, engine=engine)
        nblk = (-(-h // b)) * (-(-w // b))
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


@pytest.mark.parametrize("h,w,gop,n_gops,b,m,iters,beta,mu", [
    (96, 160, 6, 2, 32, 102, 60, 0.125, 1.0),    # 32x32: 150 blocks, 2 tiles (last 22)
    (40, 56, 3, 2, 8, 24, 100, 0.125, 1.0),      # 8x8, cropped edges, two GOPs, 140 blocks: 2 tiles
    (72, 104, 2, 1, 8, 30, 40, 0.125, 1.0),      # 8x8, 117 blocks: one tile, ragged
    (80, 112, 3, 1, 16, 200, 50, 0.125, 1.0),    # 16x16 with M > 128
    (64, 96, 3, 1, 32, 300, 30, 0.125, 1.0),     # 32x32, M16 = 304: GEMM1 in two column chunks
    (64, 128, 3, 1, 32, 60, 3, 0.125, 1.0),      # third iteration reads the stored lambda
    (64, 128, 3, 1, 32, 60, 1, 0.125, 1.0),      # a single step
    (64, 96, 3, 1, 8, 16, 80, 0.3, 2.5),         # other penalties (P scaled for mu > 1)
])
def test_streaming_tv_matches_the_oracle(B, ctx, h, w, gop, n_gops, b, m, iters, beta, mu):
    frames = scenes.surveillance_video(gop * n_gops, h, w, seed=4)
    got, u8 = _decode(B, ctx, frames, gop, n_gops, b, m, iters, B.CS_ENGINE_TC_STREAM, beta, mu)
    oplan = O.Plan(b * b, m, 4)
    ref = O.decode_tv(oplan, frames[::gop], O.encode(oplan, frames, gop), gop, gop * n_gops, iters,
                      beta, mu)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    cs = frames[[t for t in range(frames.shape[0]) if t % gop]]
    dpsnr = O.psnr(cs, got) - O.psnr(cs, ref)
    keys = np.repeat(frames[::gop].astype(np.float64), gop - 1, axis=0)
    res_err = np.linalg.norm((got - keys) - (ref - keys)) / max(np.linalg.norm(ref - keys), 1e-30)
    print("TV tcs b=%d M=%d K=%d: frame rel-l2 %.3g residual rel-l2 %.3g dPSNR %.3g dB"
          % (b, m, iters, err, res_err, dpsnr))
    assert err <= 1e-4 and abs(dpsnr) <= 0.01
    assert res_err <= 1e-3
    assert np.array_equal(u8, np.clip(np.rint(got), 0, 255).astype(np.uint8))


def test_streaming_tv_agrees_with_the_plain_kernel_and_auto(B, ctx):
    frames = scenes.surveillance_video(8, 96, 160, seed=12)
    tcs, _ = _decode(B, ctx, frames, 4, 2, 32, 102, 120, B.CS_ENGINE_TC_STREAM, seed=12)
    plain, _ = _decode(B, ctx, frames, 4, 2, 32, 102, 120, B.CS_ENGINE_PLAIN, seed=12)
    auto, _ = _decode(B, ctx, frames, 4, 2, 32, 102, 120, B.CS_ENGINE_AUTO, seed=12)
    keys = np.repeat(frames[::4].astype(np.float64), 3, axis=0)
    rel = np.linalg.norm(tcs - plain) / np.linalg.norm(plain - keys)
    print("TV tcs vs plain: residual rel-l2 %.3g" % rel)
    assert rel <= 1e-4
    assert np.array_equal(auto, tcs)          # AUTO takes the streaming kernel for 32x32


def test_streaming_tv_zero_iterations_return_the_key(B, ctx):
    frames = scenes.surveillance_video(3, 64, 96, seed=2)
    got, u8 = _decode(B, ctx, frames, 3, 1, 32, 51, 0, B.CS_ENGINE_TC_STREAM)
    assert np.array_equal(got, np.repeat(frames[:1].astype(np.float64), 2, axis=0))
    assert np.array_equal(u8, np.repeat(frames[:1], 2, axis=0))


def test_streaming_tv_more_tiles_than_sms(B, ctx):
    # 4 CS frames of 70 x 70 blocks of 8 x 8: 19600 blocks, 154 tiles, more than one
    # round of the persistent grid on any GB300; the plain kernel is the check
    frames = scenes.surveillance_video(6, 560, 556, seed=21)
    tcs, u8 = _decode(B, ctx, frames, 3, 2, 8, 20, 40, B.CS_ENGINE_TC_STREAM, seed=21)
    plain, _ = _decode(B, ctx, frames, 3, 2, 8, 20, 40, B.CS_ENGINE_PLAIN, seed=21)
    keys = np.repeat(frames[::3].astype(np.float64), 2, axis=0)
    rel = np.linalg.norm(tcs - plain) / np.linalg.norm(plain - keys)
    worst = np.abs(tcs - plain).max()
    print("TV tcs vs plain, 19600 blocks: residual rel-l2 %.3g, max |diff| %.3g" % (rel, worst))
    assert np.isfinite(tcs).all()
    assert rel <= 1e-4 and worst <= 0.05
    assert np.array_equal(u8, np.clip(np.rint(tcs), 0, 255).astype(np.uint8))


def test_streaming_tv_withheld_arrival_times_out_and_recovers(B):
    c = B.cs_ctx_create(0)
    plan = B.cs_make_phi(c, 1024, 60, 5)
    try:
        h, w = 64, 128
        frames = scenes.surveillance_video(2, h, w, seed=5)
        p = B.make_params(h, w, 2, 32, 60, iters=20, engine=B.CS_ENGINE_TC_STREAM)
        s = torch.cuda.current_stream()
        f = torch.from_numpy(frames).cuda()
        y = torch.empty((1, 8, 60), dtype=torch.float32, device="cuda")
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
