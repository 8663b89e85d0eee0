"""TV recovery on the GPU (cs_decode_gop_tv) against the FP64 oracle's TV
augmented-Lagrangian decode: 8x8, 16x16 and 32x32 blocks on the plain kernel and
on the tensor cores, several GOPs, cropped edge blocks, the uint8 rule, zero
residual and argument errors."""
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


@pytest.mark.parametrize("h,w,gop,n_gops,b,m,iters,engine", [
    (144, 176, 4, 1, 16, 64, 100, "PLAIN"),   # QCIF, 16x16 on the plain kernel
    (144, 176, 4, 1, 16, 64, 100, "AUTO"),    # the same on the on-chip tensor-core kernel
    (40, 56, 3, 2, 8, 24, 150, "PLAIN"),      # 8x8, cropped edge blocks, two GOPs
    (40, 56, 3, 2, 8, 24, 150, "AUTO"),       # the same on the streaming tensor-core kernel
    (64, 96, 3, 1, 32, 102, 60, "PLAIN"),     # 32x32
    (64, 96, 3, 1, 32, 102, 60, "AUTO"),      # streaming
])
def test_tv_matches_oracle(B, ctx, h, w, gop, n_gops, b, m, iters, engine):
    frames = scenes.surveillance_video(gop * n_gops, h, w, seed=3)
    plan = B.cs_make_phi(ctx, b * b, m, 3)
    try:
        p = B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops,
                          engine=getattr(B, "CS_ENGINE_" + engine))
        nblk = (-(-h // b)) * (-(-w // b))
        y = torch.empty((n_gops * (gop - 1), nblk, m), dtype=torch.float32, device="cuda")
        B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
        keys = torch.from_numpy(np.ascontiguousarray(frames[::gop])).cuda()
        out = torch.full((y.shape[0], h, w), float("nan"), dtype=torch.float32, device="cuda")
        u8 = torch.zeros((y.shape[0], h, w), dtype=torch.uint8, device="cuda")
        B.cs_decode_gop_tv(plan, p, keys, y, out, u8, torch.cuda.current_stream())
        B.cs_ctx_status(ctx)
        got = out.cpu().numpy().astype(np.float64)
        oplan = O.Plan(b * b, m, 3)
        ref = O.decode_tv(oplan, frames[::gop], O.encode(oplan, frames, gop), gop, gop * n_gops, iters)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        cs = frames[[t for t in range(frames.shape[0]) if t % gop]]
        dpsnr = O.psnr(cs, got) - O.psnr(cs, ref)
        print("TV b=%d M=%d: rel-l2 %.3g dPSNR %.3g dB (PSNR %.2f)" % (b, m, err, dpsnr, O.psnr(cs, ref)))
        assert err <= 1e-4 and abs(dpsnr) <= 0.01
        assert np.array_equal(u8.cpu().numpy(), np.clip(np.rint(got), 0, 255).astype(np.uint8))
    finally:
        B.cs_plan_destroy(plan)


def test_tv_zero_residual_returns_key(B, ctx):
    frames = np.repeat(scenes.surveillance_video(1, 48, 64, seed=1), 3, axis=0)
    plan = B.cs_make_phi(ctx, 256, 32, 1)
    try:
        p = B.make_params(48, 64, 3, 16, 32, iters=50)
        y = torch.empty((2, 12, 32), dtype=torch.float32, device="cuda")
        B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
        out = torch.zeros((2, 48, 64), dtype=torch.float32, device="cuda")
        B.cs_decode_gop_tv(plan, p, torch.from_numpy(frames[:1]).cuda(), y, out, None,
                           torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), frames[1:].astype(np.float32))
        with pytest.raises(B.CsError) as ei:
            B.cs_decode_gop_tv(plan, p, torch.from_numpy(frames[:1]).cuda(), y, out, None,
                               torch.cuda.current_stream(), beta=0.0)
        assert ei.value.status == B.CS_EINVAL
        with pytest.raises(B.CsError) as ei:
            B.cs_decode_gop_tv(plan, B.make_params(48, 64, 3, 16, 32, iters=50, precision=1),
                               torch.from_numpy(frames[:1]).cuda(), y, out, None,
                               torch.cuda.current_stream())
        assert ei.value.status == B.CS_EINVAL
    finally:
        B.cs_plan_destroy(plan)
