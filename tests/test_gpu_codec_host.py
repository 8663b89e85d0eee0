"""cs_codec_host: the whole codec of a clip from host memory (copy-in, one
batched encode under every plan, one batched decode, PSNR, copy-out) gives, bit
for bit, what the device-pointer calls give, and matches the FP64 oracle;
mismatched clip shapes are refused before anything is enqueued."""
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


@pytest.mark.parametrize("h,w,gop,n_gops,b,ms,iters", [
    (144, 176, 4, 2, 16, [26, 64], 40),     # two plans of 16 x 16 blocks, QCIF
    (96, 160, 3, 2, 32, [102], 30),         # 32 x 32 blocks, ragged frame
])
def test_codec_host_equals_device_path(B, h, w, gop, n_gops, b, ms, iters):
    ctx = B.cs_ctx_create(0)
    plans = [B.cs_make_phi(ctx, b * b, m, 7) for m in ms]
    try:
        frames = scenes.surveillance_video(gop * n_gops, h, w, seed=3)
        params = [B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops) for m in ms]
        n_cs = n_gops * (gop - 1)
        clip = torch.from_numpy(frames).pin_memory()
        u8 = [torch.zeros((n_cs, h, w), dtype=torch.uint8).pin_memory() for _ in ms]
        ps = [torch.zeros(n_cs, dtype=torch.float64).pin_memory() for _ in ms]
        s = torch.cuda.Stream()
        for _ in range(2):                        # the second call reuses the staging
            B.cs_codec_host(ctx, plans, params, clip, u8, ps, s)
        s.synchronize()
        B.cs_ctx_status(ctx)
        # the same through device pointers
        nblk = (-(-h // b)) * (-(-w // b))
        f_dev = torch.from_numpy(frames).cuda()
        keys = f_dev[::gop].contiguous()
        cs_idx = [t for t in range(gop * n_gops) if t % gop]
        cs_dev = f_dev[cs_idx].contiguous()
        ys = [torch.empty((n_cs, nblk, m), dtype=torch.float32, device="cuda") for m in ms]
        B.cs_encode_batch(ctx, plans, params, f_dev, ys)
        for i, m in enumerate(ms):
            y = ys[i]
            of = torch.empty((n_cs, h, w), dtype=torch.float32, device="cuda")
            ou = torch.empty((n_cs, h, w), dtype=torch.uint8, device="cuda")
            B.cs_decode_gop(plans[i], params[i], keys, y, of, ou)
            pd = torch.empty(n_cs, dtype=torch.float64, device="cuda")
            B.cs_psnr(cs_dev, of, n_cs, h, w, pd)
            torch.cuda.synchronize()
            assert torch.equal(u8[i], ou.cpu()), m
            assert torch.equal(ps[i], pd.cpu()), m
            # and the oracle: uint8 frames within one level except at rounding ties
            plan = O.Plan(b * b, m, 7)
            want, _ = O.decode(plan, frames[::gop], O.encode(plan, frames, gop), gop,
                               gop * n_gops, iters)
            rel = np.linalg.norm(of.cpu().numpy() - want) / np.linalg.norm(want)
            assert rel <= 1e-4
            assert np.abs(u8[i].numpy().astype(int) - O.to_uint8(want).astype(int)).max() <= 1
            assert np.abs(ps[i].numpy() - [O.psnr(frames[t], want[j][None])
                                           for j, t in enumerate(cs_idx)]).max() < 0.01
    finally:
        for p in plans:
            B.cs_plan_destroy(p)
        B.cs_ctx_destroy(ctx)


def test_codec_host_rejects_mismatched_shapes(B):
    ctx = B.cs_ctx_create(0)
    plans = [B.cs_make_phi(ctx, 256, 26, 0), B.cs_make_phi(ctx, 256, 51, 0)]
    try:
        params = [B.make_params(144, 176, 4, 16, 26), B.make_params(144, 160, 4, 16, 51)]
        clip = np.zeros((4, 144, 176), dtype=np.uint8)
        u8 = [np.zeros((3, 144, 176), dtype=np.uint8)] * 2
        ps = [np.zeros(3)] * 2
        with pytest.raises(B.CsError) as e:
            B.cs_codec_host(ctx, plans, params, clip, u8, ps)
        assert e.value.status == B.CS_EINVAL
    finally:
        for p in plans:
            B.cs_plan_destroy(p)
        B.cs_ctx_destroy(ctx)
