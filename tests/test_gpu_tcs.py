"""The streaming tensor-core decode (operands streamed from L2, iterates in
global memory) against the FP64 oracle: 8 x 8, 16 x 16 and 32 x 32 blocks, M
up to 512 (one and two GEMM1 column chunks, partial last K slices), one and
several tiles with a ragged tail, zero and one iteration, mixed precision, the
shapes the on-chip kernels also take, and inside a heterogeneous batch."""
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


def _run(B, ctx, h, w, gop, b, m, iters, seed, precision=0, tail=0, engine=None, n_gops=1):
    frames = scenes.surveillance_video(gop * n_gops, h, w, seed=seed)
    plan = B.cs_make_phi(ctx, b * b, m, seed)
    try:
        eng = B.CS_ENGINE_TC_STREAM if engine is None else engine
        p = B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops, precision=precision,
                          fp32_tail_iters=tail, engine=eng)
        nblk = (-(-h // b)) * (-(-w // b))
        y = torch.empty((n_gops * (gop - 1), nblk, m), dtype=torch.float32, device="cuda")
        B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
        keys = torch.from_numpy(np.ascontiguousarray(frames[::gop])).cuda()
        out = torch.full((y.shape[0], h, w), float("nan"), dtype=torch.float32, device="cuda")
        u8 = torch.zeros((y.shape[0], h, w), dtype=torch.uint8, device="cuda")
        B.cs_decode_gop(plan, p, keys, y, out, u8, torch.cuda.current_stream())
        B.cs_ctx_status(ctx)
        return frames, out.cpu().numpy().astype(np.float64), u8.cpu().numpy()
    finally:
        B.cs_plan_destroy(plan)


def _oracle(frames, b, gop, n_gops, m, iters, seed):
    plan = O.Plan(b * b, m, seed)
    y = O.encode(plan, frames, gop)
    ref, _ = O.decode(plan, frames[::gop], y, gop, gop * n_gops, iters)
    return ref


def _cs(frames, gop):
    return frames[[t for t in range(frames.shape[0]) if t % gop]]


@pytest.mark.parametrize("h,w,gop,n_gops,b,m,iters", [
    (160, 224, 5, 1, 32, 200, 30),   # 140 blocks: two tiles (ragged), M16 = 208, K slices 64+64+64+16
    (96, 128, 3, 1, 32, 300, 25),    # M16 = 304: two GEMM1 chunks of 152
    (64, 96, 3, 1, 32, 512, 20),     # M = 512: two chunks of 256, the largest operands
    (100, 130, 4, 2, 8, 16, 60),     # N = 64: 8 x 8 blocks, cropped, 1 - 2 tiles per GOP call
    (72, 72, 3, 1, 8, 32, 40),       # N = 64, M = 32 (M = N / 2)
    (80, 112, 3, 1, 16, 200, 30),    # N = 256, M > 128 (no on-chip kernel)
    (144, 176, 3, 1, 16, 77, 40),    # N = 256, M = 77: a shape the on-chip kernel also takes
    (96, 128, 3, 1, 32, 51, 30),     # N = 1024, M = 51: a shape the cluster kernel also takes
])
def test_tcs_fp32_matches_oracle(B, ctx, h, w, gop, n_gops, b, m, iters):
    frames, got, u8 = _run(B, ctx, h, w, gop, b, m, iters, seed=11, n_gops=n_gops)
    ref = _oracle(frames, b, gop, n_gops, m, iters, 11)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    dpsnr = O.psnr(_cs(frames, gop), got) - O.psnr(_cs(frames, gop), ref)
    print("N=%d M=%d: rel-l2 %.3g dPSNR %.3g dB" % (b * b, m, err, dpsnr))
    assert err <= 1e-4 and abs(dpsnr) <= 0.01
    assert np.array_equal(u8, np.clip(np.rint(got), 0, 255).astype(np.uint8))


@pytest.mark.parametrize("iters", [0, 1, 2])
def test_tcs_few_iterations(B, ctx, iters):
    # K = 0: the key comes back; K = 1: no GEMM1 at all; K = 2: one of each
    h, w, gop, b, m = 64, 96, 3, 32, 150
    frames, got, _ = _run(B, ctx, h, w, gop, b, m, iters, seed=12)
    ref = _oracle(frames, b, gop, 1, m, iters, 12)
    if iters == 0:
        assert np.array_equal(got, np.repeat(frames[:1].astype(np.float64), gop - 1, axis=0))
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-4, err


@pytest.mark.parametrize("precision,tail", [(3, 10), (1, 10), (2, 0)])   # FP16, BF16, BF16X2
def test_tcs_mixed_precision_within_tolerance(B, ctx, precision, tail):
    h, w, gop, b, m, iters = 96, 128, 4, 32, 256, 40
    frames, got, _ = _run(B, ctx, h, w, gop, b, m, iters, seed=13, precision=precision, tail=tail)
    ref = _oracle(frames, b, gop, 1, m, iters, 13)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    dpsnr = O.psnr(_cs(frames, gop), got) - O.psnr(_cs(frames, gop), ref)
    print("N=1024 M=256 precision %d tail %d: rel-l2 %.3g dPSNR %.3g dB" % (precision, tail, err, dpsnr))
    assert abs(dpsnr) <= 0.1 and err <= 2e-3


def test_tcs_unsupported_shape_is_refused(B, ctx):
    # N = 4096 (64 x 64 blocks) has no tensor-core kernel: an explicit request fails
    plan = B.cs_make_phi(ctx, 4096, 64, 1)
    try:
        p = B.make_params(64, 64, 2, 64, 64, iters=1, engine=B.CS_ENGINE_TC_STREAM)
        y = torch.zeros((1, 1, 64), dtype=torch.float32, device="cuda")
        key = torch.zeros((1, 64, 64), dtype=torch.uint8, device="cuda")
        out = torch.zeros((1, 64, 64), dtype=torch.float32, device="cuda")
        with pytest.raises(B.CsError):
            B.cs_decode_gop(plan, p, key, y, out, None, torch.cuda.current_stream())
    finally:
        B.cs_plan_destroy(plan)


def test_tcs_in_a_batch_equals_alone(B, ctx):
    # streaming jobs of three block sizes and both operand types beside an
    # on-chip tensor-core job and a plain job
    jobs = [(96, 128, 3, 32, 300, 15, 3, 0, B.CS_ENGINE_AUTO),
            (72, 80, 3, 8, 20, 20, 4, 0, B.CS_ENGINE_AUTO),
            (80, 96, 3, 16, 160, 15, 5, 2, B.CS_ENGINE_AUTO),
            (48, 64, 3, 16, 40, 20, 6, 0, B.CS_ENGINE_AUTO),
            (48, 64, 3, 16, 40, 10, 7, 0, B.CS_ENGINE_PLAIN)]
    prepared = []
    try:
        for h, w, gop, b, m, iters, seed, prec, eng in jobs:
            frames = scenes.surveillance_video(gop, h, w, seed=seed)
            plan = B.cs_make_phi(ctx, b * b, m, seed)
            p = B.make_params(h, w, gop, b, m, iters=iters, precision=prec, engine=eng)
            nblk = (-(-h // b)) * (-(-w // b))
            y = torch.empty((gop - 1, nblk, m), dtype=torch.float32, device="cuda")
            B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
            key = torch.from_numpy(np.ascontiguousarray(frames[:1])).cuda()
            alone = torch.zeros((gop - 1, h, w), dtype=torch.float32, device="cuda")
            B.cs_decode_gop(plan, p, key, y, alone, None, torch.cuda.current_stream())
            prepared.append((plan, p, key, y, alone))
        outs = [torch.zeros_like(x[4]) for x in prepared]
        B.cs_decode_batch(ctx, [x[0] for x in prepared], [x[1] for x in prepared],
                          [x[2] for x in prepared], [x[3] for x in prepared], outs, None,
                          torch.cuda.current_stream())
        B.cs_ctx_status(ctx)
        for i, (x, o) in enumerate(zip(prepared, outs)):
            assert np.array_equal(x[4].cpu().numpy().view(np.uint32), o.cpu().numpy().view(np.uint32)), i
    finally:
        for x in prepared:
            B.cs_plan_destroy(x[0])


@pytest.mark.parametrize("precision,tol", [(0, 1e-4), (2, 2e-3)])   # FP32, split-BF16 (BF16X2)
def test_tcs_full_720p_sampled(B, ctx, precision, tol):
    """A 720p GOP (1280 x 720, G = 16: 13800 blocks of 32 x 32, the last block row
    cropped) at M = 512 and K = 300, in the precision and launch path the mixed
    bench times; 96 sampled blocks recovered by the oracle one by one, with y
    measured by the oracle."""
    h, w, gop, b, m, iters, seed = 720, 1280, 16, 32, 512, 300, 21
    frames = scenes.surveillance_video(gop, h, w, seed=seed)
    plan = B.cs_make_phi(ctx, b * b, m, seed)
    try:
        p = B.make_params(h, w, gop, b, m, iters=iters, precision=precision)
        nbr, nbc = -(-h // b), -(-w // b)
        nblk = nbr * nbc
        y = torch.empty((gop - 1, nblk, m), dtype=torch.float32, device="cuda")
        B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
        key = torch.from_numpy(np.ascontiguousarray(frames[:1])).cuda()
        out = torch.full((gop - 1, h, w), float("nan"), dtype=torch.float32, device="cuda")
        B.cs_decode_gop(plan, p, key, y, out, None, torch.cuda.current_stream())
        B.cs_ctx_status(ctx)
        out_f = out.cpu().numpy().astype(np.float64)
    finally:
        B.cs_plan_destroy(plan)
    oplan = O.Plan(b * b, m, seed)
    yo = O.encode(oplan, frames, gop)
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(yo.shape[0] * nblk, size=96, replace=False))
    rows[-1] = yo.shape[0] * nblk - 1          # the last block: the cropped bottom-right corner
    r_hat = O.decode_blocks(oplan, yo.reshape(-1, m)[rows], iters)
    key64 = frames[0].astype(np.float64)
    got, want = [], []
    for i, r in enumerate(rows):
        c, blk = divmod(int(r), nblk)
        bi, bj = divmod(blk, nbc)
        hh, ww = min(b, h - bi * b), min(b, w - bj * b)
        sl = (slice(bi * b, bi * b + hh), slice(bj * b, bj * b + ww))
        want.append((key64[sl] + r_hat[i].reshape(b, b)[:hh, :ww]).ravel())
        got.append(out_f[c][sl].ravel())
    got, want = np.concatenate(got), np.concatenate(want)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    print("720p M=512 precision %d: sampled blocks rel-l2 %.3g" % (precision, err))
    assert err <= tol


@pytest.mark.parametrize("h,w,b,m", [(1, 1, 32, 300), (3, 5, 8, 20), (17, 9, 16, 150)])
def test_tcs_tiny_frames(B, ctx, h, w, b, m):
    # frames smaller than one block: every block is mostly padding, one row per tile
    gop, iters = 3, 25
    frames, got, u8 = _run(B, ctx, h, w, gop, b, m, iters, seed=14)
    ref = _oracle(frames, b, gop, 1, m, iters, 14)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err <= 1e-4, err
    assert np.array_equal(u8, np.clip(np.rint(got), 0, 255).astype(np.uint8))


def test_batch_of_no_jobs_is_a_no_op(B, ctx):
    B.cs_decode_batch(ctx, [], [], [], [], None, None, torch.cuda.current_stream())
    B.cs_ctx_status(ctx)
