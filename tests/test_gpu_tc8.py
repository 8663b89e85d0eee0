"""The tensor-core decode of 32 x 32 blocks (N = 1024) on clusters of 8 CTAs
against the FP64 oracle: FP32-grade and mixed precision, one and several
tiles, every owner split of the measurement rows (M16 = 16 .. 128), and inside
a heterogeneous cs_decode_batch."""
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


def _run(B, ctx, h, w, gop, n_gops, m, iters, seed, precision=0, tail=0, engine=None):
    b = 32
    frames = scenes.surveillance_video(gop * n_gops, h, w, seed=seed)
    plan = B.cs_make_phi(ctx, b * b, m, seed)
    try:
        eng = B.CS_ENGINE_TC if engine is None else engine
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


def _oracle(frames, gop, n_gops, m, iters, seed):
    plan = O.Plan(1024, m, seed)
    y = O.encode(plan, frames, gop)
    ref, _ = O.decode(plan, frames[::gop], y, gop, gop * n_gops, iters)
    return ref


def _cs(frames, gop):
    return frames[[t for t in range(frames.shape[0]) if t % gop]]


@pytest.mark.parametrize("h,w,gop,n_gops,m,iters", [
    (96, 128, 4, 2, 102, 40),     # 72 blocks: one ragged tile, M16 = 112 (owners of 16 and 8 rows)
    (192, 256, 5, 1, 51, 30),     # 192 blocks: two tiles, M16 = 64 (8 rows per owner)
    (64, 96, 3, 1, 10, 30),       # M16 = 16: two owners hold every row
    (80, 100, 3, 1, 128, 25),     # M16 = 128 (16 rows per owner), cropped blocks
])
def test_tc8_fp32_matches_oracle(B, ctx, h, w, gop, n_gops, m, iters):
    frames, got, u8 = _run(B, ctx, h, w, gop, n_gops, m, iters, seed=7)
    ref = _oracle(frames, gop, n_gops, m, iters, 7)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    dpsnr = O.psnr(_cs(frames, gop), got) - O.psnr(_cs(frames, gop), ref)
    print("N=1024 M=%d: rel-l2 %.3g dPSNR %.3g dB" % (m, err, dpsnr))
    assert err <= 1e-4 and abs(dpsnr) <= 0.01
    assert np.array_equal(u8, np.clip(np.rint(got), 0, 255).astype(np.uint8))


@pytest.mark.parametrize("precision,tail", [(3, 10), (1, 10), (2, 0)])   # FP16, BF16, BF16X2
def test_tc8_mixed_precision_within_tolerance(B, ctx, precision, tail):
    h, w, gop, n_gops, m, iters = 96, 128, 4, 1, 102, 40
    frames, got, _ = _run(B, ctx, h, w, gop, n_gops, m, iters, seed=9, precision=precision,
                          tail=tail)
    ref = _oracle(frames, gop, n_gops, m, iters, 9)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    dpsnr = O.psnr(_cs(frames, gop), got) - O.psnr(_cs(frames, gop), ref)
    print("N=1024 precision %d tail %d: rel-l2 %.3g dPSNR %.3g dB" % (precision, tail, err, dpsnr))
    assert abs(dpsnr) <= 0.1 and err <= 2e-3


def test_tc8_in_a_batch_equals_alone(B, ctx):
    jobs = [(96, 128, 4, 32, 102, 20, 3), (48, 64, 3, 16, 40, 20, 4), (64, 64, 3, 32, 20, 15, 5)]
    prepared = []
    try:
        for h, w, gop, b, m, iters, seed in jobs:
            frames = scenes.surveillance_video(gop, h, w, seed=seed)
            plan = B.cs_make_phi(ctx, b * b, m, seed)
            p = B.make_params(h, w, gop, b, m, iters=iters)
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


def test_tc8_large_job_tail_on_idle_sms(B, ctx):
    """The 720p workload (96 frames, G = 16: 82800 blocks, 647 tiles; M = 102, K = 300):
    whole clusters leave SMs idle, so a tail of the job runs on the streaming kernel
    there.  Sampled blocks of the head and of the tail match the oracle, and the
    tail is bit for bit the streaming kernel's own decode of those blocks."""
    h, w, gop, n_gops, m, iters, seed = 720, 1280, 16, 6, 102, 300, 31
    b = 32
    frames = scenes.surveillance_video(gop * n_gops, h, w, seed=seed)
    plan = B.cs_make_phi(ctx, b * b, m, seed)
    nbr, nbc = -(-h // b), -(-w // b)
    nblk = nbr * nbc
    n_cs = n_gops * (gop - 1)
    try:
        outs = {}
        for name, eng in (("tc", B.CS_ENGINE_TC), ("tcs", B.CS_ENGINE_TC_STREAM)):
            p = B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops, engine=eng)
            y = torch.empty((n_cs, nblk, m), dtype=torch.float32, device="cuda")
            B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
            keys = torch.from_numpy(np.ascontiguousarray(frames[::gop])).cuda()
            out = torch.full((n_cs, h, w), float("nan"), dtype=torch.float32, device="cuda")
            B.cs_decode_gop(plan, p, keys, y, out, None, torch.cuda.current_stream())
            B.cs_ctx_status(ctx)
            outs[name] = out.cpu().numpy()
    finally:
        B.cs_plan_destroy(plan)
    total = n_cs * nblk
    tiles = -(-total // 128)
    # the tail is a whole number of rounds of two CTAs per idle SM: with 15 of 19
    # possible clusters resident that is 64 tiles; the last 32 tiles are in it on
    # any part that leaves at least 16 SMs idle
    first_tail = total - (32 * 128 - (tiles * 128 - total))

    def block(o, r):
        c, blk = divmod(int(r), nblk)
        bi, bj = divmod(blk, nbc)
        return o[c, bi * b:min(h, bi * b + b), bj * b:min(w, bj * b + b)]
    for r in range(first_tail, total, 97):
        assert np.array_equal(block(outs["tc"], r).view(np.uint32), block(outs["tcs"], r).view(np.uint32)), r
    # and the head did not: the cluster kernel's arithmetic differs in the last bits
    assert not all(np.array_equal(block(outs["tc"], r), block(outs["tcs"], r)) for r in range(0, 6400, 101))
    oplan = O.Plan(b * b, m, seed)
    yo = O.encode(oplan, frames, gop)
    rng = np.random.default_rng(seed)
    rows = np.concatenate([rng.choice(first_tail, 48, replace=False),
                           first_tail + rng.choice(total - first_tail, 48, replace=False)])
    r_hat = O.decode_blocks(oplan, yo.reshape(-1, m)[rows], iters)
    got, want = [], []
    for i, r in enumerate(rows):
        c, blk = divmod(int(r), nblk)
        bi, bj = divmod(blk, nbc)
        hh, ww = min(b, h - bi * b), min(b, w - bj * b)
        key = frames[(c // (gop - 1)) * gop].astype(np.float64)
        sl = (slice(bi * b, bi * b + hh), slice(bj * b, bj * b + ww))
        want.append((key[sl] + r_hat[i].reshape(b, b)[:hh, :ww]).ravel())
        got.append(outs["tc"][c][sl].astype(np.float64).ravel())
    got, want = np.concatenate(got), np.concatenate(want)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    print("720p M=102 head + streaming tail, sampled blocks rel-l2 %.3g" % err)
    assert err <= 1e-4
