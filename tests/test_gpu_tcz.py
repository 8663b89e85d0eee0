"""The chunked tensor-core decode (CS_ENGINE_TC_CHUNK: A streamed from L2,
GEMM1 in 128-coefficient chunks from tensor memory, s^{k-1} and s^{k-2} in
global memory) against the FP64 oracle: 16 x 16 and 32 x 32 blocks, M from one
16-row step to 128 (partial last K slices), ragged tiles, cropped edges, two
GOPs, iteration counts 0 .. 3, mixed precision, more tiles than SMs, a short last
round handed to the cluster kernel (also inside a CUDA graph), the full 720p clip
at K = 300 on sampled blocks, inside a batch (one and both operand types), the
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


def _inputs(B, plan, frames, gop, n_gops, b, m, p):
    h, w = frames.shape[1:]
    nblk = (-(-h // b)) * (-(-w // b))
    y = torch.empty((n_gops * (gop - 1), nblk, m), dtype=torch.float32, device="cuda")
    B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
    keys = torch.from_numpy(np.ascontiguousarray(frames[::gop])).cuda()
    return keys, y


def _run(B, ctx, h, w, gop, b, m, iters, seed, precision=0, tail=0, engine=None, n_gops=1):
    frames = scenes.surveillance_video(gop * n_gops, h, w, seed=seed)
    plan = B.cs_make_phi(ctx, b * b, m, seed)
    try:
        eng = B.CS_ENGINE_TC_CHUNK if engine is None else engine
        p = B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops, precision=precision,
                          fp32_tail_iters=tail, engine=eng)
        keys, y = _inputs(B, plan, frames, gop, n_gops, b, m, p)
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
    (160, 224, 5, 1, 32, 102, 40),   # 140 blocks: two tiles (last 12), M16 = 112: K slices 32+32+32+16
    (96, 128, 3, 2, 32, 128, 30),    # two GOPs, M = 128: the widest U
    (100, 130, 4, 1, 32, 16, 50),    # cropped edges, M = 16: one 16-row K step
    (64, 96, 3, 1, 32, 51, 30),      # M16 = 64
    (144, 176, 3, 1, 16, 77, 40),    # N = 256: two chunks, 297 blocks in 3 tiles
    (80, 112, 3, 1, 16, 128, 30),    # N = 256, M = 128
])
def test_tcz_fp32_matches_oracle(B, ctx, h, w, gop, n_gops, b, m, iters):
    frames, got, u8 = _run(B, ctx, h, w, gop, b, m, iters, seed=21, n_gops=n_gops)
    ref = _oracle(frames, b, gop, n_gops, m, iters, 21)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    keys = np.repeat(frames[::gop].astype(np.float64), gop - 1, axis=0)
    res = np.linalg.norm(got - ref) / max(np.linalg.norm(ref - keys), 1e-30)
    dpsnr = O.psnr(_cs(frames, gop), got) - O.psnr(_cs(frames, gop), ref)
    print("tcz N=%d M=%d: frame rel-l2 %.3g residual rel-l2 %.3g dPSNR %.3g dB" % (b * b, m, err, res, dpsnr))
    assert err <= 1e-4 and abs(dpsnr) <= 0.01
    assert np.array_equal(u8, np.clip(np.rint(got), 0, 255).astype(np.uint8))


@pytest.mark.parametrize("iters", [0, 1, 2, 3])
def test_tcz_few_iterations(B, ctx, iters):
    # K = 0: the key comes back; K = 1: no GEMM1; K = 2: z^1 from s^0 alone;
    # K = 3: the first step that reads both s^{k-1} and s^{k-2}
    h, w, gop, b, m = 64, 96, 3, 32, 90
    frames, got, _ = _run(B, ctx, h, w, gop, b, m, iters, seed=22)
    ref = _oracle(frames, b, gop, 1, m, iters, 22)
    if iters == 0:
        assert np.array_equal(got, np.repeat(frames[:1].astype(np.float64), gop - 1, axis=0))
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    print("tcz K=%d: rel-l2 %.3g" % (iters, err))
    assert err <= 1e-4, err


@pytest.mark.parametrize("precision,tail", [(3, 10), (1, 10), (2, 0)])   # FP16, BF16, BF16X2
def test_tcz_mixed_precision_within_tolerance(B, ctx, precision, tail):
    h, w, gop, b, m, iters = 96, 128, 4, 32, 102, 40
    frames, got, _ = _run(B, ctx, h, w, gop, b, m, iters, seed=23, precision=precision, tail=tail)
    ref = _oracle(frames, b, gop, 1, m, iters, 23)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    dpsnr = O.psnr(_cs(frames, gop), got) - O.psnr(_cs(frames, gop), ref)
    print("tcz N=1024 M=102 precision %d tail %d: rel-l2 %.3g dPSNR %.3g dB" % (precision, tail, err, dpsnr))
    assert abs(dpsnr) <= 0.1 and err <= 2e-3


def test_tcz_more_tiles_than_sms_agrees_with_the_streaming_kernel(B, ctx):
    # two 720p GOPs of 16 frames: 27600 blocks, 216 tiles, so CTAs take several
    # tiles; the streaming kernel (checked against the oracle elsewhere) is the check
    h, w, gop, n_gops, b, m, iters = 720, 1280, 16, 2, 32, 102, 12
    _, tcz, _ = _run(B, ctx, h, w, gop, b, m, iters, seed=24, n_gops=n_gops)
    frames, tcs, _ = _run(B, ctx, h, w, gop, b, m, iters, seed=24, n_gops=n_gops, engine=B.CS_ENGINE_TC_STREAM)
    keys = np.repeat(frames[::gop].astype(np.float64), gop - 1, axis=0)
    rel = np.linalg.norm(tcz - tcs) / np.linalg.norm(tcs - keys)
    print("tcz vs tcs, 27600 blocks: residual rel-l2 %.3g" % rel)
    assert np.isfinite(tcz).all()
    assert rel <= 1e-4


def test_tcz_short_last_round_goes_to_the_cluster_kernel(B, ctx):
    # three 720p GOPs of 16 frames: 41400 blocks, 324 tiles.  On 152 SMs with 15
    # co-resident clusters of 8 the last round would hold 20 tiles: the cluster kernel
    # decodes the first 20 tiles instead (bit for bit its own decode of them, which the
    # on-chip engine gives for those rows too) and this kernel the other 304 in two
    # whole rounds; everything matches the streaming kernel
    h, w, gop, n_gops, b, m, iters = 720, 1280, 16, 3, 32, 102, 12
    _, tcz, _ = _run(B, ctx, h, w, gop, b, m, iters, seed=25, n_gops=n_gops)
    _, tc, _ = _run(B, ctx, h, w, gop, b, m, iters, seed=25, n_gops=n_gops, engine=B.CS_ENGINE_TC)
    frames, tcs, _ = _run(B, ctx, h, w, gop, b, m, iters, seed=25, n_gops=n_gops, engine=B.CS_ENGINE_TC_STREAM)
    keys = np.repeat(frames[::gop].astype(np.float64), gop - 1, axis=0)
    rel = np.linalg.norm(tcz - tcs) / np.linalg.norm(tcs - keys)
    print("tcz (with a cluster head) vs tcs, 41400 blocks: residual rel-l2 %.3g" % rel)
    assert np.isfinite(tcz).all() and rel <= 1e-4
    if torch.cuda.get_device_properties(0).multi_processor_count == 152:
        # rows 0 .. 2559: CS frames 0 and 1 whole (920 blocks each)
        assert np.array_equal(tcz[:2].astype(np.float32).view(np.uint32), tc[:2].astype(np.float32).view(np.uint32))
        # and the chunked kernel's rows differ from the cluster kernel's in the last bits
        assert not np.array_equal(tcz[5:], tc[5:])


def test_tcz_in_a_batch_equals_alone(B, ctx):
    # two chunked jobs of different N and M in one cs_decode_batch (one launch) give
    # the bits each gives alone
    cams = [(96, 160, 3, 32, 102, 20, 31), (144, 176, 4, 16, 64, 25, 32)]
    plans, params, keys, ys, alone = [], [], [], [], []
    try:
        for h, w, gop, b, m, iters, seed in cams:
            frames = scenes.surveillance_video(gop, h, w, seed=seed)
            plan = B.cs_make_phi(ctx, b * b, m, seed)
            plans.append(plan)
            p = B.make_params(h, w, gop, b, m, iters=iters, engine=B.CS_ENGINE_TC_CHUNK)
            params.append(p)
            k, y = _inputs(B, plan, frames, gop, 1, b, m, p)
            keys.append(k)
            ys.append(y)
            o = torch.empty((gop - 1, h, w), dtype=torch.float32, device="cuda")
            B.cs_decode_gop(plan, p, k, y, o, None, torch.cuda.current_stream())
            alone.append(o)
        outs = [torch.full_like(o, float("nan")) for o in alone]
        B.cs_decode_batch(ctx, plans, params, keys, ys, outs, None, torch.cuda.current_stream())
        B.cs_ctx_status(ctx)
        for a, o in zip(alone, outs):
            assert np.array_equal(a.cpu().numpy().view(np.uint32), o.cpu().numpy().view(np.uint32))
    finally:
        for p in plans:
            B.cs_plan_destroy(p)


def test_tcz_with_a_cluster_head_replays_from_a_cuda_graph(B, ctx):
    # three 720p GOPs (324 tiles): on 152 SMs the first 20 tiles go to the cluster
    # kernel and the rest to this kernel; the captured call replays to the eager bits
    h, w, gop, n_gops, b, m, iters = 720, 1280, 16, 3, 32, 102, 6
    frames = scenes.surveillance_video(gop * n_gops, h, w, seed=26)
    plan = B.cs_make_phi(ctx, b * b, m, 26)
    try:
        p = B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops, engine=B.CS_ENGINE_TC_CHUNK)
        keys, y = _inputs(B, plan, frames, gop, n_gops, b, m, p)
        eager = torch.zeros((y.shape[0], h, w), dtype=torch.float32, device="cuda")
        B.cs_decode_gop(plan, p, keys, y, eager, None, torch.cuda.current_stream())
        torch.cuda.synchronize()
        B.cs_ctx_status(ctx)
        graphed = torch.zeros_like(eager)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
                B.cs_decode_gop(plan, p, keys, y, graphed, None, side)
        torch.cuda.current_stream().wait_stream(side)
        for rep in range(2):
            graphed.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            B.cs_ctx_status(ctx)
            assert np.array_equal(eager.cpu().numpy().view(np.uint32), graphed.cpu().numpy().view(np.uint32)), rep
    finally:
        B.cs_plan_destroy(plan)


def test_tcz_batch_of_both_operand_types_equals_alone(B, ctx):
    # FP32-grade (fp16 operands) and split-BF16 chunked jobs in one cs_decode_batch:
    # one launch per operand type, each job's bits as alone
    cams = [(96, 160, 3, 32, 102, 20, 41, 0, 0), (96, 128, 4, 32, 64, 20, 42, 2, 0),
            (144, 176, 3, 16, 77, 20, 43, 1, 8), (80, 112, 3, 16, 40, 20, 44, 0, 0)]
    plans, params, keys, ys, alone = [], [], [], [], []
    try:
        for h, w, gop, b, m, iters, seed, prec, tail in cams:
            frames = scenes.surveillance_video(gop, h, w, seed=seed)
            plan = B.cs_make_phi(ctx, b * b, m, seed)
            plans.append(plan)
            p = B.make_params(h, w, gop, b, m, iters=iters, precision=prec, fp32_tail_iters=tail,
                              engine=B.CS_ENGINE_TC_CHUNK)
            params.append(p)
            k, y = _inputs(B, plan, frames, gop, 1, b, m, p)
            keys.append(k)
            ys.append(y)
            o = torch.empty((gop - 1, h, w), dtype=torch.float32, device="cuda")
            B.cs_decode_gop(plan, p, k, y, o, None, torch.cuda.current_stream())
            alone.append(o)
        outs = [torch.full_like(o, float("nan")) for o in alone]
        B.cs_decode_batch(ctx, plans, params, keys, ys, outs, None, torch.cuda.current_stream())
        B.cs_ctx_status(ctx)
        for i, (a, o) in enumerate(zip(alone, outs)):
            assert np.array_equal(a.cpu().numpy().view(np.uint32), o.cpu().numpy().view(np.uint32)), i
    finally:
        for p in plans:
            B.cs_plan_destroy(p)


def test_tcz_engine_rules(B, ctx):
    s = torch.cuda.current_stream()
    # N = 64 and M > 128 have no chunked kernel; TV recovery has none either
    for b, m in [(8, 24), (32, 200), (16, 144)]:
        plan = B.cs_make_phi(ctx, b * b, m, 1)
        try:
            p = B.make_params(64, 64, 2, b, m, iters=5, engine=B.CS_ENGINE_TC_CHUNK)
            y = torch.zeros((1, (64 // b) ** 2, m), dtype=torch.float32, device="cuda")
            key = torch.zeros((1, 64, 64), dtype=torch.uint8, device="cuda")
            out = torch.empty((1, 64, 64), dtype=torch.float32, device="cuda")
            with pytest.raises(B.CsError) as ei:
                B.cs_decode_gop(plan, p, key, y, out, None, s)
            assert ei.value.status == B.CS_EINVAL
        finally:
            B.cs_plan_destroy(plan)
    plan = B.cs_make_phi(ctx, 1024, 64, 1)
    try:
        p = B.make_params(64, 64, 2, 32, 64, iters=5, engine=B.CS_ENGINE_TC_CHUNK)
        y = torch.zeros((1, 4, 64), dtype=torch.float32, device="cuda")
        key = torch.zeros((1, 64, 64), dtype=torch.uint8, device="cuda")
        out = torch.empty((1, 64, 64), dtype=torch.float32, device="cuda")
        with pytest.raises(B.CsError) as ei:
            B.cs_decode_gop_tv(plan, p, key, y, out, None, s)
        assert ei.value.status == B.CS_EINVAL
    finally:
        B.cs_plan_destroy(plan)


def test_tcz_withheld_arrival_times_out_and_recovers(B):
    c = B.cs_ctx_create(0)
    plan = B.cs_make_phi(c, 1024, 102, 5)
    try:
        h, w = 96, 128
        frames = scenes.surveillance_video(2, h, w, seed=5)
        p = B.make_params(h, w, 2, 32, 102, iters=20, engine=B.CS_ENGINE_TC_CHUNK)
        s = torch.cuda.current_stream()
        f = torch.from_numpy(frames).cuda()
        y = torch.empty((1, 12, 102), dtype=torch.float32, device="cuda")
        B.cs_encode_gop(plan, p, f, y, s)
        ref = torch.empty((1, h, w), dtype=torch.float32, device="cuda")
        B.cs_decode_gop(plan, p, f[:1], y, ref, None, s)
        B.cs_ctx_status(c)

        B.cs_ctx_set_debug(c, B.CS_DEBUG_DROP_ARRIVAL)
        out = torch.full((1, h, w), -1.0, dtype=torch.float32, device="cuda")
        t0 = time.time()
        B.cs_decode_gop(plan, p, f[:1], y, out, None, s)
        with pytest.raises(B.CsError) as ei:
            B.cs_ctx_status(c)
        assert ei.value.status == B.CS_ETIMEDOUT
        assert time.time() - t0 < 30
        B.cs_ctx_status(c)

        again = torch.empty((1, h, w), dtype=torch.float32, device="cuda")
        B.cs_decode_gop(plan, p, f[:1], y, again, None, s)
        B.cs_ctx_status(c)
        assert np.array_equal(again.cpu().numpy(), ref.cpu().numpy())
    finally:
        B.cs_plan_destroy(plan)
        B.cs_ctx_destroy(c)


def test_tcz_full_720p_clip_sampled_blocks_match_the_oracle(B, ctx):
    """The 720p workload as the bench decodes it (96 frames, G = 16: 82,800 blocks,
    647 tiles of 128; M = 102, K = 300) on the chunked engine, the cluster kernel
    taking the short last round's worth of tiles first where the SM count leaves
    one.  Blocks sampled from the first tiles, the middle and the ragged last tile
    (112 rows) match the oracle block by block, and the uint8 frames are the
    rounded float frames."""
    h, w, gop, n_gops, b, m, iters, seed = 720, 1280, 16, 6, 32, 102, 300, 41
    frames, out, u8 = _run(B, ctx, h, w, gop, b, m, iters, seed, n_gops=n_gops)
    nbr, nbc = -(-h // b), -(-w // b)
    nblk = nbr * nbc
    total = n_gops * (gop - 1) * nblk
    assert total == 82800
    rng = np.random.default_rng(seed)
    rows = np.concatenate([rng.choice(39 * 128, 32, replace=False),          # the first tiles
                           39 * 128 + rng.choice(total - 40 * 128, 32, replace=False),
                           (total // 128) * 128 + rng.choice(total % 128, 16, replace=False)])
    oplan = O.Plan(b * b, m, seed)
    yo = O.encode(oplan, frames, gop)
    r_hat = O.decode_blocks(oplan, yo.reshape(-1, m)[rows], iters)
    got, want, res_got, res_want = [], [], [], []
    for i, r in enumerate(rows):
        c, blk = divmod(int(r), nblk)
        bi, bj = divmod(blk, nbc)
        hh, ww = min(b, h - bi * b), min(b, w - bj * b)              # 720 = 22.5 blocks
        sl = (slice(bi * b, bi * b + hh), slice(bj * b, bj * b + ww))
        key = frames[(c // (gop - 1)) * gop].astype(np.float64)
        g = out[c][sl].ravel()
        rb = r_hat[i].reshape(b, b)[:hh, :ww].ravel()
        want.append(key[sl].ravel() + rb)
        got.append(g)
        res_got.append(g - key[sl].ravel())
        res_want.append(rb)
        assert np.array_equal(u8[c][sl].ravel(), np.clip(np.rint(g), 0, 255).astype(np.uint8)), r
    got, want = np.concatenate(got), np.concatenate(want)
    res_got, res_want = np.concatenate(res_got), np.concatenate(res_want)
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    res_err = np.linalg.norm(res_got - res_want) / np.linalg.norm(res_want)
    print("720p M=102 K=300 chunked, %d sampled blocks: frame rel-l2 %.3g, residual rel-l2 %.3g"
          % (len(rows), err, res_err))
    assert err <= 1e-4
    assert res_err <= 1e-3
