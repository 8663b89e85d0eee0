"""The decode autotuner and CUDA-graph capture of the batched decode.

cs_autotune times the launch shapes a plan's (N, M) admits and records the
fastest; FP32 AUTO decodes then use it and still match the FP64 oracle.  A
cs_decode_batch of jobs on both kernels, captured into a CUDA graph, replays to
the same bits as the eager call."""
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


def _case(B, ctx, h, w, gop, b, m, iters, seed, precision=0, tail=0):
    frames = scenes.surveillance_video(gop, h, w, seed=seed)
    plan = B.cs_make_phi(ctx, b * b, m, seed)
    p = B.make_params(h, w, gop, b, m, iters=iters, precision=precision, fp32_tail_iters=tail)
    nblk = (-(-h // b)) * (-(-w // b))
    y = torch.empty((gop - 1, nblk, m), dtype=torch.float32, device="cuda")
    B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
    key = torch.from_numpy(np.ascontiguousarray(frames[:1])).cuda()
    return frames, plan, p, key, y


@pytest.mark.parametrize("h,w,gop,b,m,iters", [(48, 64, 3, 8, 16, 60),      # N = 64
                                               (64, 96, 2, 32, 102, 40),    # N = 1024
                                               (64, 96, 2, 32, 300, 30),    # N = 1024, M > 128: streaming
                                               (48, 80, 3, 16, 40, 50)])    # N = 256
def test_autotuned_decode_matches_oracle(B, ctx, h, w, gop, b, m, iters):
    frames, plan, p, key, y = _case(B, ctx, h, w, gop, b, m, iters, seed=5)
    try:
        eng, thr, blk, ns = B.cs_autotune(ctx, plan)
        assert eng in (B.CS_ENGINE_TC, B.CS_ENGINE_TC_STREAM, B.CS_ENGINE_TC_CHUNK, B.CS_ENGINE_PLAIN) and ns > 0
        if eng == B.CS_ENGINE_PLAIN:
            assert thr in (64, 128, 256, 512, 1024) and blk in (1, 2, 4, 8, 16)
        else:
            assert thr == 0 and blk == 0
            if eng in (B.CS_ENGINE_TC, B.CS_ENGINE_TC_CHUNK):
                assert b in (16, 32) and m <= 128
        print("N=%d M=%d: engine %d threads %d blocks/CTA %d, %.2f ns per block-iteration"
              % (b * b, m, eng, thr, blk, ns))
        out = torch.full((gop - 1, h, w), float("nan"), dtype=torch.float32, device="cuda")
        B.cs_decode_gop(plan, p, key, y, out, None, torch.cuda.current_stream())
        B.cs_ctx_status(ctx)
        oplan = O.Plan(b * b, m, 5)
        ref, _ = O.decode(oplan, frames[:1], O.encode(oplan, frames, gop), gop, gop, iters)
        got = out.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4
        assert abs(O.psnr(frames[1:], got) - O.psnr(frames[1:], ref)) <= 0.01
    finally:
        B.cs_plan_destroy(plan)


def test_batched_decode_replays_from_a_cuda_graph(B, ctx):
    # two tensor-core layouts (M16 <= 96 and M = 128: launches forked onto the
    # context's streams and joined), the 32 x 32 cluster kernel and the plain kernel
    cases = [_case(B, ctx, 144, 176, 4, 16, 26, 40, 1),
             _case(B, ctx, 96, 112, 5, 16, 64, 30, 2, precision=3, tail=10),
             _case(B, ctx, 80, 96, 3, 16, 128, 30, 6),
             _case(B, ctx, 64, 96, 3, 32, 51, 20, 7),
             _case(B, ctx, 48, 64, 3, 8, 16, 30, 3)]
    try:
        plans = [c[1] for c in cases]
        params = [c[2] for c in cases]
        keys = [c[3] for c in cases]
        ys = [c[4] for c in cases]
        shapes = [(c[4].shape[0], c[0].shape[1], c[0].shape[2]) for c in cases]
        eager = [torch.zeros(s, dtype=torch.float32, device="cuda") for s in shapes]
        B.cs_decode_batch(ctx, plans, params, keys, ys, eager, None, torch.cuda.current_stream())
        torch.cuda.synchronize()
        B.cs_ctx_status(ctx)

        graphed = [torch.zeros(s, dtype=torch.float32, device="cuda") for s in shapes]
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
                B.cs_decode_batch(ctx, plans, params, keys, ys, graphed, None, side)
        torch.cuda.current_stream().wait_stream(side)
        for rep in range(2):
            for t in graphed:
                t.fill_(float("nan"))
            g.replay()
            torch.cuda.synchronize()
            B.cs_ctx_status(ctx)
            for i, (a, b_) in enumerate(zip(eager, graphed)):
                assert np.array_equal(a.cpu().numpy().view(np.uint32),
                                      b_.cpu().numpy().view(np.uint32)), "replay %d job %d" % (rep, i)
    finally:
        for c in cases:
            B.cs_plan_destroy(c[1])
