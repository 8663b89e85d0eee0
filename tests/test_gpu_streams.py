"""Many decodes in flight at once on many caller streams: the decode kernels
take per-launch device resources (tile counters, the streaming kernel's
iterate scratch, the cluster kernel's all-gather scratch) from rings of a few
slots, and a slot is handed to a new launch only after its previous holder has
finished.  20 launches on 20 streams, more than any ring has slots, each give
bit for bit what they give alone."""
import numpy as np
import pytest

from paper_1311_1419_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_STREAMS = 20


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


def _jobs(B, ctx, b, m, engine, iters, h=224, w=288, gop=3):
    jobs = []
    for i in range(N_STREAMS):
        frames = scenes.surveillance_video(gop, h, w, seed=100 + i)
        plan = B.cs_make_phi(ctx, b * b, m, 100 + i)
        p = B.make_params(h, w, gop, b, m, iters=iters, engine=engine)
        nblk = (-(-h // b)) * (-(-w // b))
        y = torch.empty((gop - 1, nblk, m), dtype=torch.float32, device="cuda")
        B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
        key = torch.from_numpy(np.ascontiguousarray(frames[:1])).cuda()
        jobs.append((plan, p, key, y, (gop - 1, h, w)))
    torch.cuda.synchronize()
    return jobs


def _alone_then_together(B, ctx, jobs):
    alone = []
    for plan, p, key, y, shape in jobs:
        out = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
        B.cs_decode_gop(plan, p, key, y, out, None, torch.cuda.current_stream())
        torch.cuda.synchronize()
        alone.append(out.cpu())
    streams = [torch.cuda.Stream() for _ in jobs]
    outs = [torch.full(j[4], float("nan"), dtype=torch.float32, device="cuda") for j in jobs]
    torch.cuda.synchronize()
    for (plan, p, key, y, _), s, out in zip(jobs, streams, outs):
        B.cs_decode_gop(plan, p, key, y, out, None, s)       # no synchronisation in between
    torch.cuda.synchronize()
    B.cs_ctx_status(ctx)                                      # raises on a device-side timeout
    for i, (a, o) in enumerate(zip(alone, outs)):
        assert torch.equal(a, o.cpu()), "stream %d differs from its decode alone" % i
    for plan, *_ in jobs:
        B.cs_plan_destroy(plan)


def test_streaming_decodes_on_20_streams_equal_each_alone(B, ctx):
    # 32 x 32 blocks, M = 200: the streaming kernel (its scratch ring has 8 slots)
    _alone_then_together(B, ctx, _jobs(B, ctx, 32, 200, B.CS_ENGINE_TC_STREAM, 40))


def test_cluster_decodes_on_20_streams_equal_each_alone(B, ctx):
    # 32 x 32 blocks, M = 102: the 8-CTA cluster kernel (its scratch ring has 16 slots)
    _alone_then_together(B, ctx, _jobs(B, ctx, 32, 102, B.CS_ENGINE_TC, 40))


def test_onchip_decodes_on_20_streams_equal_each_alone(B, ctx):
    # 16 x 16 blocks, M = 64: the on-chip kernel (tile counters)
    _alone_then_together(B, ctx, _jobs(B, ctx, 16, 64, B.CS_ENGINE_TC, 60))
