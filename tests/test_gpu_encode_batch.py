"""cs_encode_batch: several plans of one block size measure one clip in shared
tensor-core launches (the clip read once per launch).  Each plan's y matches its
own cs_encode_gop to FP32 rounding (a launch with room sums a plan's hi and lo
products in separate accumulators, a crowded one in one: the order of the sums
differs) and the FP64 oracle; plans whose images exceed one launch split into
several; a plain-engine plan runs on the SIMT encode beside them; calls that
differ in their clip are refused."""
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


def _run(B, ctx, frames, gop, b, ms, engines=None, seed=7):
    n_f, h, w = frames.shape
    n_gops = n_f // gop
    nblk = (-(-h // b)) * (-(-w // b))
    engines = engines or [B.CS_ENGINE_AUTO] * len(ms)
    plans = [B.cs_make_phi(ctx, b * b, m, seed + i) for i, m in enumerate(ms)]
    try:
        params = [B.make_params(h, w, gop, b, m, n_gops=n_gops, engine=e) for m, e in zip(ms, engines)]
        s = torch.cuda.current_stream()
        f = torch.from_numpy(frames).cuda()
        yb = [torch.full((n_gops * (gop - 1), nblk, m), float("nan"), dtype=torch.float32, device="cuda")
              for m in ms]
        B.cs_encode_batch(ctx, plans, params, f, yb, s)
        ys = []
        for plan, p, m in zip(plans, params, ms):
            y = torch.full((n_gops * (gop - 1), nblk, m), float("nan"), dtype=torch.float32, device="cuda")
            B.cs_encode_gop(plan, p, f, y, s)
            ys.append(y)
        B.cs_ctx_status(ctx)
        return [y.cpu().numpy() for y in yb], [y.cpu().numpy() for y in ys]
    finally:
        for p in plans:
            B.cs_plan_destroy(p)


@pytest.mark.parametrize("h,w,gop,n_f,b,ms", [
    (288, 352, 8, 16, 16, [26, 51, 77, 128]),   # the CIF sweep's plans: one launch, 304 columns
    (144, 176, 4, 8, 16, [200, 150]),           # 208 + 160 columns: two launches
    (100, 90, 3, 6, 16, [26, 13, 64]),          # cropped edges, byte loads
    (72, 96, 3, 6, 8, [5, 19, 32]),             # 8 x 8 blocks
    (96, 160, 4, 4, 32, [102, 51]),             # 32 x 32 blocks
])
def test_batch_equals_single_calls_and_the_oracle(B, ctx, h, w, gop, n_f, b, ms):
    frames = scenes.surveillance_video(n_f, h, w, seed=9)
    yb, ys = _run(B, ctx, frames, gop, b, ms)
    for i, m in enumerate(ms):
        d = np.linalg.norm(yb[i] - ys[i]) / np.linalg.norm(ys[i])
        assert d <= 1e-6, "plan %d (M=%d) differs from its own call: %.3g" % (i, m, d)
        ref = O.encode(O.Plan(b * b, m, 7 + i), frames, gop)
        err = np.linalg.norm(yb[i] - ref) / np.linalg.norm(ref)
        print("batch encode b=%d M=%d: rel-l2 %.3g" % (b, m, err))
        assert err <= 1e-5


def test_batch_with_a_plain_engine_plan(B, ctx):
    frames = scenes.surveillance_video(8, 144, 176, seed=2)
    ms = [64, 32, 96]
    engines = [B.CS_ENGINE_AUTO, B.CS_ENGINE_PLAIN, B.CS_ENGINE_AUTO]
    yb, ys = _run(B, ctx, frames, 4, 16, ms, engines)
    for i, m in enumerate(ms):
        assert np.linalg.norm(yb[i] - ys[i]) / np.linalg.norm(ys[i]) <= 1e-6
        ref = O.encode(O.Plan(256, m, 7 + i), frames, 4)
        assert np.linalg.norm(yb[i] - ref) / np.linalg.norm(ref) <= 1e-5


def test_batch_refuses_calls_on_different_clips(B, ctx):
    plans = [B.cs_make_phi(ctx, 256, 32, 1), B.cs_make_phi(ctx, 256, 48, 2)]
    try:
        s = torch.cuda.current_stream()
        f = torch.zeros((4, 64, 64), dtype=torch.uint8, device="cuda")
        y = [torch.empty((3, 16, 32), device="cuda"), torch.empty((3, 16, 48), device="cuda")]
        params = [B.make_params(64, 64, 4, 16, 32), B.make_params(64, 48, 4, 16, 48)]
        with pytest.raises(B.CsError) as ei:
            B.cs_encode_batch(ctx, plans, params, f, y, s)
        assert ei.value.status == B.CS_EINVAL
        B.cs_encode_batch(ctx, [], [], f, [], s)     # nothing to do
    finally:
        for p in plans:
            B.cs_plan_destroy(p)
