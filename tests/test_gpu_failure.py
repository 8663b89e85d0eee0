"""Failure detection without a GPU fault: a barrier arrival withheld on purpose
(a test hook) makes one bounded device-side wait run out; the kernel drains,
cs_ctx_status reports CS_ETIMEDOUT once, and the context keeps decoding
correctly afterwards."""
import time

import numpy as np
import pytest

from paper_1311_1419_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1311_1419_gb300 import binding
    return binding


@pytest.mark.parametrize("b,m,engine", [(16, 32, "TC"), (32, 200, "TC_STREAM"), (32, 102, "TC")])
def test_withheld_arrival_times_out_and_the_context_recovers(B, b, m, engine):
    # the on-chip kernel (16 x 16 blocks), the streaming kernel (32 x 32, M > 128) and
    # the 8-CTA cluster kernel (32 x 32, M <= 128: one CTA stops, its peers' waits for
    # its data run out in turn, and every CTA drains its inbound copies before leaving)
    eng = getattr(B, "CS_ENGINE_" + engine)
    ctx = B.cs_ctx_create(0)
    plan = B.cs_make_phi(ctx, b * b, m, 3)
    try:
        h, w = 64, 128
        nblk = (h // b) * (w // b)                                    # one tile
        frames = scenes.surveillance_video(2, h, w, seed=5)
        p = B.make_params(h, w, 2, b, m, iters=20, engine=eng)
        s = torch.cuda.current_stream()
        f = torch.from_numpy(frames).cuda()
        y = torch.empty((1, nblk, m), dtype=torch.float32, device="cuda")
        B.cs_encode_gop(plan, p, f, y, s)
        ref = torch.empty((1, h, w), dtype=torch.float32, device="cuda")
        B.cs_decode_gop(plan, p, f[:1], y, ref, None, s)
        B.cs_ctx_status(ctx)                                          # healthy

        B.cs_ctx_set_debug(ctx, B.CS_DEBUG_DROP_ARRIVAL)
        out = torch.full((1, h, w), -1.0, dtype=torch.float32, device="cuda")
        t0 = time.time()
        B.cs_decode_gop(plan, p, f[:1], y, out, None, s)
        with pytest.raises(B.CsError) as ei:
            B.cs_ctx_status(ctx)
        assert ei.value.status == B.CS_ETIMEDOUT
        assert time.time() - t0 < 30
        B.cs_ctx_status(ctx)                                          # reported once

        again = torch.empty((1, h, w), dtype=torch.float32, device="cuda")
        B.cs_decode_gop(plan, p, f[:1], y, again, None, s)
        B.cs_ctx_status(ctx)
        assert np.array_equal(again.cpu().numpy(), ref.cpu().numpy())
    finally:
        B.cs_plan_destroy(plan)
        B.cs_ctx_destroy(ctx)
