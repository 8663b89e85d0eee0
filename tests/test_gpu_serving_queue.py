"""Serving through the device work queue: the tiles of every admitted request
join one queue that a persistent launch of the streaming tensor-core decode
drains.  Each request gives, bit for bit, what it gives decoded alone by that
kernel; a request that arrives while a large one is on the GPU is admitted and
finishes first (its tiles run beside the large one's); the launch ends itself
when idle and is started again by the next request."""
import time

import numpy as np
import pytest

from paper_1311_1419_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BUDGET = 4 << 30   # room for the streaming kernel's scratch beside the pool

CAMERAS = [  # (h, w, gop, block, m, iters, precision, tail, seed)
    (144, 176, 4, 16, 26, 60, 0, 0, 21),
    (288, 352, 5, 16, 64, 40, 3, 10, 22),     # FP16 bulk, FP32-grade tail
    (96, 128, 6, 8, 12, 80, 0, 0, 23),        # 8 x 8 blocks
    (288, 352, 3, 32, 102, 40, 0, 0, 24),
    (160, 192, 4, 32, 200, 30, 0, 0, 25),     # M > 128
    (120, 200, 3, 32, 256, 20, 3, 5, 26),
]


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1311_1419_gb300 import binding
    return binding


def _camera(B, ctx, cam):
    h, w, gop, b, m, iters, prec, tail, seed = cam
    frames = scenes.surveillance_video(gop, h, w, seed=seed)
    plan = B.cs_make_phi(ctx, b * b, m, seed)
    p = B.make_params(h, w, gop, b, m, iters=iters, precision=prec, fp32_tail_iters=tail)
    nblk = (-(-h // b)) * (-(-w // b))
    y = torch.empty((gop - 1, nblk, m), dtype=torch.float32, device="cuda")
    B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
    key = torch.from_numpy(np.ascontiguousarray(frames[:1])).pin_memory()
    # alone: the streaming kernel's own decode of this request
    pa = B.make_params(h, w, gop, b, m, iters=iters, precision=prec, fp32_tail_iters=tail,
                       engine=B.CS_ENGINE_TC_STREAM)
    alone = torch.zeros((gop - 1, h, w), dtype=torch.uint8, device="cuda")
    B.cs_decode_gop(plan, pa, key.cuda(), y, None, alone, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return plan, p, key, y.cpu().pin_memory(), alone.cpu().numpy()


def _submit(B, ctx, cam_state):
    plan, p, key, y_host, _ = cam_state
    out = torch.zeros(y_host.shape[0:1] + key.shape[1:], dtype=torch.uint8).pin_memory()
    while True:
        try:
            return B.cs_submit(ctx, plan, p, key, y_host, out), out
        except B.CsError as e:
            if e.status != B.CS_EAGAIN:
                raise
            time.sleep(0.001)


def _wait(B, ctx, tickets, timeout_s=60.0):
    done_at = {}
    t0 = time.time()
    while len(done_at) < len(tickets):
        for t in tickets:
            if t not in done_at and B.cs_poll(ctx, t)[0]:
                done_at[t] = time.time()
        assert time.time() - t0 < timeout_s
    return done_at


def test_queue_requests_equal_each_alone(B):
    ctx = B.cs_ctx_create(0, BUDGET)
    cams = [_camera(B, ctx, c) for c in CAMERAS]
    try:
        subs = []
        for rep in range(3):                     # 18 requests in flight at once
            for c in cams:
                subs.append(_submit(B, ctx, c))
        _wait(B, ctx, [t for t, _ in subs])
        for i, (_, out) in enumerate(subs):
            assert np.array_equal(out.numpy(), cams[i % len(cams)][4]), "request %d" % i
        B.cs_ctx_status(ctx)
    finally:
        for c in cams:
            B.cs_plan_destroy(c[0])
        B.cs_ctx_destroy(ctx)


def test_request_arriving_while_a_large_one_runs_finishes_first(B):
    ctx = B.cs_ctx_create(0, BUDGET)
    # 720p GOP of 16 frames, 32 x 32 blocks, M = 102, K = 300: 108 tiles, each
    # about 30 ms on the streaming kernel; then a small QCIF request
    big = _camera(B, ctx, (720, 1280, 16, 32, 102, 300, 0, 0, 31))
    small = _camera(B, ctx, (144, 176, 3, 16, 40, 50, 0, 0, 32))
    try:
        tb, out_b = _submit(B, ctx, big)
        time.sleep(0.005)
        assert not B.cs_poll(ctx, tb)[0]         # the large request is on the GPU
        ts, out_s = _submit(B, ctx, small)
        done = _wait(B, ctx, [tb, ts])
        assert done[ts] < done[tb]
        assert np.array_equal(out_b.numpy(), big[4])
        assert np.array_equal(out_s.numpy(), small[4])
        B.cs_ctx_status(ctx)
    finally:
        B.cs_plan_destroy(big[0])
        B.cs_plan_destroy(small[0])
        B.cs_ctx_destroy(ctx)


def test_queue_launch_restarts_after_idle(B):
    ctx = B.cs_ctx_create(0, BUDGET)
    cam = _camera(B, ctx, CAMERAS[0])
    try:
        for _ in range(3):
            t, out = _submit(B, ctx, cam)
            _wait(B, ctx, [t])
            assert np.array_equal(out.numpy(), cam[4])
            time.sleep(0.05)                     # longer than the launch's idle limit
        B.cs_ctx_status(ctx)
    finally:
        B.cs_plan_destroy(cam[0])
        B.cs_ctx_destroy(ctx)
