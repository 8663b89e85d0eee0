"""Serving: requests from several cameras admitted while others are in flight
give, bit for bit, what each request gives decoded alone; admission by slots
and HBM budget; failures (refusal, unknown ticket) reported on the host."""
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


CAMERAS = [  # (h, w, gop, m, iters, precision, tail, seed, block)
    (144, 176, 4, 26, 80, 0, 0, 11, 16),
    (288, 352, 6, 64, 60, 0, 0, 12, 16),
    (96, 128, 8, 13, 100, 3, 20, 13, 16),
    (144, 176, 5, 51, 40, 0, 0, 14, 16),
    (288, 352, 4, 102, 40, 0, 0, 15, 32),    # the 8-CTA cluster kernel
    (160, 192, 3, 200, 30, 0, 0, 16, 32),    # M > 128: the streaming kernel's scratch does not
                                             # fit this context's budget, so the plain kernel
]


def _camera(B, ctx, cam):
    h, w, gop, m, iters, prec, tail, seed = cam[:8]
    b = cam[8] if len(cam) > 8 else 16
    frames = scenes.surveillance_video(gop, h, w, seed=seed)
    plan = B.cs_make_phi(ctx, b * b, m, seed)
    p = B.make_params(h, w, gop, b, m, iters=iters, precision=prec, fp32_tail_iters=tail)
    nblk = (-(-h // b)) * (-(-w // b))
    y = torch.empty((gop - 1, nblk, m), dtype=torch.float32, device="cuda")
    B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
    torch.cuda.synchronize()
    key = torch.from_numpy(np.ascontiguousarray(frames[:1])).pin_memory()
    y_host = y.cpu().pin_memory()
    alone = torch.zeros((gop - 1, h, w), dtype=torch.uint8, device="cuda")
    B.cs_decode_gop(plan, p, key.cuda(), y, None, alone, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return plan, p, key, y_host, alone.cpu().numpy()


def _wait(B, ctx, tickets, timeout_s=30.0):
    lat = {}
    t0 = time.time()
    while len(lat) < len(tickets):
        for t in tickets:
            if t in lat:
                continue
            done, ms = B.cs_poll(ctx, t)
            if done:
                lat[t] = ms
        assert time.time() - t0 < timeout_s
    return lat


def test_requests_in_the_mix_equal_each_request_alone(B):
    ctx = B.cs_ctx_create(0, 256 << 20)
    cams = [_camera(B, ctx, c) for c in CAMERAS]
    try:
        outs, tickets = [], []
        for rep in range(3):                       # 18 requests in flight at once
            for plan, p, key, y_host, _ in cams:
                out = torch.zeros(y_host.shape[0:1] + key.shape[1:], dtype=torch.uint8).pin_memory()
                tickets.append(B.cs_submit(ctx, plan, p, key, y_host, out))
                outs.append(out)
        lat = _wait(B, ctx, tickets)
        assert all(v > 0 for v in lat.values())
        for i, out in enumerate(outs):
            assert np.array_equal(out.numpy(), cams[i % len(cams)][4]), "request %d" % i
        B.cs_ctx_status(ctx)
    finally:
        for c in cams:
            B.cs_plan_destroy(c[0])
        B.cs_ctx_destroy(ctx)


def test_admission_by_hbm_budget_and_slots(B):
    h, w, gop, m = 144, 176, 4, 26
    # budget for about one QCIF request: key 25 KB + y 30 KB + out 76 KB
    ctx = B.cs_ctx_create(0, 160 << 10)
    cam = _camera(B, ctx, (h, w, gop, m, 400, 0, 0, 21))
    plan, p, key, y_host, ref = cam
    try:
        out1 = torch.zeros((gop - 1, h, w), dtype=torch.uint8).pin_memory()
        out2 = torch.zeros((gop - 1, h, w), dtype=torch.uint8).pin_memory()
        t1 = B.cs_submit(ctx, plan, p, key, y_host, out1)
        with pytest.raises(B.CsError) as ei:
            B.cs_submit(ctx, plan, p, key, y_host, out2)
        assert ei.value.status == B.CS_EAGAIN
        _wait(B, ctx, [t1])
        t2 = B.cs_submit(ctx, plan, p, key, y_host, out2)     # memory was returned
        _wait(B, ctx, [t2])
        assert np.array_equal(out1.numpy(), ref) and np.array_equal(out2.numpy(), ref)
        with pytest.raises(B.CsError) as ei:
            B.cs_poll(ctx, t2)                                  # retired
        assert ei.value.status == B.CS_ENOTFOUND
        big = B.make_params(1080, 1920, 4, 16, m, iters=10)
        with pytest.raises(B.CsError) as ei:
            B.cs_submit(ctx, plan, big, np.zeros((1, 1080, 1920), np.uint8),
                        np.zeros((3, 8160, m), np.float32), np.zeros((3, 1080, 1920), np.uint8))
        assert ei.value.status == B.CS_ENOMEM
    finally:
        B.cs_plan_destroy(plan)
        B.cs_ctx_destroy(ctx)

    # slots: 64 requests in flight at most
    ctx = B.cs_ctx_create(0, 512 << 20)
    plan, p, key, y_host, ref = _camera(B, ctx, (48, 64, 2, 16, 3000, 0, 0, 22))
    try:
        outs, tickets = [], []
        refused = 0
        for i in range(70):
            out = torch.zeros((1, 48, 64), dtype=torch.uint8).pin_memory()
            try:
                tickets.append(B.cs_submit(ctx, plan, p, key, y_host, out))
                outs.append(out)
            except B.CsError as e:
                assert e.status == B.CS_EAGAIN
                refused += 1
        assert len(tickets) <= 64 and refused >= 6
        _wait(B, ctx, tickets, timeout_s=120)
        for out in outs:
            assert np.array_equal(out.numpy(), ref)
    finally:
        B.cs_plan_destroy(plan)
        B.cs_ctx_destroy(ctx)
