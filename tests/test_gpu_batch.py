"""cs_decode_batch: one persistent launch over jobs of different plans (M), frame
sizes, GOP sizes, iteration counts and precisions gives, bit for bit, what
cs_decode_gop gives for each job alone; and it matches the FP64 oracle."""
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


JOBS = [  # (h, w, gop, n_gops, block, m, iters, precision, tail, seed)
    (144, 176, 4, 2, 16, 26, 60, 0, 0, 1),
    (288, 352, 8, 1, 16, 128, 40, 0, 0, 2),
    (48, 80, 3, 2, 16, 64, 75, 3, 10, 3),     # FP16 with an FP32-grade tail
    (64, 64, 2, 1, 8, 20, 30, 0, 0, 4),       # 8 x 8 blocks: the plain kernel
    (96, 112, 5, 1, 16, 51, 50, 1, 10, 5),    # BF16: the other operand type
    (40, 56, 4, 1, 16, 77, 20, 0, 0, 6),
]


def _prepare(B, ctx, job):
    h, w, gop, n_gops, b, m, iters, prec, tail, seed = job
    frames = scenes.surveillance_video(gop * n_gops, h, w, seed=seed)
    plan = B.cs_make_phi(ctx, b * b, m, seed)
    p = B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops, precision=prec,
                      fp32_tail_iters=tail)
    nblk = (-(-h // b)) * (-(-w // b))
    f = torch.from_numpy(frames).cuda()
    keys = torch.from_numpy(np.ascontiguousarray(frames[::gop])).cuda()
    y = torch.empty((n_gops * (gop - 1), nblk, m), dtype=torch.float32, device="cuda")
    B.cs_encode_gop(plan, p, f, y, torch.cuda.current_stream())
    return frames, plan, p, keys, y


def test_batch_equals_each_job_alone_and_matches_oracle(B, ctx):
    prepared = [_prepare(B, ctx, j) for j in JOBS]
    try:
        outs_alone, outs_batch = [], []
        for frames, plan, p, keys, y in prepared:
            shape = (y.shape[0], frames.shape[1], frames.shape[2])
            a = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
            B.cs_decode_gop(plan, p, keys, y, a, None, torch.cuda.current_stream())
            outs_alone.append(a)
            outs_batch.append(torch.full(shape, float("nan"), dtype=torch.float32, device="cuda"))
        u8 = [torch.zeros(o.shape, dtype=torch.uint8, device="cuda") for o in outs_batch]
        B.cs_decode_batch(ctx, [x[1] for x in prepared], [x[2] for x in prepared],
                          [x[3] for x in prepared], [x[4] for x in prepared], outs_batch, u8,
                          torch.cuda.current_stream())
        B.cs_ctx_status(ctx)
        for i, (a, bb, uu) in enumerate(zip(outs_alone, outs_batch, u8)):
            a, bb = a.cpu().numpy(), bb.cpu().numpy()
            assert np.array_equal(a.view(np.uint32), bb.view(np.uint32)), "job %d" % i
            assert np.array_equal(uu.cpu().numpy(), np.clip(np.rint(bb), 0, 255).astype(np.uint8))
        # the FP32 jobs also against the oracle
        for i, job in enumerate(JOBS):
            h, w, gop, n_gops, b, m, iters, prec, tail, seed = job
            if prec != 0 or h * w > 50000:
                continue
            frames = prepared[i][0]
            oplan = O.Plan(b * b, m, seed)
            yr = O.encode(oplan, frames, gop)
            ref, _ = O.decode(oplan, frames[::gop], yr, gop, frames.shape[0], iters)
            got = outs_batch[i].cpu().numpy().astype(np.float64)
            err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            print("job %d rel-l2 %.3g" % (i, err))
            assert err <= 1e-4
    finally:
        for x in prepared:
            B.cs_plan_destroy(x[1])


def test_batch_rejects_a_bad_job_and_enqueues_nothing(B, ctx):
    frames, plan, p, keys, y = _prepare(B, ctx, JOBS[0])
    try:
        bad = B.make_params(144, 176, 4, 16, 27, iters=10, n_gops=2)   # M does not match
        out = torch.zeros((6, 144, 176), dtype=torch.float32, device="cuda")
        with pytest.raises(B.CsError) as ei:
            B.cs_decode_batch(ctx, [plan, plan], [p, bad], [keys, keys], [y, y], [out, out])
        assert ei.value.status == B.CS_EINVAL
        assert "job 1" in B.cs_last_error()
    finally:
        B.cs_plan_destroy(plan)
