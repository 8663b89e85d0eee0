"""GPU path vs the FP64 oracle, through the C ABI, on seeded synthetic inputs.

Bars: Phi bit-exact; y relative l2 <= 1e-5; recovered frames relative l2 <=
1e-4 and PSNR within 0.01 dB (FP32 decode); uint8 frames are the float frames
rounded, and differ from the oracle's only at rounding ties within the float
error.
"""
import math

import numpy as np
import pytest

from oracle import cs_oracle as O
from paper_1311_1419_gb300 import scenes

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

Y_TOL = 1e-5
F_TOL = 1e-4
PSNR_TOL = 0.01


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


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


class _DeviceView:
    """A borrowed device buffer exposed through __cuda_array_interface__."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3}


def dev_array(ptr, shape, dtype):
    """Copy a library-owned float32 device buffer into a numpy array."""
    assert dtype == torch.float32
    view = torch.as_tensor(_DeviceView(ptr, shape, "<f4"), device="cuda")
    return view.clone().cpu().numpy()


def gpu_encode(B, plan, frames, gop, b, m):
    n_f, h, w = frames.shape
    n_gops = n_f // gop
    nblk = (-(-h // b)) * (-(-w // b))
    p = B.make_params(h, w, gop, b, m, n_gops=n_gops)
    f = torch.from_numpy(frames).cuda()
    y = torch.full((n_gops * (gop - 1), nblk, m), float("nan"), dtype=torch.float32, device="cuda")
    B.cs_encode_gop(plan, p, f, y, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return y


def gpu_decode(B, plan, frames, y, gop, b, m, iters, lambda_rel=0.01, engine=0, precision=0):
    n_f, h, w = frames.shape
    n_gops = n_f // gop
    p = B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops, lambda_rel=lambda_rel,
                      engine=engine, precision=precision)
    keys = torch.from_numpy(np.ascontiguousarray(frames[::gop])).cuda()
    out_f = torch.full((n_gops * (gop - 1), h, w), float("nan"), dtype=torch.float32, device="cuda")
    out_u = torch.zeros((n_gops * (gop - 1), h, w), dtype=torch.uint8, device="cuda")
    B.cs_decode_gop(plan, p, keys, y, out_f, out_u, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out_f.cpu().numpy(), out_u.cpu().numpy()


@pytest.mark.parametrize("n,m,seed", [(256, 64, 0), (256, 26, 0), (256, 51, 0), (256, 77, 0),
                                      (256, 128, 0), (1024, 102, 0), (9, 3, 11), (16, 16, 4),
                                      (64, 5, 2**63 + 12345), (4096, 1, 7)])
def test_phi_bit_exact_and_plan(B, ctx, n, m, seed):
    plan = B.cs_make_phi(ctx, n, m, seed)
    try:
        phi = dev_array(B.cs_plan_phi(plan), (m, n), torch.float32)
        ref = O.gaussian_phi(n, m, seed)
        assert np.array_equal(phi.view(np.uint32), ref.view(np.uint32))
        if n <= 1024:
            oplan = O.Plan(n, m, seed)
            a = dev_array(B.cs_plan_a(plan), (m, n), torch.float32)
            assert rel_l2(a, oplan.a) <= 2e-7
            assert B.cs_plan_lipschitz(plan) == pytest.approx(oplan.lipschitz, rel=1e-10)
    finally:
        B.cs_plan_destroy(plan)


@pytest.mark.parametrize("h,w,gop,n_f,b,m", [(144, 176, 4, 12, 16, 64), (37, 45, 3, 6, 8, 20),
                                             (20, 33, 2, 2, 4, 16), (64, 96, 5, 10, 32, 102)])
def test_encode_matches_oracle(B, ctx, h, w, gop, n_f, b, m):
    frames = scenes.surveillance_video(n_f, h, w, seed=1)
    plan = B.cs_make_phi(ctx, b * b, m, 0)
    try:
        y = gpu_encode(B, plan, frames, gop, b, m).cpu().numpy()
        oplan = O.Plan(b * b, m, 0)
        y_ref = O.encode(oplan, frames, gop)
        assert y.shape == y_ref.shape
        assert rel_l2(y, y_ref) <= Y_TOL
    finally:
        B.cs_plan_destroy(plan)


def test_encode_zero_residual_is_exactly_zero(B, ctx):
    key = scenes.surveillance_video(1, 50, 70, seed=2)[0]
    frames = np.stack([key] * 6)
    plan = B.cs_make_phi(ctx, 256, 64, 0)
    try:
        y = gpu_encode(B, plan, frames, 3, 16, 64).cpu().numpy()
        assert np.count_nonzero(y) == 0
    finally:
        B.cs_plan_destroy(plan)


def _decode_case(B, ctx, h, w, gop, n_f, b, m, iters, seed=0, engine=0, lambda_rel=0.01):
    frames = scenes.surveillance_video(n_f, h, w, seed=seed)
    plan = B.cs_make_phi(ctx, b * b, m, 0)
    try:
        y = gpu_encode(B, plan, frames, gop, b, m)
        out_f, out_u = gpu_decode(B, plan, frames, y, gop, b, m, iters, lambda_rel, engine)
    finally:
        B.cs_plan_destroy(plan)
    oplan = O.Plan(b * b, m, 0)
    y_ref = O.encode(oplan, frames, gop)
    ref_f, ref_u = O.decode(oplan, frames[::gop], y_ref, gop, n_f, iters, lambda_rel)
    return frames, out_f, out_u, ref_f, ref_u


def _check_frames(frames, gop, out_f, out_u, ref_f, ref_u, f_tol=F_TOL, psnr_tol=PSNR_TOL):
    assert rel_l2(out_f, ref_f) <= f_tol
    orig = frames[[t for t in range(frames.shape[0]) if t % gop]]
    assert abs(O.psnr(orig, out_f) - O.psnr(orig, ref_f)) <= psnr_tol
    # uint8: the GPU's own float frame rounded half-even and clamped, bit for
    # bit; it differs from the oracle's only where the FP64 value lies within
    # the float error of a rounding tie, and then by one level
    assert np.array_equal(out_u, np.clip(np.rint(out_f), 0, 255).astype(np.uint8))
    diff = out_u.astype(np.int64) - ref_u.astype(np.int64)
    dist_to_tie = np.abs(np.abs(ref_f - np.floor(ref_f)) - 0.5)
    allowed = dist_to_tie <= np.abs(out_f.astype(np.float64) - ref_f) + 1e-6
    assert np.all((diff == 0) | (allowed & (np.abs(diff) == 1)))


@pytest.mark.parametrize("engine", [1, 0])
def test_decode_qcif_matches_oracle(B, ctx, engine):
    """QCIF 176x144, 12 frames, GOP 4, B 16, M 64, 200 iterations."""
    frames, out_f, out_u, ref_f, ref_u = _decode_case(B, ctx, 144, 176, 4, 12, 16, 64, 200,
                                                      engine=engine)
    _check_frames(frames, 4, out_f, out_u, ref_f, ref_u)


@pytest.mark.parametrize("h,w,gop,n_f,b,m,iters", [
    (37, 45, 3, 6, 8, 20, 60),       # ragged frame, 8x8 blocks
    (20, 33, 2, 2, 4, 16, 300),      # 4x4 blocks, M = N
    (64, 96, 3, 3, 32, 102, 80),     # 32x32 blocks (N = 1024)
    (16, 16, 2, 2, 16, 1, 10),       # M = 1
    (30, 40, 4, 4, 16, 64, 0),       # zero iterations: output is the key
])
def test_decode_edge_shapes(B, ctx, h, w, gop, n_f, b, m, iters):
    frames, out_f, out_u, ref_f, ref_u = _decode_case(B, ctx, h, w, gop, n_f, b, m, iters)
    _check_frames(frames, gop, out_f, out_u, ref_f, ref_u)


def test_decode_zero_residual_returns_key_exactly(B, ctx):
    key = scenes.surveillance_video(1, 48, 64, seed=5)[0]
    frames = np.stack([key] * 4)
    plan = B.cs_make_phi(ctx, 256, 64, 0)
    try:
        y = gpu_encode(B, plan, frames, 4, 16, 64)
        out_f, out_u = gpu_decode(B, plan, frames, y, 4, 16, 64, 50)
    finally:
        B.cs_plan_destroy(plan)
    assert np.array_equal(out_f, np.stack([key] * 3).astype(np.float32))
    assert np.array_equal(out_u, frames[1:])


def test_decode_lambda_zero(B, ctx):
    frames, out_f, out_u, ref_f, ref_u = _decode_case(B, ctx, 32, 48, 2, 2, 16, 64, 100,
                                                      lambda_rel=0.0)
    _check_frames(frames, 2, out_f, out_u, ref_f, ref_u)


def test_psnr_kernel_matches_oracle(B, ctx):
    rng = np.random.default_rng(0)
    ref = rng.integers(0, 256, size=(3, 37, 45), dtype=np.uint8)
    test = ref.astype(np.float32) + rng.normal(0, 3, size=ref.shape).astype(np.float32)
    test[2] = ref[2]
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    B.cs_psnr(torch.from_numpy(ref).cuda(), torch.from_numpy(test).cuda(), 3, 37, 45, out,
              torch.cuda.current_stream())
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i in range(2):
        assert got[i] == pytest.approx(O.psnr(ref[i], test[i]), abs=1e-9)
    assert math.isinf(got[2])


def test_argument_errors(B, ctx):
    plan = B.cs_make_phi(ctx, 256, 64, 0)
    try:
        f = torch.zeros((4, 32, 32), dtype=torch.uint8, device="cuda")
        y = torch.zeros((3, 4, 64), dtype=torch.float32, device="cuda")
        for bad in [B.make_params(32, 32, 4, 8, 64), B.make_params(32, 32, 4, 16, 63),
                    B.make_params(32, 32, 1, 16, 64), B.make_params(0, 32, 4, 16, 64)]:
            with pytest.raises(B.CsError) as ei:
                B.cs_encode_gop(plan, bad, f, y)
            assert ei.value.status == B.CS_EINVAL
        with pytest.raises(B.CsError) as ei:
            B.cs_decode_gop(plan, B.make_params(32, 32, 4, 16, 64), f[0:1], y, None, None)
        assert ei.value.status == B.CS_EINVAL
        with pytest.raises(B.CsError) as ei:
            B.cs_decode_gop(plan, B.make_params(32, 32, 4, 16, 64, iters=-1), f[0:1], y, y)
        assert ei.value.status == B.CS_EINVAL
    finally:
        B.cs_plan_destroy(plan)
    for n, m in [(200, 10), (256, 0), (256, 257)]:
        with pytest.raises(B.CsError) as ei:
            B.cs_make_phi(ctx, n, m, 0)
        assert ei.value.status == B.CS_EINVAL
