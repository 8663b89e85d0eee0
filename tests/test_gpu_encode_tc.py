"""The tensor-core encode against the FP64 oracle and against the SIMT encode,
on every block size (8x8, 16x16 with M <= 128 on the on-chip kernels' Phi
images, 16x16 with M > 128, 32x32; Phi streamed in 64-pixel K chunks): vector
loads and the cropped-edge path, ragged last tiles, every M16 class, several
GOPs."""
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


def _encode(B, plan, frames, gop, m, engine, b=16):
    n_f, h, w = frames.shape
    p = B.make_params(h, w, gop, b, m, n_gops=n_f // gop, engine=engine)
    nblk = (-(-h // b)) * (-(-w // b))
    y = torch.full(((n_f // gop) * (gop - 1), nblk, m), float("nan"), dtype=torch.float32, device="cuda")
    B.cs_encode_gop(plan, p, torch.from_numpy(frames).cuda(), y, torch.cuda.current_stream())
    torch.cuda.synchronize()
    return y.cpu().numpy()


@pytest.mark.parametrize("h,w,gop,n_f,m", [
    (144, 176, 4, 12, 64),     # QCIF: 16-byte loads
    (288, 352, 8, 16, 128),    # CIF, M16 = 128, 2 GOPs: 1386 blocks, ragged last tile
    (100, 90, 3, 6, 26),       # width not a multiple of 16: cropped blocks, byte loads
    (48, 64, 5, 5, 1),         # M = 1
    (40, 56, 2, 4, 77),
])
def test_tc_encode_matches_oracle_and_simt(B, ctx, h, w, gop, n_f, m):
    frames = scenes.surveillance_video(n_f, h, w, seed=4)
    plan = B.cs_make_phi(ctx, 256, m, 2)
    try:
        y_tc = _encode(B, plan, frames, gop, m, B.CS_ENGINE_AUTO)
        y_simt = _encode(B, plan, frames, gop, m, B.CS_ENGINE_PLAIN)
        y_ref = O.encode(O.Plan(256, m, 2), frames, gop)
        err = np.linalg.norm(y_tc - y_ref) / np.linalg.norm(y_ref)
        assert not np.isnan(y_tc).any()
        assert err <= 1e-6, err
        assert np.linalg.norm(y_tc - y_simt) / np.linalg.norm(y_simt) <= 1e-6
    finally:
        B.cs_plan_destroy(plan)


def test_tc_encode_zero_residual_is_exactly_zero(B, ctx):
    key = scenes.surveillance_video(1, 64, 80, seed=2)[0]
    frames = np.stack([key] * 6)
    plan = B.cs_make_phi(ctx, 256, 64, 0)
    try:
        y = _encode(B, plan, frames, 3, 64, B.CS_ENGINE_AUTO)
        assert np.count_nonzero(y) == 0
    finally:
        B.cs_plan_destroy(plan)


@pytest.mark.parametrize("h,w,gop,n_f,b,m", [
    (720, 1280, 16, 16, 32, 102),  # one 720p GOP: 13800 blocks, 32x32, M16 = 112
    (100, 130, 3, 6, 32, 256),     # 32x32, M16 = 256, cropped blocks (byte loads)
    (96, 128, 4, 8, 8, 16),        # 8x8 blocks: one K chunk per block
    (72, 88, 3, 3, 8, 40),         # 8x8, width a multiple of 8 only
    (144, 176, 4, 8, 16, 200),     # 16x16 with M > 128
    (64, 96, 2, 2, 32, 1),         # M = 1
])
def test_general_tc_encode_matches_oracle_and_simt(B, ctx, h, w, gop, n_f, b, m):
    frames = scenes.surveillance_video(n_f, h, w, seed=6)
    plan = B.cs_make_phi(ctx, b * b, m, 3)
    try:
        y_tc = _encode(B, plan, frames, gop, m, B.CS_ENGINE_AUTO, b)
        y_simt = _encode(B, plan, frames, gop, m, B.CS_ENGINE_PLAIN, b)
        y_ref = O.encode(O.Plan(b * b, m, 3), frames, gop)
        assert not np.isnan(y_tc).any()
        # FP32 accumulation over up to 1024 products: within the 1e-5 y tolerance
        err = np.linalg.norm(y_tc - y_ref) / np.linalg.norm(y_ref)
        assert err <= 1e-5, err
        assert np.linalg.norm(y_tc - y_simt) / np.linalg.norm(y_simt) <= 1e-5
    finally:
        B.cs_plan_destroy(plan)
