"""The CR-PSNR configurability sweep (Table I, Fig. 5 and Fig. 6 shapes) runs
through the library: its total-CR column is Table I's closed form of the
oracle, and PSNR falls with distance from the key frame inside a GOP."""
import numpy as np
import pytest

from oracle import cs_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1311_1419_gb300 import binding as B
    c = B.cs_ctx_create(0)
    yield c
    B.cs_ctx_destroy(c)


def test_table1_shape_total_cr_matches_the_closed_form(ctx):
    from paper_1311_1419_gb300 import sweep
    rows = sweep.table1_shape(ctx, iters=20, gops=(3, 5), crs=(40, 80), n_gops=2)
    assert len(rows) == 4
    for r in rows:
        m = r["m"]
        assert m == max(1, int(np.rint(256 / int(r["rate"].split(":")[1]))))
        assert abs(r["total_cr_table_i"] - O.total_cr(r["gop"], 23.0, 256 / m)) < 1e-9
        assert abs(r["total_cr_raw_key"] - O.raw_key_cr(r["gop"], 144, 176, 16, m)) < 1e-9
        assert 15.0 < r["psnr_cs_db"] < 60.0


def test_fig5_shape_psnr_decays_within_the_gop(ctx):
    from paper_1311_1419_gb300 import sweep
    f5 = sweep.fig5_shape(ctx, iters=40, n_gops=4)
    p = f5["psnr_by_position_db"]
    assert len(p) == 4
    assert all(a > b for a, b in zip(p, p[1:])), p


def _vs_oracle(frames, dec, gop, m, iters):
    """Frame rel-l2 and PSNR difference of the library's decode against the FP64
    oracle's decode of the same clip, plan and iteration count."""
    plan = O.Plan(256, m, 0)
    y = O.encode(plan, frames, gop)
    want, _ = O.decode(plan, frames[::gop], y, gop, frames.shape[0], iters)
    cs = O.cs_frame_indices(frames.shape[0], gop)
    rel = np.linalg.norm(dec - want) / np.linalg.norm(want)
    dpsnr = O.psnr(frames[cs], dec) - O.psnr(frames[cs], want)
    return rel, dpsnr


def test_table1_shape_decodes_match_the_oracle(ctx):
    """Every decode of the Table I shape (GOP 3, 5, 7 x rate 23:40, 23:60, 23:80,
    i.e. M = 6, 4, 3 measurements per 16 x 16 block, K = 200) equals the
    oracle's within the FP32 tolerance: frame rel-l2 <= 1e-4, PSNR within 0.01 dB."""
    from paper_1311_1419_gb300 import sweep
    rows = sweep.table1_shape(ctx, iters=200, n_gops=2, keep_frames=True)
    assert sorted({r["m"] for r in rows}) == [3, 4, 6]
    for r in rows:
        rel, dpsnr = _vs_oracle(r["frames"], r["decoded"], r["gop"], r["m"], 200)
        assert rel <= 1e-4, (r["gop"], r["m"], rel)
        assert abs(dpsnr) <= 0.01, (r["gop"], r["m"], dpsnr)


def test_fig5_shape_decode_matches_the_oracle(ctx):
    """The Fig. 5 shape (1 key + 4 CS frames, CR_cs 50, M = 5, K = 200)."""
    from paper_1311_1419_gb300 import sweep
    f5 = sweep.fig5_shape(ctx, iters=200, n_gops=3, keep_frames=True)
    assert f5["m"] == 5
    rel, dpsnr = _vs_oracle(f5["frames"], f5["decoded"], 5, 5, 200)
    assert rel <= 1e-4 and abs(dpsnr) <= 0.01, (rel, dpsnr)
