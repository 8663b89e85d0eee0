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
