"""Pins for the oracle's DCT basis, plan (A, L), blocks, residuals and encode.

References: scipy.fft.dctn (orthonormal DCT-II), the DCT definition summed by
hand, LAPACK eigenvalues, explicit pixel loops, and closed forms (zero residual,
linearity).
"""
import math

import numpy as np
import pytest
from scipy.fft import dctn

from oracle import cs_oracle as O
from paper_1311_1419_gb300 import scenes


@pytest.mark.parametrize("b", [2, 4, 8, 16, 32])
def test_dct_orthonormal_and_matches_scipy(b):
    c = O.dct_matrix(b)
    assert np.allclose(c @ c.T, np.eye(b), atol=1e-14)
    psi = O.psi_matrix(b)
    assert np.allclose(psi.T @ psi, np.eye(b * b), atol=1e-13)
    rng = np.random.default_rng(b)
    r = rng.normal(size=(b, b))
    # forward transform s = Psi^T r must be the 2-D orthonormal DCT-II
    assert np.allclose(psi.T @ r.reshape(-1), dctn(r, norm="ortho").reshape(-1), atol=1e-12)


def test_dct_definition_sum_4x4():
    b = 4
    rng = np.random.default_rng(0)
    r = rng.normal(size=(b, b))
    s = np.zeros((b, b))
    for k in range(b):
        for l in range(b):
            ak = math.sqrt((1 if k == 0 else 2) / b)
            al = math.sqrt((1 if l == 0 else 2) / b)
            acc = 0.0
            for p in range(b):
                for q in range(b):
                    acc += r[p, q] * math.cos(math.pi * (2 * p + 1) * k / (2 * b)) * \
                        math.cos(math.pi * (2 * q + 1) * l / (2 * b))
            s[k, l] = ak * al * acc
    psi = O.psi_matrix(b)
    assert np.allclose(psi.T @ r.reshape(-1), s.reshape(-1), atol=1e-13)
    assert np.allclose(psi @ s.reshape(-1), r.reshape(-1), atol=1e-13)


@pytest.mark.parametrize("n,m", [(256, 64), (256, 26), (1024, 102), (64, 16)])
def test_plan_a_rows_are_dct_of_phi_rows_and_l_is_top_eigenvalue(n, m):
    plan = O.Plan(n, m, seed=1)
    b = plan.b
    for i in [0, m // 2, m - 1]:
        want = dctn(plan.phi[i].reshape(b, b), norm="ortho").reshape(-1)
        assert np.allclose(plan.a[i], want, atol=1e-12)
    lam = np.linalg.eigvalsh(plan.phi @ plan.phi.T).max()
    assert abs(plan.lam_max / lam - 1.0) < 1e-9
    # A A^T = Phi Phi^T because Psi is orthonormal, so ||A||_2^2 is the same number
    assert abs(np.linalg.norm(plan.a, 2) ** 2 / lam - 1.0) < 1e-9
    assert plan.lipschitz == pytest.approx(1.0001 * plan.lam_max, rel=1e-15)


def test_plan_rejects_bad_shapes():
    with pytest.raises(ValueError):
        O.Plan(200, 10, 0)
    with pytest.raises(ValueError):
        O.Plan(16, 17, 0)


def test_blockify_matches_pixel_loops_and_roundtrips():
    h, w, b = 37, 45, 8
    rng = np.random.default_rng(4)
    img = rng.integers(-255, 256, size=(h, w)).astype(np.float64)
    blocks = O.blockify(img, b)
    br, bc = O.block_grid(h, w, b)
    assert blocks.shape == (br * bc, b * b) and (br, bc) == (5, 6)
    for bi in range(br):
        for bj in range(bc):
            for p in range(b):
                for q in range(b):
                    y, x = bi * b + p, bj * b + q
                    v = img[y, x] if (y < h and x < w) else 0.0
                    assert blocks[bi * bc + bj, p * b + q] == v
    assert np.array_equal(O.unblockify(blocks, h, w, b), img)


def test_residuals_use_the_gop_key_for_every_cs_frame():
    frames = scenes.surveillance_video(10, 20, 24, seed=3)
    gop = 4
    res = O.residuals(frames, gop)
    cs = O.cs_frame_indices(10, gop)
    assert cs == [1, 2, 3, 5, 6, 7, 9]
    for i, t in enumerate(cs):
        key = (t // gop) * gop
        for y in range(20):
            for x in range(24):
                assert res[i, y, x] == int(frames[t, y, x]) - int(frames[key, y, x])


def test_encode_zero_residual_gives_zero():
    plan = O.Plan(64, 16, seed=0)
    frame = scenes.surveillance_video(1, 30, 30, seed=0)[0]
    frames = np.stack([frame] * 5)
    y = O.encode(plan, frames, gop=5)
    assert y.shape == (4, 16, 16)
    assert np.count_nonzero(y) == 0


def test_encode_is_linear_in_the_residual():
    plan = O.Plan(256, 64, seed=2)
    rng = np.random.default_rng(5)
    r1 = rng.integers(-255, 256, size=(40, 256)).astype(np.float64)
    r2 = rng.integers(-255, 256, size=(40, 256)).astype(np.float64)
    a, c = 3.0, -0.5
    lhs = (a * r1 + c * r2) @ plan.phi.T
    rhs = a * (r1 @ plan.phi.T) + c * (r2 @ plan.phi.T)
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * np.max(np.abs(lhs))


def test_encode_4x4_blocks_by_explicit_loops():
    b, m, gop = 4, 8, 3
    plan = O.Plan(b * b, m, seed=9)
    frames = scenes.surveillance_video(6, 10, 9, seed=1)
    y = O.encode(plan, frames, gop)
    br, bc = O.block_grid(10, 9, b)
    cs = O.cs_frame_indices(6, gop)
    for i, t in enumerate(cs):
        key = frames[(t // gop) * gop].astype(np.int64)
        cur = frames[t].astype(np.int64)
        for bi in range(br):
            for bj in range(bc):
                for row in range(m):
                    acc = 0.0
                    for p in range(b):
                        for q in range(b):
                            yy, xx = bi * b + p, bj * b + q
                            r = (cur[yy, xx] - key[yy, xx]) if (yy < 10 and xx < 9) else 0
                            acc += float(plan.phi32[row, p * b + q]) * r
                    assert y[i, bi * bc + bj, row] == pytest.approx(acc, rel=1e-12, abs=1e-9)
