"""Pins for the oracle's recovery (Eq. 1 read as l1-DCT LASSO, solved by FISTA),
the add-back of Eq. (4), the multiple-residual identity of Eqs. (2)-(4), the
Table I compression ratios and PSNR.

References: LAPACK linear solves, brute-force enumeration of LASSO supports and
signs with their KKT conditions, exactly sparse signals, closed forms.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import cs_oracle as O
from paper_1311_1419_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_cr.txt")


def test_zero_residual_decodes_to_the_key_exactly():
    plan = O.Plan(256, 64, seed=0)
    key = scenes.surveillance_video(1, 40, 50, seed=7)[0]
    frames = np.stack([key] * 4)
    y = O.encode(plan, frames, gop=4)
    out_f, out_u8 = O.decode(plan, key[None], y, gop=4, n_frames=4, iters=50)
    assert np.array_equal(out_f, np.stack([key.astype(np.float64)] * 3))
    assert np.array_equal(out_u8, frames[1:])


def test_each_gop_adds_back_its_own_key():
    """Two static GOPs with different keys: every CS frame decodes to its own
    GOP's key (frame t uses key floor(t/G) G, Sec. 3.2)."""
    plan = O.Plan(64, 16, seed=1)
    keys = scenes.surveillance_video(2, 24, 16, seed=9)
    gop = 3
    frames = np.stack([keys[0]] * gop + [keys[1]] * gop)
    y = O.encode(plan, frames, gop)
    out_f, _ = O.decode(plan, keys, y, gop=gop, n_frames=2 * gop, iters=10)
    assert np.array_equal(out_f[:2], np.stack([keys[0]] * 2).astype(np.float64))
    assert np.array_equal(out_f[2:], np.stack([keys[1]] * 2).astype(np.float64))


@pytest.mark.parametrize("k", [2, 4, 8])
def test_exactly_sparse_dct_residual_is_recovered(k):
    plan = O.Plan(256, 64, seed=11)
    rng = np.random.default_rng(k)
    s_true = np.zeros(256)
    support = rng.choice(256, size=k, replace=False)
    s_true[support] = rng.choice([-1.0, 1.0], size=k) * rng.uniform(20, 60, size=k)
    y = plan.a @ s_true
    lam = O.block_lambda(plan.a, y[None], 1e-4)
    s_hat = O.fista(plan.a, y[None], plan.lipschitz, lam, 5000)[0]
    found = np.flatnonzero(np.abs(s_hat) > 1e-3 * np.abs(s_true).max())
    assert set(found) == set(support)
    assert np.linalg.norm(s_hat - s_true) <= 1e-3 * np.linalg.norm(s_true)
    # the same through the pixel domain: r = Psi s, recovered as Psi s_hat
    r_hat = O.decode_blocks(plan, y[None], 5000, lambda_rel=1e-4)[0]
    assert np.linalg.norm(r_hat - plan.psi @ s_true) <= 1e-3 * np.linalg.norm(s_true)


def test_square_a_with_zero_lambda_reduces_to_a_linear_solve():
    n = 16
    plan = O.Plan(n, n, seed=4)
    rng = np.random.default_rng(6)
    y = rng.normal(size=(3, n)) * 10
    s = O.fista(plan.a, y, plan.lipschitz, np.zeros(3), 60000)
    want = np.linalg.solve(plan.a, y.T).T
    assert np.max(np.abs(s - want)) <= 1e-8 * np.max(np.abs(want))


def _lasso_brute_force(a, y, lam):
    """Every (support, sign) candidate whose KKT conditions hold."""
    m, n = a.shape
    found = []
    if np.max(np.abs(a.T @ y)) <= lam:
        found.append(np.zeros(n))
    for k in range(1, m + 1):
        signs = np.array(list(itertools.product([-1.0, 1.0], repeat=k)))  # [2^k][k]
        for supp in itertools.combinations(range(n), k):
            a_s = a[:, supp]
            gram = a_s.T @ a_s
            rhs = (a_s.T @ y)[:, None] - lam * signs.T               # [k][2^k]
            sol = np.linalg.solve(gram, rhs)                          # [k][2^k]
            ok = np.all(np.sign(sol) == signs.T, axis=0)
            for j in np.flatnonzero(ok):
                x = np.zeros(n)
                x[list(supp)] = sol[:, j]
                corr = a.T @ (y - a @ x)
                off = np.setdiff1d(np.arange(n), supp)
                if off.size == 0 or np.max(np.abs(corr[off])) <= lam * (1 + 1e-12):
                    found.append(x)
    return found


def test_fista_matches_brute_force_lasso_on_a_4x4_block():
    plan = O.Plan(16, 8, seed=21)
    rng = np.random.default_rng(8)
    r = rng.integers(-40, 41, size=16).astype(np.float64)
    y = plan.phi @ r
    lam = 0.1 * np.max(np.abs(plan.a.T @ y))
    cands = _lasso_brute_force(plan.a, y, lam)
    assert len(cands) == 1
    s = O.fista(plan.a, y[None], plan.lipschitz, np.array([lam]), 20000)[0]
    assert np.max(np.abs(s - cands[0])) <= 1e-8 * max(1.0, np.max(np.abs(cands[0])))


def test_fista_result_satisfies_lasso_kkt():
    plan = O.Plan(256, 64, seed=3)
    frames = scenes.surveillance_video(2, 32, 32, seed=2)
    y = O.encode(plan, frames, gop=2)[0]
    lam = O.block_lambda(plan.a, y, 0.01)
    s = O.fista(plan.a, y, plan.lipschitz, lam, 20000)
    corr = (y - s @ plan.a.T) @ plan.a                   # A^T (y - A s) per block
    for b in range(y.shape[0]):
        on = np.abs(s[b]) > 0
        scale = max(lam[b], 1e-12)
        assert np.all(np.abs(corr[b][~on]) <= lam[b] + 1e-6 * scale)
        assert np.allclose(corr[b][on], lam[b] * np.sign(s[b][on]), atol=1e-6 * scale, rtol=0)


def test_fista_first_step_by_hand():
    """One FISTA iteration from zero, written out for a 2-coefficient problem."""
    a = np.array([[1.0, 2.0], [0.5, -1.0]])
    y = np.array([[3.0, 1.0]])
    lip = 7.0
    lam = np.array([0.7])
    s1 = O.fista(a, y, lip, lam, 1)[0]
    g = a.T @ (a @ np.zeros(2) - y[0])                  # = -A^T y
    v = -g / lip
    want = np.sign(v) * np.maximum(np.abs(v) - lam[0] / lip, 0)
    assert np.allclose(s1, want, atol=0, rtol=1e-15)
    # two iterations: t_2 = (1 + sqrt 5)/2, momentum (t_1 - 1)/t_2 = 0 on step 1
    s2 = O.fista(a, y, lip, lam, 2)[0]
    z2 = want
    g2 = a.T @ (a @ z2 - y[0])
    v2 = z2 - g2 / lip
    want2 = np.sign(v2) * np.maximum(np.abs(v2) - lam[0] / lip, 0)
    assert np.allclose(s2, want2, atol=0, rtol=1e-14)


def test_multiple_residual_cancels_key_error_eqs_2_to_4():
    """Encoding against the reconstructed key F'_key = F_key + e (Eq. 2) and
    adding the recovered residual back to the same F'_key (Eq. 4) leaves
    F'_t - F_t equal to the CS recovery error alone (Eq. 3): no e term."""
    plan = O.Plan(16, 16, seed=4)            # M = N, lambda = 0: exact recovery (cond(A) = 12)
    frames = scenes.surveillance_video(4, 16, 24, seed=4)
    rng = np.random.default_rng(1)
    e_key = rng.integers(-6, 7, size=frames.shape[1:])
    key_rec = np.clip(frames[0].astype(np.int64) + e_key, 0, 255).astype(np.uint8)
    coded = frames.copy()
    coded[0] = key_rec                          # the encoder subtracts F'_key
    y = O.encode(plan, coded, gop=4)
    out_f, _ = O.decode(plan, key_rec[None], y, gop=4, n_frames=4, iters=5000,
                        lambda_rel=0.0)
    assert np.max(np.abs(out_f - frames[1:].astype(np.float64))) < 1e-6
    # with the original key at the encoder but F'_key at the decoder the key
    # error does show up: F'_t - F_t = (F'_key - F_key)
    y_orig = O.encode(plan, frames, gop=4)
    out_bad, _ = O.decode(plan, key_rec[None], y_orig, gop=4, n_frames=4, iters=5000,
                          lambda_rel=0.0)
    diff = out_bad - frames[1:].astype(np.float64)
    assert np.allclose(diff, (key_rec.astype(np.int64) - frames[0].astype(np.int64))[None], atol=1e-6)


def test_multiple_residual_with_lossy_recovery_error_is_the_residual_error():
    """With lambda > 0 recovery is lossy; Eq. (4) still holds exactly: the frame
    error equals the error of the recovered residual D'_N."""
    plan = O.Plan(256, 64, seed=6)
    frames = scenes.surveillance_video(3, 32, 48, seed=8)
    y = O.encode(plan, frames, gop=3)
    out_f, _ = O.decode(plan, frames[0][None], y, gop=3, n_frames=3, iters=100)
    for i, t in enumerate([1, 2]):
        r_true = frames[t].astype(np.float64) - frames[0].astype(np.float64)
        r_hat = O.unblockify(O.decode_blocks(plan, y[i], 100), 32, 48, plan.b)
        assert np.allclose(out_f[i] - frames[t], r_hat - r_true, atol=1e-9)


def test_table_i_total_cr():
    rows = [list(map(float, ln.split())) for ln in open(GOLDEN) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 9
    for gop, cr_key, cr_cs, want in rows:
        assert round(O.total_cr(int(gop), cr_key, cr_cs), 2) == pytest.approx(want, abs=1e-9)


def test_raw_key_cr_closed_forms():
    assert O.raw_key_cr(4, 144, 176, 16, 64) == pytest.approx(4 / (1 + 3 * 0.25))
    assert round(O.raw_key_cr(4, 144, 176, 16, 64), 3) == 2.286
    assert round(O.raw_key_cr(8, 288, 352, 16, 26), 3) == 4.676
    assert round(O.raw_key_cr(16, 720, 1280, 32, 102), 3) == 6.331
    # every pixel per block at M = N and G = 1 + 1: CR = 1 when blocks tile the frame
    assert O.raw_key_cr(2, 32, 32, 16, 256) == pytest.approx(1.0)


def test_psnr_closed_form_and_uint8_rounding():
    ref = np.full((4, 4), 100, dtype=np.uint8)
    test = ref.astype(np.float64) + 5.0
    assert O.psnr(ref, test) == pytest.approx(10 * math.log10(255 ** 2 / 25.0))
    assert O.psnr(ref, ref) == math.inf
    x = np.array([-3.0, 0.5, 1.5, 2.5, 254.5, 255.4, 300.0])
    assert list(O.to_uint8(x)) == [0, 0, 2, 2, 254, 255, 255]


def test_block_lambda_by_explicit_loops():
    """lambda_b = lambda_rel * max_j |sum_i A_ij y_bi| on a hand-built 3 x 4 A.
    The second row's largest entry of A^T y is negative, so a maximum taken
    without the absolute value gives a different number."""
    a = np.array([[1.0, -2.0, 0.5, 3.0],
                  [0.0, 4.0, -1.0, 1.0],
                  [2.0, 1.0, 1.0, -0.5]])
    y = np.array([[1.0, 1.0, 1.0],
                  [0.0, -3.0, 0.5]])
    want = []
    for b in range(y.shape[0]):
        best = 0.0
        for j in range(a.shape[1]):
            acc = 0.0
            for i in range(a.shape[0]):
                acc += a[i, j] * y[b, i]
            best = max(best, abs(acc))
        want.append(0.01 * best)
    # A^T y_0 = (3, 3, 0.5, 3.5); A^T y_1 = (1, -11.5, 3.5, -3.25)
    assert want == pytest.approx([0.035, 0.115], abs=1e-15)
    assert np.array_equal(O.block_lambda(a, y, 0.01), np.array(want))


def test_lambda_at_the_lasso_threshold_gives_the_zero_solution():
    """For the LASSO, s = 0 is optimal exactly when lambda >= ||A^T y||_inf (the
    subgradient condition at 0).  So lambda_rel = 1 must decode every block to
    zero, and lambda_rel just below 1 must leave the coefficient of largest
    |A^T y| nonzero: a norm other than the max-abs one fails one of the two."""
    plan = O.Plan(64, 16, seed=12)
    frames = scenes.surveillance_video(2, 24, 24, seed=5)
    y = O.encode(plan, frames, gop=2)[0]                  # 9 blocks of 8 x 8
    corr = y @ plan.a                                     # A^T y per block
    assert np.any(np.argmax(corr, axis=1) != np.argmax(np.abs(corr), axis=1))
    s_at = O.fista(plan.a, y, plan.lipschitz, O.block_lambda(plan.a, y, 1.0), 200)
    assert np.array_equal(s_at, np.zeros_like(s_at))
    assert np.array_equal(O.decode_blocks(plan, y, 200, lambda_rel=1.0), np.zeros((9, 64)))
    s_below = O.fista(plan.a, y, plan.lipschitz, O.block_lambda(plan.a, y, 0.999), 200)
    top = np.argmax(np.abs(corr), axis=1)
    assert np.all(s_below[np.arange(9), top] != 0.0)
    # at lambda_rel = 0.01 the decode is the FISTA run with the loop-built lambda
    lam = np.array([0.01 * max(abs(sum(plan.a[i, j] * y[b, i] for i in range(16)))
                               for j in range(64)) for b in range(9)])
    want = O.fista(plan.a, y, plan.lipschitz, lam, 60) @ plan.psi.T
    assert np.allclose(O.decode_blocks(plan, y, 60, lambda_rel=0.01), want, rtol=0, atol=1e-9)
