"""Pins for the oracle's Philox stream, log/sincos and Gaussian Phi.

Independent references: numpy's Philox bit generator (a separate
implementation of Philox4x64-10), mpmath / long-double elementary functions,
scipy's normal CDF and the Marchenko-Pastur edge.
"""
import math

import mpmath
import numpy as np
import pytest
from scipy import stats

from oracle import cs_oracle as O


def _numpy_block(counter_words, key):
    """numpy's Philox emits Philox(c + 1) first when seeded with counter c."""
    value = sum(int(w) << (64 * i) for i, w in enumerate(counter_words))
    bg = np.random.Philox(counter=(value - 1) % (1 << 256), key=np.array(key, dtype=np.uint64))
    return bg.random_raw(4)


@pytest.mark.parametrize("key", [(0, 0), (1, 0), (0xDEADBEEF12345678, 0), (7, 0xFFFFFFFFFFFFFFFF)])
def test_philox_matches_numpy(key):
    rng = np.random.default_rng(1)
    ctrs = rng.integers(0, 2**63, size=(16, 4), dtype=np.uint64) * np.uint64(2) + np.uint64(1)
    ctrs[0] = [0, 0, 0, 0]
    ctrs[1] = [1, 0, 0, 0]
    ctrs[2] = [0, (256 << 16) | 64, 0, 0]
    ctrs[3] = [2**64 - 1, 5, 0, 0]
    got = O.philox4x64_10(ctrs, key)
    for i in range(ctrs.shape[0]):
        want = _numpy_block(ctrs[i], key)
        assert np.array_equal(got[i], want), (i, ctrs[i])


def _ulps(got, want):
    want = np.asarray(want, dtype=np.float64)
    spacing = np.spacing(np.abs(want))
    return np.abs(np.asarray(got) - want) / spacing


def test_log_within_two_ulp():
    rng = np.random.default_rng(2)
    k = rng.integers(1, 2**53 + 1, size=200_000, dtype=np.int64)
    x = k.astype(np.float64) * 2.0 ** -53
    edge = np.array([2.0 ** -53, 0.5, 1.0, 1.0 - 2.0 ** -53, O.SQRT2 / 2, math.sqrt(0.5) + 2 ** -53,
                     0.70710678118654746, 0.70710678118654757, 0.25, 1e-9, 0.999999])
    x = np.concatenate([x, edge])
    ref = np.log(x.astype(np.longdouble)).astype(np.float64)
    got = O.log_fp64(x)
    assert np.max(_ulps(got, ref)) <= 2.0
    assert O.log_fp64(np.array([1.0]))[0] == 0.0
    # mpmath at 100 bits on a subsample, independent of the platform's long double
    mpmath.mp.prec = 100
    for xi, gi in zip(x[:2000], got[:2000]):
        r = float(mpmath.log(mpmath.mpf(float(xi))))
        assert abs(gi - r) <= 2 * np.spacing(abs(r)), xi


def test_sincos_within_two_ulp():
    rng = np.random.default_rng(3)
    k = rng.integers(0, 2**53, size=4000, dtype=np.int64)
    special = np.array([0, 2**50, 2**51, 2**52, 3 * 2**51, 2**53 - 1, 1, 2**49, 5 * 2**50, 7 * 2**50,
                        2**51 - 1, 2**51 + 1, 2**52 + 12345])
    u = np.concatenate([k, special]).astype(np.float64) * 2.0 ** -53
    s, c = O.sincos_2pi(u)
    mpmath.mp.prec = 120
    tp = 2 * mpmath.pi
    for ui, si, ci in zip(u, s, c):
        rs = float(mpmath.sin(tp * mpmath.mpf(float(ui))))
        rc = float(mpmath.cos(tp * mpmath.mpf(float(ui))))
        # 2 ulp of the exact value; the 2^-100 floor covers mpmath's own error
        # at exact quarter turns, where the true value is 0
        assert abs(si - rs) <= 2 * np.spacing(abs(rs)) + 2.0 ** -100, (ui, si, rs)
        assert abs(ci - rc) <= 2 * np.spacing(abs(rc)) + 2.0 ** -100, (ui, ci, rc)
    s0, c0 = O.sincos_2pi(np.array([0.0, 0.25, 0.5, 0.75]))
    assert list(s0) == [0.0, 1.0, 0.0, -1.0]
    assert list(c0) == [1.0, 0.0, -1.0, 0.0]


def test_phi_entry_layout_against_library_box_muller():
    """Entries 2q, 2q+1 of the row-major Phi come from pair q's Philox block."""
    n, m, seed = 256, 64, 5
    phi = O.gaussian_phi(n, m, seed)
    assert phi.shape == (m, n) and phi.dtype == np.float32
    flat = phi.reshape(-1)
    for q in [0, 1, 2, 1000, n * m // 2 - 1]:
        w = O.philox4x64_10(np.array([[q, (n << 16) | m, 0, 0]], dtype=np.uint64), (seed, 0))[0]
        u1 = (int(w[0]) >> 11) + 1
        u2 = int(w[1]) >> 11
        u1 = u1 * 2.0 ** -53
        u2 = u2 * 2.0 ** -53
        rad = math.sqrt(-2.0 * math.log(u1))
        z0 = rad * math.cos(2 * math.pi * u2) / math.sqrt(m)
        z1 = rad * math.sin(2 * math.pi * u2) / math.sqrt(m)
        assert flat[2 * q] == pytest.approx(z0, rel=2e-7, abs=1e-12)
        assert flat[2 * q + 1] == pytest.approx(z1, rel=2e-7, abs=1e-12)


def test_phi_odd_size_and_determinism():
    a = O.gaussian_phi(9, 3, 11)
    b = O.gaussian_phi(9, 3, 11)
    assert a.shape == (3, 9)
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    c = O.gaussian_phi(9, 3, 12)
    assert not np.array_equal(a, c)
    # the plan tag separates (N, M) pairs even under one seed
    d = O.gaussian_phi(9, 4, 11)
    assert not np.array_equal(a.reshape(-1)[:20], d.reshape(-1)[:20])


def test_phi_is_standard_gaussian_after_scaling():
    vals = np.concatenate([O.gaussian_phi(1024, 128, s).reshape(-1) * math.sqrt(128) for s in range(4)])
    vals = vals.astype(np.float64)
    n = vals.size
    assert abs(vals.mean()) < 5 / math.sqrt(n)
    assert abs(vals.var() - 1.0) < 5 * math.sqrt(2.0 / n)
    kurt = np.mean(vals ** 4) / vals.var() ** 2
    assert abs(kurt - 3.0) < 5 * math.sqrt(24.0 / n)
    assert stats.kstest(vals, "norm").pvalue > 1e-4
    # odd moment / symmetry between the cos and sin halves of each pair
    assert abs(np.mean(vals[0::2] * vals[1::2])) < 5 / math.sqrt(n / 2)


def test_phi_spectrum_marchenko_pastur_edge():
    n, m = 1024, 256
    phi = O.gaussian_phi(n, m, 3).astype(np.float64)
    lam = np.linalg.eigvalsh(phi @ phi.T)
    edge = (math.sqrt(n / m) + 1.0) ** 2
    low = (math.sqrt(n / m) - 1.0) ** 2
    assert abs(lam.max() / edge - 1.0) < 0.05
    assert abs(lam.min() / low - 1.0) < 0.15
    assert abs(lam.mean() / (n / m) - 1.0) < 0.02
