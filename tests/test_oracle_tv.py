"""Pins of the oracle's TV recovery (Eq. 1 with the total variation, the TVAL3
choice of Sec. 4) against what the mathematics fixes: the difference operator
against numpy's diff, one augmented-Lagrangian step in closed form, exact
recovery of constant and gradient-sparse residuals, and the minimiser of the
4 x 4 problem solved as a linear program by scipy."""
import numpy as np
import pytest

from oracle import cs_oracle as O


def test_difference_matrix_is_forward_differences_with_zero_last():
    rng = np.random.default_rng(0)
    b = 5
    u = rng.standard_normal((b, b))
    d = O.tv_difference_matrix(b)
    du = d @ u.reshape(-1)
    dx = np.zeros((b, b))
    dy = np.zeros((b, b))
    dx[:, :-1] = np.diff(u, axis=1)
    dy[:-1, :] = np.diff(u, axis=0)
    assert np.array_equal(du[: b * b], dx.reshape(-1))
    assert np.array_equal(du[b * b:], dy.reshape(-1))
    # ||D||^2 <= 8, the bound the step length uses
    assert np.linalg.eigvalsh(d.T @ d).max() <= 8.0


def test_one_step_in_closed_form():
    # from r = nu = lam = 0: w = 0, g = -mu Phi^T y, r1 = alpha mu Phi^T y,
    # nu1 = -beta D r1, lam1 = -mu (Phi r1 - y)
    plan = O.Plan(16, 8, 3)
    rng = np.random.default_rng(1)
    y = rng.standard_normal((2, 8))
    beta, mu = 0.5, 3.0
    r1 = O.tv_adm(plan.phi, y, plan.lipschitz, 1, beta, mu)
    alpha = 1.0 / (8 * beta + mu * plan.lipschitz)
    assert np.allclose(r1, alpha * mu * y @ plan.phi, rtol=1e-13, atol=1e-15)
    # the second step's shrinkage sees D r1 - nu1 / beta = 2 D r1
    d = O.tv_difference_matrix(4)
    dr = r1 @ d.T
    w2 = O.soft(2 * dr, 1 / beta)
    lam1 = -mu * (r1 @ plan.phi.T - y)
    nu1 = -beta * dr
    g2 = (beta * (dr - w2) - nu1) @ d + (mu * (r1 @ plan.phi.T - y) - lam1) @ plan.phi
    r2 = O.tv_adm(plan.phi, y, plan.lipschitz, 2, beta, mu)
    assert np.allclose(r2, r1 - alpha * g2, rtol=1e-12, atol=1e-14)


def test_zero_residual_stays_zero():
    plan = O.Plan(64, 16, 2)
    r = O.tv_adm(plan.phi, np.zeros((3, 16)), plan.lipschitz, 50)
    assert np.array_equal(r, np.zeros((3, 64)))


def test_constant_block_recovered():
    # TV(c 1) = 0 and Phi 1 != 0: the constant block is the unique minimiser
    plan = O.Plan(64, 16, 5)
    truth = np.full((1, 64), 7.0)
    r = O.tv_adm(plan.phi, truth @ plan.phi.T, plan.lipschitz, 20000)
    assert np.abs(r - truth).max() < 1e-6


def test_gradient_sparse_block_recovered():
    # a bright rectangle on a flat background (a mover of the synthetic scenes):
    # 2 levels, a sparse gradient, recovered exactly from M = N/2 measurements
    b = 16
    img = np.zeros((b, b))
    img[3:11, 5:13] = 30.0
    truth = img.reshape(1, -1)
    plan = O.Plan(b * b, 128, 7)
    r = O.tv_adm(plan.phi, truth @ plan.phi.T, plan.lipschitz, 6000)
    assert np.linalg.norm(r - truth) / np.linalg.norm(truth) < 1e-3


def test_4x4_matches_linear_program():
    # min ||D r||_1 s.t. Phi r = y as an LP in (r, s): -s <= D r <= s, min 1^T s
    linprog = pytest.importorskip("scipy.optimize").linprog
    b, m = 4, 8
    n = b * b
    plan = O.Plan(n, m, 11)
    rng = np.random.default_rng(4)
    truth = np.zeros((b, b))
    truth[1:3, 2:4] = 5.0
    truth += 0.3 * rng.standard_normal((b, b))
    y = plan.phi @ truth.reshape(-1)
    d = O.tv_difference_matrix(b)
    k = d.shape[0]
    c = np.concatenate([np.zeros(n), np.ones(k)])
    a_ub = np.block([[d, -np.eye(k)], [-d, -np.eye(k)]])
    b_ub = np.zeros(2 * k)
    a_eq = np.hstack([plan.phi, np.zeros((m, k))])
    res = linprog(c, A_ub=a_ub, b_ub=b_ub, A_eq=a_eq, b_eq=y,
                  bounds=[(None, None)] * n + [(0, None)] * k, method="highs")
    assert res.status == 0
    tv_star = res.fun
    r = O.tv_adm(plan.phi, y[None, :], plan.lipschitz, 40000)[0]
    # the optimal value is unique (the minimiser need not be): compare it, and feasibility
    assert np.abs(d @ r).sum() == pytest.approx(tv_star, rel=1e-4)
    assert np.linalg.norm(plan.phi @ r - y) / np.linalg.norm(y) < 1e-5


def test_tv_decode_adds_back_each_gops_own_key():
    """Two static GOPs with different keys: the residuals are zero, TV recovery
    keeps them zero, and every CS frame decodes to its own GOP's key
    (frame t uses key floor(t/G) G, Sec. 3.2, Eq. 4)."""
    from paper_1311_1419_gb300 import scenes

    plan = O.Plan(64, 16, seed=1)
    keys = scenes.surveillance_video(2, 24, 16, seed=9)
    assert not np.array_equal(keys[0], keys[1])
    gop = 3
    frames = np.stack([keys[0]] * gop + [keys[1]] * gop)
    y = O.encode(plan, frames, gop)
    out = O.decode_tv(plan, keys, y, gop, 2 * gop, 20)
    assert np.array_equal(out[:2], np.stack([keys[0]] * 2).astype(np.float64))
    assert np.array_equal(out[2:], np.stack([keys[1]] * 2).astype(np.float64))


def test_tv_decode_is_key_plus_recovered_residual():
    """With moving content the decoded frame minus its key is the TV recovery of
    that frame's residual blocks, cropped (Eq. 4), for every GOP."""
    from paper_1311_1419_gb300 import scenes

    plan = O.Plan(64, 32, seed=3)
    frames = scenes.surveillance_video(6, 20, 28, seed=4)
    gop = 3
    y = O.encode(plan, frames, gop)
    keys = frames[::gop]
    out = O.decode_tv(plan, keys, y, gop, 6, 15)
    for i, t in enumerate([1, 2, 4, 5]):
        r = O.tv_adm(plan.phi, y[i], plan.lipschitz, 15)
        want = frames[(t // gop) * gop].astype(np.float64) + O.unblockify(r, 20, 28, 8)
        assert np.array_equal(out[i], want)
