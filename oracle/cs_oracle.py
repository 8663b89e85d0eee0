"""Plain FP64 CPU oracle of the multiple-residual block-CS codec hot path.

TEST INFRASTRUCTURE ONLY.  This module is the correctness reference for the
CUDA library.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import or call it; the library and its Python binding
never do, and it shares no code, constant table or helper with them.  It is
deliberately slow and written to be checked against the paper by eye.

Paper: "Increasing compression ratio of low complexity compressive sensing
video encoder with application-aware configurable mechanism" (Yu, Qiao, Luo,
Yang, arXiv 1311.1419).

What each function follows
--------------------------
* GOP split, key frame + CS frames, every CS frame minus the SAME key frame
  (the multiple-residual scheme): Sec. 3 intro, Sec. 3.1, Sec. 3.2 and
  Eqs. (2)-(4).  Key frames pass raw (no intra codec), so the reconstructed key
  equals the original key.
* Gaussian random measurement matrix, each CS frame measured separately:
  Sec. 1 (Fig. 1 text), Sec. 3.1, Sec. 4.  Measurement per B x B block with one
  matrix Phi of shape M x N (N = B^2) shared by all blocks: y_b = Phi r_b.
* Sparse recovery, Eq. (1): min Phi(x) s.t. Ax = y with the regulariser left
  generic.  Read as the l1-regularised least-squares problem in the orthonormal
  2-D DCT basis, min_s 1/2 ||A s - y||^2 + lambda ||s||_1 with A = Phi Psi,
  solved by FISTA (Beck & Teboulle, SIAM J. Imaging Sci. 2009) for a fixed
  number of iterations.
* The paper's own recovery, TVAL3 (Sec. 4): Eq. (1) with Phi(x) the total
  variation of the residual block, min TV(r) s.t. Phi r = y, by the augmented
  Lagrangian / alternating-direction scheme of Li, Yin, Jiang and Zhang
  (Comput. Optim. Appl. 2013), read as: anisotropic TV with forward differences
  (zero at the last row and column), one shrinkage step for the splitting
  variable w, one gradient step of fixed length 1 / (8 beta + mu L) for r and
  one update of each multiplier per iteration, a fixed number of iterations.
* Add the recovered residual back to the key frame: Sec. 3.2, Eq. (4).
* Total compression ratio of a GOP: Sec. 3.1 and Table I (Sec. 4).

Readings of points the paper leaves open (all listed in the design notes):
Phi ~ N(0, 1/M) drawn by Philox4x64-10 + Box-Muller with the log and sincos
algorithms defined below; lambda_b = lambda_rel * ||A^T y_b||_inf per block;
step 1/L with L = 1.0001 * lambda_max(Phi Phi^T) from 1000 FP64 power
iterations; residuals zero-padded to whole blocks; uint8 output by
round-half-even and clamp.

Pinned by ``tests/test_oracle_*.py`` against numpy's Philox, long-double
sin/cos/log, scipy's DCT, LAPACK eigenvalues and solves, brute-force LASSO
enumeration, a linear-programming solution of the TV problem, closed forms and
the Table I compression ratios.
"""
from __future__ import annotations

import math

import numpy as np

# ---------------------------------------------------------------------------
# Philox4x64-10, counter-based generator of Salmon, Moraes, Dror and Shaw,
# "Parallel random numbers: as easy as 1, 2, 3" (SC'11).  Round function:
#   (hi0, lo0) = M0 * X0,  (hi1, lo1) = M1 * X2   (full 128-bit products)
#   X <- (hi1 ^ X1 ^ K0,  lo1,  hi0 ^ X3 ^ K1,  lo0)
# with the key bumped by the Weyl increments (W0, W1) between rounds.
# ---------------------------------------------------------------------------
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B
PHILOX_ROUNDS = 10
_MASK32 = np.uint64(0xFFFFFFFF)
_SH32 = np.uint64(32)


def _mulhilo64(a: int, b: np.ndarray):
    """(high, low) 64-bit halves of the 128-bit product a*b, b a uint64 array."""
    a_lo = np.uint64(a & 0xFFFFFFFF)
    a_hi = np.uint64(a >> 32)
    b_lo = b & _MASK32
    b_hi = b >> _SH32
    ll = a_lo * b_lo
    hl = a_hi * b_lo
    lh = a_lo * b_hi
    hh = a_hi * b_hi
    cross = (ll >> _SH32) + (hl & _MASK32) + (lh & _MASK32)
    lo = (ll & _MASK32) | (cross << _SH32)
    hi = hh + (hl >> _SH32) + (lh >> _SH32) + (cross >> _SH32)
    return hi, lo


def philox4x64_10(counter: np.ndarray, key) -> np.ndarray:
    """Philox4x64-10 blocks for counters [n][4] (uint64) under key (k0, k1)."""
    x = [np.array(counter[:, i], dtype=np.uint64) for i in range(4)]
    k0, k1 = int(key[0]), int(key[1])
    with np.errstate(over="ignore"):
        for _ in range(PHILOX_ROUNDS):
            hi0, lo0 = _mulhilo64(PHILOX_M0, x[0])
            hi1, lo1 = _mulhilo64(PHILOX_M1, x[2])
            x = [hi1 ^ x[1] ^ np.uint64(k0), lo1, hi0 ^ x[3] ^ np.uint64(k1), lo0]
            k0 = (k0 + PHILOX_W0) & 0xFFFFFFFFFFFFFFFF
            k1 = (k1 + PHILOX_W1) & 0xFFFFFFFFFFFFFFFF
    return np.stack(x, axis=1)


# ---------------------------------------------------------------------------
# Natural log and sincos(2*pi*u) written out from textbook methods, using only
# correctly rounded IEEE double +, -, *, / (numpy never fuses them), so that an
# independent implementation of the same steps reproduces every bit.
# ---------------------------------------------------------------------------
LN2_HI = float.fromhex("0x1.62e42fefa2000p-1")   # ln 2 cut to 40 bits
LN2_LO = float.fromhex("0x1.9ef35793c7673p-41")  # ln 2 - LN2_HI, rounded
SQRT2 = float.fromhex("0x1.6a09e667f3bcdp+0")    # sqrt(2), rounded
PIO2 = float.fromhex("0x1.921fb54442d18p+0")     # pi/2, rounded
LOG_TERMS = 11   # atanh series s^(2j+1)/(2j+1), j = 1..LOG_TERMS
SIN_TERMS = 9    # sin Taylor terms (-1)^k t^(2k+1)/(2k+1)!, k = 1..SIN_TERMS
COS_TERMS = 10   # cos Taylor terms (-1)^k t^(2k)/(2k)!,    k = 1..COS_TERMS


def _log_coeff(j: int) -> float:
    return 1.0 / float(2 * j + 1)


def _sin_coeff(k: int) -> float:
    c = 1.0 / float(math.factorial(2 * k + 1))  # (2k+1)! is exact in a double
    return -c if k % 2 else c


def _cos_coeff(k: int) -> float:
    c = 1.0 / float(math.factorial(2 * k))
    return -c if k % 2 else c


def log_fp64(x: np.ndarray) -> np.ndarray:
    """ln x for positive normal doubles.

    x = 2^e f with f in [1, 2); if f > sqrt(2) then f /= 2, e += 1.
    s = (f - 1)/(f + 1);  ln f = 2 atanh(s) = 2s + 2s * (s^2 * q(s^2)) with
    q(w) = sum_{j=1..11} w^(j-1)/(2j+1) by Horner;  ln x = e*LN2_HI +
    (ln f + e*LN2_LO).
    """
    x = np.asarray(x, dtype=np.float64)
    mant, ex = np.frexp(x)               # x = mant * 2^ex, mant in [0.5, 1)
    f = mant * 2.0
    e = (ex - 1).astype(np.float64)
    big = f > SQRT2
    f = np.where(big, f * 0.5, f)
    e = np.where(big, e + 1.0, e)
    s = (f - 1.0) / (f + 1.0)
    s2 = s * s
    q = np.full_like(s, _log_coeff(LOG_TERMS))
    for j in range(LOG_TERMS - 1, 0, -1):
        q = q * s2 + _log_coeff(j)
    two_s = 2.0 * s
    ln_f = two_s + two_s * (s2 * q)
    return e * LN2_HI + (ln_f + e * LN2_LO)


def sincos_2pi(u: np.ndarray):
    """(sin 2 pi u, cos 2 pi u) for u in [0, 1) given with at most 53 bits.

    t = 4u (exact), n = rint(t) (ties to even), d = t - n (exact, |d| <= 1/2),
    theta = d * PIO2;  sin(theta) = theta + theta*(theta^2 p), cos(theta) =
    1 + theta^2 q with p, q the Taylor tails by Horner; then rotate by the
    quadrant n mod 4.
    """
    u = np.asarray(u, dtype=np.float64)
    t = 4.0 * u
    n = np.rint(t)
    d = t - n
    th = d * PIO2
    th2 = th * th
    p = np.full_like(th, _sin_coeff(SIN_TERMS))
    for k in range(SIN_TERMS - 1, 0, -1):
        p = p * th2 + _sin_coeff(k)
    s = th + th * (th2 * p)
    q = np.full_like(th, _cos_coeff(COS_TERMS))
    for k in range(COS_TERMS - 1, 0, -1):
        q = q * th2 + _cos_coeff(k)
    c = 1.0 + th2 * q
    quad = n.astype(np.int64) & 3
    sin_out = np.choose(quad, [s, c, -s, -c])
    cos_out = np.choose(quad, [c, -s, -c, s])
    return sin_out, cos_out


# ---------------------------------------------------------------------------
# Gaussian measurement matrix (Sec. 3.1 / Sec. 4: "Gaussian random matrix").
# ---------------------------------------------------------------------------
def plan_tag(n: int, m: int) -> int:
    return (int(n) << 16) | int(m)


def gaussian_phi(n: int, m: int, seed: int) -> np.ndarray:
    """Phi in float32 [m][n], entries N(0, 1/m), row-major.

    Pair q = 0, 1, ... covers entries 2q and 2q+1 (row-major).  Its Philox
    block uses counter (q, (n << 16) | m, 0, 0) and key (seed, 0); words x0, x1
    give u1 = ((x0 >> 11) + 1) 2^-53 in (0, 1] and u2 = (x1 >> 11) 2^-53 in
    [0, 1).  Box-Muller: rad = sqrt(-2 ln u1), entry 2q = rad cos 2 pi u2,
    entry 2q+1 = rad sin 2 pi u2; each divided by sqrt(m) in double and
    rounded to float32.
    """
    total = int(n) * int(m)
    pairs = (total + 1) // 2
    ctr = np.zeros((pairs, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(pairs, dtype=np.uint64)
    ctr[:, 1] = np.uint64(plan_tag(n, m))
    words = philox4x64_10(ctr, (int(seed) & 0xFFFFFFFFFFFFFFFF, 0))
    u1 = ((words[:, 0] >> np.uint64(11)) + np.uint64(1)).astype(np.float64) * 2.0 ** -53
    u2 = (words[:, 1] >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    rad = np.sqrt(-2.0 * log_fp64(u1))
    sn, cs = sincos_2pi(u2)
    z = np.empty(2 * pairs, dtype=np.float64)
    z[0::2] = rad * cs
    z[1::2] = rad * sn
    phi = (z[:total] / math.sqrt(float(m))).astype(np.float32)
    return phi.reshape(m, n)


# ---------------------------------------------------------------------------
# Sparsifying basis: orthonormal 2-D DCT-II of a B x B block, vec row-major.
# ---------------------------------------------------------------------------
def dct_matrix(b: int) -> np.ndarray:
    """C[k][j] = alpha_k cos(pi (2j+1) k / (2B)), alpha_0 = sqrt(1/B), else sqrt(2/B)."""
    k = np.arange(b, dtype=np.float64)[:, None]
    j = np.arange(b, dtype=np.float64)[None, :]
    c = np.cos(np.pi * (2.0 * j + 1.0) * k / (2.0 * b))
    c[0, :] *= math.sqrt(1.0 / b)
    c[1:, :] *= math.sqrt(2.0 / b)
    return c


def psi_matrix(b: int) -> np.ndarray:
    """Psi (N x N) with r = Psi s  <=>  R = C^T S C for row-major vec."""
    c = dct_matrix(b)
    return np.kron(c.T, c.T)


class Plan:
    """Phi (float32, widened to float64), A = Phi Psi, and the step constant L."""

    def __init__(self, n: int, m: int, seed: int, power_iters: int = 1000):
        b = math.isqrt(n)
        if b * b != n or m < 1 or m > n:
            raise ValueError("need N = B^2 and 1 <= M <= N")
        self.n, self.m, self.b, self.seed = n, m, b, seed
        self.phi32 = gaussian_phi(n, m, seed)
        self.phi = self.phi32.astype(np.float64)
        self.psi = psi_matrix(b)
        self.a = self.phi @ self.psi
        self.lam_max = power_iteration_lambda_max(self.phi, power_iters)
        self.lipschitz = 1.0001 * self.lam_max


def power_iteration_lambda_max(phi: np.ndarray, iters: int = 1000) -> float:
    """lambda_max(Phi Phi^T) = ||A||_2^2 (Psi orthonormal) by power iteration.

    v0 = ones / sqrt(M); v <- G v / ||G v||; result = v^T G v, G = Phi Phi^T.
    """
    g = phi @ phi.T
    v = np.ones(g.shape[0]) / math.sqrt(g.shape[0])
    for _ in range(iters):
        w = g @ v
        v = w / np.linalg.norm(w)
    return float(v @ (g @ v))


# ---------------------------------------------------------------------------
# GOP structure and blocks (Sec. 3, Sec. 3.1).
# ---------------------------------------------------------------------------
def block_grid(height: int, width: int, b: int):
    """(block rows, block cols) of the zero-padded frame."""
    return -(-height // b), -(-width // b)


def key_index(t: int, gop: int) -> int:
    """Index of the key frame a frame t is coded against: floor(t/G)*G."""
    return (t // gop) * gop


def cs_frame_indices(n_frames: int, gop: int):
    """Frame indices that are CS frames (every frame that is not a key frame)."""
    return [t for t in range(n_frames) if t % gop != 0]


def blockify(img: np.ndarray, b: int) -> np.ndarray:
    """[H][W] -> [nblk][B*B]: zero-pad to whole blocks, raster block order,
    row-major inside a block."""
    h, w = img.shape
    br, bc = block_grid(h, w, b)
    pad = np.zeros((br * b, bc * b), dtype=np.float64)
    pad[:h, :w] = img
    return pad.reshape(br, b, bc, b).transpose(0, 2, 1, 3).reshape(br * bc, b * b)


def unblockify(blocks: np.ndarray, height: int, width: int, b: int) -> np.ndarray:
    """Inverse of blockify followed by the crop to [H][W]."""
    br, bc = block_grid(height, width, b)
    full = blocks.reshape(br, bc, b, b).transpose(0, 2, 1, 3).reshape(br * b, bc * b)
    return full[:height, :width]


def residuals(frames: np.ndarray, gop: int) -> np.ndarray:
    """int64 [n_cs][H][W]: each CS frame minus its GOP's key frame (the same key
    for all CS frames of a GOP: the multiple-residual scheme, Sec. 3.2)."""
    frames = np.asarray(frames)
    out = []
    for t in cs_frame_indices(frames.shape[0], gop):
        out.append(frames[t].astype(np.int64) - frames[key_index(t, gop)].astype(np.int64))
    if not out:
        return np.zeros((0,) + frames.shape[1:], dtype=np.int64)
    return np.stack(out)


def encode(plan: Plan, frames: np.ndarray, gop: int) -> np.ndarray:
    """y [n_cs][nblk][M] float64: y_b = Phi r_b for every block of every CS frame."""
    frames = np.asarray(frames)
    h, w = frames.shape[1:]
    res = residuals(frames, gop)
    br, bc = block_grid(h, w, plan.b)
    y = np.empty((res.shape[0], br * bc, plan.m))
    for i in range(res.shape[0]):
        y[i] = blockify(res[i].astype(np.float64), plan.b) @ plan.phi.T
    return y


# ---------------------------------------------------------------------------
# Recovery (Sec. 3.2, Eq. 1) by FISTA on 1/2 ||A s - y||^2 + lambda ||s||_1.
# ---------------------------------------------------------------------------
def soft(v: np.ndarray, tau) -> np.ndarray:
    """Soft threshold sign(v) max(|v| - tau, 0)."""
    return np.sign(v) * np.maximum(np.abs(v) - tau, 0.0)


def block_lambda(a: np.ndarray, y: np.ndarray, lambda_rel: float) -> np.ndarray:
    """lambda_b = lambda_rel * ||A^T y_b||_inf for each row y_b of y [nb][M]."""
    return lambda_rel * np.max(np.abs(y @ a), axis=1)


def fista(a: np.ndarray, y: np.ndarray, lipschitz: float, lam: np.ndarray,
          iters: int) -> np.ndarray:
    """Fixed-count FISTA for each row y_b of y [nb][M]; returns s^K [nb][N].

    s^0 = 0, z^1 = 0, t_1 = 1; for k = 1..K:
      g = A^T (A z^k - y);  s^k = soft(z^k - g/L, lambda/L);
      t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2;
      z^{k+1} = s^k + ((t_k - 1)/t_{k+1}) (s^k - s^{k-1}).
    """
    y = np.atleast_2d(np.asarray(y, dtype=np.float64))
    nb, n = y.shape[0], a.shape[1]
    tau = (np.asarray(lam, dtype=np.float64) / lipschitz).reshape(nb, 1)
    s_prev = np.zeros((nb, n))
    z = np.zeros((nb, n))
    s = s_prev
    t = 1.0
    for _ in range(iters):
        grad = (z @ a.T - y) @ a
        s = soft(z - grad / lipschitz, tau)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = s + ((t - 1.0) / t_next) * (s - s_prev)
        s_prev = s
        t = t_next
    return s


def decode(plan: Plan, key_frames: np.ndarray, y: np.ndarray, gop: int,
           n_frames: int, iters: int, lambda_rel: float = 0.01):
    """Recover every CS frame: F'_t = F_key + Psi s_hat, cropped (Eq. 4).

    key_frames: uint8 [n_gops][H][W] (raw keys); y: [n_cs][nblk][M].
    Returns (float64 [n_cs][H][W], uint8 [n_cs][H][W]).
    """
    key_frames = np.asarray(key_frames)
    h, w = key_frames.shape[1:]
    cs = cs_frame_indices(n_frames, gop)
    out = np.empty((len(cs), h, w))
    for i, t in enumerate(cs):
        yb = np.asarray(y[i], dtype=np.float64)
        lam = block_lambda(plan.a, yb, lambda_rel)
        s_hat = fista(plan.a, yb, plan.lipschitz, lam, iters)
        r_hat = s_hat @ plan.psi.T
        out[i] = key_frames[t // gop].astype(np.float64) + unblockify(r_hat, h, w, plan.b)
    return out, to_uint8(out)


def decode_blocks(plan: Plan, y_blocks: np.ndarray, iters: int,
                  lambda_rel: float = 0.01) -> np.ndarray:
    """Recovered residual blocks r_hat [nb][N] for measurement rows y [nb][M]."""
    yb = np.atleast_2d(np.asarray(y_blocks, dtype=np.float64))
    lam = block_lambda(plan.a, yb, lambda_rel)
    return fista(plan.a, yb, plan.lipschitz, lam, iters) @ plan.psi.T


def tv_difference_matrix(b: int) -> np.ndarray:
    """D = [Dx; Dy] (2N x N) of a B x B block in row-major vec order: forward
    differences along rows (Dx) and columns (Dy), zero at the last column / row."""
    n = b * b
    d = np.zeros((2 * n, n))
    for i in range(b):
        for j in range(b):
            k = i * b + j
            if j < b - 1:
                d[k, k + 1], d[k, k] = 1.0, -1.0
            if i < b - 1:
                d[n + k, k + b], d[n + k, k] = 1.0, -1.0
    return d


def tv_adm(phi: np.ndarray, y: np.ndarray, lipschitz: float, iters: int,
           beta: float = 0.125, mu: float = 1.0) -> np.ndarray:
    """TV recovery of every block (Eq. 1 with Phi(x) = TV, the TVAL3 choice of
    Sec. 4): min ||D r||_1 s.t. Phi r = y by the augmented Lagrangian
    ||w||_1 - nu^T (D r - w) + beta/2 ||D r - w||^2 - lam^T (Phi r - y)
    + mu/2 ||Phi r - y||^2, minimised alternately in w (shrinkage) and r (one
    gradient step of length 1 / (8 beta + mu L); 8 bounds ||D||^2, L the plan's
    Lipschitz constant of Phi Phi^T), then nu -= beta (D r - w) and
    lam -= mu (Phi r - y); r, nu, lam start at zero.

    phi: [M][N]; y: [blocks][M].  Returns r: [blocks][N] (pixel domain).
    """
    n = phi.shape[1]
    b = int(round(np.sqrt(n)))
    d = tv_difference_matrix(b)
    alpha = 1.0 / (8.0 * beta + mu * lipschitz)
    r = np.zeros((y.shape[0], n))
    nu = np.zeros((y.shape[0], 2 * n))
    lam = np.zeros_like(y, dtype=np.float64)
    for _ in range(iters):
        dr = r @ d.T
        w = soft(dr - nu / beta, 1.0 / beta)
        g = (beta * (dr - w) - nu) @ d + (mu * (r @ phi.T - y) - lam) @ phi
        r = r - alpha * g
        nu = nu - beta * (r @ d.T - w)
        lam = lam - mu * (r @ phi.T - y)
    return r


def decode_tv(plan: Plan, key_frames: np.ndarray, y: np.ndarray, gop: int, n_frames: int,
              iters: int, beta: float = 0.125, mu: float = 1.0) -> np.ndarray:
    """Every CS frame by TV recovery of its residual blocks, added back to its
    GOP's key (Sec. 3.2, Eq. 4).  Returns float64 [n_cs][H][W]."""
    _, h, w = key_frames.shape
    cs = cs_frame_indices(n_frames, gop)
    out = np.empty((len(cs), h, w))
    for i, t in enumerate(cs):
        r = tv_adm(plan.phi, y[i], plan.lipschitz, iters, beta, mu)
        out[i] = key_frames[key_index(t, gop) // gop].astype(np.float64) + unblockify(r, h, w, plan.b)
    return out


def to_uint8(frames: np.ndarray) -> np.ndarray:
    """clamp(rint(x), 0, 255) with ties to even."""
    return np.clip(np.rint(frames), 0, 255).astype(np.uint8)


# ---------------------------------------------------------------------------
# Reporting: compression ratio (Table I) and PSNR.
# ---------------------------------------------------------------------------
def total_cr(gop: int, cr_key: float, cr_cs: float) -> float:
    """Total CR of a GOP of 1 key + (G-1) CS frames: G / (1/CR_key + (G-1)/CR_cs)."""
    return gop / (1.0 / cr_key + (gop - 1) / cr_cs)


def raw_key_cr(gop: int, height: int, width: int, b: int, m: int) -> float:
    """Samples in / samples out for a GOP whose key frame is sent raw."""
    br, bc = block_grid(height, width, b)
    return gop * height * width / (height * width + (gop - 1) * br * bc * m)


def psnr(ref_u8: np.ndarray, test: np.ndarray) -> float:
    """10 log10(255^2 / MSE) in FP64; inf when the two are identical."""
    diff = np.asarray(ref_u8, dtype=np.float64) - np.asarray(test, dtype=np.float64)
    mse = float(np.mean(diff * diff))
    return math.inf if mse == 0.0 else 10.0 * math.log10(255.0 ** 2 / mse)
