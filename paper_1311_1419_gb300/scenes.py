"""Seeded synthetic surveillance video, shared by the tests, the bench and users.

The paper measures on QCIF surveillance sequences (a static, well defined
background with few moving objects, Sec. 2.1 and Sec. 4).  Those sequences are
not shipped here; this module makes stand-ins of the same shape:

* background: i.i.d. uniform[0,1) noise smoothed by a 2-D Gaussian low-pass
  filter (sigma 8 px, radius 24, reflecting border), min-max scaled to [40, 200];
* movers: bright 12x12 rectangles of value 230 that move at a constant integer
  velocity in {+-1, +-2, +-3}^2 px/frame and bounce off the frame border;
* sensor noise: i.i.d. N(0, 2^2) per pixel and frame;
* output: clamp(rint(.), 0, 255) as uint8, frames laid out [F][H][W].

Every random draw comes from numpy's Philox bit generator keyed by
(seed, stream): stream 1 for the background, 2 for the movers, 3 for the noise.
Nothing here is part of the codec's arithmetic: the module only makes inputs.
"""
from __future__ import annotations

import numpy as np

MOVER_SIZE = 12
MOVER_VALUE = 230.0
BG_LO, BG_HI = 40.0, 200.0
BLUR_SIGMA = 8.0
NOISE_SIGMA = 2.0

RESOLUTIONS = {
    "qcif": (144, 176),
    "cif": (288, 352),
    "720p": (720, 1280),
    "1080p": (1080, 1920),
}


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=[int(seed), int(stream)]))


def background(height: int, width: int, seed: int) -> np.ndarray:
    """Low-pass filtered uniform noise scaled to [40, 200], float64 [H][W]."""
    from scipy.ndimage import gaussian_filter

    noise = _rng(seed, 1).random((height, width))
    smooth = gaussian_filter(noise, sigma=BLUR_SIGMA, mode="reflect", truncate=3.0)
    lo, hi = smooth.min(), smooth.max()
    if hi <= lo:
        return np.full((height, width), 0.5 * (BG_LO + BG_HI))
    return BG_LO + (smooth - lo) * ((BG_HI - BG_LO) / (hi - lo))


def _mover_tracks(n_frames: int, height: int, width: int, n_movers: int, seed: int):
    """Top-left corners [F][n_movers][2] (row, col) of each mover in each frame."""
    rng = _rng(seed, 2)
    span = np.array([max(height - MOVER_SIZE, 0), max(width - MOVER_SIZE, 0)])
    pos = np.stack([rng.integers(0, span[0] + 1, n_movers),
                    rng.integers(0, span[1] + 1, n_movers)], axis=1)
    speeds = np.array([-3, -2, -1, 1, 2, 3])
    vel = speeds[rng.integers(0, len(speeds), (n_movers, 2))]
    tracks = np.empty((n_frames, n_movers, 2), dtype=np.int64)
    for t in range(n_frames):
        tracks[t] = pos
        pos = pos + vel
        for d in range(2):
            low = pos[:, d] < 0
            pos[low, d] = -pos[low, d]
            vel[low, d] = -vel[low, d]
            high = pos[:, d] > span[d]
            pos[high, d] = 2 * span[d] - pos[high, d]
            vel[high, d] = -vel[high, d]
        pos = np.clip(pos, 0, span)
    return tracks


def surveillance_video(n_frames: int, height: int, width: int, seed: int = 0,
                       n_movers: int | None = None) -> np.ndarray:
    """uint8 [n_frames][height][width] synthetic surveillance clip.

    n_movers defaults to 2 for frames no larger than QCIF and 4 otherwise.
    """
    if n_frames < 0 or height <= 0 or width <= 0:
        raise ValueError("bad video shape")
    if n_movers is None:
        n_movers = 2 if height * width <= 176 * 144 else 4
    bg = background(height, width, seed)
    tracks = _mover_tracks(n_frames, height, width, n_movers, seed)
    noise = _rng(seed, 3).normal(0.0, NOISE_SIGMA, (n_frames, height, width))
    out = np.empty((n_frames, height, width), dtype=np.uint8)
    for t in range(n_frames):
        frame = bg.copy()
        for r, c in tracks[t]:
            frame[r:r + MOVER_SIZE, c:c + MOVER_SIZE] = MOVER_VALUE
        frame += noise[t]
        out[t] = np.clip(np.rint(frame), 0, 255).astype(np.uint8)
    return out
