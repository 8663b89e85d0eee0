"""Configurability sweep of the codec (the experiments of Sec. 4 on synthetic video).

The paper configures the GOP size and the CS frames' compression ratio and
reports, on QCIF surveillance video, the total compression ratio and PSNR
(Table I, Fig. 6) and the per-frame PSNR inside a GOP of 1 key + 4 CS frames
(Fig. 5).  This module runs the same sweeps through the library on synthetic
QCIF scenes (the paper's videos are not available): the CS frames' ratio
CR_cs = N / M samples per block, so M = rint(256 / CR_cs) for 16 x 16 blocks,
and the total CR uses Table I's closed form with the key frame at CR 23.  The
PSNR and tracking columns of Table I are not reproduced (other video, H.264
key frames and a tracker).

  python -m paper_1311_1419_gb300.sweep        (needs a GPU and the built library)
"""
from __future__ import annotations

import numpy as np

from . import binding as B
from . import scenes

H, W, BLK, N = 144, 176, 16, 256
CR_KEY = 23.0


def _decode(ctx, frames, gop, m, iters, seed=0):
    import torch

    n_gops = frames.shape[0] // gop
    plan = B.cs_make_phi(ctx, N, m, seed)
    try:
        p = B.make_params(H, W, gop, BLK, m, iters=iters, n_gops=n_gops)
        nblk = (-(-H // BLK)) * (-(-W // BLK))
        f = torch.from_numpy(frames[:n_gops * gop]).cuda()
        keys = torch.from_numpy(np.ascontiguousarray(frames[:n_gops * gop:gop])).cuda()
        y = torch.empty((n_gops * (gop - 1), nblk, m), dtype=torch.float32, device="cuda")
        out = torch.empty((n_gops * (gop - 1), H, W), dtype=torch.float32, device="cuda")
        s = torch.cuda.current_stream()
        B.cs_encode_gop(plan, p, f, y, s)
        B.cs_decode_gop(plan, p, keys, y, out, None, s)
        B.cs_ctx_status(ctx)
        return out.cpu().numpy().astype(np.float64)
    finally:
        B.cs_plan_destroy(plan)


def _psnr(ref, test):
    mse = np.mean((ref.astype(np.float64) - test) ** 2)
    return float("inf") if mse == 0 else 10 * np.log10(255.0 ** 2 / mse)


def table1_shape(ctx, iters=200, gops=(3, 5, 7), crs=(40, 60, 80), n_gops=6, seed=0,
                 keep_frames=False):
    """One row per (GOP, CS-frame CR); with keep_frames each row also carries
    the clip ("frames") and the decoded CS frames ("decoded", float64)."""
    rows = []
    for g in gops:
        frames = scenes.surveillance_video(g * n_gops, H, W, seed=seed)
        cs = [t for t in range(g * n_gops) if t % g]
        for cr in crs:
            m = max(1, int(np.rint(N / cr)))
            dec = _decode(ctx, frames, g, m, iters)
            rows.append({"gop": g, "rate": "23:%d" % cr, "m": m,
                         "total_cr_table_i": B.cs_total_cr(g, CR_KEY, N / m),
                         "total_cr_raw_key": B.cs_raw_key_cr(g, H, W, BLK, m),
                         "psnr_cs_db": _psnr(frames[cs], dec)})
            if keep_frames:
                rows[-1].update(frames=frames[:g * n_gops], decoded=dec)
    return rows


def fig5_shape(ctx, iters=200, cr=50, gop=5, n_gops=8, seed=0, keep_frames=False):
    m = max(1, int(np.rint(N / cr)))
    frames = scenes.surveillance_video(gop * n_gops, H, W, seed=seed)
    dec = _decode(ctx, frames, gop, m, iters)
    per_pos = []
    for pos in range(1, gop):
        idx = [g * (gop - 1) + pos - 1 for g in range(n_gops)]
        ref = frames[[g * gop + pos for g in range(n_gops)]]
        per_pos.append(_psnr(ref, dec[idx]))
    out = {"gop": gop, "cr_cs": cr, "m": m, "psnr_by_position_db": per_pos}
    if keep_frames:
        out.update(frames=frames, decoded=dec)
    return out


def fig6_shape(ctx, iters=200, gop=5, crs=(10, 20, 30, 40, 50, 60, 70, 80), n_gops=6, seed=0):
    frames = scenes.surveillance_video(gop * n_gops, H, W, seed=seed)
    cs = [t for t in range(gop * n_gops) if t % gop]
    out = []
    for cr in crs:
        m = max(1, int(np.rint(N / cr)))
        dec = _decode(ctx, frames, gop, m, iters)
        out.append({"cr_cs": cr, "m": m, "total_cr_table_i": B.cs_total_cr(gop, CR_KEY, N / m),
                    "psnr_cs_db": _psnr(frames[cs], dec)})
    return out


def main():
    ctx = B.cs_ctx_create(0)
    try:
        print("Table I shape (synthetic QCIF, K = 200, FP32)")
        print("| GOP | rate | M | total CR (Table I form) | total CR (raw key) | PSNR CS frames (dB) |")
        print("|---|---|---|---|---|---|")
        for r in table1_shape(ctx):
            print("| %d | %s | %d | %.2f | %.2f | %.2f |" % (r["gop"], r["rate"], r["m"],
                  r["total_cr_table_i"], r["total_cr_raw_key"], r["psnr_cs_db"]))
        f5 = fig5_shape(ctx)
        print("\nFig. 5 shape: 1 key + 4 CS frames, CR_cs = %d (M = %d): PSNR by position %s" % (
            f5["cr_cs"], f5["m"], ", ".join("%.2f" % v for v in f5["psnr_by_position_db"])))
        print("\nFig. 6 shape (GOP 5)")
        print("| CR_cs | M | total CR (Table I form) | PSNR CS frames (dB) |")
        print("|---|---|---|---|")
        for r in fig6_shape(ctx):
            print("| %d | %d | %.2f | %.2f |" % (r["cr_cs"], r["m"], r["total_cr_table_i"],
                                               r["psnr_cs_db"]))
    finally:
        B.cs_ctx_destroy(ctx)


if __name__ == "__main__":
    main()
