#!/usr/bin/env python
"""Recovered Mpixel/s of the block-CS video codec hot path on GB300.

Default workload: the 720p clip (1280x720, 96 frames, GOP 16, 32x32 blocks,
M = 102, FISTA 300 iterations, FP32-grade products).  One step = the whole hot
path over the clip: encode every CS frame (y = Phi r per block), decode all of
them in one batched call, score the result (PSNR).  The plan (Phi, A, L) is
built and the decode shape autotuned once before timing, like weights; their
times are reported as plan_ms and autotune.  value = recovered CS-frame pixels
per second over the device-resident step; e2e = the same through the
host-buffer entry point cs_codec_host (copies inside the timed region).

Beside the headline, the same JSON line carries the other workloads: the CIF
M-sweep (cif_sweep), the plain per-block FP32 decode of the 720p clip
(plain_engine, and the tensor path's ratio to it), the 64-GOP heterogeneous
batch (mixed64), the mixed-precision decodes of the clip, TV recovery and a
serving sweep.  --workload cif or mixed64 puts that workload in the headline
instead; --no-extras leaves the others out.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one process per GPU) every rank decodes its own copy of
the clip (replicas, weak scaling); value = pixels of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    "720p": {
        "workload": "720p 1280x720, 96 frames, GOP 16 (1 raw key + 15 CS), 32x32 blocks (N=1024), "
                    "M=102 (10%), Gaussian Phi N(0,1/M) Philox seed 0, FISTA 300 iters, "
                    "lambda=0.01*||A^T y||_inf, synthetic surveillance scene, FP32-grade products",
        "metric": "recovered Mpixel/s at fixed iters (720p, 32x32 blocks, FISTA 300 iters)",
        "height": 720, "width": 1280, "frames": 96, "gop": 16, "block": 32,
        "ms": [102], "iters": 300, "lambda_rel": 0.01, "seed": 0, "oracle_frames": 1,
    },
    "cif": {
        "workload": "CIF 352x288, 64 frames, GOP 8 (1 raw key + 7 CS), 16x16 blocks (N=256), "
                    "M in {26,51,77,128} (CR sweep), Gaussian Phi N(0,1/M) Philox seed 0, "
                    "FISTA 300 iters, lambda=0.01*||A^T y||_inf, synthetic surveillance scene",
        "metric": "recovered Mpixel/s at fixed iters (CIF M-sweep, FISTA 300 iters)",
        "height": 288, "width": 352, "frames": 64, "gop": 8, "block": 16,
        "ms": [26, 51, 77, 128], "iters": 300, "lambda_rel": 0.01, "seed": 0, "oracle_frames": 2,
    },
}
WORKLOADS["mixed64"] = {
    "workload": "64 GOPs (seeds 0..63) of QCIF/CIF/720p, 8x8/16x16/32x32 blocks, M/N uniform in "
                "5%..50%, GOP uniform in 4..32, FISTA 300 iters, synthetic surveillance scenes; "
                "split-BF16 on the tensor-core kernels (on-chip, streaming or chunked), FP32 on the plain "
                "kernel for any shape they do not cover; one cs_decode_batch captured in a CUDA graph",
    "metric": "recovered Mpixel/s at fixed iters (64 heterogeneous GOPs, one graph-captured batch)",
    "iters": 300, "lambda_rel": 0.01, "seed": 0, "jobs": 64,
}
DEFAULT_WORKLOAD = "720p"
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the decode of one
# step, from one ncu capture of that exact configuration (FP32-grade, batched) on
# the engine it ran (2 = on-chip tensor cores; 4 = chunked, whose 720p decode is
# one cluster-kernel launch for the first 39 tiles and one chunked launch for the
# other 608); reported as roofline.traffic when the step's decode ran on that
# engine, null otherwise
DECODE_DRAM_BYTES = {"cif": (2, 62_840_000), "720p": (4, 236_941_000_000)}


def decode_traffic(workload, res):
    engine, nbytes = DECODE_DRAM_BYTES.get(workload, (None, None))
    return nbytes if res["engines"] == [engine] else None
FP32_LANES_PER_SM = 128


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(x: float, world: int, device="cpu") -> float:
    """The slowest rank's time: every rank times its own replica of the work, and
    the job takes as long as its slowest rank (all_reduce MAX over the process
    group; nccl with a CUDA device, gloo with the CPU)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, units_per_rank_step: float, steps: int, max_ms: float) -> float:
    """Whole-job throughput in units per second: the units all ranks processed
    over the slowest rank's time (weak scaling: each rank a fixed share)."""
    return world * units_per_rank_step * steps / (max_ms / 1e3)


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while the timed region runs."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "bench_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for ln in f:
                parts = [p.strip() for p in ln.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        loaded = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def decode_flops(blocks: int, m: int, n: int, iters: int) -> float:
    """Algorithmic flops of the recovery: 4MN per block per iteration (A z and
    A^T rho) plus 2MN once per block for lambda (A^T y)."""
    return float(blocks) * (4.0 * m * n * iters + 2.0 * m * n)


SERVING = {
    "workload": "256 synthetic cameras, resolution QCIF/CIF/720p/1080p (p = .4/.3/.2/.1), "
                "GOP uniform 4..32, 16x16 or 32x32 blocks (p = .5/.5), M/N uniform 5%..25%, "
                "Phi seed = camera id, FISTA 200 iters; one request = one GOP decode; Poisson "
                "arrivals; every shape of the mix has a tensor-core kernel (on chip for M <= 128, "
                "streaming above)",
    "cameras": 256, "iters": 200, "seed": 7,
}


def serving_run(B, torch, dev, configs, rates, seconds, hbm_budget=8 << 30, batch_ref=True):
    """Open-loop serving: Poisson arrivals over the camera mix.  configs: list of
    (name, serving mode, precision, FP32-grade tail); every config runs every
    rate on the same cameras.  Returns {name: [one dict per rate: p50/p99
    latency, Mpixel/s, admitted, refused]}, plus, with batch_ref, the same
    cameras' GOPs decoded in one cs_decode_batch per precision (the throughput
    the serving loop is compared with)."""
    from paper_1311_1419_gb300 import scenes

    rng = np.random.default_rng(SERVING["seed"])
    res = [scenes.RESOLUTIONS[k] for k in ("qcif", "cif", "720p", "1080p")]
    base = {r: scenes.surveillance_video(32, r[0], r[1], seed=i) for i, r in enumerate(res)}
    ctx = B.cs_ctx_create(dev.index, hbm_budget)
    cams = []
    stream = torch.cuda.Stream(dev)
    out = {}
    try:
        for cid in range(SERVING["cameras"]):
            h, w = res[rng.choice(4, p=[0.4, 0.3, 0.2, 0.1])]
            gop = int(rng.integers(4, 33))
            b = (16, 32)[rng.integers(2)]
            m = max(1, int(np.rint(b * b * rng.uniform(0.05, 0.25))))
            plan = B.cs_make_phi(ctx, b * b, m, cid)
            off = cid % (33 - gop)
            clip = base[(h, w)][off:off + gop]
            nblk = (-(-h // b)) * (-(-w // b))
            p32 = B.make_params(h, w, gop, b, m, iters=SERVING["iters"])
            y = torch.empty((gop - 1, nblk, m), dtype=torch.float32, device=dev)
            B.cs_encode_gop(plan, p32, torch.from_numpy(np.ascontiguousarray(clip)).to(dev), y, stream)
            stream.synchronize()
            cams.append({"plan": plan, "dims": (h, w, gop, b, m), "y_dev": y,
                         "key_dev": torch.from_numpy(np.ascontiguousarray(clip[:1])).to(dev),
                         "key": torch.from_numpy(np.ascontiguousarray(clip[:1])).pin_memory(),
                         "y": y.cpu().pin_memory(), "shape": (gop - 1, h, w),
                         "pixels": (gop - 1) * h * w, "free": []})

        def params(c, precision, tail):
            h, w, gop, b, m = c["dims"]
            return B.make_params(h, w, gop, b, m, iters=SERVING["iters"], precision=precision,
                                 fp32_tail_iters=tail)

        for name, mode, precision, tail in configs:
            B.cs_ctx_set_serving(ctx, mode)
            prm = [params(c, precision, tail) for c in cams]
            rows = []
            for rate in rates:
                t_next = 0.0
                arrivals = []
                while t_next < seconds:
                    t_next += rng.exponential(1.0 / rate)
                    arrivals.append((t_next, int(rng.integers(len(cams)))))
                inflight, lat, pixels, refused = {}, [], 0, 0
                backlog = []
                t0 = time.perf_counter()
                i = 0
                while i < len(arrivals) or backlog or inflight:
                    now = time.perf_counter() - t0
                    while i < len(arrivals) and arrivals[i][0] <= now:
                        backlog.append((arrivals[i][1], t0 + arrivals[i][0]))
                        i += 1
                    while backlog:                      # admit as slots and memory free up
                        c = cams[backlog[0][0]]
                        o = c["free"].pop() if c["free"] else torch.empty(
                            c["shape"], dtype=torch.uint8).pin_memory()
                        try:
                            t = B.cs_submit(ctx, c["plan"], prm[backlog[0][0]], c["key"], c["y"], o)
                        except B.CsError as e:
                            c["free"].append(o)
                            if e.status != B.CS_EAGAIN:
                                raise
                            refused += 1
                            break
                        cid, t_arr = backlog.pop(0)
                        inflight[t] = (cid, o, time.perf_counter() - t_arr)
                    for t in list(inflight):
                        done, ms = B.cs_poll(ctx, t)
                        if done:
                            cid, o, queued = inflight.pop(t)
                            # arrival to completion: admission queueing + submit-to-done
                            lat.append(1e3 * queued + ms)
                            pixels += cams[cid]["pixels"]
                            cams[cid]["free"].append(o)
                wall = time.perf_counter() - t0
                B.cs_ctx_status(ctx)
                lat_ms = np.array(lat)
                rows.append({"rate_per_s": rate, "requests": len(lat), "refused_retries": refused,
                             "p50_ms": float(np.percentile(lat_ms, 50)),
                             "p99_ms": float(np.percentile(lat_ms, 99)),
                             "mpixel_per_s": pixels / wall / 1e6})
            out[name] = rows
        if batch_ref:
            # every camera's GOP once, in one batched call on the best kernels
            for precision, tail, name in ((B.CS_FP32, 0, "batched_fp32"),
                                          (B.CS_FP16, 20, "batched_fp16_tail20")):
                prm = [params(c, precision, tail) for c in cams]
                outs = [torch.empty(c["shape"], dtype=torch.uint8, device=dev) for c in cams]
                args_ = ([c["plan"] for c in cams], prm, [c["key_dev"] for c in cams],
                         [c["y_dev"] for c in cams], None, outs)
                with torch.cuda.stream(stream):
                    B.cs_decode_batch(ctx, *args_, stream)
                    torch.cuda.synchronize(dev)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    B.cs_decode_batch(ctx, *args_, stream)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                ms = e0.elapsed_time(e1)
                out[name] = {"gops": len(cams), "ms": ms,
                             "mpixel_per_s": sum(c["pixels"] for c in cams) / (ms / 1e3) / 1e6}
        return out
    finally:
        for c in cams:
            B.cs_plan_destroy(c["plan"])
        B.cs_ctx_destroy(ctx)


def oracle_sample(frames, wl, n_cs_frames: int):
    """Time the FP64 oracle on the first n_cs_frames CS frames at every M.

    Returns (seconds, recovered pixels, decoded frames per M)."""
    from oracle import cs_oracle as O

    gop, b = wl["gop"], wl["block"]
    clip = frames[:gop]
    t0 = time.perf_counter()
    out = {}
    for m in wl["ms"]:
        plan = O.Plan(b * b, m, wl["seed"])
        y = O.encode(plan, clip, gop)[:n_cs_frames]
        dec = []
        for i in range(n_cs_frames):
            r_hat = O.decode_blocks(plan, y[i], wl["iters"], wl["lambda_rel"])
            dec.append(clip[0].astype(np.float64) +
                       O.unblockify(r_hat, wl["height"], wl["width"], b))
        out[m] = np.stack(dec)
    secs = time.perf_counter() - t0
    pixels = len(wl["ms"]) * n_cs_frames * wl["height"] * wl["width"]
    return secs, pixels, out


def parity(frames, got, want):
    """Error of decoded CS frames 1.. (got) against the oracle's (want), both
    [n][H][W] of the first GOP: whole-frame rel-l2, rel-l2 of the recovered
    residual (the key frame taken out of the denominator), and PSNR difference."""
    from oracle import cs_oracle as O

    n = want.shape[0]
    orig = frames[1:1 + n]
    key = frames[0].astype(np.float64)
    return {"frame_rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
            "residual_rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want - key)),
            "dpsnr_db": float(O.psnr(orig, got) - O.psnr(orig, want))}


def run_reference(args, wl, frames):
    """The reference arm: the FP64 CPU oracle as it stands, bounded samples."""
    n_cs = 1
    for _ in range(args.warmup):
        oracle_sample(frames, wl, n_cs)
    secs = []
    pixels = 0
    for _ in range(args.steps):
        s, pixels, _ = oracle_sample(frames, wl, n_cs)
        secs.append(s)
    total = sum(secs)
    value = pixels * args.steps / total / 1e6
    nblk = (-(-wl["height"] // wl["block"])) * (-(-wl["width"] // wl["block"]))
    sample = ("first CS frame of the clip (%d blocks) at each M in %s, %d iters, per step"
              % (nblk, wl["ms"], wl["iters"]))
    line = {
        "impl": "reference", "metric": wl["metric"], "value": value, "unit": "Mpixel/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {k: wl[k] for k in ("workload",)},
        "cpu_baseline": {"value": value, "unit": "Mpixel/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Mpixel/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def mixed_launches(jobs, clusters=15, kappa=13, n_sm=152) -> int:
    """Kernels one cs_decode_batch of the mix launches, from each job's engine
    (j["engine"]: 1 plain, 2 on chip, 3 streaming, 4 chunked): one per group of up
    to 48 jobs of each tensor-core kernel (16x16 on chip by shared-memory layout,
    32x32 cluster, streaming, chunked; one operand type here), one for the
    streaming tail of the cluster jobs when one of them has more tiles than
    clusters x kappa, one for the cluster-kernel heads of the chunked 32x32 jobs
    whose last round of tiles is short (more tiles than SMs, at most 4 x clusters
    left over) (the library's rules; 15 clusters of 8 are co-resident on this
    part), and one per plain-kernel job."""
    groups = {}
    for j in jobs:
        b, m, eng = j["p"].block, j["p"].m, j["engine"]
        m16 = (m + 15) // 16 * 16
        if eng == 1:
            key = ("plain", len(groups))
        elif eng == 4:
            key = ("tcz",)
            t = -(-j.get("blocks", 0) // 128)
            if b == 32 and t > n_sm and 0 < t % n_sm <= 4 * clusters:
                groups[("tc8 head",)] = groups.get(("tc8 head",), 0) + 1
        elif eng == 3:
            key = ("tcs",)
        elif b == 16:
            key = ("tc", m16 <= 96)
        else:
            key = ("tc8",)
            if -(-j.get("blocks", 0) // 128) > clusters * kappa:
                groups[("tc8 tail",)] = 1
        groups[key] = groups.get(key, 0) + 1
    return sum(-(-c // 48) for c in groups.values())


def mixed64_oracle(O, job, iters, lambda_rel, max_blocks=8):
    """Oracle check of one job of the mix on sampled blocks: the first row of
    blocks (up to max_blocks) of the job's first CS frame, recovered by the FP64
    oracle from its own measurements and compared with the library's frame."""
    p, clip = job["p"], job["clip"]
    b, h, w = p.block, p.height, p.width
    plan = O.Plan(b * b, p.m, job["seed"])
    res = clip[1].astype(np.int64) - clip[0].astype(np.int64)
    k = min(max_blocks, -(-w // b))
    y = O.blockify(res.astype(np.float64), b)[:k] @ plan.phi.T
    r_hat = O.decode_blocks(plan, y, iters, lambda_rel)
    rows = min(b, h)
    cols = min(k * b, w)
    want = np.zeros((rows, k * b))
    for j in range(k):
        want[:, j * b:(j + 1) * b] = r_hat[j].reshape(b, b)[:rows]
    key = clip[0][:rows, :cols].astype(np.float64)
    want = key + want[:, :cols]
    got = job["out"][0, :rows, :cols].cpu().numpy().astype(np.float64)
    orig = clip[1][:rows, :cols]
    return {"blocks": k, "frame_rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
            "residual_rel_l2": float(np.linalg.norm(got - want) / max(np.linalg.norm(want - key), 1e-30)),
            "dpsnr_db": float(O.psnr(orig, got) - O.psnr(orig, want))}


def run_mixed64(args, wl, B, torch, dev, steps, warmup, with_oracle=True):
    """The heterogeneous batch: every GOP a job of its own plan, one batched call
    captured in a CUDA graph and replayed; returns the measurement as a dict
    (value = CS pixels per second), with the oracle's error on sampled blocks of
    one job per (N, M) bucket."""
    from paper_1311_1419_gb300 import scenes

    rng = np.random.default_rng(wl["seed"])
    res = [scenes.RESOLUTIONS[k] for k in ("qcif", "cif", "720p")]
    ctx = B.cs_ctx_create(dev.index)
    stream = torch.cuda.Stream(dev)
    jobs = []
    t0 = time.perf_counter()
    try:
        for i in range(wl["jobs"]):
            h, w = res[rng.integers(3)]
            b = (8, 16, 32)[rng.integers(3)]
            n = b * b
            m = max(1, int(np.rint(n * rng.uniform(0.05, 0.5))))
            gop = int(rng.integers(4, 33))
            plan = B.cs_make_phi(ctx, n, m, i)
            # every shape of the mix has a tensor-core kernel: on chip (16 x 16 and
            # 32 x 32 blocks, M <= 128) or streaming (8 x 8 .. 32 x 32, M <= 512)
            tc = (b in (16, 32) and m <= 128) or (b in (8, 16, 32) and (m + 15) // 16 * 16 <= 512)
            p = B.make_params(h, w, gop, b, m, iters=wl["iters"], lambda_rel=wl["lambda_rel"],
                              precision=B.CS_BF16X2 if tc else B.CS_FP32)
            clip = scenes.surveillance_video(gop, h, w, seed=i)
            nblk = (-(-h // b)) * (-(-w // b))
            y = torch.empty((gop - 1, nblk, m), dtype=torch.float32, device=dev)
            B.cs_encode_gop(plan, p, torch.from_numpy(clip).to(dev), y, stream)
            jobs.append({"plan": plan, "p": p, "seed": i, "clip": clip[:2],
                         "key": torch.from_numpy(np.ascontiguousarray(clip[:1])).to(dev),
                         "y": y, "out": torch.empty((gop - 1, h, w), dtype=torch.float32, device=dev),
                         "pixels": (gop - 1) * h * w, "tc": tc, "blocks": (gop - 1) * nblk,
                         "flops": (gop - 1) * nblk * (4.0 * m * n * wl["iters"] + 2.0 * m * n)})
        stream.synchronize()
        # the decode shape of every (N, M) is picked by timing, once, before capture
        tuned = {}
        for j in jobs:
            key = (j["p"].block, j["p"].m)
            if key not in tuned:
                tuned[key] = B.cs_autotune(ctx, j["plan"])
            # the library's rule for CS_ENGINE_AUTO: the tuned engine, except that a
            # mixed-precision job whose tuned engine is the (FP32-only) plain kernel
            # takes the on-chip tensor-core kernel, else the streaming one
            eng = tuned[key][0]
            if j["p"].precision != B.CS_FP32 and eng == B.CS_ENGINE_PLAIN:
                b, m = key
                eng = B.CS_ENGINE_TC if (b in (16, 32) and m <= 128) else B.CS_ENGINE_TC_STREAM
            j["engine"] = eng
        setup_s = time.perf_counter() - t0
        args_ = ([j["plan"] for j in jobs], [j["p"] for j in jobs], [j["key"] for j in jobs],
                 [j["y"] for j in jobs], [j["out"] for j in jobs])
        with torch.cuda.stream(stream):
            B.cs_decode_batch(ctx, *args_, None, stream)       # eager warm-up
            torch.cuda.synchronize(dev)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
                B.cs_decode_batch(ctx, *args_, None, stream)
            for _ in range(warmup):
                g.replay()
            torch.cuda.synchronize(dev)
            times = []
            with ClockSampler(dev.index) as clocks:
                for _ in range(steps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    g.replay()
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    times.append(e0.elapsed_time(e1))
        B.cs_ctx_status(ctx)
        ms = sum(times) / len(times)
        pixels = sum(j["pixels"] for j in jobs)
        tc_pix = sum(j["pixels"] for j in jobs if j["tc"])
        gflop = sum(j["flops"] for j in jobs) / 1e9
        out = {
            "metric": wl["metric"], "value": pixels / (ms / 1e3) / 1e6, "unit": "Mpixel/s",
            "ms_per_step": ms, "steps": steps, "warmup": warmup, "dtype": "bf16x2/f32",
            "workload": wl["workload"], "jobs": len(jobs),
            "tensor_core_jobs": sum(j["tc"] for j in jobs), "pixels_per_step": pixels,
            "tensor_core_pixel_share": tc_pix / pixels, "gflop_per_step": gflop,
            "achieved_tflops": gflop / ms, "gpu_launches": mixed_launches(jobs, n_sm=torch.cuda.get_device_properties(dev).multi_processor_count) * steps,
            "clocks": clocks.summary(), "setup_s": setup_s, "autotuned_shapes": len(tuned),
        }
        if with_oracle:
            from oracle import cs_oracle as O
            seen, errs = set(), {}
            for j in jobs:
                key = (j["p"].block * j["p"].block, j["p"].m)
                if key in seen:
                    continue
                seen.add(key)
                errs["N=%d,M=%d" % key] = mixed64_oracle(O, j, wl["iters"], wl["lambda_rel"])
            out["vs_oracle"] = {
                "sample": "first block row (up to 8 blocks) of the first CS frame of one job per "
                          "(N, M) bucket, FP64 oracle from its own measurements",
                "buckets": errs,
                "max_frame_rel_l2": max(e["frame_rel_l2"] for e in errs.values()),
                "max_residual_rel_l2": max(e["residual_rel_l2"] for e in errs.values()),
                "max_abs_dpsnr_db": max(abs(e["dpsnr_db"]) for e in errs.values())}
        return out
    finally:
        for j in jobs:
            B.cs_plan_destroy(j["plan"])
        B.cs_ctx_destroy(ctx)


def codec_run(wl, B, torch, dev, world, barrier, steps, warmup, engine, want_e2e=True,
              want_mixed=True, no_batch=False):
    """Plans, autotune, then `steps` timed steps of the whole hot path over the
    clip (encode every M, one batched decode, PSNR), device-resident with L2
    flushed before each step; then the same through cs_codec_host from pinned
    host memory (e2e); then the mixed-precision decodes.  Returns a dict of the
    measurements and the live buffers (release with codec_free)."""
    from paper_1311_1419_gb300 import scenes

    h, w, gop, b, iters = wl["height"], wl["width"], wl["gop"], wl["block"], wl["iters"]
    n = b * b
    n_gops = wl["frames"] // gop
    n_cs = n_gops * (gop - 1)
    nblk = (-(-h // b)) * (-(-w // b))
    cs_idx = [t for t in range(wl["frames"]) if t % gop]
    frames = scenes.surveillance_video(wl["frames"], h, w, seed=wl["seed"])
    ms = wl["ms"]

    ctx = B.cs_ctx_create(dev.index)
    t0 = time.perf_counter()
    plans = {m: B.cs_make_phi(ctx, n, m, wl["seed"]) for m in ms}
    plan_ms = 1e3 * (time.perf_counter() - t0)
    params = {m: B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops,
                               lambda_rel=wl["lambda_rel"], engine=engine) for m in ms}
    t0 = time.perf_counter()
    tuned = {str(m): dict(zip(("engine", "plain_threads", "plain_blocks_per_cta", "ns_per_block_iter"),
                              B.cs_autotune(ctx, plans[m]))) for m in ms}
    autotune_s = time.perf_counter() - t0

    stream = torch.cuda.Stream(dev)
    frames_dev = torch.from_numpy(frames).to(dev)
    keys_dev = torch.from_numpy(np.ascontiguousarray(frames[::gop])).to(dev)
    cs_dev = torch.from_numpy(np.ascontiguousarray(frames[cs_idx])).to(dev)
    y_dev = {m: torch.empty((n_cs, nblk, m), dtype=torch.float32, device=dev) for m in ms}
    out_f = {m: torch.empty((n_cs, h, w), dtype=torch.float32, device=dev) for m in ms}
    out_u = {m: torch.empty((n_cs, h, w), dtype=torch.uint8, device=dev) for m in ms}
    psnr_dev = {m: torch.empty(n_cs, dtype=torch.float64, device=dev) for m in ms}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    plan_list = [plans[m] for m in ms]
    param_list = [params[m] for m in ms]
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count

    # our kernels per step: the encode (tensor-core plans share launches of up to 4
    # plans and 320 accumulator columns; plain-engine plans one each), one PSNR per
    # M, and the decode: one
    # launch per call with no_batch, else one per (operand type, shared-memory
    # layout) group of the 16x16 tensor path (M16 <= 96 or <= 128), one per group
    # of the 32x32 cluster path (and its streaming tail), one per group of the
    # streaming path, one per group of the chunked path, one per plain-kernel job
    # (FP32: one operand type)
    def decode_launches():
        if no_batch:
            return len(ms)
        groups, plain = set(), 0
        for m in ms:
            m16 = (m + 15) // 16 * 16
            eng = engine if engine != B.CS_ENGINE_AUTO else tuned[str(m)]["engine"]
            if eng == B.CS_ENGINE_PLAIN:
                plain += 1
            elif eng == B.CS_ENGINE_TC_STREAM:
                groups.add(("tcs",))
            elif eng == B.CS_ENGINE_TC_CHUNK:
                groups.add(("tcz",))
                # the library hands a short last round of a 32x32 job to the cluster
                # kernel (more tiles than SMs, at most 4 x 15 clusters left over)
                tiles = -(-(n_cs * nblk) // 128)
                if n == 1024 and tiles > n_sm and 0 < tiles % n_sm <= 4 * 15:
                    groups.add(("tc8 head",))
            elif n == 256:
                groups.add(("tc", m16 <= 96))
            else:
                groups.add(("tc8",))
                # a large 32x32 job also launches its streaming tail on the SMs whole
                # clusters leave idle (the library's rule: a tail once the job has more
                # tiles than clusters x 13; 15 clusters of 8 are co-resident on this part)
                tiles = -(-(n_cs * nblk) // 128)
                if n_sm - 8 * 15 > 0 and tiles > 15 * 13:
                    groups.add(("tc8 tail",))
        return len(groups) + plain
    def encode_launches():
        if engine == B.CS_ENGINE_PLAIN:
            return len(ms)
        count, cols, k = 0, 0, 0
        for m in ms:
            m16 = (m + 15) // 16 * 16
            if k == 0 or k == 4 or cols + m16 > 320:
                count, cols, k = count + 1, 0, 0
            cols, k = cols + m16, k + 1
        return count
    launches_per_step = encode_launches() + len(ms) + decode_launches()

    enc_ev, dec_ev, psnr_ev = [], [], []

    def ev_pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step(record):
        if record:
            a0, a1 = ev_pair()
            a0.record(stream)
        B.cs_encode_batch(ctx, plan_list, param_list, frames_dev, [y_dev[m] for m in ms], stream)
        if record:
            a1.record(stream)
            enc_ev.append((a0, a1))
            d0, d1 = ev_pair()
            d0.record(stream)
        if no_batch:
            for m in ms:
                B.cs_decode_gop(plans[m], params[m], keys_dev, y_dev[m], out_f[m], out_u[m], stream)
        else:
            B.cs_decode_batch(ctx, plan_list, param_list, [keys_dev] * len(ms),
                              [y_dev[m] for m in ms], [out_f[m] for m in ms],
                              [out_u[m] for m in ms], stream)
        if record:
            d1.record(stream)
            dec_ev.append((d0, d1))
            c0, c1 = ev_pair()
            c0.record(stream)
        for m in ms:
            B.cs_psnr(cs_dev, out_f[m], n_cs, h, w, psnr_dev[m], stream)
        if record:
            c1.record(stream)
            psnr_ev.append((c0, c1))

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step(False)
        torch.cuda.synchronize(dev)
        step_ms = []
        with ClockSampler(dev.index) as clocks:
            for _ in range(steps):
                flush.zero_()
                torch.cuda.synchronize(dev)
                barrier()
                e0, e1 = ev_pair()
                e0.record(stream)
                step(True)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                barrier()
                step_ms.append(e0.elapsed_time(e1))
        clock_info = clocks.summary()

        # the encode launch's own duration: each launch is queued behind the L2 flush
        # (a 256 MB fill that outlasts the host's enqueueing), so its events bracket
        # the kernel alone, cold L2, with no host launch gap inside
        enc_q = []
        for _ in range(5):
            flush.zero_()
            q0, q1 = ev_pair()
            q0.record(stream)
            B.cs_encode_batch(ctx, plan_list, param_list, frames_dev, [y_dev[m] for m in ms], stream)
            q1.record(stream)
            enc_q.append((q0, q1))
        torch.cuda.synchronize(dev)

        # end to end through the C ABI's host-buffer entry point: the clip in
        # from pinned host memory, encode, batched decode, PSNR, uint8 frames
        # and PSNRs out, all inside the timed region
        e2e_ms, h2d, d2h = [], 0, 0
        if want_e2e:
            clip_pin = torch.from_numpy(frames).pin_memory()
            u8_pin = [torch.empty((n_cs, h, w), dtype=torch.uint8).pin_memory() for _ in ms]
            ps_pin = [torch.empty(n_cs, dtype=torch.float64).pin_memory() for _ in ms]
            h2d = clip_pin.numel()
            d2h = sum(u.numel() + 8 * p.numel() for u, p in zip(u8_pin, ps_pin))
            for it in range(warmup + steps):
                flush.zero_()
                torch.cuda.synchronize(dev)
                barrier()
                e0, e1 = ev_pair()
                e0.record(stream)
                B.cs_codec_host(ctx, plan_list, param_list, clip_pin, u8_pin, ps_pin, stream)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                barrier()
                if it >= warmup:
                    e2e_ms.append(e0.elapsed_time(e1))
            # the host path decodes to the same bytes as the device-resident step
            for i, m in enumerate(ms):
                assert torch.equal(u8_pin[i], out_u[m].cpu()), "cs_codec_host differs (M=%d)" % m
    B.cs_ctx_status(ctx)

    def avg(evs):
        return sum(a.elapsed_time(b_) for a, b_ in evs) / len(evs)
    res = {"ctx": ctx, "plans": plans, "params": params, "frames": frames, "stream": stream,
           "keys_dev": keys_dev, "cs_dev": cs_dev, "y_dev": y_dev, "out_f": out_f, "flush": flush,
           "tuned": tuned, "plan_ms": plan_ms, "autotune_s": autotune_s, "step_ms": step_ms,
           "e2e_ms": e2e_ms, "h2d": h2d, "d2h": d2h, "clocks": clock_info,
           "launches_per_step": launches_per_step, "dec_ms": avg(dec_ev), "enc_ms": avg(enc_ev),
           "enc_kernel_ms": avg(enc_q),
           "psnr_ms": avg(psnr_ev), "n_cs": n_cs, "nblk": nblk,
           "pixels_step": len(ms) * n_cs * h * w,
           "flops": sum(decode_flops(n_cs * nblk, m, n, iters) for m in ms),
           "psnr": {str(m): float(np.mean(psnr_dev[m].cpu().numpy())) for m in ms},
           "enc_bytes": frames.nbytes + sum(4 * n_cs * nblk * m for m in ms),
           "psnr_bytes": len(ms) * n_cs * h * w * (1 + 4)}
    res["engines"] = sorted({engine if engine != B.CS_ENGINE_AUTO else tuned[str(m)]["engine"] for m in ms})
    tc_engines = (B.CS_ENGINE_TC, B.CS_ENGINE_TC_STREAM, B.CS_ENGINE_TC_CHUNK)
    res["tc_used"] = engine in tc_engines or (
        engine == B.CS_ENGINE_AUTO and all(t["engine"] in tc_engines for t in tuned.values()))
    res["mixed"], res["mixed_out"] = {}, {}
    if want_mixed and res["tc_used"]:
        # the same batched decode with mixed precision: bulk products in one 16-bit
        # MMA, the last 20 iterations FP32-grade (or split bf16 throughout)
        for name, prec, tail in (("fp16_tail20", B.CS_FP16, 20), ("bf16_tail20", B.CS_BF16, 20),
                                 ("bf16x2", B.CS_BF16X2, 0)):
            mp = [B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops,
                                lambda_rel=wl["lambda_rel"], engine=engine, precision=prec,
                                fp32_tail_iters=tail) for m in ms]
            mo = [torch.empty((n_cs, h, w), dtype=torch.float32, device=dev) for _ in ms]
            evs = []
            with torch.cuda.stream(stream):
                for it in range(2 + 3):
                    flush.zero_()
                    a0, a1 = ev_pair()
                    a0.record(stream)
                    B.cs_decode_batch(ctx, plan_list, mp, [keys_dev] * len(ms),
                                      [y_dev[m] for m in ms], mo, None, stream)
                    a1.record(stream)
                    if it >= 2:
                        evs.append((a0, a1))
                torch.cuda.synchronize(dev)
            B.cs_ctx_status(ctx)
            res["mixed"][name] = {"decode_ms_per_step": avg(evs),
                                  "achieved_tflops": res["flops"] / (avg(evs) / 1e3) / 1e12,
                                  "vs_fp32_decode": res["dec_ms"] / avg(evs)}
            res["mixed_out"][name] = {m: mo[i] for i, m in enumerate(ms)}
    return res


def codec_free(B, res):
    for p in res["plans"].values():
        B.cs_plan_destroy(p)
    B.cs_ctx_destroy(res["ctx"])


def roofline(flops, ms, peaks, peak_kind, tc_used, clock_info, n_sm, traffic=None):
    """The decode's achieved algorithmic TFLOP/s against the tensor peak (the
    measured bf16 burst figure: the decode launch lasts well under a second; the
    kind::f16 MMAs with fp16 operands run at the bf16 rate), or, on the plain
    kernel, against the FP32 FMA peak of the SIMT lanes."""
    achieved = flops / (ms / 1e3) / 1e12
    if tc_used:
        peak, bound = peaks["bf16_tflops"], "tensor"
        src = "%s bf16 dense, burst (MEASURED_PEAKS.json bf16_tflops)" % peak_kind
    else:
        clk = clock_info.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak, bound = n_sm * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12, "alu"
        src = "FP32 FMA: SMs x 128 lanes x 2 x max SM clock"
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": "decode", "peak_source": src}


def hbm_kernels(res, peaks):
    def gbs(ms_, nbytes):
        return {"ms_per_step": ms_, "bytes_per_step": nbytes, "achieved_gbs": nbytes / (ms_ / 1e3) / 1e9,
                "peak_gbs": peaks["hbm_gbs"], "frac": nbytes / (ms_ / 1e3) / 1e9 / peaks["hbm_gbs"]}
    enc = gbs(res["enc_kernel_ms"], res["enc_bytes"])
    enc["ms_in_step"] = res["enc_ms"]
    return {"encode": enc, "psnr": gbs(res["psnr_ms"], res["psnr_bytes"]),
            "note": "algorithmic bytes: the step's one encode call (cs_encode_batch, every M in one "
                    "launch) reads the clip once and writes every M's y. encode.ms_per_step is the "
                    "launch's own duration (queued behind an L2 flush: cold L2, no host gap); "
                    "ms_in_step is the same call timed inside the step (idle GPU before it)"}


def tv_run(B, torch, dev, res, wl, iters, with_oracle):
    """TV recovery (the paper's TVAL3 regulariser) of the clip at its largest M:
    on the on-chip tensor-core TV kernel where the shape fits it (16x16 blocks,
    M <= 128), else on the streaming tensor-core one (blocks of 64, 256 or 1024
    pixels), else on the plain per-block kernel, each timed once after a warm-up
    call; with the tensor cores, the plain kernel is timed beside them on the same
    input.  The oracle checks the first block row of the first CS frame."""
    h, w, b = wl["height"], wl["width"], wl["block"]
    m = max(wl["ms"])
    n_cs, stream = res["n_cs"], res["stream"]
    n_gops = wl["frames"] // wl["gop"]

    def timed(engine):
        p = B.make_params(h, w, wl["gop"], b, m, iters=iters, n_gops=n_gops, engine=engine)
        out = torch.empty((n_cs, h, w), dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            for _ in range(2):
                a0 = torch.cuda.Event(enable_timing=True)
                a1 = torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                B.cs_decode_gop_tv(res["plans"][m], p, res["keys_dev"], res["y_dev"][m], out, None,
                                   stream)
                a1.record(stream)
                torch.cuda.synchronize(dev)
        B.cs_ctx_status(res["ctx"])
        return out, a0.elapsed_time(a1)

    tv_out = None
    for engine, kernel in [
            (B.CS_ENGINE_TC, "on-chip tensor-core TV kernel (k_tv_tc, FP32-grade split-fp16 products)"),
            (B.CS_ENGINE_TC_STREAM, "streaming tensor-core TV kernel (k_tv_tcs, FP32-grade split-fp16 "
                                    "products, Phi images streamed from L2)"),
            (B.CS_ENGINE_PLAIN, "plain FP32 TV kernel (k_tv_plain)")]:
        try:
            tv_out, tv_ms = timed(engine)
            break
        except B.CsError as e:
            if e.status != B.CS_EINVAL or engine == B.CS_ENGINE_PLAIN:
                raise
    tv_psnr = torch.empty(n_cs, dtype=torch.float64, device=dev)
    B.cs_psnr(res["cs_dev"], tv_out, n_cs, h, w, tv_psnr, stream)
    torch.cuda.synchronize(dev)
    flops = 4.0 * m * b * b * iters * n_cs * res["nblk"]
    out = {"workload": "the clip at M=%d, %d iters, beta=1/8, mu=1" % (m, iters), "kernel": kernel,
           "decode_ms": tv_ms, "mpixel_per_s": n_cs * h * w / (tv_ms / 1e3) / 1e6,
           "achieved_tflops": flops / (tv_ms / 1e3) / 1e12,
           "psnr_db": float(np.mean(tv_psnr.cpu().numpy()))}
    if "tensor-core" in kernel:
        plain_out, plain_ms = timed(B.CS_ENGINE_PLAIN)
        keys = res["keys_dev"].repeat_interleave(wl["gop"] - 1, dim=0).to(torch.float64)
        d = (tv_out.to(torch.float64) - plain_out.to(torch.float64)).norm()
        out["plain_kernel"] = {"decode_ms": plain_ms,
                               "mpixel_per_s": n_cs * h * w / (plain_ms / 1e3) / 1e6,
                               "tensor_speedup": plain_ms / tv_ms,
                               "residual_rel_l2_vs_tensor": float(d / (plain_out.to(torch.float64) - keys).norm())}
        del plain_out
    if with_oracle:
        from oracle import cs_oracle as O
        frames = res["frames"]
        oplan = O.Plan(b * b, m, wl["seed"])
        k = min(8, -(-w // b))
        res1 = frames[1].astype(np.int64) - frames[0].astype(np.int64)
        y0 = O.blockify(res1.astype(np.float64), b)[:k] @ oplan.phi.T
        r0 = O.tv_adm(oplan.phi, y0, oplan.lipschitz, iters)
        rows = min(b, h)
        full = np.zeros((rows, k * b))
        for j in range(k):
            full[:, j * b:(j + 1) * b] = r0[j].reshape(b, b)[:rows]
        cols = min(k * b, w)
        want = frames[0][:rows, :cols].astype(np.float64) + full[:, :cols]
        got = tv_out[0, :rows, :cols].cpu().numpy().astype(np.float64)
        key = frames[0][:rows, :cols].astype(np.float64)
        out["vs_oracle"] = {"sample": "first %d blocks of the first CS frame's first block row" % k,
                            "frame_rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
                            "residual_rel_l2": float(np.linalg.norm(got - want) /
                                                     max(np.linalg.norm(want - key), 1e-30)),
                            "dpsnr_db": float(O.psnr(frames[1][:rows, :cols], got) -
                                                  O.psnr(frames[1][:rows, :cols], want))}
    return out


def plain_run(B, torch, dev, res, wl):
    """The plain per-block FP32 decode (one CTA per block group, SIMT) of the
    same clip, one batched call, timed once after a warm-up call."""
    h, w, gop, b, iters = wl["height"], wl["width"], wl["gop"], wl["block"], wl["iters"]
    ms = wl["ms"]
    n_gops = wl["frames"] // gop
    stream = res["stream"]
    pp = [B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops, lambda_rel=wl["lambda_rel"],
                        engine=B.CS_ENGINE_PLAIN) for m in ms]
    outs = [torch.empty((res["n_cs"], h, w), dtype=torch.float32, device=dev) for _ in ms]
    with torch.cuda.stream(stream):
        for it in range(2):
            res["flush"].zero_()
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            B.cs_decode_batch(res["ctx"], [res["plans"][m] for m in ms], pp,
                              [res["keys_dev"]] * len(ms), [res["y_dev"][m] for m in ms], outs,
                              None, stream)
            a1.record(stream)
            torch.cuda.synchronize(dev)
    B.cs_ctx_status(res["ctx"])
    pms = a0.elapsed_time(a1)
    err = max(float(torch.linalg.norm(outs[i] - res["out_f"][m]) / torch.linalg.norm(res["out_f"][m]))
              for i, m in enumerate(ms))
    return {"engine": "plain FP32 SIMT kernel (CS_ENGINE_PLAIN) at its default launch shape",
            "decode_ms": pms, "mpixel_per_s": res["pixels_step"] / (pms / 1e3) / 1e6,
            "achieved_tflops": res["flops"] / (pms / 1e3) / 1e12,
            "tensor_decode_speedup": pms / res["dec_ms"],
            "rel_l2_vs_tensor_decode": err}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--engine", choices=["auto", "plain", "tc", "tcs", "tcz"], default="auto")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD,
                    help="720p (default): 32x32 blocks, M = 102; cif: the CIF M-sweep; "
                         "mixed64: the heterogeneous batch")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-m", type=int, default=0,
                    help="run a single M of the sweep (profiling runs)")
    ap.add_argument("--frames", type=int, default=0,
                    help="use only the clip's first F frames, a multiple of the GOP (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end loop")
    ap.add_argument("--no-batch", action="store_true",
                    help="one decode call per M instead of one batched launch")
    ap.add_argument("--no-extras", action="store_true",
                    help="leave out the other workloads (CIF sweep, plain engine, mixed64, serving)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-tv", action="store_true", help="skip the TV-recovery measurement")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision decode measurement")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps, always
    rank, world, local = dist_env()
    wl = dict(WORKLOADS[args.workload])
    if args.only_m and args.workload != "mixed64":
        if args.only_m not in wl["ms"]:
            ap.error("--only-m must be one of %s" % wl["ms"])
        wl["ms"] = [args.only_m]
    if args.frames and args.workload != "mixed64":
        if args.frames % wl["gop"] or not 0 < args.frames <= wl["frames"]:
            ap.error("--frames must be a multiple of the GOP (%d), at most %d" % (wl["gop"], wl["frames"]))
        wl["frames"] = args.frames

    if args.impl == "reference":
        if rank == 0:
            if args.workload == "mixed64":
                print(json.dumps({"impl": "reference", "unavailable":
                                  "the oracle arm is measured on the 720p and cif workloads"}))
            else:
                from paper_1311_1419_gb300 import scenes
                frames = scenes.surveillance_video(wl["frames"], wl["height"], wl["width"],
                                                   seed=wl["seed"])
                run_reference(args, wl, frames)
        return

    import torch

    import __graft_entry__
    from paper_1311_1419_gb300 import binding as B

    __graft_entry__.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    peaks, peak_kind = read_peaks()
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    if args.workload == "mixed64":
        if rank == 0:
            r = run_mixed64(args, wl, B, torch, dev, args.steps, args.warmup)
            line = dict(r)
            line.update({"n_gpus": 1, "higher_is_better": True, "scaling": "weak",
                         "vs_baseline": None, "data": "synthetic",
                         "config": {"workload": wl["workload"]}})
            line.pop("workload")
            print(json.dumps(line), flush=True)
        return

    engine = {"auto": B.CS_ENGINE_AUTO, "plain": B.CS_ENGINE_PLAIN, "tc": B.CS_ENGINE_TC,
              "tcs": B.CS_ENGINE_TC_STREAM, "tcz": B.CS_ENGINE_TC_CHUNK}[args.engine]
    res = codec_run(wl, B, torch, dev, world, barrier, args.steps, args.warmup, engine,
                    want_e2e=not args.no_e2e, want_mixed=not args.no_mixed, no_batch=args.no_batch)
    total_ms = max_over_ranks(sum(res["step_ms"]), world, dev)
    e2e_total = max_over_ranks(sum(res["e2e_ms"]), world, dev) if res["e2e_ms"] else float("nan")
    value = job_throughput(world, res["pixels_step"], args.steps, total_ms) / 1e6
    e2e_value = job_throughput(world, res["pixels_step"], args.steps, e2e_total) / 1e6
    all_fp32 = all(p.precision == B.CS_FP32 for p in res["params"].values())
    traffic = decode_traffic(args.workload, res) if (
        res["tc_used"] and all_fp32 and not args.no_batch and not args.only_m and not args.frames) else None
    roof = roofline(res["flops"], res["dec_ms"], peaks, peak_kind, res["tc_used"], res["clocks"],
                    n_sm, traffic)
    mixed = res["mixed"]
    for name in mixed:
        mixed[name]["frac"] = mixed[name]["achieved_tflops"] / roof["peak"]
    solo = rank == 0 and world == 1
    extras = solo and not args.no_extras

    tv = None
    if not args.no_tv and args.engine != "tc" and rank == 0:
        tv = tv_run(B, torch, dev, res, wl, wl["iters"], with_oracle=solo and not args.no_cpu_baseline)
    plain = plain_run(B, torch, dev, res, wl) if (extras and res["tc_used"]) else None

    cif = None
    if extras and args.workload != "cif":
        cwl = dict(WORKLOADS["cif"])
        cres = codec_run(cwl, B, torch, dev, 1, barrier, 5, 3, B.CS_ENGINE_AUTO, want_e2e=False,
                         want_mixed=False)
        cif = {"workload": cwl["workload"], "steps": 5, "warmup": 3,
               "value": cres["pixels_step"] * 5 / (sum(cres["step_ms"]) / 1e3) / 1e6,
               "unit": "Mpixel/s", "ms_per_step": sum(cres["step_ms"]) / 5,
               "decode_ms_per_step": cres["dec_ms"], "decode_gflop_per_step": cres["flops"] / 1e9,
               "roofline": roofline(cres["flops"], cres["dec_ms"], peaks, peak_kind, cres["tc_used"],
                                    cres["clocks"], n_sm, decode_traffic("cif", cres)),
               "gpu_launches": cres["launches_per_step"] * 5, "psnr_db": cres["psnr"]}
        if not args.no_tv:
            cif["tv_recovery"] = tv_run(B, torch, dev, cres, cwl, cwl["iters"],
                                        with_oracle=not args.no_cpu_baseline)
        if not args.no_cpu_baseline:
            _, _, cref = oracle_sample(cres["frames"], cwl, cwl["oracle_frames"])
            cif["parity_vs_oracle"] = {
                str(m): parity(cres["frames"],
                               cres["out_f"][m][:cwl["oracle_frames"]].cpu().numpy().astype(np.float64),
                               cref[m]) for m in cwl["ms"]}
        codec_free(B, cres)

    mixed64 = None
    if extras:
        mwl = dict(WORKLOADS["mixed64"])
        mixed64 = run_mixed64(args, mwl, B, torch, dev, 3, 3, with_oracle=not args.no_cpu_baseline)

    serving = None
    if solo and not args.no_serving:
        rates = [50, 100, 200, 400] if extras else [100]
        cfgs = [("queue_fp32", B.CS_SERVING_QUEUE, B.CS_FP32, 0)]
        if extras:
            cfgs += [("launch_fp32", B.CS_SERVING_LAUNCH, B.CS_FP32, 0),
                     ("queue_fp16_tail20", B.CS_SERVING_QUEUE, B.CS_FP16, 20)]
        serving = {"workload": SERVING["workload"],
                   "modes": "queue: the device work queue (one persistent streaming-kernel launch "
                            "drains the tiles of every request in flight); launch: one decode launch "
                            "per request on the kernel its shape picks"}
        serving.update(serving_run(B, torch, dev, cfgs, rates, 2.0, batch_ref=extras))

    cpu = parity_d = None
    if solo and not args.no_cpu_baseline:
        n_sample = wl["oracle_frames"]
        secs, pix, ref = oracle_sample(res["frames"], wl, n_sample)
        nblk = res["nblk"]
        cpu = {"value": pix / secs / 1e6, "unit": "Mpixel/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": "first %d CS frame(s) (%d blocks) at each M in %s, %d iters; numpy "
                         "FP64 (BLAS threads = cores)" % (n_sample, n_sample * nblk, wl["ms"],
                                                          wl["iters"])}
        parity_d = {str(m): parity(res["frames"],
                                   res["out_f"][m][:n_sample].cpu().numpy().astype(np.float64), ref[m])
                    for m in wl["ms"]}
        parity_d["sample"] = "first %d CS frame(s), every block, FP64 oracle" % n_sample
        for name, outs in res["mixed_out"].items():
            mixed[name]["vs_oracle"] = {
                str(m): parity(res["frames"], outs[m][:n_sample].cpu().numpy().astype(np.float64), ref[m])
                for m in wl["ms"]}

    if rank == 0:
        line = {
            "metric": wl["metric"], "value": value, "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl["workload"], "engine": args.engine,
                       "decode": "per-M calls" if args.no_batch else
                       "one batched cs_decode_batch call (%d plan%s)" % (len(wl["ms"]), "" if len(wl["ms"]) == 1 else "s"),
                       "l2": "flushed before every timed step (256 MB write)",
                       "parallelism": "replicas x%d" % world},
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": None if not res["e2e_ms"] else {
                "value": e2e_value, "unit": "Mpixel/s", "h2d_bytes_per_step": res["h2d"],
                "d2h_bytes_per_step": res["d2h"], "entry_point": "cs_codec_host"},
            "gpu_launches": res["launches_per_step"] * args.steps,
            "clocks": res["clocks"],
            "plan_ms": res["plan_ms"],
            "autotune": res["tuned"],
            "decode_ms_per_step": res["dec_ms"],
            "decode_gflop_per_step": res["flops"] / 1e9,
            "psnr_db": res["psnr"],
            "parity_vs_oracle": parity_d,
            "mixed_precision": mixed or None,
            "hbm_kernels": hbm_kernels(res, peaks),
            "plain_engine": plain,
            "cif_sweep": cif,
            "mixed64": mixed64,
            "tv_recovery": tv,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)

    codec_free(B, res)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
