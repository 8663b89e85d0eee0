#!/usr/bin/env python
"""Recovered Mpixel/s of the block-CS video codec hot path on GB300.

One step = the whole hot path over the CIF M-sweep clip: for each M in
{26, 51, 77, 128}, encode all 8 GOPs (64 frames, 352x288, GOP 8, 16x16 blocks)
then decode them with 300 FISTA iterations and score the result (PSNR).  The
four plans (Phi, A, L) are built once before timing, like weights; their build
time is reported as plan_ms.  value = recovered CS-frame pixels per second.

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
    "cif": {
        "workload": "CIF 352x288, 64 frames, GOP 8 (1 raw key + 7 CS), 16x16 blocks (N=256), "
                    "M in {26,51,77,128} (CR sweep), Gaussian Phi N(0,1/M) Philox seed 0, "
                    "FISTA 300 iters, lambda=0.01*||A^T y||_inf, synthetic surveillance scene",
        "metric": "recovered Mpixel/s at fixed iters (CIF M-sweep, FISTA 300 iters)",
        "height": 288, "width": 352, "frames": 64, "gop": 8, "block": 16,
        "ms": [26, 51, 77, 128], "iters": 300, "lambda_rel": 0.01, "seed": 0, "oracle_frames": 5,
    },
    "720p": {
        "workload": "720p 1280x720, 96 frames, GOP 16 (1 raw key + 15 CS), 32x32 blocks (N=1024), "
                    "M=102 (10%), Gaussian Phi N(0,1/M) Philox seed 0, FISTA 300 iters, "
                    "lambda=0.01*||A^T y||_inf, synthetic surveillance scene",
        "metric": "recovered Mpixel/s at fixed iters (720p, 32x32 blocks, FISTA 300 iters)",
        "height": 720, "width": 1280, "frames": 96, "gop": 16, "block": 32,
        "ms": [102], "iters": 300, "lambda_rel": 0.01, "seed": 0, "oracle_frames": 1,
    },
}
WORKLOADS["mixed64"] = {
    "workload": "64 GOPs (seeds 0..63) of QCIF/CIF/720p, 8x8/16x16/32x32 blocks, M/N uniform in "
                "5%..50%, GOP uniform in 4..32, FISTA 300 iters, synthetic surveillance scenes; "
                "split-BF16 on the tensor-core kernels (on-chip or streaming), FP32 on the plain "
                "kernel for any shape they do not cover; one cs_decode_batch captured in a CUDA graph",
    "metric": "recovered Mpixel/s at fixed iters (64 heterogeneous GOPs, one graph-captured batch)",
    "iters": 300, "lambda_rel": 0.01, "seed": 0, "jobs": 64,
}
WORKLOAD = WORKLOADS["cif"]
METRIC = WORKLOAD["metric"]
L2_FLUSH_BYTES = 256 << 20
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of the CIF step's decode, its
# two tensor-core launches together, from one ncu capture of that exact configuration;
# reported as roofline.traffic for it only (null for any other configuration or kernel)
CIF_DECODE_DRAM_BYTES = 62_840_000
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


def serving_run(B, torch, dev, precision, tail, rates, seconds, hbm_budget=8 << 30):
    """Open-loop serving: Poisson arrivals over the camera mix at each rate;
    returns one dict per rate (p50/p99 latency, Mpixel/s, admitted, refused)."""
    from paper_1311_1419_gb300 import scenes

    rng = np.random.default_rng(SERVING["seed"])
    res = [scenes.RESOLUTIONS[k] for k in ("qcif", "cif", "720p", "1080p")]
    base = {r: scenes.surveillance_video(32, r[0], r[1], seed=i) for i, r in enumerate(res)}
    ctx = B.cs_ctx_create(dev.index, hbm_budget)
    cams = []
    stream = torch.cuda.Stream(dev)
    try:
        for cid in range(SERVING["cameras"]):
            h, w = res[rng.choice(4, p=[0.4, 0.3, 0.2, 0.1])]
            gop = int(rng.integers(4, 33))
            b = (16, 32)[rng.integers(2)]
            m = max(1, int(np.rint(b * b * rng.uniform(0.05, 0.25))))
            plan = B.cs_make_phi(ctx, b * b, m, cid)
            tc = (m + 15) // 16 * 16 <= 512       # on-chip or streaming tensor-core kernel
            p = B.make_params(h, w, gop, b, m, iters=SERVING["iters"],
                              precision=precision if tc else B.CS_FP32,
                              fp32_tail_iters=tail if tc else 0)
            off = cid % (33 - gop)
            clip = base[(h, w)][off:off + gop]
            nblk = (-(-h // b)) * (-(-w // b))
            y = torch.empty((gop - 1, nblk, m), dtype=torch.float32, device=dev)
            B.cs_encode_gop(plan, p, torch.from_numpy(np.ascontiguousarray(clip)).to(dev), y,
                            stream)
            stream.synchronize()
            cams.append({"plan": plan, "p": p, "key": torch.from_numpy(
                np.ascontiguousarray(clip[:1])).pin_memory(), "y": y.cpu().pin_memory(),
                "shape": (gop - 1, h, w), "pixels": (gop - 1) * h * w, "free": []})
        results = []
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
                    out = c["free"].pop() if c["free"] else torch.empty(
                        c["shape"], dtype=torch.uint8).pin_memory()
                    try:
                        t = B.cs_submit(ctx, c["plan"], c["p"], c["key"], c["y"], out)
                    except B.CsError as e:
                        c["free"].append(out)
                        if e.status != B.CS_EAGAIN:
                            raise
                        refused += 1
                        break
                    cid, t_arr = backlog.pop(0)
                    inflight[t] = (cid, out, time.perf_counter() - t_arr)
                for t in list(inflight):
                    done, ms = B.cs_poll(ctx, t)
                    if done:
                        cid, out, queued = inflight.pop(t)
                        # arrival to completion: admission queueing + submit-to-done
                        lat.append(1e3 * queued + ms)
                        pixels += cams[cid]["pixels"]
                        cams[cid]["free"].append(out)
            wall = time.perf_counter() - t0
            B.cs_ctx_status(ctx)
            lat_ms = np.array(lat)
            results.append({"rate_per_s": rate, "requests": len(lat), "refused_retries": refused,
                            "p50_ms": float(np.percentile(lat_ms, 50)),
                            "p99_ms": float(np.percentile(lat_ms, 99)),
                            "mpixel_per_s": pixels / wall / 1e6})
        return results
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
    sample = ("first CS frame of the clip (396 blocks) at each M in %s, %d iters, per step"
              % (wl["ms"], wl["iters"]))
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


def mixed_launches(jobs) -> int:
    """Kernels one cs_decode_batch of the mix launches: one per group of up to 48
    jobs of each tensor-core kernel (16x16 on chip by shared-memory layout, 32x32
    cluster, streaming; one operand type here) and one per plain-kernel job."""
    groups = {}
    for j in jobs:
        b, m = j["p"].block, j["p"].m
        m16 = (m + 15) // 16 * 16
        if not j["tc"]:
            key = ("plain", len(groups))
        elif b == 16 and m <= 128:
            key = ("tc", m16 <= 96)
        elif b == 32 and m <= 128:
            key = ("tc8",)
        else:
            key = ("tcs",)
        groups[key] = groups.get(key, 0) + 1
    return sum(-(-c // 48) for c in groups.values())


def run_mixed64(args, wl):
    """The heterogeneous batch: every GOP a job of its own plan, one batched call
    captured in a CUDA graph and replayed; value = CS pixels per second."""
    import torch

    import __graft_entry__
    from paper_1311_1419_gb300 import binding as B
    from paper_1311_1419_gb300 import scenes

    __graft_entry__.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rng = np.random.default_rng(wl["seed"])
    res = [scenes.RESOLUTIONS[k] for k in ("qcif", "cif", "720p")]
    ctx = B.cs_ctx_create(0)
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
            jobs.append({"plan": plan, "p": p, "key": torch.from_numpy(np.ascontiguousarray(clip[:1])).to(dev),
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
        setup_s = time.perf_counter() - t0
        args_ = ([j["plan"] for j in jobs], [j["p"] for j in jobs], [j["key"] for j in jobs],
                 [j["y"] for j in jobs], [j["out"] for j in jobs])
        with torch.cuda.stream(stream):
            B.cs_decode_batch(ctx, *args_, None, stream)       # eager warm-up
            torch.cuda.synchronize(dev)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream, capture_error_mode="thread_local"):
                B.cs_decode_batch(ctx, *args_, None, stream)
            for _ in range(args.warmup):
                g.replay()
            torch.cuda.synchronize(dev)
            times = []
            with ClockSampler(0) as clocks:
                for _ in range(args.steps):
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
        line = {
            "metric": wl["metric"], "value": pixels / (ms / 1e3) / 1e6, "unit": "Mpixel/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x2/f32",
            "data": "synthetic", "config": {"workload": wl["workload"]},
            "jobs": len(jobs), "tensor_core_jobs": sum(j["tc"] for j in jobs),
            "pixels_per_step": pixels, "tensor_core_pixel_share": tc_pix / pixels,
            "gflop_per_step": sum(j["flops"] for j in jobs) / 1e9,
            "gpu_launches": mixed_launches(jobs), "clocks": clocks.summary(), "setup_s": setup_s,
            "autotuned_shapes": len(tuned),
        }
        print(json.dumps(line), flush=True)
    finally:
        for j in jobs:
            B.cs_plan_destroy(j["plan"])
        B.cs_ctx_destroy(ctx)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--engine", choices=["auto", "plain", "tc", "tcs"], default="auto")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="cif",
                    help="cif: the CIF M-sweep (default); 720p: 32x32 blocks, M = 102")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--only-m", type=int, default=0,
                    help="run a single M of the sweep (profiling runs)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end loop")
    ap.add_argument("--no-batch", action="store_true",
                    help="one decode call per M instead of one batched launch")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-tv", action="store_true", help="skip the TV-recovery measurement")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision decode measurement")
    ap.add_argument("--serving-sweep", action="store_true",
                    help="sweep the arrival rate to saturation, FP32 and mixed precision")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up steps, always
    rank, world, local = dist_env()
    wl = dict(WORKLOADS[args.workload])
    if args.workload == "mixed64":
        if args.impl == "reference":
            if rank == 0:
                print(json.dumps({"impl": "reference", "unavailable":
                                  "the oracle arm is measured on the cif and 720p workloads"}))
            return
        if rank == 0:
            run_mixed64(args, wl)
        return
    if args.only_m:
        if args.only_m not in wl["ms"]:
            ap.error("--only-m must be one of %s" % wl["ms"])
        wl["ms"] = [args.only_m]

    from paper_1311_1419_gb300 import scenes

    frames = scenes.surveillance_video(wl["frames"], wl["height"], wl["width"], seed=wl["seed"])

    if args.impl == "reference":
        if rank == 0:
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

    engine = {"auto": B.CS_ENGINE_AUTO, "plain": B.CS_ENGINE_PLAIN, "tc": B.CS_ENGINE_TC,
              "tcs": B.CS_ENGINE_TC_STREAM}[args.engine]
    h, w, gop, b, iters = wl["height"], wl["width"], wl["gop"], wl["block"], wl["iters"]
    n = b * b
    n_gops = wl["frames"] // gop
    n_cs = n_gops * (gop - 1)
    nblk = (-(-h // b)) * (-(-w // b))
    cs_idx = [t for t in range(wl["frames"]) if t % gop]

    ctx = B.cs_ctx_create(local)
    t0 = time.perf_counter()
    plans = {m: B.cs_make_phi(ctx, n, m, wl["seed"]) for m in wl["ms"]}
    plan_ms = 1e3 * (time.perf_counter() - t0)
    params = {m: B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops,
                               lambda_rel=wl["lambda_rel"], engine=engine) for m in wl["ms"]}
    # the decode shape of every (N, M) is picked by timing, once, before the timed region
    tuned = {str(m): dict(zip(("engine", "plain_threads", "plain_blocks_per_cta", "ns_per_block_iter"),
                              B.cs_autotune(ctx, plans[m]))) for m in wl["ms"]}

    stream = torch.cuda.Stream(dev)
    frames_dev = torch.from_numpy(frames).to(dev)
    keys_host = np.ascontiguousarray(frames[::gop])
    keys_dev = torch.from_numpy(keys_host).to(dev)
    cs_dev = torch.from_numpy(np.ascontiguousarray(frames[cs_idx])).to(dev)
    y_dev = {m: torch.empty((n_cs, nblk, m), dtype=torch.float32, device=dev) for m in wl["ms"]}
    out_f = {m: torch.empty((n_cs, h, w), dtype=torch.float32, device=dev) for m in wl["ms"]}
    out_u = {m: torch.empty((n_cs, h, w), dtype=torch.uint8, device=dev) for m in wl["ms"]}
    psnr_dev = {m: torch.empty(n_cs, dtype=torch.float64, device=dev) for m in wl["ms"]}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    dec_ev = []
    plan_list = [plans[m] for m in wl["ms"]]
    param_list = [params[m] for m in wl["ms"]]
    # our kernels per step: one encode and one PSNR per M, and the decode: one
    # launch per call with --no-batch, else one per (operand type, shared-memory
    # layout) group of the 16x16 tensor path (M16 <= 96 or <= 128), one per group
    # of the 32x32 cluster path, one per group of the streaming path, one per
    # plain-kernel job (FP32: one operand type)
    def decode_launches():
        if args.no_batch:
            return len(wl["ms"])
        groups, plain = set(), 0
        for m in wl["ms"]:
            m16 = (m + 15) // 16 * 16
            eng = engine if engine != B.CS_ENGINE_AUTO else tuned[str(m)]["engine"]
            if eng == B.CS_ENGINE_PLAIN:
                plain += 1
            elif eng == B.CS_ENGINE_TC_STREAM:
                groups.add(("tcs",))
            elif n == 256:
                groups.add(("tc", m16 <= 96))
            else:
                groups.add(("tc8",))
                # a large 32x32 job also launches its streaming tail on the SMs whole
                # clusters leave idle (the library's rule: a tail once the job has more
                # tiles than clusters x 30; 15 clusters of 8 are co-resident on this part)
                tiles = -(-(n_cs * nblk) // 128)
                idle = 2 * (torch.cuda.get_device_properties(dev).multi_processor_count - 8 * 15)
                if idle > 0 and tiles > 15 * 30:
                    groups.add(("tc8 tail",))
        return len(groups) + plain
    launches_per_step = 2 * len(wl["ms"]) + decode_launches()

    enc_ev, psnr_ev = [], []

    def ev_pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def step(record_decode: bool, fr, keys):
        if record_decode:
            a0, a1 = ev_pair()
            a0.record(stream)
        for m in wl["ms"]:
            B.cs_encode_gop(plans[m], params[m], fr, y_dev[m], stream)
        if record_decode:
            a1.record(stream)
            enc_ev.append((a0, a1))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        if args.no_batch:
            for m in wl["ms"]:
                B.cs_decode_gop(plans[m], params[m], keys, y_dev[m], out_f[m], out_u[m], stream)
        else:
            B.cs_decode_batch(ctx, plan_list, param_list, [keys] * len(wl["ms"]),
                              [y_dev[m] for m in wl["ms"]], [out_f[m] for m in wl["ms"]],
                              [out_u[m] for m in wl["ms"]], stream)
        if record_decode:
            e1.record(stream)
            dec_ev.append((e0, e1))
        if record_decode:
            c0, c1 = ev_pair()
            c0.record(stream)
        for m in wl["ms"]:
            B.cs_psnr(cs_dev, out_f[m], n_cs, h, w, psnr_dev[m], stream)
        if record_decode:
            c1.record(stream)
            psnr_ev.append((c0, c1))

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step(False, frames_dev, keys_dev)
        torch.cuda.synchronize(dev)

        # device-resident timed region, L2 flushed before every step
        step_ms = []
        with ClockSampler(local) as clocks:
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize(dev)
                barrier()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step(True, frames_dev, keys_dev)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                barrier()
                step_ms.append(e0.elapsed_time(e1))
        clock_info = clocks.summary()

        # end to end through the C ABI from pinned host memory
        frames_pin = torch.from_numpy(frames).pin_memory()
        keys_pin = torch.from_numpy(keys_host).pin_memory()
        u8_pin = {m: torch.empty((n_cs, h, w), dtype=torch.uint8).pin_memory() for m in wl["ms"]}
        ps_pin = {m: torch.empty(n_cs, dtype=torch.float64).pin_memory() for m in wl["ms"]}
        fr_in = torch.empty_like(frames_dev)
        key_in = torch.empty_like(keys_dev)
        h2d = frames_pin.numel() + keys_pin.numel()
        d2h = sum(u8_pin[m].numel() + 8 * ps_pin[m].numel() for m in wl["ms"])
        e2e_ms = []
        for it in range(0 if args.no_e2e else args.warmup + args.steps):
            flush.zero_()
            torch.cuda.synchronize(dev)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fr_in.copy_(frames_pin, non_blocking=True)
            key_in.copy_(keys_pin, non_blocking=True)
            step(False, fr_in, key_in)
            for m in wl["ms"]:
                u8_pin[m].copy_(out_u[m], non_blocking=True)
                ps_pin[m].copy_(psnr_dev[m], non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            barrier()
            if it >= args.warmup:
                e2e_ms.append(e0.elapsed_time(e1))

    total_ms = max_over_ranks(sum(step_ms), world, dev)
    e2e_total = max_over_ranks(sum(e2e_ms), world, dev) if e2e_ms else float("nan")
    pixels_step = len(wl["ms"]) * n_cs * h * w
    value = job_throughput(world, pixels_step, args.steps, total_ms) / 1e6
    e2e_value = job_throughput(world, pixels_step, args.steps, e2e_total) / 1e6

    # roofline of the dominant kernel (the decode), from its own launch events
    dec_ms = sum(a.elapsed_time(b_) for a, b_ in dec_ev) / len(dec_ev)
    blocks = n_cs * nblk
    flops = sum(decode_flops(blocks, m, n, iters) for m in wl["ms"])
    peaks, peak_kind = read_peaks()
    # the tensor-core roofline applies when every plan decodes on the tensor cores
    tc_used = engine == B.CS_ENGINE_TC or (
        engine == B.CS_ENGINE_AUTO and all(t["engine"] == B.CS_ENGINE_TC for t in tuned.values()))
    achieved = flops / (dec_ms / 1e3) / 1e12
    # the captured traffic belongs to the CIF sweep's batched FP32 tensor-core decode only
    traffic = CIF_DECODE_DRAM_BYTES if (tc_used and args.workload == "cif" and not args.no_batch
                                        and not args.only_m and
                                        all(p.precision == B.CS_FP32 for p in params.values())) else None
    if tc_used:
        # kind::f16 MMAs (fp16 operands): the measured bf16 peak x the nominal
        # fp16:bf16 ratio of 1; sustained, as the decode runs inside a long step
        peak = peaks["bf16_tflops_sustained"]
        bound = "tensor"
    else:
        clk = clock_info.get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = n_sm * FP32_LANES_PER_SM * 2 * clk * 1e6 / 1e12
        bound = "alu"
    psnr = {m: float(np.mean(psnr_dev[m].cpu().numpy())) for m in wl["ms"]}

    # the HBM-bound kernels beside the decode: encode (frames in, y out, per M) and
    # the PSNR tail (uint8 reference + float32 frames in), achieved algorithmic GB/s
    def gbs(evs, nbytes):
        ms_ = sum(a.elapsed_time(b_) for a, b_ in evs) / len(evs)
        return {"ms_per_step": ms_, "bytes_per_step": nbytes, "achieved_gbs": nbytes / (ms_ / 1e3) / 1e9,
                "peak_gbs": peaks["hbm_gbs"], "frac": nbytes / (ms_ / 1e3) / 1e9 / peaks["hbm_gbs"]}
    enc_bytes = sum(frames.nbytes + 4 * n_cs * nblk * m for m in wl["ms"])
    psnr_bytes = len(wl["ms"]) * n_cs * h * w * (1 + 4)
    hbm_kernels = {"encode": gbs(enc_ev, enc_bytes), "psnr": gbs(psnr_ev, psnr_bytes),
                   "note": "algorithmic bytes (each encode call reads the clip once and writes "
                           "its y; frames re-read by later calls may hit L2)"}

    # the same batched decode with mixed precision: bulk products in one 16-bit
    # MMA, the last 20 iterations FP32-grade (or split bf16 throughout)
    mixed, mixed_out = None, {}
    if tc_used and not args.no_mixed:
        mixed = {}
        for name, prec, tail in (("fp16_tail20", B.CS_FP16, 20), ("bf16_tail20", B.CS_BF16, 20),
                                 ("bf16x2", B.CS_BF16X2, 0)):
            mp = [B.make_params(h, w, gop, b, m, iters=iters, n_gops=n_gops,
                                lambda_rel=wl["lambda_rel"], engine=engine, precision=prec,
                                fp32_tail_iters=tail) for m in wl["ms"]]
            mo = [torch.empty((n_cs, h, w), dtype=torch.float32, device=dev) for _ in wl["ms"]]
            evs = []
            with torch.cuda.stream(stream):
                for it in range(2 + 3):
                    flush.zero_()
                    a0 = torch.cuda.Event(enable_timing=True)
                    a1 = torch.cuda.Event(enable_timing=True)
                    a0.record(stream)
                    B.cs_decode_batch(ctx, plan_list, mp, [keys_dev] * len(wl["ms"]),
                                      [y_dev[m] for m in wl["ms"]], mo, None, stream)
                    a1.record(stream)
                    if it >= 2:
                        evs.append((a0, a1))
                torch.cuda.synchronize(dev)
            B.cs_ctx_status(ctx)
            mms = sum(a.elapsed_time(b_) for a, b_ in evs) / len(evs)
            ach = flops / (mms / 1e3) / 1e12
            mixed[name] = {"decode_ms_per_step": mms, "achieved_tflops": ach,
                           "frac": ach / peak,
                           "vs_fp32_decode": dec_ms / mms}
            mixed_out[name] = {m: mo[i] for i, m in enumerate(wl["ms"])}

    # TV recovery (the paper's TVAL3 regulariser) on the plain per-block kernel:
    # the clip at the largest M, timed once after a warm-up call
    tv = None
    tv_m = max(wl["ms"])
    if not args.no_tv and args.engine != "tc":
        tv_out = torch.empty((n_cs, h, w), dtype=torch.float32, device=dev)
        with torch.cuda.stream(stream):
            B.cs_decode_gop_tv(plans[tv_m], params[tv_m], keys_dev, y_dev[tv_m], tv_out, None, stream)
            torch.cuda.synchronize(dev)
            a0, a1 = ev_pair()
            a0.record(stream)
            B.cs_decode_gop_tv(plans[tv_m], params[tv_m], keys_dev, y_dev[tv_m], tv_out, None, stream)
            a1.record(stream)
            torch.cuda.synchronize(dev)
        B.cs_ctx_status(ctx)
        tv_ms = a0.elapsed_time(a1)
        tv_psnr = torch.empty(n_cs, dtype=torch.float64, device=dev)
        B.cs_psnr(cs_dev, tv_out, n_cs, h, w, tv_psnr, stream)
        torch.cuda.synchronize(dev)
        tv = {"workload": "the clip at M=%d, %d iters, beta=1/8, mu=1, plain FP32 kernel" % (tv_m, iters),
              "decode_ms": tv_ms, "mpixel_per_s": n_cs * h * w / (tv_ms / 1e3) / 1e6,
              "psnr_db": float(np.mean(tv_psnr.cpu().numpy()))}

    serving = None
    if rank == 0 and world == 1 and not args.no_serving:
        rates = [50, 100, 200, 300, 400, 600] if args.serving_sweep else [100]
        secs = 3.0 if args.serving_sweep else 2.0
        serving = {"workload": SERVING["workload"],
                   "fp32": serving_run(B, torch, dev, B.CS_FP32, 0, rates, secs)}
        if args.serving_sweep:
            serving["fp16_tail20"] = serving_run(B, torch, dev, B.CS_FP16, 20, rates, secs)

    cpu = None
    parity = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        n_sample = wl["oracle_frames"]
        secs, pix, ref = oracle_sample(frames, wl, n_sample)
        cpu = {"value": pix / secs / 1e6, "unit": "Mpixel/s", "cores": os.cpu_count(),
               "kind": "oracle",
               "sample": "first %d CS frames (%d blocks) at each M in %s, %d iters; numpy "
                         "FP64 (BLAS threads = cores)" % (n_sample, n_sample * nblk, wl["ms"],
                                                          iters)}
        from oracle import cs_oracle as O
        parity = {}
        for m in wl["ms"]:
            got = out_f[m][:n_sample].cpu().numpy().astype(np.float64)
            want = ref[m]
            orig = frames[1:1 + n_sample]
            parity[str(m)] = {
                "frame_rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
                "dpsnr_db": float(O.psnr(orig, got) - O.psnr(orig, want)),
            }
        for name, outs in mixed_out.items():
            errs = {}
            for m in wl["ms"]:
                got = outs[m][:n_sample].cpu().numpy().astype(np.float64)
                want = ref[m]
                orig = frames[1:1 + n_sample]
                errs[str(m)] = {
                    "frame_rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
                    "dpsnr_db": float(O.psnr(orig, got) - O.psnr(orig, want))}
            mixed[name]["vs_oracle"] = errs
        if tv is not None:
            # the oracle's TV decode of the first CS frame
            oplan = O.Plan(n, tv_m, wl["seed"])
            y0 = O.encode(oplan, frames[:gop], gop)[:1]
            r0 = O.tv_adm(oplan.phi, y0[0], oplan.lipschitz, iters)
            want = frames[0].astype(np.float64) + O.unblockify(r0, h, w, b)
            got = tv_out[0].cpu().numpy().astype(np.float64)
            tv["vs_oracle"] = {"frame_rel_l2": float(np.linalg.norm(got - want) / np.linalg.norm(want)),
                               "dpsnr_db": float(O.psnr(frames[1:2], got[None]) -
                                                 O.psnr(frames[1:2], want[None]))}

    if rank == 0:
        line = {
            "metric": wl["metric"], "value": value, "unit": "Mpixel/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl["workload"], "engine": args.engine,
                       "decode": "per-M calls" if args.no_batch else
                       "one batched launch (%d plans)" % len(wl["ms"]),
                       "l2": "flushed before every timed step (256 MB write)",
                       "parallelism": "replicas x%d" % world},
            "roofline": {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "decode",
                         "peak_source": ("%s bf16 dense, sustained" % peak_kind) if bound == "tensor"
                         else "FP32 FMA: SMs x 128 lanes x 2 x max SM clock"},
            "cpu_baseline": cpu,
            "e2e": None if not e2e_ms else {
                "value": e2e_value, "unit": "Mpixel/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
            "gpu_launches": launches_per_step * args.steps,
            "clocks": clock_info,
            "plan_ms": plan_ms,
            "autotune": tuned,
            "decode_ms_per_step": dec_ms,
            "decode_gflop_per_step": flops / 1e9,
            "psnr_db": {str(m): psnr[m] for m in wl["ms"]},
            "parity_vs_oracle": parity,
            "mixed_precision": mixed,
            "hbm_kernels": hbm_kernels,
            "tv_recovery": tv,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)

    for p in plans.values():
        B.cs_plan_destroy(p)
    B.cs_ctx_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
