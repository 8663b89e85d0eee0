"""The bench's multi-rank aggregation on CPU: two gloo ranks, each timing its
own replica of the work, agree on the slowest rank's time, and the whole-job
throughput counts both ranks' units over that time (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(times[rank], world, "cpu")
        out[rank] = (t, bench.job_throughput(world, 1000.0, 4, t))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = torch.multiprocessing.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    times = [12.5, 20.0]                      # ms of the two replicas
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, v = out[r]
        assert t == 20.0
        # 2 ranks x 1000 units x 4 steps in the slowest rank's 20 ms
        assert v == pytest.approx(2 * 1000 * 4 / 0.020)


def test_one_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.0, 1) == 7.0
    assert bench.job_throughput(1, 10.0, 2, 5.0) == pytest.approx(4000.0)


def test_mixed_launch_count():
    """The mixed bench's launch count, from each job's engine (1 plain, 2 on chip,
    3 streaming, 4 chunked): one launch per group of up to 48 jobs of each
    tensor-core kernel (16x16 on chip by shared-memory layout, 32x32 cluster,
    streaming, chunked) and one per plain-kernel job."""
    import bench

    class P:
        def __init__(self, block, m):
            self.block, self.m = block, m

    def job(b, m, engine):
        return {"p": P(b, m), "engine": engine}
    jobs = ([job(16, 40, 2)] * 50 + [job(16, 128, 2)] + [job(32, 102, 2)] * 3 + [job(32, 300, 3)] * 2 +
            [job(8, 16, 3)] + [job(16, 40, 1)] * 2)
    # on chip: 50 jobs of M16 <= 96 (2 launches) + 1 of M16 = 128; cluster: 1;
    # streaming: 3 (32x32 M > 128, 8x8) in 1; plain: 2
    assert bench.mixed_launches(jobs) == 2 + 1 + 1 + 1 + 2
    # a cluster job of more than 15 x 13 tiles adds the streaming tail's launch
    big = dict(job(32, 102, 2), blocks=196 * 128)
    assert bench.mixed_launches(jobs + [big]) == 2 + 1 + 1 + 1 + 2 + 1
    # chunked jobs of any block size share one launch per 48
    assert bench.mixed_launches(jobs + [job(32, 102, 4)] * 49 + [job(16, 64, 4)]) == 2 + 1 + 1 + 1 + 2 + 2
    # a chunked 32x32 job of 647 tiles (39 left over on 152 SMs) adds the cluster head's
    # launch; one of 216 tiles (64 left over) does not
    assert bench.mixed_launches(jobs + [dict(job(32, 102, 4), blocks=82800)]) == 2 + 1 + 1 + 1 + 2 + 1 + 1
    assert bench.mixed_launches(jobs + [dict(job(32, 102, 4), blocks=27600)]) == 2 + 1 + 1 + 1 + 2 + 1


def test_decode_traffic_only_for_the_captured_engine():
    """roofline.traffic is the stored ncu figure of a workload only when the step's
    decode ran on the engine that capture measured (the chunked engine for 720p, the
    on-chip one for the CIF sweep); any other engine, or a mix, reports null."""
    import bench
    eng_720p, bytes_720p = bench.DECODE_DRAM_BYTES["720p"]
    assert bench.decode_traffic("720p", {"engines": [eng_720p]}) == bytes_720p
    assert bench.decode_traffic("720p", {"engines": [1]}) is None
    assert bench.decode_traffic("720p", {"engines": [2, eng_720p]}) is None
    eng_cif, bytes_cif = bench.DECODE_DRAM_BYTES["cif"]
    assert bench.decode_traffic("cif", {"engines": [eng_cif]}) == bytes_cif
    assert bench.decode_traffic("cif", {"engines": [3]}) is None
    assert bench.decode_traffic("mixed64", {"engines": [eng_cif]}) is None
