"""Multi-rank host logic of bench.py on CPU with two gloo processes: each rank
gets its own instance (seed = rank), the reported time is the slowest rank's,
and the job's throughput counts both ranks' unknowns."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "WORLD_SIZE": str(world),
                       "RANK": str(rank), "LOCAL_RANK": str(rank)})
    import bench
    w, r, lr = bench.rank_env()
    dist.init_process_group("gloo", init_method="env://", rank=r, world_size=w)
    ms_local = 10.0 + 5.0 * r                       # rank 1 is the slower one
    ms = bench.max_over_ranks(ms_local, dist)
    from paper_2303_01163_gb300 import workloads as wl
    p = wl.random_fourier_2d(33, bench.instance_seed(r))
    out[r] = (w, r, lr, ms, bench.job_throughput(w, 31 * 31, 3, ms), float(p.s[5, 7]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing_and_split_instances():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=120)
            assert pr.exitcode == 0
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in range(world):
        w, rr, lr, ms, thr, sample = res[r]
        assert (w, rr, lr) == (2, r, r)
        assert ms == 15.0                            # max over ranks on every rank
        assert thr == pytest.approx(2 * 31 * 31 * 3 / 15e-3)
    assert res[0][5] != res[1][5]                    # different instances per rank


def test_single_rank_defaults(monkeypatch):
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    import bench
    assert bench.rank_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(1, 100, 2, 10.0) == pytest.approx(2e4)


def test_family_roofline_arithmetic():
    """bench.py's roofline entries: achieved = algorithmic work / summed event
    time, peaks from the measured figures (TF32 = bf16 x 1.1/2.25) or the
    derived FP32 FMA peak; the tensor-core Filler against HBM."""
    import bench
    peaks = {"hbm_gbs": 6756.2, "bf16_tflops": 1914.9}
    r = bench.family_roofline("residual", {"launches": 2, "ms": 0.4, "bytes": 1.24e9, "flops": 0.0},
                              peaks, "measured", 152, 2070.0)
    assert r["bound"] == "hbm" and abs(r["achieved"] - 3100.0) < 1e-9 and abs(r["frac"] - 3100.0 / 6756.2) < 1e-12
    assert abs(r["avg_launch_us"] - 200.0) < 1e-9
    r = bench.family_roofline("bcr_aniso", {"launches": 10, "ms": 1.0, "bytes": 0.0, "flops": 2.0e10},
                              peaks, "measured", 152, 2070.0)
    fp32 = 152 * 128 * 2 * 2070e6 / 1e12
    assert r["bound"] == "alu" and abs(r["peak"] - fp32) < 1e-9 and abs(r["achieved"] - 20.0) < 1e-9
    # The tensor-core Filler (~24 flop/byte, below the TF32 ridge) against HBM, its tensor rate beside.
    r = bench.family_roofline("fill_tc", {"launches": 1, "ms": 0.03, "bytes": 7.5e7, "flops": 1.77e9},
                              peaks, "measured", 152, 2070.0)
    assert r["bound"] == "hbm" and abs(r["achieved"] - 2500.0) < 1e-9 and abs(r["peak"] - 6756.2) < 1e-12
    assert abs(r["tensor"]["peak_tflops"] - 1914.9 * 1.1 / 2.25) < 1e-9
    assert abs(r["tensor"]["achieved_tflops"] - 59.0) < 1e-9
