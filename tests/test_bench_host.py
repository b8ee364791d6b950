"""Host-side logic of bench.py's N > 1 replica mode, on CPU with two gloo ranks: the timing is
the maximum over ranks and the throughput aggregates every rank's units."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = bench.max_over_ranks(10.0 * (rank + 1), world)
    thr = bench.job_throughput(1000.0, world, ms)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, thr))


def test_replica_timing_two_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [20.0, 20.0]          # max over ranks on every rank
    assert res[0][2] == pytest.approx(2 * 1000.0 / 0.020)


def test_single_rank_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(10.0, 1, 1000.0) == pytest.approx(10.0)


def test_tc_algorithmic_bytes_small():
    import bench
    import gen
    # K4 (no degree sort): U = the 6 pairs (u < v); d+ = 3, 2, 1, 0
    # 4(n+1) + 4 m_L + sum over U edges of 8 + 4 d+(v) = 20 + 24 + 48 + 4 (2 + 1 + 0 + 1 + 0 + 0)
    assert bench.tc_algorithmic_bytes(gen.complete(4)) == 108
    # star with 5 leaves (n = 6): mean degree 5/3 is not above 4 * median 1, so no sort; the hub
    # is vertex 0, U(0) = the 5 leaves (d+ 0 each): 5 edges of 8 bytes
    assert bench.tc_algorithmic_bytes(gen.star(5)) == 4 * 7 + 4 * 5 + 8 * 5


def test_clock_sampler_window():
    sys.path.insert(0, ROOT)
    import datetime
    import bench

    def line(t, sm, slow="Not Active", cap="Not Active"):
        ts = datetime.datetime.fromtimestamp(t).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return f"{ts}, 0, {sm}, 2070, 900.5, 0x0, {slow}, Not Active, Not Active, {cap}"

    c = bench.ClockSampler(0)
    c.lines = [line(100.00, 1400), line(100.05, 2070), line(100.10, 2065, cap="Active"), line(100.15, 1200,
               slow="Active"), "garbage", ""]
    s = c.summary((100.04, 100.12))
    assert s["window"] == "timed" and s["samples"] == 2 and s["sm_mhz"] == 2067.5
    assert s["reasons"] == ["sw_power_cap"] and s["sm_max_mhz"] == 2070
    s = c.summary((100.06, 100.08))  # between two samples: the ones around it
    assert s["window"] == "around the timed window" and s["samples"] == 2
    assert c.summary()["samples"] == 4 and "hw_slowdown" in c.summary()["reasons"]
    c.lines = []
    assert c.summary((0, 1))["reasons"] == ["unsampled"]


def test_clock_sampler_process(tmp_path, monkeypatch):
    # the sampler's process plumbing against a stand-in nvidia-smi that prints timestamped samples
    sys.path.insert(0, ROOT)
    import time
    import bench
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/usr/bin/env python3\n"
                    "import datetime, sys, time\n"
                    "while True:\n"
                    "    ts = datetime.datetime.now().strftime('%Y/%m/%d %H:%M:%S.%f')[:-3]\n"
                    "    print(f'{ts}, 0, 2070, 2070, 800.0, 0x0, Not Active, Not Active, Not Active, Not Active',"
                    " flush=True)\n"
                    "    time.sleep(0.02)\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ["PATH"])
    with bench.ClockSampler(0) as c:
        time.sleep(0.5)
        t0 = time.time()
        time.sleep(0.2)
        t1 = time.time()
        time.sleep(0.2)
    s = c.summary((t0, t1))
    assert s["window"] == "timed" and s["samples"] >= 3 and s["sm_mhz"] == 2070 and s["reasons"] == []
