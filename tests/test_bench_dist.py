"""bench.py's multi-rank host logic on CPU: two gloo ranks (replicas, as with
`--gpus 2` under torchrun), the barrier, the max-over-ranks time and the
whole-job throughput of all replicas."""
import os
import socket

import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import bench as b
    r, w, _ = b.dist_env()
    dist = b.init_dist(w, "gloo")
    b.barrier(dist)
    t = b.max_over_ranks(dist, 10.0 + 5.0 * r)  # rank 1 is the slow one
    q.put((r, t, b.whole_job_value(w, t)))
    b.barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, t, v in res:
        assert t == 15.0
        assert v == pytest.approx(2 * bench.FLOPS_PER_STEP / 15e-3 / 1e12)


def test_single_rank_needs_no_process_group():
    assert bench.init_dist(1, "gloo") is None
    assert bench.max_over_ranks(None, 3.5) == 3.5
    assert bench.whole_job_value(1, 1000.0) == pytest.approx(bench.FLOPS_PER_STEP / 1.0 / 1e12)


def test_launch_count_of_the_fixed_point_stepper():
    # expm (one launch), E images at full and half tile width (rows + image
    # each: 4 per mode), U -> fixed point (2), 300 mode products: the 315
    # launches of the stepper's ncu launch list
    assert bench.launches_per_step("fx32") == 1 + 12 + 2 + 300
    assert bench.launches_per_step("fx32h") == 1 + 12 + 2 + 300


def test_clock_summary_counts_only_the_timed_region():
    """Samples outside [mark, stop] are left out; throttle reasons are reported."""
    import bench
    c = bench.ClockSampler(0)
    idle = ["0", "1200", "2070", "150", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"]
    busy = ["0", "2070", "2070", "900", "0x0", "Not Active", "Not Active", "Not Active", "Active"]
    c.samples = [(1.0, idle), (2.0, busy), (3.0, busy), (9.0, idle)]
    c.t0, c.t1 = 1.5, 3.5
    s = c.summary()
    assert s["samples"] == 2 and s["sm_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    c.t0, c.t1 = 4.0, 5.0
    assert c.summary()["reasons"] == ["no samples in the timed region"]
