"""Host-side pieces of bench.py: the cross-rank aggregation (max time, summed
units) over a world of 2 gloo ranks, and the roofline arithmetic."""

import os
import socket

import pytest
import torch.multiprocessing as tmp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs, units = bench.reduce_max_sum(1.0 + rank, 100.0 * (rank + 1))
    out[rank] = (secs, units)
    dist.destroy_process_group()


def test_reduce_max_sum_two_gloo_ranks():
    ctx = tmp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == (2.0, 300.0) and out[1] == (2.0, 300.0)


def test_reduce_max_sum_single_process_is_identity():
    assert bench.reduce_max_sum(1.5, 7.0) == (1.5, 7.0)


def test_roofline_picks_the_longest_phase():
    stats = {"gemm_xv_link": dict(ms=10.0, launches=10, work=2e10),
             "prox_fista": dict(ms=2.0, launches=10, work=1e9),
             "reopt": dict(ms=50.0, launches=1, work=0.0)}
    r = bench.roofline(stats, "fp32", {"hbm_gbs": 6795.1, "sm_max_mhz": 2070.0, "source": "measured"})
    assert r["kernel"] == "gemm_xv_link" and r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    # 2e9 flops per launch in 1 ms -> 2 TFLOP/s
    assert r["achieved"] == pytest.approx(2.0)
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
