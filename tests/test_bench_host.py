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


def test_roofline_tensor_peaks_per_product_type():
    stats = {"gemm_xtr": dict(ms=10.0, launches=10, work=1e13)}    # 1e12 flops per 1 ms launch
    pk = {"hbm_gbs": 6792.7, "bf16_tflops": 1961.0, "bf16_tflops_sustained": 1730.1, "source": "measured"}
    r = bench.roofline(stats, "bf16", pk)
    assert r["bound"] == "tensor" and r["achieved"] == pytest.approx(1000.0)
    assert r["peak"] == pytest.approx(1730.1) and r["frac"] == pytest.approx(1000.0 / 1730.1)
    r32 = bench.roofline(stats, "tf32x3", pk)
    assert r32["peak"] == pytest.approx(1730.1 * 1.1 / 2.25 / 3.0)
    # the FP64 products and the certificate's exact products are held to the FP64 rate
    r64 = bench.roofline(stats, "fp64", pk)
    assert r64["bound"] == "alu" and r64["peak"] == pytest.approx(bench.FP64_NOMINAL_TFLOPS)


def test_roofline_memory_bound_phase_against_the_copy_bandwidth():
    stats = {"prox_fista": dict(ms=5.0, launches=100, work=100 * 123e6),
             "gemm_xtr": dict(ms=1.0, launches=100, work=100 * 1e9)}
    r = bench.roofline(stats, "bf16", {"hbm_gbs": 6792.7, "source": "measured"})
    # 123 MB per 50 us launch
    assert r["kernel"] == "prox_fista" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(123e6 / 50e-6 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6792.7)
    assert bench.roofline({"reopt": dict(ms=3.0, launches=1, work=0.0)}, "bf16", {"hbm_gbs": 1.0,
                                                                                    "source": "x"}) is None


def test_traffic_is_reported_only_for_the_captured_kernel_sources(tmp_path, monkeypatch):
    import json
    (tmp_path / "profiles").mkdir()
    entry = {"w/bf16/m8192": {"gemm_xtr": {"dram_bytes_per_launch": 375329280, "source_sha": "abc"}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(entry))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_sha", lambda files: "abc")
    assert bench.traffic_for("gemm_xtr", "w", "bf16", 8192) == 375329280
    assert bench.traffic_for("gemm_xtr", "w", "bf16", 4096) is None      # another batch size
    assert bench.traffic_for("prox_fista", "w", "bf16", 8192) is None    # not captured
    monkeypatch.setattr(bench, "source_sha", lambda files: "changed")
    assert bench.traffic_for("gemm_xtr", "w", "bf16", 8192) is None      # kernel changed since


def test_committed_traffic_entries_name_known_phases():
    import json
    d = json.load(open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")))
    for key, phases in d.items():
        if key.startswith("_"):
            continue
        workload, prec, m = key.split("/")
        assert prec in bench.DTYPE and m.startswith("m") and int(m[1:]) > 0
        for ph, e in phases.items():
            if ph.startswith("_"):          # a note on the entry
                continue
            assert ph in bench.PHASE_KERNEL_SOURCES
            assert e["dram_bytes_per_launch"] > 0 and len(e["source_sha"]) == 16


def test_clock_summary_reads_the_samples_and_throttle_reasons():
    s = bench.ClockSampler(0)
    fd, s.path = __import__("tempfile").mkstemp(suffix=".csv")
    os.close(fd)
    with open(s.path, "w") as f:
        f.write("0, 2070, 2070, 910.5, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 1980, 2070, 1200.0, 0x4, Not Active, Not Active, Not Active, Active\n")
        f.write("0, 2025, 2070, 700.25, 0x0, Not Active, Not Active, Not Active, Not Active\n")
        f.write("garbage line\n")
    out = s.summary()
    assert out["samples"] == 3 and out["sm_mhz"] == 2025.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["power_w_max"] == 1200.0
    assert not os.path.exists(s.path)
    empty = bench.ClockSampler(0)
    assert empty.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
