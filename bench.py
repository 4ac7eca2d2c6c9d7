#!/usr/bin/env python
"""Certified node bounds per second of the batched node-bound engine (one JSON line).

A step is one pass of the whole hot path over one node batch: layout of the
batch's fixing masks, `iters` FISTA iterations (X*V with the fused link,
X^T*R, masked prox), the FP64 certificate, rounding, re-optimization,
branching index, pruning and branching.

Headline workload: the node-bound microbenchmark, X 10000 x 2000 (Toeplitz
rho = 0.5, columns standardized), k = 20, lambda2 = 1e-3, M = 2, least
squares, 8192 nodes per batch with random fixing patterns (|J1| ~ U{0..k},
|J0| ~ U{0..p/2}), T = 50 iterations, BF16 tensor-core products with FP32
accumulate and the FP64 certificate (the largest single-GPU configuration).

  value  nodes certified per second with the instance and the node batches
         already in device memory (kglm_push_nodes_dev);
  e2e    the same through kglm_push_nodes from pinned host buffers, the
         host->device copy of the batch and the device->host read of the
         per-node results inside each timed step.

Extra keys of the default run (untimed for the headline, each measured on
its own): the same workload with logistic loss, with FP32-accurate and with
FP64 products; the error of the BF16 bounds against the FP64 oracle on
sampled nodes; the time to zero gap of a full certified solve of the hard
correlated least-squares instance (n = 5000, p = 1000, rho = 0.9) in BF16
and in FP64; the logistic n = 2000, p = 200 line with FP32-accurate
products; the serving mix (p50/p99 time to certified optimality); the
batch-size sweep at the paper's Fig. 3 setting.

Launch: python bench.py [--gpus N --steps K --warmup W]; for N > 1 under
torch.distributed.run, one rank per GPU, each rank evaluating its own
batches (node batches are independent: weak scaling, no data-path
collective).  --impl reference times the FP64 oracle on the host cores on
bounded samples of the same workload.
"""

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2605_22188_gb300 import synth  # noqa: E402

WORKLOAD = "c4_micro_n10000_p2000_k20"
METRIC = "certified node bounds/sec"
UNIT = "nodes/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Fallback peaks of the profiling recipe when MEASURED_PEAKS.json is absent.
FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}
SMS = 152
# arithmetic type of the products per engine mode (tf32x3: FP32 values carried as TF32 hi + lo pairs)
DTYPE = {"fp64": "f64", "fp32": "f32", "tf32x3": "f32", "bf16": "bf16", "tf32": "tf32"}
PRODUCTS = {"fp64": "fp64 (CUDA cores)", "fp32": "fp32 (CUDA cores)",
            "tf32x3": "fp32-accurate: TF32 hi+lo split, 3 tcgen05 products, FP32 accumulate",
            "bf16": "bf16 tcgen05, FP32 accumulate", "tf32": "tf32 tcgen05, FP32 accumulate"}
FP32_LANES_PER_SM = 128          # FP32 FMA lanes per SM (4 partitions x 32)
FP64_NOMINAL_TFLOPS = 1.25       # GB300 FP64, nominal


# ------------------------------------------------------------------ helpers

def peaks():
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    d = dict(FALLBACK)
    d["source"] = "fallback"
    return d


def rank_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def reduce_max_sum(seconds, units):
    """Max of the elapsed times and sum of the units over ranks (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return seconds, units
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        pw = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "power_w_max": max(pw) if pw else None}


def source_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


PHASE_KERNEL_SOURCES = {
    "gemm_xv_link": ["paper_2605_22188_gb300/csrc/gemm_simt.cu", "paper_2605_22188_gb300/csrc/gemm_tc.cu",
                     "paper_2605_22188_gb300/csrc/common.cuh"],
    "gemm_xtr": ["paper_2605_22188_gb300/csrc/gemm_simt.cu", "paper_2605_22188_gb300/csrc/gemm_tc.cu"],
    "prox_fista": ["paper_2605_22188_gb300/csrc/prox.cu", "paper_2605_22188_gb300/csrc/prox_stream.cu",
                   "paper_2605_22188_gb300/csrc/common.cuh"],
    "cert_xtzeta": ["paper_2605_22188_gb300/csrc/gemm_simt.cu", "paper_2605_22188_gb300/csrc/gemm_tc.cu",
                    "paper_2605_22188_gb300/csrc/cert_exact.cu"],
    "cert_xb": ["paper_2605_22188_gb300/csrc/gemm_simt.cu", "paper_2605_22188_gb300/csrc/gemm_tc.cu",
                "paper_2605_22188_gb300/csrc/layout.cu"],
    "cert_bound": ["paper_2605_22188_gb300/csrc/cert.cu", "paper_2605_22188_gb300/csrc/common.cuh"],
    "cert_dual_point": ["paper_2605_22188_gb300/csrc/cert.cu", "paper_2605_22188_gb300/csrc/common.cuh"],
    "reopt": ["paper_2605_22188_gb300/csrc/reopt.cu"],
}


def traffic_for(phase, workload, prec, nodes):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.json) for this
    workload, product precision and batch size, if the kernel's source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    d = json.load(open(path))
    e = d.get("%s/%s/m%d" % (workload, prec, nodes), {}).get(phase)
    if not e or phase not in PHASE_KERNEL_SOURCES:
        return None
    if e.get("source_sha") != source_sha(PHASE_KERNEL_SOURCES[phase]):
        return None
    return e.get("dram_bytes_per_launch")


def roofline(stats, prec, pk, workload=WORKLOAD, nodes=8192):
    """Achieved rate of the phase with the largest device time, against its peak."""
    best = None
    for name, s in stats.items():
        if s["launches"] > 0 and s["work"] > 0 and s["ms"] > 0:
            if best is None or s["ms"] > stats[best]["ms"]:
                best = name
    if best is None:
        return None
    s = stats[best]
    per_launch_s = s["ms"] / 1e3 / s["launches"]
    work = s["work"] / s["launches"]
    sm_max = pk.get("sm_max_mhz", 2070.0) * 1e6
    if best in ("gemm_xv_link", "gemm_xtr") and prec in ("bf16", "tf32", "tf32x3"):
        # tensor-core products inside a long step: the sustained BF16 peak (TF32:
        # times the nominal TF32/BF16 dense ratio 1.1/2.25; the FP32-accurate
        # TF32 hi + lo split issues three TF32 products per product: a third of that)
        base = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops", 1700.0))
        peak = {"bf16": base, "tf32": base * 1.1 / 2.25, "tf32x3": base * 1.1 / 2.25 / 3.0}[prec]
        src = pk["source"]
        note = {"bf16": "BF16 sustained dense peak (%s)" % src,
                "tf32": "TF32: BF16 sustained (%s) x nominal TF32/BF16 ratio 1.1/2.25" % src,
                "tf32x3": "FP32-accurate 3xTF32: BF16 sustained (%s) x 1.1/2.25 / 3" % src}[prec]
        achieved = work / per_launch_s / 1e12
        return {"kernel": best, "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_for(best, workload, prec, nodes),
                "peak_note": note,
                "launches": s["launches"], "avg_launch_us": per_launch_s * 1e6}
    if best in ("gemm_xv_link", "gemm_xtr", "cert_xb", "cert_xtzeta"):
        fp64 = prec == "fp64" or best == "cert_xtzeta"
        if fp64:
            peak, note = FP64_NOMINAL_TFLOPS, "FP64 nominal of the recipe"
        else:
            peak = SMS * FP32_LANES_PER_SM * 2 * sm_max / 1e12
            note = "FP32 FMA: 152 SMs x 128 lanes x 2 x max SM clock"
        achieved = work / per_launch_s / 1e12
        return {"kernel": best, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_for(best, workload, prec, nodes),
                "peak_note": note, "launches": s["launches"], "avg_launch_us": per_launch_s * 1e6}
    peak = pk["hbm_gbs"]
    achieved = work / per_launch_s / 1e9
    return {"kernel": best, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic_for(best, workload, prec, nodes),
            "peak_note": "HBM copy bandwidth, %s" % pk["source"], "launches": s["launches"],
            "avg_launch_us": per_launch_s * 1e6}


# ------------------------------------------------------------------ oracle (CPU baseline / reference arm)

_ORACLE_STATE = {}


def _oracle_init(X, y, c, L):
    os.environ["OMP_NUM_THREADS"] = "1"
    _ORACLE_STATE.update(X=X, y=y, c=c, L=L)


def _oracle_node(args):
    """One node through the oracle: T FISTA iterations, certificate, rounding, re-opt, branch index."""
    from oracle import node as on
    from oracle import reopt as ro
    J0, J1, T, full = args
    s = _ORACLE_STATE
    c = s["c"]
    nd = on.Node(c["p"], c["k"], J0, J1)
    r = on.solve_node(s["X"], s["y"], nd, c["lam2"], c["M"], c["kind"], s["L"], T)
    if full:
        S = on.round_support(r["beta"], nd)
        ro.reopt(s["X"], s["y"], S, c["lam2"], c["M"], c["kind"], beta0=r["beta"])
        on.branch_index(r["beta"], nd)
    return r["lb"]


def oracle_pool(X, y, c, cores):
    from oracle import node as on
    L = on.lipschitz(X, c["kind"])
    ctx = mp.get_context("spawn")
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    return ctx.Pool(cores, initializer=_oracle_init, initargs=(X, y, c, L))


def oracle_run(pool, nodes, T, full=True):
    t0 = time.perf_counter()
    lbs = pool.map(_oracle_node, [(J0, J1, T, full) for J0, J1 in nodes], chunksize=1)
    return lbs, time.perf_counter() - t0


def workload_config(name, c, m, T, world):
    """The workload (identical in both arms): what is evaluated, not how."""
    return {"workload": name, "n": c["n"], "p": c["p"], "k": c["k"], "lambda2": c["lam2"], "M": c["M"],
            "loss": "logistic" if c["kind"] == synth.LOGISTIC else "least_squares", "nodes_per_batch": m,
            "iters": T, "masks": "|J1|~U{0..k}, |J0|~U{0..p/2}",
            "parallelism": "replicas" if world > 1 else "single"}


# ------------------------------------------------------------------ the engine arm

def loss_kind(args):
    return None if args.loss is None else (synth.LSQ if args.loss == "lsq" else synth.LOGISTIC)


def make_batches(c, nb, m, seed):
    rng = np.random.default_rng(seed)
    return [synth.random_nodes(m, c["p"], c["k"], rng) for _ in range(nb)]


class Arm:
    """One workload on the engine: its instance, device-resident and pinned node batches,
    and the timed step (push + evaluate + prune + branch)."""

    def __init__(self, name, prec, m, T, stream, kind=None, tune="auto", seed=1000):
        import torch
        from paper_2605_22188_gb300 import kglm
        self.torch = torch
        self.c, self.X, self.y, _ = synth.config_instance(name, seed=0, kind=kind)
        self.name, self.prec, self.m, self.T, self.stream = name, prec, m, T, stream
        c = self.c
        self.eng = kglm.Engine(self.X, self.y, c["k"], c["lam2"], c["M"], c["kind"], prec=prec, max_batch=m,
                               stream=stream.cuda_stream)
        if isinstance(tune, str) and tune == "auto":
            self.tune = self.eng.autotune(iters=T, seed=1)   # tiles, split cap, launch mode (setup, untimed)
            self.tune["batch"] = m
        elif isinstance(tune, dict):
            cfg = {k: tune[k] for k in ("link_tile_cols", "grad_tile_cols", "grad_split_cap", "sub_batches", "pdl",
                                        "prox_threads", "pair") if k in tune}
            self.eng.configure(**cfg)
            self.tune = dict(tune, fixed=True)
        else:
            self.tune = None
        self.batches = make_batches(c, 8, m, seed=seed)
        self.dev = []
        for (ip, ii, op, oi) in self.batches:
            t = [torch.from_numpy(a).to("cuda") for a in (ip, ii, op, oi)]
            self.dev.append((t, int(ip[-1]), int(op[-1])))
        self.pinned = [tuple(torch.from_numpy(a).pin_memory().numpy() for a in bt) for bt in self.batches]
        self.flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        self.ub = math.inf

    def step_dev(self, i):
        t, nin, nout = self.dev[i % len(self.dev)]
        self.eng.push_dev(self.m, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), t[3].data_ptr(), nin, nout)
        res = self.eng.evaluate(self.T)
        self.eng.prune(self.ub)
        self.eng.branch(self.ub)
        return res

    def step_host(self, i):
        self.eng.push(*self.pinned[i % len(self.pinned)])
        res = self.eng.evaluate(self.T)
        self.eng.prune(self.ub)
        self.eng.branch(self.ub)
        return res

    def timed(self, fn, steps):
        """Device time of `steps` steps (CUDA events on the engine's stream), L2 flushed between steps."""
        torch = self.torch
        total = 0.0
        with torch.cuda.stream(self.stream):
            for i in range(steps):
                self.flush.zero_()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(self.stream)
                fn(i)
                b.record(self.stream)
                b.synchronize()
                total += a.elapsed_time(b) / 1e3
        return total

    def warm(self, n):
        for i in range(n):
            r = self.step_dev(i)
            self.ub = min(self.ub, float(np.min(r["ub"])))
        self.torch.cuda.synchronize()

    def rate(self, steps):
        """Nodes per second over `steps` device-resident steps, with the per-phase
        breakdown and the roofline from a second, event-instrumented pass."""
        dt = self.timed(self.step_dev, steps)
        self.eng.stats_enable(True)
        self.timed(self.step_dev, steps)
        st = self.eng.stats()
        self.eng.stats_enable(False)
        return {"value": self.m * steps / dt, "unit": UNIT, "steps": steps, "ms_per_step": dt / steps * 1e3,
                "nodes_per_batch": self.m, "products": PRODUCTS[self.prec],
                "phase_ms_per_step": {k: round(v["ms"] / steps, 4) for k, v in st.items() if v["ms"] > 0},
                "roofline": roofline(st, self.prec, peaks(), self.name, self.m)}

    def close(self):
        self.eng.close()


def guarded(label, fn):
    """Run one extra measurement; a failure is recorded in its key instead of ending the run."""
    t0 = time.perf_counter()
    try:
        out = fn()
    except Exception as e:  # noqa: BLE001 - reported in the line
        out = {"error": "%s: %s" % (type(e).__name__, str(e)[:300])}
    if isinstance(out, dict):
        out["wall_s"] = round(time.perf_counter() - t0, 2)
    print("[bench] %s done in %.1f s" % (label, time.perf_counter() - t0), file=sys.stderr, flush=True)
    return out


def run_ours(args):
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    c0 = synth.CONFIGS[args.workload]
    m = args.nodes or c0.get("m", 1024)
    T = args.iters or c0.get("T", 50)
    extras = args.extras and rank == 0 and world == 1 and args.workload == WORKLOAD

    pool, cores, cpu = None, os.cpu_count() or 1, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        c, X, y, _ = synth.config_instance(args.workload, seed=0, kind=loss_kind(args))
        pool = oracle_pool(X, y, c, cores)              # spawn pool before the first CUDA call
        cpu = cpu_baseline(pool, c, T, cores, args)

    stream = torch.cuda.Stream()
    tune = "auto"
    if args.tiles:
        v = [int(x) for x in args.tiles.split(",")]
        tune = {"link_tile_cols": v[0], "grad_tile_cols": v[1], "grad_split_cap": v[2], "sub_batches": v[3]}
        if len(v) > 4:
            tune["pair"] = v[4]
    elif args.no_autotune:
        tune = None
    arm = Arm(args.workload, args.prec, m, T, stream, kind=loss_kind(args), tune=tune, seed=1000 + rank)
    c = arm.c
    arm.warm(max(args.warmup, 3))

    # timed region: the bare step (kernel launches are counted, no timing events)
    arm.eng.stats_enable(False)
    barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        dt = arm.timed(arm.step_dev, args.steps)
    torch.cuda.synchronize()
    barrier()
    launches = sum(s["launches"] for s in arm.eng.stats().values())
    secs, units = reduce_max_sum(dt, float(m * args.steps))
    value = units / secs
    # the same steps again with CUDA events around every kernel on the engine's
    # stream (per-phase device time for the roofline; events inside the CUDA
    # graph of the iterations cost a few microseconds each, so they stay out of
    # the timed region above)
    arm.eng.stats_enable(True)
    arm.timed(arm.step_dev, args.steps)
    stats = arm.eng.stats()
    arm.eng.stats_enable(False)

    # end to end from pinned host buffers
    for i in range(2):
        arm.step_host(i)
    barrier()
    dt_e2e = arm.timed(arm.step_host, args.steps)
    secs_e, units_e = reduce_max_sum(dt_e2e, float(m * args.steps))
    ip, ii, op, oi = arm.batches[0]
    h2d = 4 * (len(ip) + len(ii) + len(op) + len(oi))
    d2h = m * (8 * 3 + 4 * c["k"] + 8 * c["k"] + 4 + 4) + m      # lb, primal, ub, support, beta_re, j*, iters, pruned
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[args.prec], "data": "synthetic",
        "config": workload_config(args.workload, c, m, T, world),
        "impl_config": {"products": PRODUCTS[args.prec], "certificate": "fp64",
                        "l2": "flushed between steps (256 MiB write)", "autotune": arm.tune},
        "e2e": {"value": units_e / secs_e, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "roofline": roofline(stats, args.prec, peaks(), args.workload, m),
        "cpu_baseline": cpu,
        "clocks": clocks,
        "phase_ms_per_step": {k: round(v["ms"] / args.steps, 4) for k, v in stats.items() if v["ms"] > 0},
    }
    if extras:
        line["bf16_bound_error_vs_fp64_oracle"] = guarded("bound error", lambda: bound_error(arm, pool, cores))
        tuned = arm.tune if isinstance(arm.tune, dict) else None
        arm.close()
        line["logistic"] = guarded("logistic", lambda: other_arm(args.workload, args.prec, m, T, stream,
                                                                 synth.LOGISTIC, tuned, args))
        line["fp32_accurate_products"] = guarded("tf32x3", lambda: other_arm(args.workload, "tf32x3", m, T, stream,
                                                                             None, None, args))
        line["fp64_products"] = guarded("fp64", lambda: other_arm(args.workload, "fp64", 256, T, stream, None, None,
                                                                  args, steps=2))
        if isinstance(line["fp64_products"], dict) and "value" in line["fp64_products"]:
            line["mixed_over_fp64"] = value / line["fp64_products"]["value"]
        line["time_to_zero_gap"] = guarded("time to zero gap", lambda: time_to_zero_gap(
            "c3_lsq_n5000_p1000_k15", "bf16", stream, 4096))
        line["c2"] = guarded("c2", lambda: c2_line(stream, args))
        line["serving"] = guarded("serving", lambda: serving_summary(args))
        line["batch_sweep"] = guarded("sweep", lambda: sweep_summary(args))
    else:
        arm.close()
    if pool is not None:
        pool.close()
        pool.join()
    if rank == 0:
        print(json.dumps(line), flush=True)


def other_arm(name, prec, m, T, stream, kind, tune, args, steps=None):
    """The same workload in another precision or loss: a shorter timed run on its own engine."""
    arm = Arm(name, prec, m, T, stream, kind=kind, tune=tune if tune else None, seed=2000)
    try:
        arm.warm(2)
        out = arm.rate(steps or max(3, args.steps // 4))
        out["loss"] = "logistic" if arm.c["kind"] == synth.LOGISTIC else "least_squares"
        return out
    finally:
        arm.close()


def bound_error(arm, pool, cores):
    """The BF16 bounds of one batch against the FP64 oracle's after the same T (the
    oracle's FISTA from the same start), on nodes sampled across the batch: per-node
    relative difference (LB_oracle - LB_gpu) / max(1, |LB_oracle|)."""
    if pool is None:
        return {"skipped": "no oracle pool (--no-cpu-baseline)"}
    from paper_2605_22188_gb300 import kglm  # noqa: F401
    arm.eng.push(*arm.batches[0])
    res = arm.eng.evaluate(arm.T)
    nodes = synth.csr_to_sets(*arm.batches[0])
    idx = sorted(set(np.linspace(0, arm.m - 1, min(cores, arm.m)).astype(int).tolist()))
    ref, dt = oracle_run(pool, [nodes[i] for i in idx], arm.T, full=False)
    rel = [(r - float(res["lb"][i])) / max(1.0, abs(r)) for i, r in zip(idx, ref)]
    return {"nodes": len(idx), "iters": arm.T, "median_rel": float(np.median(rel)), "max_abs_rel": float(np.max(np.abs(rel))),
            "min_rel": float(np.min(rel)), "per_node": [round(v, 8) for v in rel], "node_index": idx,
            "note": "positive = the GPU bound is below the oracle's (same T, same start); both are valid bounds"}


def time_to_zero_gap(name, prec, stream, m):
    """Wall time of a full certified solve (kglm_solve, the hybrid loop of Fig. 1) of the
    instance in the mixed precision and with FP64 products.  Each solve runs once
    untimed (CUDA-graph capture) and once timed; both must close the gap and agree
    on the support."""
    from paper_2605_22188_gb300 import kglm
    c, X, y, _ = synth.config_instance(name, seed=0)
    out = {"workload": name, "batch": m, "iters": 200, "check_every": 10}
    sols = {}
    for label, pr, limit in (("mixed", prec, 120.0), ("fp64", "fp64", 240.0)):
        with kglm.Engine(X, y, c["k"], c["lam2"], c["M"], c["kind"], prec=pr, max_batch=m,
                         stream=stream.cuda_stream) as e:
            e.solve(m, 200, 10, limit)
            stream.synchronize()
            t0 = time.perf_counter()
            r = e.solve(m, 200, 10, limit)
            dt = time.perf_counter() - t0
        sols[label] = r
        out[label + "_s"] = dt
        out[label + "_nodes"] = r["nodes"]
        out[label + "_gap"] = r["gap"]
        out[label + "_opt"] = r["opt"]
    out["mixed_products"] = PRODUCTS[prec]
    out["support"] = sols["mixed"]["support"]
    out["support_equal"] = sols["mixed"]["support"] == sols["fp64"]["support"]
    out["fp64_over_mixed_time"] = out["fp64_s"] / out["mixed_s"]
    # c1 (n 200, p 30, k 5, FP64): the batched solve of the sequential-vs-batched
    # comparison; the oracle's sequential BnB of the same instance is in
    # cpu_baseline["sequential_bnb"]
    c, X, y, _ = synth.config_instance(C1, seed=0)
    with kglm.Engine(X, y, c["k"], c["lam2"], c["M"], c["kind"], prec="fp64", max_batch=64,
                     stream=stream.cuda_stream) as e:
        e.solve(64, 200, 10, 60.0)
        stream.synchronize()
        t0 = time.perf_counter()
        r = e.solve(64, 200, 10, 60.0)
        dt = time.perf_counter() - t0
    out["c1"] = {"workload": C1, "products": "fp64", "batch": 64, "seconds": dt, "nodes": r["nodes"],
                 "gap": r["gap"], "opt": r["opt"], "support": r["support"]}
    return out


def c2_line(stream, args):
    """The logistic n = 2000, p = 200, k = 10 workload (1024 nodes, T = 50) with
    FP32-accurate products: device-resident and end-to-end rates, and FP64 products."""
    arm = Arm("c2_logistic_n2000_p200_k10", "tf32x3", 1024, 50, stream, tune="auto", seed=3000)
    try:
        arm.warm(3)
        out = arm.rate(max(10, args.steps))
        dt = arm.timed(arm.step_host, max(10, args.steps))
        out["e2e_value"] = arm.m * max(10, args.steps) / dt
    finally:
        arm.close()
    f = other_arm("c2_logistic_n2000_p200_k10", "fp64", 1024, 50, stream, None, None, args, steps=3)
    out["fp64_products_value"] = f["value"]
    out["mixed_over_fp64"] = out["value"] / f["value"]
    return out


SERVING = "c5_serving_mix64"
SWEEP = "sweep_batch_n1000_p1000_k10"


def sweep_summary(args):
    """Node-evaluation throughput against the batch size at the paper's Fig. 3 setting
    (n = p = 1000, rho = 0.9, k = 10, lambda2 = 1, M = 2): least squares 2^0..2^15,
    logistic 2^7..2^16.  Each point: the same random fixing patterns, T iterations +
    certificate + re-optimization, device time by CUDA events (best of 3 after one
    untimed run).  The plateau batch is the smallest reaching 95% of the best rate."""
    import torch
    from paper_2605_22188_gb300 import kglm
    out = {"n": 1000, "p": 1000, "k": 10, "lambda2": 1.0, "M": 2.0, "rho": 0.9, "iters": args.sweep_iters,
           "products": PRODUCTS["bf16"]}
    for kind, lo, hi in ((synth.LSQ, 0, 15), (synth.LOGISTIC, 7, 16)):
        X, y, _ = synth.instance(1000, 1000, 10, kind, rho=0.9, snr=5.0, seed=0)
        mmax = 1 << hi
        rng = np.random.default_rng(5)
        ip, ii, op, oi = synth.random_nodes(mmax, 1000, 10, rng)
        stream = torch.cuda.Stream()
        pts = []
        with kglm.Engine(X, y, 10, 1.0, 2.0, kind, prec="bf16", max_batch=mmax, stream=stream.cuda_stream) as eng:
            for e in range(lo, hi + 1):
                mb = 1 << e
                eng.push(ip[:mb + 1], ii[:ip[mb]], op[:mb + 1], oi[:op[mb]])
                best = None
                for r in range(4):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    with torch.cuda.stream(stream):
                        a.record(stream)
                        eng.evaluate(args.sweep_iters)
                        b.record(stream)
                    b.synchronize()
                    if r > 0:
                        ms = a.elapsed_time(b)
                        best = ms if best is None else min(best, ms)
                pts.append({"batch": mb, "ms": round(best, 4), "nodes_per_s": mb / (best * 1e-3)})
        top = max(p["nodes_per_s"] for p in pts)
        plateau = min(p["batch"] for p in pts if p["nodes_per_s"] >= 0.95 * top)
        key = "least_squares" if kind == synth.LSQ else "logistic"
        out[key] = {"points": pts, "best_nodes_per_s": top, "plateau_batch": plateau,
                    "plateau_log2": int(round(math.log2(plateau))),
                    "paper_plateau_log2": 10 if kind == synth.LSQ else 15}
    return out


def run_sweep(args):
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    if rank != 0:
        return
    out = sweep_summary(args)
    line = {"metric": "node bounds/sec against batch size", "value": out["logistic"]["best_nodes_per_s"],
            "unit": "nodes/s", "n_gpus": world, "steps": 3, "warmup": 1, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE["bf16"], "data": "synthetic",
            "config": {"workload": SWEEP, "n": 1000, "p": 1000, "k": 10, "lambda2": 1.0, "M": 2.0, "rho": 0.9,
                       "iters": args.sweep_iters},
            "sweep": out}
    print(json.dumps(line), flush=True)


def serving_summary(args):
    """The serving mix: 64 instances (synth.serving_specs) arriving as a Poisson
    stream, certified by the kglm_server loop with HBM-budgeted admission.
    value = aggregate nodes evaluated per second over the makespan; latency =
    time from submission to certified optimality (p50/p99 over the requests
    that closed their gap within the per-request limit)."""
    from paper_2605_22188_gb300 import kglm
    rank, world, local = rank_info()
    specs = synth.serving_specs(64, seed=rank)
    arrivals = synth.poisson_arrivals(len(specs), args.rate, seed=rank)
    data = []
    for sp in specs:                       # drawn before the timed region
        X, y, _ = synth.instance(sp["n"], sp["p"], sp["k"], sp["kind"], rho=sp["rho"], snr=sp["snr"], seed=sp["seed"])
        data.append((X, y))
    srv = kglm.Server(max_active=args.max_active, hbm_budget=0, iters=200, check_every=10,
                      time_limit_s=args.request_limit, batch_cap=4096)
    local_clk = ClockSampler(local)
    with local_clk as clk:
        t0 = time.perf_counter()
        ids = []
        for sp, (X, y), ta in zip(specs, data, arrivals):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids.append(srv.submit(X, y, sp["k"], sp["lam2"], sp["M"], sp["kind"], prec=args.serve_prec, max_batch=0))
        srv.drain()
        wall = time.perf_counter() - t0
    infos = [srv.info(r) for r in ids]
    st = srv.stats()
    srv.close()
    nodes = sum(i["nodes"] for i in infos)
    cert = [i for i in infos if i["state"] == kglm.REQ_DONE and i["gap"] <= 1e-6]
    lat = sorted(i["t_done"] - i["t_submit"] for i in cert)
    pct = lambda q: float(np.percentile(lat, q)) if lat else None
    # where the latency goes: waiting for a slot (admission) and being solved
    wait = sorted(i["t_admit"] - i["t_submit"] for i in cert if i["t_admit"] >= 0)
    serve = sorted(i["t_done"] - i["t_admit"] for i in cert if i["t_admit"] >= 0)
    pq = lambda v, q: float(np.percentile(v, q)) if v else None
    return {
        "value": nodes / wall, "unit": "nodes/s", "wall_s": wall, "requests": len(specs),
        "arrival_rate_per_s": args.rate, "max_active": args.max_active, "request_time_limit_s": args.request_limit,
        "products": args.serve_prec, "budget_bytes": st["budget"],
        "latency_s": {"p50": pct(50), "p99": pct(99), "max": lat[-1] if lat else None,
                      "of": "requests certified within the limit"},
        "admission_wait_s": {"p50": pq(wait, 50), "p99": pq(wait, 99)},
        "solve_s": {"p50": pq(serve, 50), "p99": pq(serve, 99)},
        "certified": len(cert), "not_certified": len(infos) - len(cert),
        "failed": sum(1 for i in infos if i["state"] == kglm.REQ_FAILED),
        "worst_gap": max(i["gap"] for i in infos), "peak_active": st["peak_active"], "peak_bytes": st["peak_bytes"],
        "rounds": st["rounds"], "round_batches": st["round_batches"], "shared_launches": st["shared_launches"],
        "clocks": clk.summary(),
        "per_request": [{"n": sp["n"], "p": sp["p"], "k": sp["k"],
                         "loss": "lsq" if sp["kind"] == synth.LSQ else "logistic", "rho": sp["rho"],
                         "batch": i["batch"], "nodes": i["nodes"], "gap": i["gap"], "state": i["state"],
                         "latency_s": round(i["t_done"] - i["t_submit"], 3),
                         "wait_s": round(i["t_admit"] - i["t_submit"], 3) if i["t_admit"] >= 0 else None}
                        for sp, i in zip(specs, infos)],
    }


def run_serving(args):
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    barrier()
    out = serving_summary(args)
    secs, units = reduce_max_sum(out["wall_s"], out["value"] * out["wall_s"])
    if rank != 0:
        return
    line = {
        "metric": "aggregate node bounds/sec and time-to-certified-optimality p50/p99 (serving mix)",
        "value": units / secs, "unit": "nodes/s", "n_gpus": world, "steps": 1, "warmup": 0,
        "ms_per_step": secs * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.serve_prec, "data": "synthetic",
        "config": {"workload": SERVING, "requests": out["requests"], "arrival_rate_per_s": args.rate,
                   "max_active": args.max_active, "request_time_limit_s": args.request_limit,
                   "parallelism": "replicas" if world > 1 else "single"},
        "serving": out,
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(pool, c, T, cores, args):
    """The oracle as it stands on the host cores, on a bounded sample of the workload's
    nodes (one process per core), sized from a first timed node to about args.cpu_seconds."""
    rng = np.random.default_rng(77)
    probe = synth.csr_to_sets(*synth.random_nodes(cores, c["p"], c["k"], rng))
    _, dt1 = oracle_run(pool, probe, T)                # one node per core: warms the workers, times a node
    per_node = dt1
    reps = max(1, int(args.cpu_seconds / max(per_node, 1e-3)))
    nodes = synth.csr_to_sets(*synth.random_nodes(cores * reps, c["p"], c["k"], rng))
    _, dt = oracle_run(pool, nodes, T)
    return {"value": len(nodes) / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d nodes of the workload (T=%d, certificate, rounding, re-opt, branch index), "
                      "one process per core, %.1f s" % (len(nodes), T, dt),
            "sequential_bnb": oracle_sequential_bnb()}


C1 = "c1_lsq_n200_p30_k5"


def oracle_sequential_bnb():
    """The oracle's sequential best-bound BnB (one node per evaluation, one thread) on the
    c1 instance, the baseline of the sequential-vs-batched comparison: wall time, nodes,
    certified optimum and support (the GPU's batched solve of the same instance is in
    time_to_zero_gap["c1"])."""
    from oracle import bnb
    c, X, y, _ = synth.config_instance(C1, seed=0)
    t0 = time.perf_counter()
    r = bnb.solve(X, y, c["k"], c["lam2"], c["M"], c["kind"], T_max=200, check_every=10)
    return {"workload": C1, "seconds": time.perf_counter() - t0, "nodes": int(r["nodes"]), "opt": float(r["opt"]),
            "support": [int(j) for j in r["support"]], "gap": float(r["gap"]), "threads": 1,
            "T_max": 200, "check_every": 10}


def run_reference(args):
    """The FP64 oracle timed on the host cores: same metric and workload, bounded samples per step."""
    rank, world, _ = rank_info()
    if rank != 0:
        return
    if args.workload in (SERVING, SWEEP):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle is timed per node-bound workload; "
                          "this workload has no oracle arm"}))
        return
    c0 = synth.CONFIGS[args.workload]
    m = args.nodes or c0.get("m", 1024)
    T = args.iters or c0.get("T", 50)
    c, X, y, _ = synth.config_instance(args.workload, seed=0, kind=loss_kind(args))
    cores = os.cpu_count() or 1
    rng = np.random.default_rng(1000)
    pool = oracle_pool(X, y, c, cores)
    # nodes per step: one per core, more while a step stays under about args.ref_step_seconds
    probe = synth.csr_to_sets(*synth.random_nodes(cores, c["p"], c["k"], rng))
    _, dt1 = oracle_run(pool, probe, T)
    per_step = cores * max(1, int(args.ref_step_seconds / max(dt1, 1e-3)))
    total_nodes, total_s = 0, 0.0
    try:
        for i in range(args.warmup + args.steps):
            nodes = synth.csr_to_sets(*synth.random_nodes(per_step, c["p"], c["k"], rng))
            _, dt = oracle_run(pool, nodes, T)
            if i >= args.warmup:
                total_nodes += len(nodes)
                total_s += dt
    finally:
        pool.close()
        pool.join()
    value = total_nodes / total_s
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args.workload, c, m, T, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "%d nodes of the workload per step (of %d in a batch), one process per core"
                                   % (per_step, m)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--prec", default="bf16", choices=["fp64", "fp32", "bf16", "tf32", "tf32x3"])
    ap.add_argument("--iters", type=int, default=0, help="FISTA iterations per node (0: the workload's, else 50)")
    ap.add_argument("--nodes", type=int, default=0, help="nodes per batch (0: the workload's)")
    ap.add_argument("--loss", default=None, choices=[None, "lsq", "logistic"],
                    help="override the workload's loss (the microbench runs both)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="oracle CPU baseline: target wall seconds")
    ap.add_argument("--ref-step-seconds", type=float, default=2.0, help="reference arm: target seconds per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="only the headline line (no logistic/precision/solve/c2/serving/sweep keys)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default tiles (profiling runs)")
    ap.add_argument("--tiles", default="",
                    help="fixed tiles instead of tuning: link,grad,split_cap,sub_batches[,pair (1 on, -1 off)]")
    ap.add_argument("--rate", type=float, default=2.0, help="serving mix: Poisson arrivals per second")
    ap.add_argument("--max-active", type=int, default=16, help="serving mix: requests solved at once")
    ap.add_argument("--request-limit", type=float, default=20.0, help="serving mix: seconds per request")
    ap.add_argument("--serve-prec", default="bf16", help="serving mix: product precision")
    ap.add_argument("--sweep-iters", type=int, default=50, help="batch sweep: iterations per evaluation")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup
    rank, world, local = rank_info()
    if world > 1:
        import torch
        import torch.distributed as dist
        if args.impl == "ours":
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    try:
        if args.impl == "reference":
            run_reference(args)
        elif args.workload == SERVING:
            run_serving(args)
        elif args.workload == SWEEP:
            run_sweep(args)
        else:
            run_ours(args)
    finally:
        if world > 1:
            import torch.distributed as dist
            if dist.is_initialized():
                dist.destroy_process_group()


if __name__ == "__main__":
    main()
