"""GPU: the hybrid loop of Fig. 1 with the open-node queue on the device.

kglm_solve_device keeps the open nodes in a device pool sorted by (parent
bound, id) and selects, closes, branches and prunes there.  It evaluates the
nodes in the order of the host queue (best bound, ties to the older node) with
the same incumbent updates and children, so on instances whose warm-start
slots never run out it must reproduce kglm_solve exactly: the same node and
batch counts and, in FP64, the same certified objective bit for bit; in every
mode the certified optimum and support must equal brute force over all
supports (definition of problem (intro_sparse_glm)).  A pool too small for the
search stops it with a positive gap whose bound is still valid; the device
bytes include the queue exactly as the estimate says.
"""

import numpy as np
import pytest

from oracle import reopt as ro
from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu


def _instances():
    c, X, y, _ = synth.config_instance("c1_lsq_n200_p30_k5", seed=0)
    yield "c1", X, y, c["k"], c["lam2"], c["M"], c["kind"]
    X, y, _ = synth.instance(40, 16, 4, synth.LSQ, rho=0.9, snr=1.0, seed=3)
    yield "hard_lsq", X, y, 4, 1e-3, 2.0, synth.LSQ
    X, y, _ = synth.instance(60, 12, 3, synth.LOGISTIC, rho=0.7, seed=4)
    yield "logistic", X, y, 3, 0.05, 2.0, synth.LOGISTIC


@pytest.mark.parametrize("prec", ["fp64", "bf16", "tf32x3"])
@pytest.mark.parametrize("batch", [1, 8, 64])
def test_device_queue_reproduces_the_host_queue(prec, batch):
    for name, X, y, k, lam2, M, kind in _instances():
        top = ro.brute_force(X, y, k, lam2, M, kind, top=2)
        best, second = top[0], top[1]
        delta = 1e-6 * max(1.0, abs(best[0]))
        with kglm.Engine(X, y, k, lam2, M, kind, prec=prec, max_batch=64, open_cap=4096) as eng:
            host = eng.solve(batch, 300, 20)
            dev = eng.solve_device(batch, 300, 20)
        assert dev["gap"] <= 1e-6, (name, dev)
        assert abs(dev["opt"] - best[0]) <= 1e-9 * abs(best[0]) + delta, (name, dev["opt"], best[0])
        if second[0] - best[0] > delta:
            assert tuple(dev["support"]) == tuple(best[1]), name
        assert (dev["nodes"], dev["batches"]) == (host["nodes"], host["batches"]), (name, dev, host)
        assert dev["support"] == host["support"], name
        if prec == "fp64":
            assert dev["opt"] == host["opt"], name
            assert np.array_equal(dev["beta"], host["beta"]), name


def test_pool_overflow_stops_with_a_valid_gap():
    X, y, _ = synth.instance(40, 16, 4, synth.LSQ, rho=0.9, snr=1.0, seed=3)
    best = ro.brute_force(X, y, 4, 1e-3, 2.0, synth.LSQ, top=1)[0]
    with kglm.Engine(X, y, 4, 1e-3, 2.0, synth.LSQ, prec="fp64", max_batch=8, open_cap=3) as eng:
        res = eng.solve_device(2, 300, 20)
        assert res["gap"] > 1e-6
        # the reported gap bounds the distance to the optimum from below: opt - gap*max(1,|opt|) <= v*
        assert res["opt"] >= best[0] - 1e-9 * abs(best[0])
        assert res["opt"] - res["gap"] * max(1.0, abs(res["opt"])) <= best[0] + 1e-9 * abs(best[0])
        with pytest.raises(kglm.KglmError) as ei:
            eng.checkpoint("/dev/null")
        assert ei.value.status == kglm.KGLM_ESTATE
        # the context is still usable; the host queue certifies
        assert eng.solve(8, 300, 20)["gap"] <= 1e-6


def test_device_queue_needs_a_pool_and_counts_its_bytes():
    X, y, _ = synth.instance(200, 30, 5, synth.LSQ, seed=1)
    with kglm.Engine(X, y, 5, 1e-2, 2.0, synth.LSQ, prec="bf16", max_batch=64) as eng:
        with pytest.raises(kglm.KglmError) as ei:
            eng.solve_device(8, 100, 20)
        assert ei.value.status == kglm.KGLM_EINVAL
    for prec in ("fp64", "bf16"):
        with kglm.Engine(X, y, 5, 1e-2, 2.0, synth.LSQ, prec=prec, max_batch=64, open_cap=1000) as eng:
            got = eng.device_bytes()
        want = kglm.kglm_estimate_bytes(kglm.make_desc(200, 30, 5, 1e-2, 2.0, synth.LSQ, prec, 64, open_cap=1000))
        assert got == want, prec
