"""The serving loop (kglm_server_*) and the device footprint used for its admission.

* Every result is the same alone and in the mix: a request's nodes see the
  same arithmetic whatever shares its rounds and launches, so objective,
  support and node count are compared exactly with the request alone on the
  server (FP64 and reduced precision alike); requests whose iterations run
  their own launches also equal kglm_solve exactly, BF16 ones its certified
  optimum; small instances are also checked against brute force.
* Shared launches: BF16 requests in flight together are evaluated by grouped
  products and a grouped prox (the server counts the launches that carried
  more than one request).
* Admission: FIFO order, the bytes in use never pass the budget, the footprint
  kglm_estimate_bytes predicts is what kglm_create allocates.
* Failures stay inside their request: bad data fails that request only, an
  instance larger than the budget is refused at submission, destroying the
  server stops running requests at a batch boundary.
"""

import time

import numpy as np
import pytest

from oracle import reopt as ro
from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "tf32"])
@pytest.mark.parametrize("n,p,m,given_L", [(200, 30, 64, False), (2000, 200, 1024, True), (777, 333, 100, False)])
def test_device_bytes_equal_the_estimate(prec, n, p, m, given_L):
    X, y, _ = synth.instance(n, p, 5, synth.LOGISTIC, seed=1)
    L = 10.0 if given_L else 0.0
    with kglm.Engine(X, y, 5, 1e-2, 2.0, synth.LOGISTIC, prec=prec, max_batch=m, lipschitz=L) as eng:
        got = eng.device_bytes()
    want = kglm.kglm_estimate_bytes(kglm.make_desc(n, p, 5, 1e-2, 2.0, synth.LOGISTIC, prec, m, L))
    assert got == want


def _mix():
    """Six small instances of both losses, several shapes and precisions."""
    specs = [
        (synth.LSQ, 120, 18, 4, 1e-3, 0.7, 3.0, "fp64", 16),
        (synth.LOGISTIC, 150, 16, 3, 5e-2, 0.6, 5.0, "fp32", 32),
        (synth.LSQ, 300, 40, 5, 1e-3, 0.9, 3.0, "bf16", 64),
        (synth.LOGISTIC, 400, 50, 5, 1e-2, 0.5, 5.0, "bf16", 64),
        (synth.LSQ, 200, 30, 5, 1e-3, 0.5, 5.0, "tf32", 32),
        (synth.LOGISTIC, 250, 24, 4, 2e-2, 0.7, 5.0, "fp64", 16),
    ]
    out = []
    for i, (kind, n, p, k, lam2, rho, snr, prec, batch) in enumerate(specs):
        X, y, _ = synth.instance(n, p, k, kind, rho=rho, snr=snr, seed=100 + i)
        out.append(dict(X=X, y=y, k=k, lam2=lam2, M=2.0, kind=kind, prec=prec, batch=batch))
    return out


ITERS, CHECK = 200, 10


def _alone(inst):
    """The request on a server of its own (nothing shares its rounds or launches)."""
    with kglm.Server(max_active=1, iters=ITERS, check_every=CHECK) as srv:
        r = srv.submit(inst["X"], inst["y"], inst["k"], inst["lam2"], inst["M"], inst["kind"], prec=inst["prec"],
                       max_batch=inst["batch"])
        return srv.wait(r, timeout=300)


def _engine(inst):
    with kglm.Engine(inst["X"], inst["y"], inst["k"], inst["lam2"], inst["M"], inst["kind"], prec=inst["prec"],
                     max_batch=inst["batch"]) as eng:
        return eng.solve(inst["batch"], ITERS, CHECK)


def test_each_result_is_the_same_alone_and_in_the_mix():
    """Bit for bit against the request alone on the server; against kglm_solve
    (host queue, the context's own launches): identical in the precisions whose
    iterations do not share launches (the device queue evaluates the host queue's
    nodes in its order), the same certified optimum and support in BF16 (its
    grouped products tile the link product without split-K, which rounds S
    differently)."""
    mix = _mix()
    alone = [_alone(inst) for inst in mix]
    eng = [_engine(inst) for inst in mix]
    fp = [kglm.kglm_estimate_bytes(kglm.make_desc(i["X"].shape[0], i["X"].shape[1], i["k"], i["lam2"], i["M"],
                                                  i["kind"], i["prec"], i["batch"])) for i in mix]
    budget = int(sum(sorted(fp)[-3:]))          # at most three at once: later requests queue
    with kglm.Server(max_active=4, hbm_budget=budget, iters=ITERS, check_every=CHECK) as srv:
        ids = [srv.submit(i["X"], i["y"], i["k"], i["lam2"], i["M"], i["kind"], prec=i["prec"], max_batch=i["batch"])
               for i in mix]
        srv.drain(timeout=300)
        infos = [srv.info(r) for r in ids]
        st = srv.stats()
    assert st["finished"] == len(mix) and st["peak_bytes"] <= budget and st["peak_active"] <= 4
    for inst, a, b, e in zip(mix, alone, infos, eng):
        assert b["state"] == kglm.REQ_DONE and b["status"] == 0
        assert b["opt"] == a["opt"], (b["opt"], a["opt"])
        assert b["support"] == a["support"]
        assert b["nodes"] == a["nodes"] and b["batches"] == a["batches"]
        assert b["gap"] <= 1e-6
        if inst["prec"] == "bf16":
            assert abs(b["opt"] - e["opt"]) <= 2e-6 * max(1.0, abs(e["opt"])) and b["support"] == e["support"]
        else:
            assert (b["opt"], b["support"], b["nodes"], b["batches"]) == (e["opt"], e["support"], e["nodes"],
                                                                          e["batches"])
    # the two smallest are also checked against brute force
    for inst, b in list(zip(mix, infos))[:2]:
        top = ro.brute_force(inst["X"], inst["y"], inst["k"], inst["lam2"], inst["M"], inst["kind"], top=1)
        assert abs(b["opt"] - top[0][0]) <= 1e-6 * max(1.0, abs(top[0][0]))


def test_admission_is_fifo_within_the_budget():
    mix = _mix() * 2
    fp = max(kglm.kglm_estimate_bytes(kglm.make_desc(i["X"].shape[0], i["X"].shape[1], i["k"], i["lam2"], i["M"],
                                                     i["kind"], i["prec"], i["batch"])) for i in mix)
    budget = int(1.5 * fp)                      # one big request at a time, sometimes two small
    with kglm.Server(max_active=8, hbm_budget=budget, iters=ITERS, check_every=CHECK) as srv:
        ids = [srv.submit(i["X"], i["y"], i["k"], i["lam2"], i["M"], i["kind"], prec=i["prec"], max_batch=i["batch"])
               for i in mix]
        for r in ids:
            srv.wait(r, timeout=300)
        infos = [srv.info(r) for r in ids]
        st = srv.stats()
    assert st["peak_bytes"] <= budget
    adm = [i["t_admit"] for i in infos]
    assert all(adm[t] <= adm[t + 1] for t in range(len(adm) - 1)), adm
    for i in infos:
        assert i["t_submit"] <= i["t_admit"] <= i["t_done"]
        assert i["state"] == kglm.REQ_DONE


def test_automatic_batch_and_failures_stay_inside_their_request():
    X, y, _ = synth.instance(300, 40, 5, synth.LSQ, rho=0.7, snr=3.0, seed=7)
    bad = X.copy()
    bad[3, 4] = np.nan
    with kglm.Server(max_active=2, hbm_budget=1 << 30, iters=ITERS, check_every=CHECK, batch_cap=256) as srv:
        ok = srv.submit(X, y, 5, 1e-3, 2.0, synth.LSQ, prec="fp32", max_batch=0)
        nan = srv.submit(bad, y, 5, 1e-3, 2.0, synth.LSQ, prec="fp32", max_batch=16)
        with pytest.raises(kglm.KglmError) as ei:
            big = np.zeros((20000, 4000))
            srv.submit(big, np.zeros(20000), 5, 1e-3, 2.0, synth.LSQ, prec="fp64", max_batch=1024)
        assert ei.value.status == kglm.KGLM_ENOMEM
        a = srv.wait(ok, timeout=120)
        b = srv.wait(nan, timeout=120)
    assert a["state"] == kglm.REQ_DONE and a["gap"] <= 1e-6
    assert a["batch"] & (a["batch"] - 1) == 0 and 1 <= a["batch"] <= 256
    assert b["state"] == kglm.REQ_FAILED and b["status"] == kglm.KGLM_ENUMERIC


def test_destroy_stops_running_requests_at_a_batch_boundary():
    # a correlated instance that takes many batches at batch size 1
    X, y, _ = synth.instance(400, 60, 8, synth.LSQ, rho=0.9, snr=1.0, seed=3)
    srv = kglm.Server(max_active=2, hbm_budget=1 << 30, iters=50, check_every=0)
    ids = [srv.submit(X, y, 8, 1e-3, 2.0, synth.LSQ, prec="fp32", max_batch=1) for _ in range(3)]
    time.sleep(0.5)
    t0 = time.perf_counter()
    srv.close()
    assert time.perf_counter() - t0 < 30.0
    assert ids


def test_contexts_with_different_k_evaluate_concurrently():
    """Two contexts whose re-optimization needs different shared memory (k = 3 and
    k = 40) evaluate node batches from two host threads at once.  A per-launch
    shared-memory opt-in sized to one context's k could be lowered by the other
    between its setting and its launch ("too many resources requested"); the
    setting and the launch now happen under one lock."""
    import threading
    errors = []

    def run(k, seed):
        try:
            X, y, _ = synth.instance(600, 120, min(k, 10), synth.LOGISTIC, rho=0.5, seed=seed)
            rng = np.random.default_rng(seed)
            csr = synth.random_nodes(256, 120, k, rng)
            with kglm.Engine(X, y, k, 1e-2, 2.0, synth.LOGISTIC, prec="bf16", max_batch=256) as eng:
                for _ in range(25):
                    eng.push(*csr)
                    res = eng.evaluate(10)
                    assert np.all(np.isfinite(res["ub"]))
        except Exception as e:   # reported to the main thread
            errors.append(repr(e))

    ts = [threading.Thread(target=run, args=(3, 1)), threading.Thread(target=run, args=(40, 2))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors


def test_bf16_requests_share_launches_and_keep_their_results():
    """Five BF16 requests of different n, p, k and both losses run at once: their
    iterations go through grouped launches (the server counts launches that carried
    more than one request) and each result equals the request alone, bit for bit;
    the small ones equal brute force."""
    specs = [(synth.LSQ, 200, 20, 3, 1e-3, 0.8, 2.0, 32), (synth.LOGISTIC, 300, 18, 3, 2e-2, 0.6, 5.0, 64),
             (synth.LSQ, 500, 260, 6, 1e-3, 0.5, 4.0, 128), (synth.LOGISTIC, 700, 150, 5, 1e-2, 0.5, 5.0, 96),
             (synth.LSQ, 1200, 300, 8, 1e-3, 0.6, 3.0, 256)]
    mix = []
    for i, (kind, n, p, k, lam2, rho, snr, batch) in enumerate(specs):
        X, y, _ = synth.instance(n, p, k, kind, rho=rho, snr=snr, seed=300 + i)
        mix.append(dict(X=X, y=y, k=k, lam2=lam2, M=2.0, kind=kind, prec="bf16", batch=batch))
    alone = [_alone(inst) for inst in mix]
    with kglm.Server(max_active=8, iters=ITERS, check_every=CHECK) as srv:
        ids = [srv.submit(i["X"], i["y"], i["k"], i["lam2"], i["M"], i["kind"], prec="bf16", max_batch=i["batch"])
               for i in mix]
        srv.drain(timeout=300)
        infos = [srv.info(r) for r in ids]
        st = srv.stats()
    assert st["shared_launches"] > 0 and st["round_batches"] > st["rounds"], st
    for a, b in zip(alone, infos):
        assert b["state"] == kglm.REQ_DONE and b["gap"] <= 1e-6
        assert (b["opt"], b["support"], b["nodes"], b["batches"]) == (a["opt"], a["support"], a["nodes"],
                                                                      a["batches"])
    for inst, b in list(zip(mix, infos))[:2]:
        top = ro.brute_force(inst["X"], inst["y"], inst["k"], inst["lam2"], inst["M"], inst["kind"], top=1)
        assert abs(b["opt"] - top[0][0]) <= 1e-6 * max(1.0, abs(top[0][0]))
