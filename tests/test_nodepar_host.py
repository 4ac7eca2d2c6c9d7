"""Node-parallel branch and bound on 2 CPU ranks (gloo), App. D node-parallel regime.

The ranks share the incumbent (the minimum over their posted objectives) and
deal the open frontier between them each round; the node evaluator is the FP64
oracle (T FISTA iterations with periodic certificates, rounding, re-optimization,
branching index), so the host protocol is exercised without a GPU.  Cases:
both ranks to the end; one rank leaving between batches (announced); one rank
going silent between batches (its post never arrives: the survivor times out).
In every case the surviving rank(s) must certify the brute-force optimum and
its support (definition of problem (intro_sparse_glm)).
"""

import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

from oracle import node as on
from oracle import reopt as ro
from paper_2605_22188_gb300 import synth

N, P, K, LAM2, M = 40, 12, 3, 1e-3, 2.0


def _instance():
    return synth.instance(N, P, K, synth.LSQ, rho=0.9, snr=1.0, seed=11)[:2]


def _oracle_evaluator(X, y):
    L = on.lipschitz(X, synth.LSQ)

    def evaluate(nodes, ub):
        out = []
        for n in nodes:
            nd = on.Node(P, K, n.J0, n.J1)
            d = 1e-6 * max(1.0, abs(ub)) if np.isfinite(ub) else 0.0
            r = on.solve_node(X, y, nd, LAM2, M, synth.LSQ, L, 400, beta0=n.warm, check_every=10, ub=ub, delta=d,
                              gap_rtol=1e-9)
            S = on.round_support(r["beta"], nd)
            _, v = ro.reopt(X, y, S, LAM2, M, synth.LSQ, beta0=r["beta"])
            out.append(dict(lb=r["lb"], ub=v, support=S, branch_j=on.branch_index(r["beta"], nd), beta=r["beta"]))
        return out
    return evaluate


def _rank(rank, world, port, store_port, mode, q):
    import torch.distributed as dist
    from paper_2605_22188_gb300 import nodepar
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    store = dist.TCPStore("127.0.0.1", store_port, world, is_master=(rank == 0), wait_for_workers=True)
    X, y = _instance()
    comm = nodepar.StoreComm(store, rank, world, timeout_s=5.0)
    if mode == "silent" and rank == 1:
        # evaluate two rounds, then stop posting (as a process that died between batches)
        res = nodepar.node_parallel_solve(_oracle_evaluator(X, y), P, K, comm, batch=2, max_rounds=2)
        q.put((rank, res["certified"], None, None, res["rounds"]))
        store.set("rank1_done", b"1")
        return
    leave = 2 if (mode == "leave" and rank == 1) else None
    res = nodepar.node_parallel_solve(_oracle_evaluator(X, y), P, K, comm, batch=2, leave_at_round=leave)
    q.put((rank, res["certified"], res["opt"], res["support"], res["rounds"]))
    if mode == "silent" and rank == 0:
        store.wait(["rank1_done"])
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize("mode", ["both", "leave", "silent"])
def test_node_parallel_survivor_certifies_the_optimum(mode):
    X, y = _instance()
    top = ro.brute_force(X, y, K, LAM2, M, synth.LSQ, top=2)
    best = top[0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port, store_port = _free_port(), _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, store_port, mode, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    results = {}
    for _ in procs:
        r, cert, opt, sup, rounds = q.get(timeout=300)
        results[r] = (cert, opt, sup, rounds)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    delta = 1e-6 * max(1.0, abs(best[0]))
    finishers = [0, 1] if mode == "both" else [0]
    for r in finishers:
        cert, opt, sup, rounds = results[r]
        assert cert, (mode, r, results[r])
        assert abs(opt - best[0]) <= 1e-9 * abs(best[0]) + delta, (opt, best[0])
        if top[1][0] - best[0] > delta:
            assert tuple(sup) == tuple(best[1])
    if mode != "both":
        assert not results[1][0]                      # the leaver did not finish the search
        assert results[0][3] > 2                      # the survivor went on past the departure
