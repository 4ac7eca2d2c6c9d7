"""Oracle node solves on worker processes (test infrastructure).

The pool is started with the 'spawn' method, so it is safe to start after
the test process has made CUDA calls; the workers only import the oracle and
the seeded input generators.
"""

import multiprocessing as mp
import os

_STATE = {}


def _init(X, y, p, k, lam2, M, kind, L, T):
    os.environ["OMP_NUM_THREADS"] = "1"
    _STATE.update(X=X, y=y, p=p, k=k, lam2=lam2, M=M, kind=kind, L=L, T=T)


def _solve(sets):
    from oracle import node as on
    s = _STATE
    J0, J1 = sets
    r = on.solve_node(s["X"], s["y"], on.Node(s["p"], s["k"], J0, J1), s["lam2"], s["M"], s["kind"], s["L"], s["T"])
    return r["lb"], r["primal"], r["beta"]


def solve_nodes(X, y, p, k, lam2, M, kind, L, T, nodes, procs=None):
    """[(lb, primal, beta)] of oracle.node.solve_node (T iterations, warm start 0) for each (J0, J1)."""
    procs = procs or min(len(nodes), os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs, initializer=_init, initargs=(X, y, p, k, lam2, M, kind, L, T)) as pool:
        return pool.map(_solve, [(list(J0), list(J1)) for J0, J1 in nodes], chunksize=4)
