"""Node-parallel branch and bound across ranks (App. D, node-parallel regime).

Node batches are independent, so ranks can evaluate disjoint parts of the open
frontier; the one exchange the method needs is the incumbent (a min over the
ranks' best objectives), plus the bookkeeping of which nodes were evaluated and
what children they produced.  This driver runs the hybrid loop of Fig. 1 on
every rank in rounds, communicating through a key-value store only (the TCP
store of torch.distributed), so that a rank that leaves, or stops answering,
between batches cannot hang the others in a collective:

* every live rank holds the same global frontier (open nodes with their
  parent bounds and warm starts) and the same incumbent;
* round r: the frontier, pruned against the incumbent (LB >= UB - delta,
  delta = gap_tol * max(1, |UB|)), is sorted by (bound, id) and dealt
  round-robin over the live ranks; each rank evaluates the best `batch` nodes
  of its share with its evaluator and posts the ids it evaluated, the children
  of the nodes it branched (both children inherit the node's final beta,
  Fig. 1 "warm starts") and its best re-optimized support;
* every rank then reads the posts of round r in rank order: the incumbent
  becomes the minimum over the posted objectives (the all-reduce(min) of
  App. D), the evaluated nodes leave the frontier and their children join it;
* a rank that posts "leave" instead of results, or whose post does not arrive
  within `timeout_s`, is dropped from the live set: its share of the round was
  not evaluated, so those nodes are still in the frontier and are dealt to the
  survivors in the next round; nothing is lost and the survivors still certify;
* the search ends when the frontier is empty: the incumbent is then certified
  optimal (every node was pruned, fathomed or closed as a leaf).

The evaluator is pluggable: `EngineEvaluator` runs a node batch through the
CUDA engine (kglm_push_nodes, kglm_evaluate, kglm_read_batch).
"""

import pickle
import time

import numpy as np


class Node:
    __slots__ = ("lb", "id", "J0", "J1", "warm")

    def __init__(self, lb, nid, J0, J1, warm=None):
        self.lb, self.id, self.J0, self.J1, self.warm = float(lb), int(nid), tuple(J0), tuple(J1), warm


class EngineEvaluator:
    """Evaluate a node batch on the GPU engine: `iters` FISTA iterations (certificate
    every `check_every`), the FP64 bound, rounding, re-optimization and branching index."""

    def __init__(self, engine, iters, check_every=10):
        self.eng, self.iters, self.check_every = engine, int(iters), int(check_every)

    def __call__(self, nodes, ub):
        from . import synth
        p = self.eng.p
        csr = synth.sets_to_csr([(n.J0, n.J1) for n in nodes])
        warm = None
        if any(n.warm is not None for n in nodes):
            warm = np.zeros((len(nodes), p))
            for b, n in enumerate(nodes):
                if n.warm is not None:
                    warm[b] = n.warm
        self.eng.set_incumbent(ub if np.isfinite(ub) else 1e300)
        self.eng.push(*csr, warm_B=warm)
        res = self.eng.evaluate(self.iters, self.check_every)
        B, _ = self.eng.read_batch(beta=True, zeta=False)
        out = []
        for b in range(len(nodes)):
            sup = [int(s) for s in res["support"][b] if s >= 0]
            out.append(dict(lb=float(res["lb"][b]), ub=float(res["ub"][b]), support=sup,
                            branch_j=int(res["branch_j"][b]), beta=B[b].copy()))
        return out


class StoreComm:
    """Round posts through a torch.distributed store (TCPStore)."""

    def __init__(self, store, rank, world, timeout_s=30.0, prefix="nodepar"):
        self.store, self.rank, self.world, self.timeout_s, self.prefix = store, int(rank), int(world), timeout_s, prefix

    def key(self, rnd, rank):
        return "%s/%d/%d" % (self.prefix, rnd, rank)

    def post(self, rnd, obj):
        self.store.set(self.key(rnd, self.rank), pickle.dumps(obj))

    def read(self, rnd, rank):
        """The post of `rank` for round rnd, or None if it does not arrive within the timeout."""
        k = self.key(rnd, rank)
        deadline = time.monotonic() + self.timeout_s
        while True:
            try:
                if self.store.check([k]):
                    return pickle.loads(self.store.get(k))
            except RuntimeError:
                pass
            if time.monotonic() > deadline:
                return None
            time.sleep(0.002)


def node_parallel_solve(evaluate, p, k, comm, batch, gap_tol=1e-6, max_rounds=100000, leave_at_round=None):
    """Run the node-parallel BnB on this rank; returns dict(opt, support, rounds, evaluated,
    live, certified).  `evaluate(nodes, ub)` -> per node dict(lb, ub, support, branch_j, beta).
    leave_at_round: this rank announces that it leaves before evaluating that round
    (returns immediately with certified=False)."""
    delta = lambda u: gap_tol * max(1.0, abs(u)) if np.isfinite(u) else 0.0
    frontier = {0: Node(-np.inf, 0, (), ())}
    next_ids = {}
    ub, best_sup = np.inf, None
    live = list(range(comm.world))
    evaluated = 0
    rnd = 0
    while frontier and rnd < max_rounds:
        if comm.rank not in live:
            break
        if leave_at_round is not None and rnd == leave_at_round:
            comm.post(rnd, {"leave": True})
            return dict(opt=ub, support=best_sup, rounds=rnd, evaluated=evaluated, live=live, certified=False)
        order = sorted((n for n in frontier.values() if not (n.lb >= ub - delta(ub))), key=lambda n: (n.lb, n.id))
        mine = [n for i, n in enumerate(order) if live[i % len(live)] == comm.rank][:batch]
        post = {"evaluated": [], "children": [], "ub": np.inf, "support": None}
        if mine:
            res = evaluate(mine, ub)
            for n, r in zip(mine, res):
                post["evaluated"].append(n.id)
                if r["ub"] < post["ub"]:
                    post["ub"], post["support"] = r["ub"], r["support"]
                lbb = max(r["lb"], n.lb)
                cand = min(ub, post["ub"])
                leaf = r["branch_j"] < 0
                if leaf or lbb >= cand - delta(cand) or r["ub"] - lbb <= delta(r["ub"]):
                    continue                         # closed: leaf, pruned or fathomed
                j = r["branch_j"]
                warm = np.asarray(r["beta"], dtype=np.float64)
                post["children"].append(Node(lbb, 2 * n.id + 1, n.J0 + (j,), n.J1, warm))
                post["children"].append(Node(lbb, 2 * n.id + 2, n.J0, n.J1 + (j,), warm))
            evaluated += len(mine)
        comm.post(rnd, post)
        # merge every live rank's post, in rank order (the same on every rank)
        survivors = []
        for r in live:
            got = post if r == comm.rank else comm.read(rnd, r)
            if got is None or got.get("leave"):
                continue                             # left or silent: its share stays open
            survivors.append(r)
            if got["ub"] < ub:
                ub, best_sup = got["ub"], got["support"]
            for nid in got["evaluated"]:
                frontier.pop(nid, None)
            for c in got["children"]:
                frontier[c.id] = c
        live = survivors
        frontier = {i: n for i, n in frontier.items() if not (n.lb >= ub - delta(ub))}
        rnd += 1
    return dict(opt=ub, support=sorted(best_sup) if best_sup is not None else None, rounds=rnd,
                evaluated=evaluated, live=live, certified=not frontier)
