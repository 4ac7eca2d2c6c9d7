"""Sequential best-bound branch and bound with one node per evaluation (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

Fig. 1 of §4.1 with a batch of one node: pop the open node with the smallest
bound, solve its relaxation and certify a lower bound (§3), round to a support
and re-optimize (§4.3) to offer an incumbent, prune if LB >= UB - delta
(§3 "Safe Lower Bound and Pruning"), otherwise branch on j* (§4.3) and insert
both children.  Readings where the paper is silent:

* delta = gap_tol * max(1, |UB|): pruning with ">=" in floating point;
* a leaf (kbar = 0 or |J1| + pf <= k) is closed after its evaluation, and a
  node whose own rounded solution is within delta of its bound is fathomed;
* node order is best-bound on the parent's bound, ties to the older node;
* children start from the parent's final beta, with beta_{j*} = 0 in the
  z_{j*} = 0 child (that coordinate is in J0 there);
* the incumbent starts at +inf and is set by the root's rounding.
"""

import heapq
import time

import numpy as np

from .node import Node, lipschitz, solve_node, round_support, branch_index
from .reopt import reopt


def solve(X, y, k, lam2, M, kind, T_max=1000, check_every=10, gap_tol=1e-6,
          node_rtol=1e-9, time_limit=None, L=None, restart=True, log=None):
    """Certify min { F(X beta) + lambda2 ||beta||^2 : ||beta||_0 <= k, ||beta||_inf <= M }.

    Returns dict(opt, support, beta, nodes, gap, certified, seconds).
    """
    t0 = time.perf_counter()
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p = X.shape[1]
    if L is None:
        L = lipschitz(X, kind)
    ub = np.inf
    inc_support, inc_beta = None, None
    counter = 0
    heap = [(-np.inf, counter, Node(p, k), np.zeros(p))]
    nodes = 0

    def delta_of(u):
        return gap_tol * max(1.0, abs(u)) if np.isfinite(u) else 0.0

    while heap:
        if time_limit is not None and time.perf_counter() - t0 > time_limit:
            break
        lb_parent, _, nd, warm = heapq.heappop(heap)
        if lb_parent >= ub - delta_of(ub):
            continue                                   # pruned by the parent's bound
        nodes += 1
        res = solve_node(X, y, nd, lam2, M, kind, L, T_max, beta0=warm, restart=restart,
                         check_every=check_every, ub=ub, delta=delta_of(ub), gap_rtol=node_rtol)
        beta, lb = res["beta"], res["lb"]
        lb = max(lb, lb_parent)                        # the parent's bound also holds here
        S = round_support(beta, nd)
        b_re, v = reopt(X, y, S, lam2, M, kind, beta0=beta)
        if v < ub:
            ub, inc_support, inc_beta = v, S, b_re
        if log is not None:
            log.append(dict(node=nodes, J0=nd.J0, J1=nd.J1, lb=lb, v=v, ub=ub))
        if lb >= ub - delta_of(ub):
            continue                                   # pruned
        if nd.is_leaf():
            continue                                   # leaf: its rounding is exact
        if v - lb <= delta_of(ub):
            continue                                   # fathomed by its own rounding
        j = branch_index(beta, nd)
        c0, c1 = nd.children(j)
        w0 = beta.copy()
        w0[j] = 0.0
        counter += 1
        heapq.heappush(heap, (lb, counter, c0, w0))
        counter += 1
        heapq.heappush(heap, (lb, counter, c1, beta.copy()))
    open_lb = min((h[0] for h in heap), default=np.inf)
    glb = min(open_lb, ub)
    gap = (ub - glb) / max(1.0, abs(ub)) if np.isfinite(ub) else np.inf
    return dict(opt=ub, support=inc_support, beta=inc_beta, nodes=nodes,
                gap=gap, certified=not heap, seconds=time.perf_counter() - t0)
