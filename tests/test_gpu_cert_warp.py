"""GPU: the certificate of the reduced-precision modes on inputs that take its
slow paths.

In the BF16/TF32 modes X^T zeta arrives as exact-splitting partial products;
the certificate kernel takes a warp per node, bounds every free coordinate's
value v_j = (|q~_j| + err_j) / (2 lambda2) from above and below in FP32, and
computes v_j exactly in FP64 only for the coordinates whose upper bound
reaches a threshold taken from per-lane samples of the lower bounds.  The same
kernel ranks |beta| over the free coordinates with ties to the smaller index.
Ties defeat the thresholds, so these cases force the fallbacks:

* y = 0: beta stays 0 and zeta = 0 on every node: every free coordinate ties
  in v and in |beta| (the support is J1 plus the smallest free indices, the
  branching index the smallest free index);
* X of rank one (column j = s_j x with s_j = +-1): |q_j| ties on every free
  coordinate, and so do the |beta_j| that the prox treats alike;
* columns repeated in groups of eight: ties inside each group only.

The checks are those of the other reduced-precision tests: the bound is a
certificate at the GPU's own dual point (never above Psi_N there, and within
1e-6 relative of it, plus for the logistic loss the FP32 conjugate terms'
rounding margins, at most 2^-21 of each |l*(-zeta_i)|: with repeated columns
the logistic sum of conjugates nearly cancels against the TopSum part, so
those margins exceed 1e-6 of Psi_N), support and branching index are the
oracle's decisions on the GPU's iterate, and the primal value is the oracle's Phi_N of that iterate to 1e-5
relative.  That bar is set by the loss term: its margins X beta come from the
split TF32 products (about 2^-22 relative per term), and on the rank-one
design the margins are sums with cancellation of up to two orders of
magnitude; g_N itself is summed in compensated FP32 (about 2^-44 relative).
p = 1029 leaves a ragged last mask word.
"""

import numpy as np
import pytest

from oracle import node as on
from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu

N, P, K = 240, 1029, 12


def _nodes(p, k, rng, m):
    nodes = [([], []),
             ([], list(range(k))),                                   # kbar = 0
             (list(range(p - k + 1)), []),                           # pf = k - 1 < kbar
             (list(range(1, p - 2)), [0]),                           # pf = 2 <= kbar
             (sorted(rng.choice(p, p // 2, replace=False).tolist()), []),
             ([j for j in range(p) if j % 3], [0, 3])]
    return nodes + synth.csr_to_sets(*synth.random_nodes(m - len(nodes), p, k, rng))


def _instance(case, kind, rng):
    if case == "zero":
        X = synth.design(N, P, 0.3, rng)
        return X, np.zeros(N)
    if case == "rank1":
        x = rng.standard_normal(N)
        X = np.outer(x, np.where(rng.random(P) < 0.5, -1.0, 1.0))
    else:
        X = np.repeat(synth.design(N, (P + 7) // 8, 0.3, rng), 8, axis=1)[:, :P]
    bstar = np.zeros(P)
    bstar[[0, 40, 400, P - 1]] = [1.0, -1.0, 1.0, -1.0]
    s = X @ bstar
    if kind == synth.LSQ:
        y = s + 0.3 * rng.standard_normal(N)
    else:
        y = np.where(rng.random(N) < 1.0 / (1.0 + np.exp(-s)), 1.0, -1.0)
    return np.ascontiguousarray(X), y


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
@pytest.mark.parametrize("case,kind", [("zero", synth.LSQ), ("rank1", synth.LSQ), ("groups", synth.LSQ),
                                       ("groups", synth.LOGISTIC)])
def test_certificate_with_ties(case, kind, prec):
    rng = np.random.default_rng(31)
    X, y = _instance(case, kind, rng)
    lam2, M, T = 1e-2, 2.0, 15
    L = on.lipschitz(X, kind)
    nodes = _nodes(P, K, rng, 24)
    with kglm.Engine(X, y, K, lam2, M, kind, prec=prec, max_batch=len(nodes), lipschitz=L) as eng:
        eng.push(*synth.sets_to_csr(nodes))
        res = eng.evaluate(T)
        B, Z = eng.read_batch()
    if case == "zero":
        assert not np.any(B) and not np.any(Z)
    for b, (J0, J1) in enumerate(nodes):
        nd = on.Node(P, K, J0, J1)
        psi = on.dual_value(X, y, Z[b], nd, lam2, M, kind)
        lb = res["lb"][b]
        assert lb <= psi + 1e-12 * max(1.0, abs(psi)), (b, lb, psi)
        tol = 1e-6 * max(1.0, abs(psi))
        if kind == synth.LOGISTIC:
            tol += 2.0 ** -21 * float(np.sum(np.abs(on.loss_conj(-Z[b], y, kind))))
        assert psi - lb <= tol, (b, lb, psi, tol)
        S = on.round_support(B[b], nd)
        assert [int(s) for s in res["support"][b] if s >= 0] == S, b
        assert res["branch_j"][b] == on.branch_index(B[b], nd), b
        phi = on.primal_value(X, y, B[b].astype(np.float64), nd, lam2, M, kind)
        if np.isfinite(phi):
            assert abs(res["primal"][b] - phi) <= 1e-5 * max(1.0, abs(phi)), (b, res["primal"][b], phi)
        else:
            assert np.isinf(res["primal"][b]), b
