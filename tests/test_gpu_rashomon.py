"""Rashomon-set collection (kglm_rashomon, §4.5) against the brute-force definition.

The engine's pool must hold exactly the supports S with |S| <= k and
v(S) <= (1 + eps) Phi* (or the N best of them with the cap), with Phi* the
certified optimum.  Supports within 1e-6 relative of the threshold are
borderline (the engine's objectives carry the re-optimization tolerance) and
are neither required nor forbidden; their count is reported.  Every stored
record's objective is the FP64 objective of its stored coefficients, and its
coefficients are in the order of its trie path (App. G).
"""

import numpy as np
import pytest

from oracle import reopt as ro
from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu

BORDER = 1e-6


def _compare(pool, info, X, y, k, lam2, M, kind, eps, N=None, obj_rtol=1e-9):
    phi, R = ro.rashomon_set(X, y, k, lam2, M, kind, eps, N)
    recs = pool.records()
    assert info["complete"]
    assert abs(info["opt"] - phi) <= obj_rtol * max(1.0, abs(phi)), (info["opt"], phi)
    tau = (1.0 + eps) * phi
    if N is not None and len(R) == N:
        tau = min(tau, R[-1][0])
    _, allv = ro.rashomon_set(X, y, k, lam2, M, kind, 1e9)
    vmap = {S: v for v, S in allv}
    border = {S for S, v in vmap.items() if abs(v - tau) <= BORDER * tau}
    got = {S for _, S, _, _ in recs}
    want = {S for _, S in R}
    assert (got - border) == (want - border), (sorted(got - want), sorted(want - got))
    for v, S, coef, labels in recs:
        beta = np.zeros(X.shape[1])
        beta[labels] = coef
        assert abs(ro.objective(X, y, beta, lam2, kind) - v) <= 1e-9 * max(1.0, v)
        assert v >= vmap[S] - 1e-9 * vmap[S] and v - vmap[S] <= obj_rtol * max(1.0, vmap[S])
    return len(border & (got ^ want))


@pytest.mark.parametrize("prec", ["fp64", "bf16", "tf32x3"])
@pytest.mark.parametrize("kind", [synth.LSQ, synth.LOGISTIC])
def test_rashomon_set_matches_brute_force(kind, prec):
    X, y, _ = synth.instance(40, 7, 3, kind, rho=0.6, snr=0.5, seed=8)
    lam2, M = 0.05, 2.0
    rtol = 1e-9 if prec == "fp64" else 2e-6
    with kglm.Engine(X, y, 3, lam2, M, kind, prec=prec, max_batch=16) as eng:
        pool, info = eng.rashomon(0.2, batch=16, iters=400, check_every=20)
        with pool:
            nb = _compare(pool, info, X, y, 3, lam2, M, kind, 0.2, obj_rtol=rtol)
            print("%s %s: %d records, %d nodes, %d borderline" % (kind, prec, len(pool.records()), info["nodes"], nb))


@pytest.mark.parametrize("kind", [synth.LSQ, synth.LOGISTIC])
def test_rashomon_top_n_cap(kind):
    X, y, _ = synth.instance(60, 12, 3, kind, rho=0.5, snr=1.0, seed=21)
    lam2, M = 0.02, 2.0
    with kglm.Engine(X, y, 3, lam2, M, kind, prec="fp64", max_batch=64) as eng:
        pool, info = eng.rashomon(0.5, max_models=5, batch=64, iters=400, check_every=20)
        with pool:
            _compare(pool, info, X, y, 3, lam2, M, kind, 0.5, N=5)
            assert len(pool.records()) <= 5
