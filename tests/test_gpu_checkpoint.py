"""GPU: checkpoint and resume of an unfinished certified solve.

A search stopped after a few node batches leaves its open queue (fixing sets,
parent bounds, warm starts) and incumbent; kglm_solve_checkpoint writes them,
and kglm_solve_resume on a fresh context of the same instance (in the same or
another precision) continues the search.  The resumed search must certify the
optimum that brute force over all supports gives (definition of problem
(intro_sparse_glm)) and that an uninterrupted solve gives, with the support of
the unique optimum; a checkpoint is refused for another instance, for a
completed search, and when the file is malformed.
"""

import os

import numpy as np
import pytest

from oracle import reopt as ro
from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu


def _instance():
    X, y, _ = synth.instance(40, 16, 4, synth.LSQ, rho=0.9, snr=1.0, seed=3)
    return X, y, 4, 1e-3, 2.0


@pytest.mark.parametrize("prec_a,prec_b", [("fp64", "fp64"), ("fp64", "bf16"), ("tf32x3", "fp32")])
def test_resumed_search_certifies_the_same_optimum(tmp_path, prec_a, prec_b):
    X, y, k, lam2, M = _instance()
    top = ro.brute_force(X, y, k, lam2, M, synth.LSQ, top=2)
    best = top[0]
    delta = 1e-6 * max(1.0, abs(best[0]))
    path = os.fspath(tmp_path / "bnb.ckp")
    with kglm.Engine(X, y, k, lam2, M, synth.LSQ, prec=prec_a, max_batch=8) as eng:
        full = eng.solve(4, 300, 20)
        eng.set_solve_limit(2)                      # two batches of four nodes, then stop
        part = eng.solve(4, 300, 20)
        assert part["batches"] == 2 and part["gap"] > 1e-6, part
        eng.checkpoint(path)
    with kglm.Engine(X, y, k, lam2, M, synth.LSQ, prec=prec_b, max_batch=8) as eng:
        res = eng.resume(path, 4, 300, 20)
    assert full["gap"] <= 1e-6 and res["gap"] <= 1e-6
    assert abs(res["opt"] - best[0]) <= 1e-9 * abs(best[0]) + delta
    assert abs(res["opt"] - full["opt"]) <= 2 * delta
    if top[1][0] - best[0] > delta:
        assert tuple(res["support"]) == tuple(best[1])
        assert res["support"] == full["support"]
    assert res["batches"] > part["batches"] and res["nodes"] > part["nodes"]


def test_checkpoint_refusals(tmp_path):
    X, y, k, lam2, M = _instance()
    path = os.fspath(tmp_path / "bnb.ckp")
    with kglm.Engine(X, y, k, lam2, M, synth.LSQ, prec="fp64", max_batch=8) as eng:
        eng.solve(4, 300, 20)                       # completes: nothing open
        with pytest.raises(kglm.KglmError) as ei:
            eng.checkpoint(path)
        assert ei.value.status == kglm.KGLM_ESTATE
        eng.set_solve_limit(1)
        eng.solve(4, 300, 20)
        eng.checkpoint(path)
    # another instance (same sizes, other data) and a truncated file are refused
    X2 = X.copy()
    X2[0, 0] += 0.5
    with kglm.Engine(X2, y, k, lam2, M, synth.LSQ, prec="fp64", max_batch=8) as eng:
        with pytest.raises(kglm.KglmError) as ei:
            eng.resume(path, 4, 300, 20)
        assert ei.value.status == kglm.KGLM_EINVAL
    data = open(path, "rb").read()
    bad = os.fspath(tmp_path / "short.ckp")
    open(bad, "wb").write(data[:len(data) // 2])
    with kglm.Engine(X, y, k, lam2, M, synth.LSQ, prec="fp64", max_batch=8) as eng:
        with pytest.raises(kglm.KglmError) as ei:
            eng.resume(bad, 4, 300, 20)
        assert ei.value.status == kglm.KGLM_EINVAL
        # the context is still usable after a refused resume
        assert eng.solve(4, 300, 20)["gap"] <= 1e-6
