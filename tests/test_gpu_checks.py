"""GPU: the bounds-checked build (KGLM_CHECKS=1, libkglm_checks.so).

In that build the prox, certificate and re-optimization kernels check the
indices they write or gather with; a failed check records its kernel and skips
the access, and the evaluation returns KGLM_EINVAL.  The test builds the checked
library and runs, in a child process that selects it:

* kglm_checks_enabled is 1, and the self-test's checked write one past the end
  of a context buffer is caught (KGLM_EINVAL), twice, with the context usable;
* evaluations on that context and others (FP64 products on a c1 batch, BF16
  tensor-core products on a c2-shaped batch, both losses) give the results the
  normal build is held to (the FP64 bound equals the oracle's to 1e-9; the BF16
  bound is the oracle's Psi at the GPU's dual point to 1e-6, never above) and no
  check fires on validated inputs.

In this process (the normal build) the self-test launches nothing and returns
KGLM_ESTATE.
"""

import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_2605_22188_gb300 import build, kglm, synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    sys.path.insert(0, %r)
    import numpy as np
    from oracle import node as on
    from paper_2605_22188_gb300 import kglm, synth

    assert kglm.lib_path().endswith("libkglm_checks.so"), kglm.lib_path()
    assert kglm.checks_enabled()
    c, X, y, _ = synth.config_instance("c1_lsq_n200_p30_k5", seed=0)
    L = on.lipschitz(X, c["kind"])
    csr = synth.random_nodes(8, c["p"], c["k"], np.random.default_rng(0), max_out=10)
    with kglm.Engine(X, y, c["k"], c["lam2"], c["M"], c["kind"], prec="fp64", max_batch=8, lipschitz=L) as eng:
        for _ in range(2):
            assert kglm.kglm_selftest_checks(eng.ctx) == kglm.KGLM_EINVAL
            assert "caught" in kglm.lib().kglm_last_error(eng.ctx).decode()
        eng.push(*csr)
        res = eng.evaluate(20)
    for b, (J0, J1) in enumerate(synth.csr_to_sets(*csr)):
        ref = on.solve_node(X, y, on.Node(c["p"], c["k"], J0, J1), c["lam2"], c["M"], c["kind"], L, 20)
        assert abs(res["lb"][b] - ref["lb"]) <= 1e-9 * max(1.0, abs(ref["lb"])), (b, res["lb"][b], ref["lb"])
    for kind in (synth.LOGISTIC, synth.LSQ):
        c, X, y, _ = synth.config_instance("c2_logistic_n2000_p200_k10", seed=0, kind=kind)
        L = on.lipschitz(X, c["kind"])
        csr = synth.random_nodes(64, c["p"], c["k"], np.random.default_rng(1))
        sets = synth.csr_to_sets(*csr)
        with kglm.Engine(X, y, c["k"], c["lam2"], c["M"], c["kind"], prec="bf16", max_batch=64, lipschitz=L) as eng:
            eng.push(*csr)
            res = eng.evaluate(20)
            _, Z = eng.read_batch(beta=False)
        for b in range(0, 64, 8):
            psi = on.dual_value(X, y, Z[b], on.Node(c["p"], c["k"], *sets[b]), c["lam2"], c["M"], c["kind"])
            assert res["lb"][b] <= psi + 1e-12 * max(1.0, abs(psi)), (kind, b)
            assert psi - res["lb"][b] <= 1e-6 * max(1.0, abs(psi)), (kind, b)
    print("checked build ok")
""") % ROOT


def test_checked_build_catches_its_self_test_and_passes_validated_batches():
    build.build(checks=True)
    env = dict(os.environ, KGLM_CHECKS="1")
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout


def test_normal_build_self_test_is_refused():
    if os.environ.get("KGLM_CHECKS") == "1":
        pytest.skip("the bounds-checked library is selected")
    c, X, y, _ = synth.config_instance("c1_lsq_n200_p30_k5", seed=0)
    with kglm.Engine(X, y, c["k"], c["lam2"], c["M"], c["kind"], prec="fp64", max_batch=4) as eng:
        assert kglm.kglm_selftest_checks(eng.ctx) == kglm.KGLM_ESTATE
        eng.push(*synth.sets_to_csr([([], []), ([1], [2])]))
        res = eng.evaluate(10)
        assert np.all(np.isfinite(res["lb"]))
