"""Failure detection without a GPU fault: a device wait that runs out.

Every wait in the engine's kernels is bounded; when one runs out the kernel
sets an error flag and returns, the launching call reports KGLM_ETIMEOUT, and
the context stays usable.  kglm_selftest_timeout launches a kernel whose wait
is on an mbarrier that nothing arrives on (a flag nothing sets); the test
checks the status and then evaluates a batch on the same context, checked
against the oracle.
"""

import numpy as np
import pytest

from oracle import node as on
from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["bf16", "fp64"])
def test_wait_that_runs_out_reports_and_the_context_survives(prec):
    c, X, y, _ = synth.config_instance("c1_lsq_n200_p30_k5", seed=4)
    L = on.lipschitz(X, c["kind"])
    nodes = [([], []), ([3, 4], [0])]
    with kglm.Engine(X, y, c["k"], c["lam2"], c["M"], c["kind"], prec=prec, max_batch=4, lipschitz=L) as eng:
        for _ in range(2):
            assert kglm.kglm_selftest_timeout(eng.ctx, 20000) == kglm.KGLM_ETIMEOUT
        eng.push(*synth.sets_to_csr(nodes))
        res = eng.evaluate(30)
        _, Z = eng.read_batch()
    for b, (J0, J1) in enumerate(nodes):
        nd = on.Node(c["p"], c["k"], J0, J1)
        psi = on.dual_value(X, y, Z[b], nd, c["lam2"], c["M"], c["kind"])
        assert res["lb"][b] <= psi + 1e-12 * max(1.0, abs(psi))
        assert psi - res["lb"][b] <= 1e-6 * max(1.0, abs(psi))
