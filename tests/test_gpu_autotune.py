"""The autotuner (kglm_autotune): tile shapes of the tensor-core products and the batch size.

Its choices are valid (tiles from the candidate sets, a power-of-two batch
within max_batch at >= 95% of the best rate it measured), and retiling changes
no result beyond rounding: after tuning, the batch still matches the oracle's
certificate at the GPU's own dual points and its rounding/branching decisions,
and kglm_solve with the tuned batch (batch 0) still certifies the brute-force
optimum.
"""

import numpy as np
import pytest

from oracle import node as on
from oracle import reopt as ro
from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["bf16", "tf32x3", "fp32"])
def test_autotune_choices_are_valid_and_results_unchanged(prec):
    n, p, k, m = 1500, 300, 8, 512
    X, y, _ = synth.instance(n, p, k, synth.LOGISTIC, rho=0.5, seed=31)
    lam2, M, T = 1e-2, 2.0, 30
    L = on.lipschitz(X, synth.LOGISTIC)
    rng = np.random.default_rng(4)
    nodes = synth.csr_to_sets(*synth.random_nodes(64, p, k, rng))
    with kglm.Engine(X, y, k, lam2, M, synth.LOGISTIC, prec=prec, max_batch=m, lipschitz=L) as eng:
        t = eng.autotune(iters=10, seed=3)
        eng.push(*synth.sets_to_csr(nodes))
        res = eng.evaluate(T)
        B, Z = eng.read_batch()
    assert 1 <= t["batch"] <= m and (t["batch"] & (t["batch"] - 1) == 0 or t["batch"] == m)
    assert t["nodes_per_s"] >= 0.95 * t["best_nodes_per_s"] > 0
    if prec in ("bf16", "tf32x3"):
        # tile widths are multiples of 16 up to 256 columns (link from 32, gradient from 64)
        assert t["link_tile_cols"] % 16 == 0 and 32 <= t["link_tile_cols"] <= 256
        assert t["grad_tile_cols"] % 16 == 0 and 64 <= t["grad_tile_cols"] <= 256
        assert t["grad_split_cap"] in (1, 2, 4, 8, 16)
    else:
        assert t["link_tile_cols"] == t["grad_tile_cols"] == t["grad_split_cap"] == 0
    for b, (J0, J1) in enumerate(nodes):
        nd = on.Node(p, k, J0, J1)
        psi = on.dual_value(X, y, Z[b], nd, lam2, M, synth.LOGISTIC)
        assert res["lb"][b] <= psi + 1e-12 * max(1.0, abs(psi))
        assert psi - res["lb"][b] <= 1e-6 * max(1.0, abs(psi))
        assert [int(s) for s in res["support"][b] if s >= 0] == on.round_support(B[b], nd)
        assert res["branch_j"][b] == on.branch_index(B[b], nd)


def test_solve_with_the_tuned_batch_matches_brute_force():
    X, y, _ = synth.instance(120, 16, 4, synth.LSQ, rho=0.8, snr=2.0, seed=13)
    with kglm.Engine(X, y, 4, 1e-3, 2.0, synth.LSQ, prec="bf16", max_batch=256) as eng:
        res = eng.solve(0, 300, 20)
    top = ro.brute_force(X, y, 4, 1e-3, 2.0, synth.LSQ, top=2)
    assert res["gap"] <= 1e-6
    assert abs(res["opt"] - top[0][0]) <= 1e-6 * max(1.0, abs(top[0][0]))
    if top[1][0] - top[0][0] > 1e-6 * abs(top[0][0]):
        assert tuple(res["support"]) == tuple(top[0][1])


@pytest.mark.parametrize("prec", ["bf16", "tf32x3"])
def test_sub_batches_give_the_same_results(prec):
    """Iterating node ranges side by side on forked streams changes no result
    beyond summation order.  With one split-K slice of X^T R the BF16 run has
    the same summation order in every product, so bounds, iterates, supports
    and branching indices are identical for 1, 2 and 4 sub-batches (ragged last
    range included).  In the TF32 split at this shape the whole-batch link
    product takes split-K (few tiles) while sub-batches do not, so its FP32
    sums are ordered differently: bounds agree to 1e-6 and iterates to 1e-5."""
    n, p, k, m = 900, 150, 6, 600
    X, y, _ = synth.instance(n, p, k, synth.LOGISTIC, rho=0.5, seed=41)
    rng = np.random.default_rng(6)
    csr = synth.random_nodes(m, p, k, rng)
    out = []
    with kglm.Engine(X, y, k, 1e-2, 2.0, synth.LOGISTIC, prec=prec, max_batch=m) as eng:
        for ns in (1, 2, 4):
            eng.configure(grad_split_cap=1, sub_batches=ns)
            eng.push(*csr)
            res = eng.evaluate(25)
            B, _ = eng.read_batch(zeta=False)
            out.append((res, B))
    r0, B0 = out[0]
    for res, B in out[1:]:
        if prec == "bf16":
            assert np.array_equal(B, B0)
            for key in ("lb", "ub", "support", "branch_j"):
                assert np.array_equal(res[key], r0[key]), key
        else:
            assert np.max(np.abs(B - B0)) <= 1e-5 * max(1.0, np.max(np.abs(B0)))
            for key in ("lb", "ub"):
                assert np.all(np.abs(res[key] - r0[key]) <= 1e-6 * np.maximum(1.0, np.abs(r0[key]))), key


@pytest.mark.parametrize("p,opts", [(1000, (0, 64, 32)), (2000, (0, 128, 64, 32))])
def test_prox_thread_options_agree(p, opts):
    """The prox kernels with fewer threads per node (more coordinates each) compute
    the same step: the certificate at the GPU's own dual point and the
    rounding/branching decisions match the oracle for every option, and with the
    FP32-accurate products (no BF16 rounding to amplify the FP32 reduction-order
    differences of the kernels) the bounds agree across options to 1e-3."""
    n, k, m = 700, 8, 40
    X, y, _ = synth.instance(n, p, k, synth.LSQ, rho=0.5, snr=5.0, seed=p)
    lam2, M = 1e-2, 2.0
    rng = np.random.default_rng(p + 1)
    nodes = synth.csr_to_sets(*synth.random_nodes(m, p, k, rng))
    nodes[0] = ([], [])
    lbs = []
    with kglm.Engine(X, y, k, lam2, M, synth.LSQ, prec="tf32x3", max_batch=m) as eng:
        for t in opts:
            eng.configure(prox_threads=t) if t else eng.configure()
            eng.push(*synth.sets_to_csr(nodes))
            res = eng.evaluate(20)
            B, Z = eng.read_batch()
            for b, (J0, J1) in enumerate(nodes):
                nd = on.Node(p, k, J0, J1)
                psi = on.dual_value(X, y, Z[b], nd, lam2, M, synth.LSQ)
                assert res["lb"][b] <= psi + 1e-12 * max(1.0, abs(psi))
                assert psi - res["lb"][b] <= 1e-6 * max(1.0, abs(psi))
                assert [int(s) for s in res["support"][b] if s >= 0] == on.round_support(B[b], nd)
                assert res["branch_j"][b] == on.branch_index(B[b], nd)
            lbs.append(res["lb"])
    for lb in lbs[1:]:
        assert np.all(np.abs(lb - lbs[0]) <= 1e-3 * np.maximum(1.0, np.abs(lbs[0])))
