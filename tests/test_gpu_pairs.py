"""GPU: the BF16 products as CTA pairs (clusters of two computing 256-row tiles
with one cta_group::2 product, each CTA holding its 128 rows of A and half of
the B tile) give bit-for-bit the results of one CTA per 128-row tile.

A pair only changes where the operand slices sit (each CTA's rows of A and half
of the B columns in its own shared memory) and which SM issues the products;
every accumulator row still sees the same K slices in the same order, so
bounds, iterates, supports and branching indices must be identical, including
an odd number of row tiles (the last pair's second CTA has no rows to store),
sub-batches (row offsets into the operand), split-K slices of G = X^T R, tile
widths whose half is not a multiple of 16 columns, and both losses.  The bound
is also checked as a certificate against the oracle at the GPU's own dual point.
"""

import numpy as np
import pytest

from oracle import node as on
from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", [synth.LSQ, synth.LOGISTIC])
@pytest.mark.parametrize("m,sub,cap,bn", [(640, 1, 1, (256, 224)), (1152, 2, 4, (256, 224)), (300, 1, 2, (256, 224)),
                                          (520, 1, 1, (112, 48))])
def test_pairs_match_single_ctas_bit_for_bit(kind, m, sub, cap, bn):
    n, p, k = 3000, 700, 10
    X, y, _ = synth.instance(n, p, k, kind, rho=0.5, snr=5.0, seed=61)
    lam2, M, T = 1e-2, 2.0, 20
    csr = synth.random_nodes(m, p, k, np.random.default_rng(62))
    out = {}
    with kglm.Engine(X, y, k, lam2, M, kind, prec="bf16", max_batch=m) as eng:
        for pair in (-1, 1):
            eng.configure(link_tile_cols=bn[0], grad_tile_cols=bn[1], grad_split_cap=cap, sub_batches=sub, pair=pair)
            eng.push(*csr)
            res = eng.evaluate(T)
            B, Z = eng.read_batch()
            out[pair] = (res, B, Z)
    (r0, B0, Z0), (r1, B1, Z1) = out[-1], out[1]
    for key in ("lb", "primal", "ub", "support", "branch_j"):
        assert np.array_equal(r0[key], r1[key]), key
    assert np.array_equal(B0, B1) and np.array_equal(Z0, Z1)
    L = None
    sets = synth.csr_to_sets(*csr)
    for b in (0, m // 2, m - 1):
        nd = on.Node(p, k, *sets[b])
        psi = on.dual_value(X, y, Z1[b], nd, lam2, M, kind)
        assert r1["lb"][b] <= psi + 1e-12 * max(1.0, abs(psi))
        assert psi - r1["lb"][b] <= 1e-6 * max(1.0, abs(psi))
