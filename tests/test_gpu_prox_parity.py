"""Element-wise parity of the FP32 proximal step against the oracle's Algorithm 1.

The FP32 prox kernel (the one every reduced-precision mode runs) selects the
kbar largest free magnitudes with code that the FP64 path never executes: a
warp per node by candidates above the kbar-th largest lane maximum (or the
kbar-round tournament when kbar > 32 or too many candidates qualify), and a
CTA per node by radix select.  These tests compare its output beta element by
element with the oracle's prox_node (Algorithm 1, App. B, in FP64), across
feature counts that reach each path: p = 64 and 512 (a warp per node), 600,
1000, 1001 and 2000 (the persistent kernel that streams nodes through shared
memory by default, with 16-byte copies when p is a multiple of 4 and 4-byte
ones at 1001; every prox_threads option selects one of the CTA-per-node or
warp-per-node kernels instead), 4093 and 8189 (a CTA per node: too few rows
of the persistent kernel fit in shared memory).

First step (exact products).  With X on a coarse dyadic grid (entries k/4,
|k| <= 2), a warm start beta0 on the grid 2^-6 inside the box, y on the grid
2^-6, and L a power of two, every product and sum of S = X beta0,
R = 2 (S - y) and G = X^T R is exact in FP32 (all partial sums are multiples
of 2^-9 below 2^15), also in the TF32 hi + lo split (every operand fits in its
two 11-bit parts), and eta G is exact.  So the GPU's
u = beta0 - eta G equals the FP64 u up to one rounding, and one FISTA step
from beta0 (which takes no momentum) returns prox(u) computed by the FP32
kernel.  Tolerance 2^-18 max(1, |u|_inf): the prox is 1-Lipschitz, the
rounding of u costs 2^-24 |u|, and the block threshold is a ratio of sums of
positive terms (a lane's sequential sum of at most 32 terms and a tree of at
most 9 levels), each carrying a relative error below 64 * 2^-24.

Later steps (inexact products).  Steps 2 and 3 start from the GPU's own
iterates; their u is formed in FP64 from those iterates (v_2 = beta_1, v_3 =
beta_2 + ((t_2 - 1)/t_3)(beta_2 - beta_1) unless the restart test fires) and
the tolerance adds twice the rigorous FP32 product bound
  |du_j| <= eta (gamma_n sum_i |X_ij| |r_i| + sum_i |X_ij| 2 gamma_p (|X| |v|)_i),
gamma_q = q 2^-24 / (1 - q 2^-24), in the max norm: beta_j moves by at most
|du_j| plus the move of the block threshold, and the threshold (the root of
f(x) = sum_tail (|u_j| - x)^+ - sum_top (h(x) - |u_j|)^+, whose slope in x is at
least the count of its active terms and in each |u_j| at most 1) moves by at
most max_j |du_j|.
"""

import numpy as np
import pytest

from oracle import node as on
from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
N_ROWS = 64
M_BOX = 2.0


def _gamma(q):
    return q * EPS32 / (1.0 - q * EPS32)


def _instance(p, seed, dup):
    """Coarse dyadic X (n x p) and y, L a power of two, lambda2 with c = 2 lambda2 / L = 2^-5."""
    rng = np.random.default_rng(seed)
    q = p // 2 if dup else p
    X = rng.integers(-2, 3, size=(N_ROWS, q)).astype(np.float64) / 4.0
    if dup:                                       # x_{2i} = x_{2i+1}: exact ties in every step
        X = np.repeat(X, 2, axis=1)
        if X.shape[1] < p:
            X = np.hstack([X, rng.integers(-2, 3, size=(N_ROWS, p - X.shape[1])) / 4.0])
    X = np.ascontiguousarray(X)
    y = rng.integers(-128, 129, size=N_ROWS).astype(np.float64) / 64.0
    L_true = 2.0 * np.linalg.norm(X, 2) ** 2
    L = 2.0 ** np.ceil(np.log2(L_true))
    lam2 = L * 2.0 ** -6
    return X, y, L, lam2


def _warm(p, nodes, rng, dup):
    """Warm starts on the grid 2^-6 inside |b| <= 2; at most 256 nonzeros per node, so
    that |X| |beta0| and |X^T| |r| stay below 2^15 (the exactness condition)."""
    B = rng.integers(-128, 129, size=(len(nodes), p)).astype(np.float64) / 64.0
    if p > 256:
        B[rng.random(B.shape) > 256.0 / p] = 0.0
    if dup:
        h = 2 * (p // 2)
        B[:, 1:h:2] = B[:, 0:h:2]
    for b, (J0, _) in enumerate(nodes):
        B[b, list(J0)] = 0.0
    return B


def _assert_exact_products(X, y, v):
    """Every partial sum of X v and X^T (2 (X v - y)) is a multiple of 2^-9 below 2^15."""
    ax = np.abs(X)
    assert np.max(ax @ np.abs(v)) < 2.0 ** 15
    r = 2.0 * (X @ v - y)
    assert np.max(ax.T @ np.abs(r)) < 2.0 ** 15


def _nodes(p, k, rng):
    """Special nodes (kbar = k, kbar = 1, kbar = 0, pf <= kbar, pf = 0, a J1-heavy node) and random ones."""
    perm = rng.permutation(p)
    nodes = [([], []),                                            # root, kbar = k
             ([], sorted(perm[:k - 1].tolist())),                 # kbar = 1
             ([], sorted(perm[:k].tolist())),                     # kbar = 0
             (sorted(perm[:p - k + 2].tolist()), []),             # pf = k - 2 < kbar
             (sorted(perm[2:].tolist()), sorted(perm[:2].tolist())),   # pf = 0
             (sorted(perm[k:k + p // 2].tolist()), sorted(perm[:k // 2].tolist()))]
    nodes += synth.csr_to_sets(*synth.random_nodes(10, p, k, rng))
    return nodes


def _u(X, y, L, v):
    return v - (X.T @ (2.0 * (X @ v - y))) / L


def _u_err(X, y, L, v, unit):
    """Rigorous bound on |u_gpu - u| for the GPU's products of X v and X^T r (least
    squares).  unit: the relative error of one product term, 2^-24 for FP32; the
    TF32 hi + lo split drops lo*lo and rounds each operand to hi + lo (22 bits):
    2^-21 covers both."""
    n, p = X.shape
    ax = np.abs(X)
    gam = lambda q: q * unit / (1.0 - q * unit)
    ds = gam(p + 1) * (ax @ np.abs(v))
    r = 2.0 * (X @ v - y)
    dr = 2.0 * ds + 4.0 * EPS32 * (np.abs(r) + 2.0 * ds)
    dg = gam(n + 1) * (ax.T @ (np.abs(r) + dr)) + ax.T @ dr
    return dg / L + 2.0 * EPS32 * (np.abs(v) + np.abs(X.T @ r) / L)


def _options(p):
    """prox_threads values accepted at this p (0: the default kernel)."""
    if p <= 512:
        return [0]
    if p <= 1024:
        return [0, 64, 32]
    if p <= 2048:
        return [0, 128, 64, 32]
    if p <= 4096:
        return [0, 256, 128]
    return [0, 256]


CASES = [(64, 12, False), (64, 40, True), (512, 20, False), (512, 40, False), (600, 10, False),
         (1000, 15, True), (1001, 30, False), (2000, 20, False), (2000, 40, False), (4093, 30, False),
         (8189, 20, False)]


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
@pytest.mark.parametrize("p,k,dup", CASES)
def test_first_step_prox_matches_algorithm1(p, k, dup, prec):
    X, y, L, lam2 = _instance(p, seed=p + k, dup=dup)
    rng = np.random.default_rng(3 * p + k)
    nodes = _nodes(p, k, rng)
    B0 = _warm(p, nodes, rng, dup)
    rho = 1.0 / (2.0 * lam2 / L)
    csr = synth.sets_to_csr(nodes)
    with kglm.Engine(X, y, k, lam2, M_BOX, synth.LSQ, prec=prec, max_batch=len(nodes), lipschitz=L) as eng:
        for opt in _options(p):
            if opt:
                eng.configure(prox_threads=opt)
            eng.push(*csr, warm_B=B0)
            eng.evaluate(1)
            B1, _ = eng.read_batch(zeta=False)
            for b, (J0, J1) in enumerate(nodes):
                nd = on.Node(p, k, J0, J1)
                _assert_exact_products(X, y, B0[b])
                u = _u(X, y, L, B0[b])
                want = on.prox_node(u, nd, rho, M_BOX)
                tol = 2.0 ** -18 * max(1.0, np.max(np.abs(u)))
                err = np.max(np.abs(B1[b] - want))
                assert err <= tol, (p, k, prec, opt, b, err, tol)
                if J0:
                    assert np.all(B1[b, J0] == 0.0)
                if dup and b == 0:              # the root keeps tied pairs equal
                    assert np.array_equal(B1[b, 0:2 * (p // 2):2], B1[b, 1:2 * (p // 2):2])


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
@pytest.mark.parametrize("p,k", [(512, 20), (2000, 20), (8189, 20)])
def test_second_and_third_steps_with_momentum(p, k, prec):
    X, y, L, lam2 = _instance(p, seed=7 * p + k, dup=False)
    rng = np.random.default_rng(11 * p + k)
    nodes = _nodes(p, k, rng)
    B0 = _warm(p, nodes, rng, False)
    rho = 1.0 / (2.0 * lam2 / L)
    csr = synth.sets_to_csr(nodes)
    iters = []
    with kglm.Engine(X, y, k, lam2, M_BOX, synth.LSQ, prec=prec, max_batch=len(nodes), lipschitz=L) as eng:
        for T in (1, 2, 3):
            eng.push(*csr, warm_B=B0)
            eng.evaluate(T)
            iters.append(eng.read_batch(zeta=False)[0])
    unit = EPS32 if prec == "fp32" else 2.0 ** -21
    t2 = 0.5 * (1.0 + np.sqrt(5.0))
    t3 = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t2 * t2))
    checked = 0
    for b, (J0, J1) in enumerate(nodes):
        nd = on.Node(p, k, J0, J1)
        b1, b2, b3 = iters[0][b], iters[1][b], iters[2][b]
        # step 2: v_2 = beta_1 (the first extrapolation takes no momentum)
        u = _u(X, y, L, b1)
        du = 2.0 * np.max(_u_err(X, y, L, b1, unit))
        tol = du + 2.0 ** -18 * max(1.0, np.max(np.abs(u)))
        assert np.max(np.abs(b2 - on.prox_node(u, nd, rho, M_BOX))) <= tol, (b, 2)
        # step 3: restart test <v_2 - beta_2, beta_2 - beta_1> > 0, taken on the GPU in FP32
        dot = float(np.dot(b1 - b2, b2 - b1))          # v_2 = beta_1: never positive
        assert dot <= 0.0
        v3 = b2 + ((t2 - 1.0) / t3) * (b2 - b1)
        u = _u(X, y, L, v3)
        du = 2.0 * np.max(_u_err(X, y, L, v3, unit) + 4.0 * EPS32 * np.abs(v3))
        tol = du + 2.0 ** -18 * max(1.0, np.max(np.abs(u)))
        assert np.max(np.abs(b3 - on.prox_node(u, nd, rho, M_BOX))) <= tol, (b, 3)
        checked += 1
    assert checked == len(nodes)


@pytest.mark.parametrize("p", [600, 2000])
def test_streaming_prox_with_several_nodes_per_warp(p):
    """6000 nodes: every warp of the streaming kernel takes several nodes in turn, its
    shared-memory rows reused from node to node; a sample of nodes spread over the
    batch, including the last, against Algorithm 1 on the same u."""
    k = 20
    X, y, L, lam2 = _instance(p, seed=5 * p, dup=False)
    rng = np.random.default_rng(13 * p)
    nodes = _nodes(p, k, rng) + synth.csr_to_sets(*synth.random_nodes(6000 - 16, p, k, rng))
    B0 = _warm(p, nodes, rng, False)
    rho = 1.0 / (2.0 * lam2 / L)
    with kglm.Engine(X, y, k, lam2, M_BOX, synth.LSQ, prec="fp32", max_batch=len(nodes), lipschitz=L) as eng:
        eng.push(*synth.sets_to_csr(nodes), warm_B=B0)
        eng.evaluate(1)
        B1, _ = eng.read_batch(zeta=False)
    for b in list(range(0, len(nodes), 97)) + [len(nodes) - 1]:
        J0, J1 = nodes[b]
        nd = on.Node(p, k, J0, J1)
        u = _u(X, y, L, B0[b])
        want = on.prox_node(u, nd, rho, M_BOX)
        tol = 2.0 ** -18 * max(1.0, np.max(np.abs(u)))
        err = np.max(np.abs(B1[b] - want))
        assert err <= tol, (p, b, err, tol)
