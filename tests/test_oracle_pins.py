"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here uses something other than the oracle's own formula: finite
differences, scipy optimisers / LP / BVLS, LAPACK solves, brute force over
supports, weak and strong duality, and the worked example of Fig. 2.
"""

import os

import numpy as np
import pytest
from scipy.optimize import linprog, minimize, minimize_scalar

from oracle import losses as ol
from oracle import node as on
from oracle import reopt as ro
from oracle import bnb as ob
from paper_2605_22188_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))
KINDS = [ol.LSQ, ol.LOGISTIC]


def _y(kind, rng, n):
    return rng.standard_normal(n) if kind == ol.LSQ else rng.choice([-1.0, 1.0], n)


# ---------------------------------------------------------------- P1 losses

@pytest.mark.parametrize("kind", KINDS)
def test_dloss_finite_difference(kind):
    rng = np.random.default_rng(1)
    s = rng.standard_normal(50) * 3
    y = _y(kind, rng, 50)
    h = 1e-6
    fd = (ol.loss(s + h, y, kind) - ol.loss(s - h, y, kind)) / (2 * h)
    assert np.allclose(ol.dloss(s, y, kind), fd, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("kind", KINDS)
def test_conjugate_fenchel_young_and_sup(kind):
    """l(s) + l*(l'(s)) = s l'(s) (equality case of Fenchel-Young), and l* = sup by scipy."""
    rng = np.random.default_rng(2)
    s = rng.standard_normal(40) * 2
    y = _y(kind, rng, 40)
    d = ol.dloss(s, y, kind)
    assert np.allclose(ol.loss(s, y, kind) + ol.loss_conj(d, y, kind), s * d, atol=1e-12)
    for i in range(8):
        w = d[i] * 0.7
        r = minimize_scalar(lambda t: -(w * t - float(ol.loss(t, y[i], kind))),
                            bounds=(-60, 60), method="bounded", options=dict(xatol=1e-12))
        assert abs(-r.fun - float(ol.loss_conj(w, y[i], kind))) < 1e-9


def test_logistic_conjugate_domain():
    assert np.isinf(ol.loss_conj(np.array([0.5]), np.array([1.0]), ol.LOGISTIC))[0]
    assert np.isinf(ol.loss_conj(np.array([-1.5]), np.array([1.0]), ol.LOGISTIC))[0]
    assert float(ol.loss_conj(np.array([0.0]), np.array([1.0]), ol.LOGISTIC)[0]) == 0.0


def test_huber_is_box_conjugate_and_prox():
    """H_M(q) = sup_{|b|<=M} qb - b^2/2; prox_{rH_M} = argmin 1/2(v-x)^2 + r H_M(v)."""
    M = 2.0
    for q in [-7.0, -2.5, -1.0, 0.0, 0.3, 1.99, 2.0, 4.2]:
        f = lambda b: q * b - 0.5 * b * b
        r = minimize_scalar(lambda b: -f(b), bounds=(-M, M), method="bounded", options=dict(xatol=1e-12))
        sup = max(f(r.x), f(-M), f(M))           # the bounded search never lands exactly on an end
        assert abs(sup - float(ol.huber(q, M))) < 1e-9
    for x in [-20.0, -3.0, 0.5, 2.9, 3.1, 30.0]:
        for rr in [0.0, 0.5, 3.0]:
            r = minimize_scalar(lambda v: 0.5 * (v - x) ** 2 + rr * float(ol.huber(v, M)),
                                bounds=(-50, 50), method="bounded", options=dict(xatol=1e-12))
            assert abs(r.x - float(ol.prox_huber(x, rr, M))) < 1e-6


# ---------------------------------------------------------------- Algorithm 1

def _isotonic_slsqp(a_sorted, rho_j, M):
    """min sum 1/2 (v_j - a_j)^2 + rho_j H_M(v_j) s.t. v_1 >= ... >= v_p >= 0, by SLSQP."""
    pf = a_sorted.size
    cons = [dict(type="ineq", fun=lambda v, j=j: v[j] - v[j + 1]) for j in range(pf - 1)]
    cons.append(dict(type="ineq", fun=lambda v: v[-1]))
    f = lambda v: float(np.sum(0.5 * (v - a_sorted) ** 2 + rho_j * ol.huber(v, M)))
    best = None
    for x0 in (a_sorted, np.full(pf, a_sorted.mean()), np.sort(a_sorted / 3)[::-1]):
        r = minimize(f, x0, constraints=cons, method="SLSQP", options=dict(ftol=1e-15, maxiter=2000))
        if best is None or r.fun < best.fun:
            best = r
    return best.x


@pytest.mark.parametrize("seed", range(12))
def test_alg1_matches_generic_isotonic_solver(seed):
    """Algorithm 1 equals a generic constrained solve of the isotonic problem of App. B."""
    rng = np.random.default_rng(100 + seed)
    pf = int(rng.integers(2, 8))
    kbar = int(rng.integers(0, pf + 1))
    M = 2.0
    rho = float(rng.choice([0.3, 1.0, 4.0]))
    w = rng.standard_normal(pf) * rng.choice([0.5, 2.0, 6.0])
    out = on.alg1_prox_gconj(w, rho, kbar, M)
    a = np.abs(w)
    pi = np.argsort(-a, kind="stable")
    v = _isotonic_slsqp(a[pi], np.where(np.arange(pf) < kbar, rho, 0.0), M)
    ref = np.empty(pf)
    ref[pi] = v
    assert np.allclose(np.abs(out), ref, atol=2e-6), (out, ref)
    assert np.all(np.sign(out)[np.abs(out) > 0] == np.sign(w)[np.abs(out) > 0])


# ---------------------------------------------------------------- g and g*

def _g_by_slsqp(beta, node, M):
    """g_N(beta) by minimising over z with SLSQP (definition of g_N, §3)."""
    Jf = np.array(node.Jf, dtype=int)
    g1 = 0.5 * float(np.sum(beta[np.array(node.J1, dtype=int)] ** 2)) if node.J1 else 0.0
    b = np.abs(beta[Jf])
    nz = b > 0
    if not np.any(nz):
        return g1
    bb = b[nz]
    lo = bb / M
    cons = [dict(type="ineq", fun=lambda z: node.kbar - np.sum(z))]
    f = lambda z: 0.5 * float(np.sum(bb ** 2 / z))
    z0 = np.clip(np.full(bb.size, node.kbar / bb.size), lo, 1.0)
    r = minimize(f, z0, bounds=list(zip(lo, np.ones(bb.size))), constraints=cons, method="SLSQP",
                 options=dict(ftol=1e-15, maxiter=2000))
    return g1 + r.fun


@pytest.mark.parametrize("seed", range(10))
def test_g_theorem41_matches_direct_minimisation(seed):
    rng = np.random.default_rng(200 + seed)
    p, k, M = 8, 4, 2.0
    perm = rng.permutation(p)
    J1 = list(perm[:int(rng.integers(0, 3))])
    J0 = list(perm[len(J1):len(J1) + int(rng.integers(0, 3))])
    nd = on.Node(p, k, J0, J1)
    beta = rng.standard_normal(p) * 0.6
    beta[J0] = 0.0
    beta[rng.random(p) < 0.2] = 0.0
    # scale the free part inside the budget so that g is finite
    Jf = np.array(nd.Jf)
    s = np.sum(np.abs(beta[Jf])) / M
    if s > nd.kbar:
        beta[Jf] *= 0.95 * nd.kbar / s
    beta = np.clip(beta, -M, M)
    g = on.g_node(beta, nd, M)
    assert np.isfinite(g)
    assert abs(g - _g_by_slsqp(beta, nd, M)) < 1e-6 * max(1.0, g)
    z = on.z_recover(beta, nd, M)
    assert np.all(z[nd.J1] == 1.0) and np.all(z[nd.J0] == 0.0)
    assert np.sum(z[Jf]) <= nd.kbar + 1e-12
    assert np.all(z[Jf] >= np.abs(beta[Jf]) / M - 1e-12) and np.all(z <= 1.0 + 1e-12)


def test_g_domain():
    nd = on.Node(5, 2, [0], [1])
    assert np.isinf(on.g_node(np.array([0.1, 0, 0, 0, 0]), nd, 2.0))       # beta_J0 != 0
    assert np.isinf(on.g_node(np.array([0, 2.5, 0, 0, 0]), nd, 2.0))       # box
    assert np.isinf(on.g_node(np.array([0, 1.0, 1.5, 1.0, 0]), nd, 2.0))   # budget: 2.5/2 > kbar=1
    assert on.g_node(np.array([0, 1.0, 1.5, 0, 0]), nd, 2.0) == pytest.approx(0.5 * (1 + 2.25))


@pytest.mark.parametrize("seed", range(8))
def test_gconj_topsum_matches_lp(seed):
    """g*(q) = max over the node polytope of sum z_j H_M(q_j): an LP (scipy HiGHS)."""
    rng = np.random.default_rng(300 + seed)
    p, k, M = 9, 4, 2.0
    perm = rng.permutation(p)
    J1 = list(perm[:int(rng.integers(0, 3))])
    J0 = list(perm[len(J1):len(J1) + int(rng.integers(0, 3))])
    nd = on.Node(p, k, J0, J1)
    q = rng.standard_normal(p) * 2.5
    h = ol.huber(q, M)
    bounds = [(0, 0) if j in J0 else (1, 1) if j in J1 else (0, 1) for j in range(p)]
    A = np.array([[1.0 if j in nd.Jf else 0.0 for j in range(p)]])
    r = linprog(-h, A_ub=A, b_ub=[nd.kbar], bounds=bounds, method="highs")
    assert abs(-r.fun - on.g_conj_node(q, nd, M)) < 1e-9


# ---------------------------------------------------------------- the prox step

def _node_problem(seed, p=10, k=4):
    rng = np.random.default_rng(seed)
    perm = rng.permutation(p)
    J1 = list(perm[:int(rng.integers(0, 3))])
    J0 = list(perm[len(J1):len(J1) + int(rng.integers(0, 4))])
    return rng, on.Node(p, k, J0, J1)


@pytest.mark.parametrize("seed", range(10))
def test_prox_is_the_minimiser(seed):
    """beta = prox_{c g}(u) minimises 1/2||beta - u||^2 + c g(beta), c = 1/rho (g by Theorem 4.1)."""
    rng, nd = _node_problem(400 + seed)
    M = 2.0
    rho = float(rng.choice([0.5, 2.0, 10.0]))
    c = 1.0 / rho
    u = rng.standard_normal(nd.p) * float(rng.choice([0.3, 1.0, 3.0]))
    beta = on.prox_node(u, nd, rho, M)
    obj = lambda b: 0.5 * float(np.sum((b - u) ** 2)) + c * on.g_node(b, nd, M)
    f0 = obj(beta)
    assert np.isfinite(f0)
    mask = np.ones(nd.p, bool)
    mask[nd.J0] = False
    for _ in range(400):
        d = rng.standard_normal(nd.p) * float(rng.choice([1e-3, 1e-2, 1e-1]))
        d[~mask] = 0.0
        f1 = obj(beta + d)
        assert f1 >= f0 - 1e-12 * max(1.0, abs(f0))


def test_prox_special_cases():
    """kbar >= pf: ridge-and-clip on every free coordinate; kbar = 0: free coordinates are 0."""
    M, rho = 2.0, 3.0
    u = np.array([0.5, -4.0, 1.0, 2.5, -0.2, 7.0])
    nd = on.Node(6, 5, J0=[0], J1=[])          # pf = 5 <= kbar = 5
    beta = on.prox_node(u, nd, rho, M)
    ref = np.clip(u / (1.0 + 1.0 / rho), -M, M)
    ref[0] = 0.0
    assert np.allclose(beta, ref, atol=1e-14)
    nd0 = on.Node(6, 2, J0=[3], J1=[1, 4])       # kbar = 0
    beta0 = on.prox_node(u, nd0, rho, M)
    assert np.all(beta0[[0, 2, 3, 5]] == 0.0)
    assert np.allclose(beta0[[1, 4]], np.clip(u[[1, 4]] / (1.0 + 1.0 / rho), -M, M))


# ---------------------------------------------------------------- node bounds

def _tiny(kind, seed=7, n=60, p=10, k=3, rho=0.5):
    X, y, _ = synth.instance(n, p, k, kind, rho=rho, snr=3.0, seed=seed)
    return X, y


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("sets", [((), ()), ((0, 5), (2,)), ((1,), (3, 7)), ((), (0, 1, 2)), ((4, 6, 8), ())])
def test_strong_duality_at_convergence(kind, sets):
    """Converged primal (g by Theorem 4.1) equals the dual (TopSum certificate)."""
    X, y = _tiny(kind)
    nd = on.Node(10, 3, *sets)
    lam2, M = 0.05, 2.0
    L = on.lipschitz(X, kind)
    r = on.solve_node(X, y, nd, lam2, M, kind, L, T=4000)
    assert r["lb"] <= r["primal"] + 1e-12 * abs(r["primal"])
    assert r["primal"] - r["lb"] <= 1e-10 * max(1.0, abs(r["primal"]))


@pytest.mark.parametrize("kind", KINDS)
def test_weak_duality_against_brute_force(kind):
    """LB(N) <= min over supports consistent with N of v(S), for every node (reading 17)."""
    X, y = _tiny(kind, seed=11, n=50, p=9, k=3)
    lam2, M = 0.02, 2.0
    L = on.lipschitz(X, kind)
    rng = np.random.default_rng(5)
    for _ in range(6):
        perm = rng.permutation(9)
        J1 = list(perm[:int(rng.integers(0, 3))])
        J0 = list(perm[len(J1):len(J1) + int(rng.integers(0, 4))])
        nd = on.Node(9, 3, J0, J1)
        for T in (5, 50, 2000):
            lb = on.solve_node(X, y, nd, lam2, M, kind, L, T=T)["lb"]
            best = ro.brute_force(X, y, 3, lam2, M, kind, J0=J0, J1=J1, top=1)[0][0]
            assert lb <= best + 1e-9 * abs(best)


def test_leaf_equals_ridge_closed_form():
    """kbar = 0 leaf with an inactive box: the bound is the ridge fit on J1 (LAPACK solve)."""
    X, y = _tiny(ol.LSQ, n=80, p=8, k=3)
    lam2, M = 0.1, 50.0
    S = [1, 4, 6]
    nd = on.Node(8, 3, J0=[j for j in range(8) if j not in S], J1=S)
    L = on.lipschitz(X, ol.LSQ)
    r = on.solve_node(X, y, nd, lam2, M, ol.LSQ, L, T=3000)
    XS = X[:, S]
    b = np.linalg.solve(XS.T @ XS + lam2 * np.eye(3), XS.T @ y)
    v = float(np.sum((XS @ b - y) ** 2)) + lam2 * float(b @ b)
    assert abs(r["lb"] - v) <= 1e-10 * v and abs(r["primal"] - v) <= 1e-10 * v
    assert np.allclose(r["beta"][S], b, atol=1e-8)


def test_root_without_cardinality_is_ridge():
    """k >= p: the relaxation at the root is plain ridge regression (no budget binds)."""
    X, y = _tiny(ol.LSQ, n=80, p=6, k=6)
    lam2, M = 0.3, 50.0
    nd = on.Node(6, 6)
    r = on.solve_node(X, y, nd, lam2, M, ol.LSQ, on.lipschitz(X, ol.LSQ), T=3000)
    b = np.linalg.solve(X.T @ X + lam2 * np.eye(6), X.T @ y)
    assert np.allclose(r["beta"], b, atol=1e-8)


# ---------------------------------------------------------------- re-opt, rounding, branching

@pytest.mark.parametrize("kind", KINDS)
def test_reopt_matches_library_solution(kind):
    X, y = _tiny(kind, n=70, p=8, k=3)
    lam2, M = 0.05, 0.6   # a tight box so that it binds
    for S in ([0, 3, 5], [1, 2], [7]):
        _, v = ro.reopt(X, y, S, lam2, M, kind)
        ref = ro.brute_force(X, y, len(S), lam2, M, kind, J0=[j for j in range(8) if j not in S], top=1)[0][0]
        assert abs(v - ref) <= 1e-9 * max(1.0, abs(ref))


def test_rounding_and_branching_ties():
    nd = on.Node(6, 3, J0=[0], J1=[5])
    beta = np.array([0.0, 0.5, -0.5, 0.2, 0.5, 1.0])
    assert on.round_support(beta, nd) == [1, 2, 5]
    assert on.branch_index(beta, nd) == 1
    assert on.branch_index(beta, on.Node(6, 1, J1=[5])) == -1     # kbar = 0


def test_fig2_padding_pattern():
    """The sentinel pattern of Fig. 2 (p=6, m=3, k=3) from the node sets."""
    rows = open(os.path.join(HERE, "golden", "fig2_padding.txt")).read().splitlines()
    sets, pad, srt = [], [], []
    for r in rows:
        if r.startswith("N"):
            parts = [s.strip() for s in r.split(":", 1)[1].split("|")]
            conv = lambda s: [] if s == "-" else [int(t) - 1 for t in s.split()]
            sets.append((conv(parts[0]), conv(parts[1]), conv(parts[2])))
        elif r.startswith("pad:"):
            pad.append([int(t) for t in r[4:].split()])
        elif r.startswith("sort:"):
            srt.append([int(t) for t in r[5:].split()])
    pad, srt = np.array(pad), np.array(srt)
    rng = np.random.default_rng(0)
    u = rng.random((6, 3)) + 0.1
    for b, (J0, J1, Jf) in enumerate(sets):
        nd = on.Node(6, 3, J0, J1)
        assert nd.Jf == Jf and nd.kbar == 3 - len(J1)
        K = np.full(6, -np.inf)
        K[nd.Jf] = np.abs(u[nd.Jf, b])
        assert np.array_equal(np.isfinite(K).astype(int), pad[:, b])
        Ks = np.sort(K)[::-1]
        assert np.array_equal(np.isfinite(Ks).astype(int), srt[:, b])


# ---------------------------------------------------------------- BnB optimum

def _check_bnb(X, y, k, lam2, M, kind):
    res = ob.solve(X, y, k, lam2, M, kind)
    top = ro.brute_force(X, y, k, lam2, M, kind, top=2)
    assert res["certified"] and res["gap"] <= 1e-6
    best, second = top[0], top[1]
    delta = 1e-6 * max(1.0, abs(best[0]))
    assert abs(res["opt"] - best[0]) <= 1e-9 * abs(best[0]) + delta
    if second[0] - best[0] > delta:                      # unique optimum: supports agree exactly
        assert tuple(res["support"]) == tuple(best[1])
    return res


def test_bnb_equals_brute_force_c1():
    """C1 (least squares, n=200, p=30, k=5): BnB optimum = brute force over all C(30,5) supports."""
    c, X, y, _ = synth.config_instance("c1_lsq_n200_p30_k5", seed=0)
    _check_bnb(X, y, c["k"], c["lam2"], c["M"], c["kind"])


def test_bnb_equals_brute_force_hard_lsq():
    """A correlated, noisy least-squares case that needs real branching."""
    X, y, _ = synth.instance(40, 16, 4, ol.LSQ, rho=0.9, snr=1.0, seed=3)
    res = _check_bnb(X, y, 4, 1e-3, 2.0, ol.LSQ)
    assert res["nodes"] > 3


def test_bnb_equals_brute_force_logistic():
    X, y, _ = synth.instance(60, 12, 3, ol.LOGISTIC, rho=0.7, seed=4)
    _check_bnb(X, y, 3, 0.05, 2.0, ol.LOGISTIC)


# --------------------------------------------------------------------------
# Rashomon set (§4.5): the brute-force definition, pinned by its properties
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", KINDS)
def test_rashomon_set_definition(kind):
    """Phi* equals the brute-force optimum; the set grows with eps; it is closed
    under adding features up to size k (v is non-increasing under inclusion);
    eps = 0 keeps exactly the minimizers; the capped set is a prefix."""
    X, y, _ = synth.instance(40, 7, 3, kind, rho=0.6, snr=0.5, seed=8)
    lam2, M = 0.05, 2.0
    phi, R1 = ro.rashomon_set(X, y, 3, lam2, M, kind, 0.05)
    best = ro.brute_force(X, y, 3, lam2, M, kind, top=1)[0]
    assert abs(phi - best[0]) <= 1e-9 * max(1.0, abs(phi))
    _, R0 = ro.rashomon_set(X, y, 3, lam2, M, kind, 0.0)
    assert [S for _, S in R0] == [S for v, S in R1 if v <= phi]
    _, R5 = ro.rashomon_set(X, y, 3, lam2, M, kind, 0.2)
    s1, s5 = {S for _, S in R1}, {S for _, S in R5}
    assert s1 <= s5 and len(s5) > len(s1)
    vmap = {S: v for v, S in ro.rashomon_set(X, y, 3, lam2, M, kind, 10.0)[1]}
    for S in s5:
        for j in range(7):
            if j not in S and len(S) < 3:
                T = tuple(sorted(S + (j,)))
                assert vmap[T] <= vmap[S] + 1e-9 * vmap[S]
                assert T in s5
    assert any(len(S) < 3 for S in s5)          # smaller supports belong to the set too
    _, Rn = ro.rashomon_set(X, y, 3, lam2, M, kind, 0.2, N=4)
    assert Rn == R5[:4]


def test_appG_trie_layout_golden():
    """The pool's trie-and-offset layout reproduces the worked example of App. G:
    o = (0, 3, 6, 9, 11), the coefficient vector, shared prefixes (18, 2) and (18),
    and supports recovered from the trie paths (through the C ABI, host only)."""
    from paper_2605_22188_gb300 import kglm
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "appG_trie.txt")
    recs, o, c, sets = [], None, None, []
    for line in open(path):
        if line.startswith("rec:"):
            seq, cf = line[4:].split("|")
            recs.append(([int(t) for t in seq.split()], [float(t) for t in cf.split()]))
        elif line.startswith("o:"):
            o = [int(t) for t in line[2:].split()]
        elif line.startswith("c:"):
            c = [float(t) for t in line[2:].split()]
        elif line.startswith("S:"):
            sets.append(tuple(sorted(int(t) for t in line[2:].split())))
    with kglm.Pool(20) as pool:
        for r, (seq, cf) in enumerate(recs):
            assert pool.insert(seq, cf, objective=float(r)) == r
        d = pool.read()
        assert d["offsets"].tolist() == o
        assert np.allclose(d["coef"], c, rtol=0, atol=0)
        # root + {18, (18,2), (18,2,7), (18,2,11), (18,9), (18,9,3), 12, (12,4)}
        assert len(d["parent"]) == 9
        paths = [pool.support(r) for r in range(4)]
        assert paths == [seq for seq, _ in recs]
        assert [tuple(sorted(p)) for p in paths] == sets
        # the first two records share the trie nodes of (18, 2); the first three share (18)
        leaf = d["leaf"]
        assert d["parent"][leaf[0]] == d["parent"][leaf[1]]
        top = lambda v: v if d["parent"][v] == 0 else top(int(d["parent"][v]))
        assert top(int(leaf[0])) == top(int(leaf[1])) == top(int(leaf[2])) != top(int(leaf[3]))
        # record 2 (second) uses c[3:6] and the support {2, 11, 18}
        recs2 = pool.records()
        assert recs2[1][1] == (2, 11, 18) and np.allclose(recs2[1][2], [0.5, -1.0, 0.1])
        # a support already held is not stored twice
        assert pool.insert([7, 18, 2], [0.0, 0.0, 0.0], 9.0) == -1
        # filtering keeps order and rebuilds the layout
        pool.filter(2.5, keep_best=2)
        d2 = pool.read()
        assert d2["offsets"].tolist() == [0, 3, 6] and np.allclose(d2["coef"], c[:6])
        assert len(d2["parent"]) == 5
