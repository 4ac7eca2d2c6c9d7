"""Pins of the oracle's FISTA trajectory, its step size and Theorem 4.1's z.

The node solver's iterates after a fixed T are what every GPU parity test
compares against, so they are pinned here by facts that do not come from the
oracle's own code:

* the step 1/L: L against the largest singular value from an iterative
  library solver (ARPACK through scipy.sparse.linalg.svds);
* the momentum schedule: the trajectory equals the accelerated scheme of
  O'Donoghue and Candes (2015, Algorithm 1 with q = 0), written in its own
  theta parametrization (theta_0 = 1, beta_{k+1} = theta_k (1 - theta_k) /
  (theta_k^2 + theta_{k+1})), whose first extrapolation takes no momentum;
  its gradient restart resets theta to 1;
* the rate of Beck and Teboulle (2009, Thm. 4.4) without restart,
  Phi(x_T) - Phi* <= 2 L ||x_0 - x*||^2 / (T + 1)^2, and the monotone energy of
  their Lemma 4.1, with Phi* from a bounded least-squares library solver;
* the restart sign: on an ill-conditioned node the restarted method ends
  closer to the optimum than the plain one (a reversed test would restart on
  useful momentum and fall behind);
* one proximal-gradient step (§3 Eq. (pgd_step_vector_form)) on a hand-made
  node, against the perspective form of the prox minimised over z directly;
* z of Theorem 4.1 against a direct minimisation over the node polytope,
  including the breakpoints where two choices of s give the same g.
"""

import numpy as np
import pytest
from scipy.optimize import lsq_linear, minimize, minimize_scalar
from scipy.sparse.linalg import svds

from oracle import losses as ol
from oracle import node as on
from paper_2605_22188_gb300 import synth


@pytest.mark.parametrize("kind", [ol.LSQ, ol.LOGISTIC])
def test_lipschitz_matches_arpack(kind):
    rng = np.random.default_rng(1)
    X = synth.design(120, 40, 0.7, rng)
    s = svds(X, k=1, return_singular_vectors=False, tol=1e-14)[0]
    want = 2.0 * s * s if kind == ol.LSQ else 0.25 * s * s
    assert abs(on.lipschitz(X, kind) - want) <= 1e-12 * want


def _oc_theta_fista(X, y, node, lam2, M, kind, L, T, beta0, restart):
    """O'Donoghue-Candes Algorithm 1 (q = 0) with the node prox after the gradient step."""
    eta = 1.0 / L
    rho = 1.0 / (2.0 * eta * lam2)
    x = np.array(beta0, dtype=np.float64)
    x[node.J0] = 0.0
    yk, theta = x.copy(), 1.0
    for _ in range(T):
        x_new = on.prox_node(yk - eta * (X.T @ ol.dloss(X @ yk, y, kind)), node, rho, M)
        th2 = theta * theta
        theta_new = 0.5 * (-th2 + np.sqrt(th2 * th2 + 4.0 * th2))   # theta'^2 = (1 - theta') theta^2
        mom = theta * (1.0 - theta) / (th2 + theta_new)
        if restart and float(np.dot(yk - x_new, x_new - x)) > 0.0:
            # restart: the next point is x_new itself and theta starts over at 1
            yk, theta = x_new.copy(), 1.0
        else:
            yk, theta = x_new + mom * (x_new - x), theta_new
        x = x_new
    return x


@pytest.mark.parametrize("kind", [ol.LSQ, ol.LOGISTIC])
@pytest.mark.parametrize("restart", [False, True])
@pytest.mark.parametrize("sets", [((), ()), ((1, 4), (0,)), ((), (2, 5, 6))])
def test_trajectory_is_the_published_accelerated_scheme(kind, restart, sets):
    X, y, _ = synth.instance(50, 9, 3, kind, rho=0.8, snr=2.0, seed=31)
    lam2, M = 0.03, 1.5
    nd = on.Node(9, 3, *sets)
    L = on.lipschitz(X, kind)
    beta0 = np.random.default_rng(2).standard_normal(9) * 0.7
    for T in (1, 2, 3, 7, 40):
        got = on.solve_node(X, y, nd, lam2, M, kind, L, T, beta0=beta0, restart=restart)["beta"]
        want = _oc_theta_fista(X, y, nd, lam2, M, kind, L, T, beta0, restart)
        assert np.max(np.abs(got - want)) <= 1e-12 * max(1.0, np.max(np.abs(want))), T


def _ridge_box_optimum(X, y, lam2, M, free):
    """min ||X b - y||^2 + lam2 ||b||^2 over |b| <= M on the free columns (BVLS)."""
    Xf = X[:, free]
    A = np.vstack([Xf, np.sqrt(lam2) * np.eye(len(free))])
    rhs = np.concatenate([y, np.zeros(len(free))])
    r = lsq_linear(A, rhs, bounds=(-M, M), method="bvls", tol=1e-15)
    b = np.zeros(X.shape[1])
    b[free] = r.x
    return b, float(np.sum((X @ b - y) ** 2) + lam2 * b @ b)


@pytest.mark.parametrize("seed", range(6))
def test_beck_teboulle_rate_and_energy_without_restart(seed):
    """A node whose budget does not bind (kbar >= pf) is ridge regression with a box,
    strongly convex: Phi* by BVLS, then the rate bound at every T and the
    non-increasing energy of Beck and Teboulle's Lemma 4.1."""
    rng = np.random.default_rng(50 + seed)
    n, p = 40, 8
    X = synth.design(n, p, 0.9, rng)
    y = 3.0 * rng.standard_normal(n)
    lam2 = float(10 ** rng.uniform(-3, 0))
    M = float(rng.choice([0.4, 50.0]))          # a binding and a loose box
    J0 = [int(rng.integers(p))]
    nd = on.Node(p, p, J0=J0)
    free = [j for j in range(p) if j not in J0]
    L = on.lipschitz(X, ol.LSQ)
    xs, phis = _ridge_box_optimum(X, y, lam2, M, free)
    beta0 = np.zeros(p)
    beta0[free] = np.clip(3.0 * rng.standard_normal(p - 1), -M, M)
    d0 = float(np.sum((beta0 - xs) ** 2))
    phi = lambda b: float(np.sum((X @ b - y) ** 2) + lam2 * b @ b)
    prev, t, energy_prev = beta0, 1.0, None
    for T in range(1, 41):
        x = on.solve_node(X, y, nd, lam2, M, ol.LSQ, L, T, beta0=beta0, restart=False)["beta"]
        gap = phi(x) - phis
        assert gap <= 2.0 * L * d0 / (T + 1) ** 2 + 1e-9 * max(1.0, phis), T
        u = t * x - (t - 1.0) * prev - xs
        energy = 2.0 / L * t * t * gap + float(u @ u)
        if energy_prev is None:
            assert energy <= d0 * (1 + 1e-9) + 1e-12
        else:
            assert energy <= energy_prev * (1 + 1e-9) + 1e-12, T
        energy_prev, prev, t = energy, x, 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))


def test_gradient_restart_helps_on_an_ill_conditioned_node():
    """Restart when momentum points uphill (O'Donoghue-Candes): on a strongly convex,
    ill-conditioned node the restarted run converges linearly and, after a few
    multiples of sqrt(condition number) iterations, ends far closer to Phi*
    than the plain one (which only has the O(1/T^2) rate)."""
    rng = np.random.default_rng(8)
    n, p = 60, 10
    X = synth.design(n, p, 0.9, rng)
    y = X @ rng.standard_normal(p) + 0.1 * rng.standard_normal(n)
    lam2, M = 0.1, 50.0          # condition number of the Hessian ~230
    nd = on.Node(p, p)
    L = on.lipschitz(X, ol.LSQ)
    xs, phis = _ridge_box_optimum(X, y, lam2, M, list(range(p)))
    phi = lambda b: float(np.sum((X @ b - y) ** 2) + lam2 * b @ b)
    for T in (200, 400):
        g_plain = phi(on.solve_node(X, y, nd, lam2, M, ol.LSQ, L, T, restart=False)["beta"]) - phis
        g_rest = phi(on.solve_node(X, y, nd, lam2, M, ol.LSQ, L, T, restart=True)["beta"]) - phis
        assert g_rest < 1e-2 * g_plain, (T, g_rest, g_plain)


def _prox_by_z(u, node, c, M):
    """prox of c g_N at u with g_N in its perspective form (§3): for fixed z the
    coordinates separate, beta_j = sign(u_j) min(|u_j| z_j / (z_j + c), M z_j);
    the budget binds at the optimum, so z runs over the segment sum_Jf z = kbar
    (here two free coordinates and kbar = 1: one scalar, minimised by Brent)."""
    Jf = node.Jf
    assert len(Jf) == 2 and node.kbar == 1

    def beta_of(z):
        b = np.zeros_like(u)
        for j in node.J1:
            b[j] = np.sign(u[j]) * min(abs(u[j]) / (1.0 + c), M)
        for j, zj in zip(Jf, (z, 1.0 - z)):
            b[j] = np.sign(u[j]) * min(abs(u[j]) * zj / (zj + c), M * zj) if zj > 0 else 0.0
        return b

    def obj(z):
        b = beta_of(z)
        val = 0.5 * float(np.sum((b - u) ** 2))
        for j, zj in zip(node.J1 + Jf, [1.0] * len(node.J1) + [z, 1.0 - z]):
            if zj > 0:
                val += c * 0.5 * b[j] ** 2 / zj
        return val

    r = minimize_scalar(obj, bounds=(0.0, 1.0), method="bounded", options=dict(xatol=1e-13))
    return beta_of(r.x)


def test_one_proximal_gradient_step_by_hand():
    """One step of §3 Eq. (pgd_step_vector_form) on p = 4: J1 = {0}, J0 = {3},
    Jf = {1, 2}, kbar = 1.  X, y and beta0 are small integers, so u = beta0 -
    eta X^T dl(X beta0) is exact; beta1 is checked against the prox minimised
    over z, and the first FISTA step of the solver is that plain step."""
    X = np.array([[1.0, 2.0, 0.0, 1.0],
                  [0.0, 1.0, -1.0, 2.0],
                  [2.0, 0.0, 1.0, 0.0]])
    y = np.array([3.0, -1.0, 2.0])
    beta0 = np.array([1.0, -1.0, 1.0, 0.0])
    lam2, M, L = 0.5, 1.25, 64.0                   # eta = 1/64, rho = 64, c = 1/64
    nd = on.Node(4, 2, J0=[3], J1=[0])
    s = X @ beta0                                  # (-1, -2, 3)
    g = X.T @ (2.0 * (s - y))                      # LS: dl = 2 (s - y) = (-8, -2, 2)
    assert np.array_equal(g, np.array([-4.0, -18.0, 4.0, -12.0]))
    u = beta0 - g / L                              # (1.0625, -0.71875, 0.9375, 0.1875)
    c = 2.0 * lam2 / L
    want = _prox_by_z(u, nd, c, M)
    got = on.solve_node(X, y, nd, lam2, M, ol.LSQ, L, 1, beta0=beta0)["beta"]
    assert np.max(np.abs(got - want)) <= 1e-9, (got, want)
    assert got[3] == 0.0


def _z_by_slsqp(beta, node, M):
    """argmin_z 1/2 sum beta_j^2 / z_j over the node polytope with z_j >= |beta_j| / M (§3)."""
    Jf = np.array(node.Jf, dtype=int)
    b = np.abs(beta[Jf])
    nz = b > 0
    bb = b[nz]
    lo = bb / M
    cons = [dict(type="ineq", fun=lambda z: node.kbar - np.sum(z))]
    z0 = np.clip(np.full(bb.size, node.kbar / bb.size), lo, 1.0)
    r = minimize(lambda z: 0.5 * float(np.sum(bb ** 2 / z)), z0, bounds=list(zip(lo, np.ones(bb.size))),
                 constraints=cons, method="SLSQP", options=dict(ftol=1e-16, maxiter=5000))
    z = np.zeros(beta.size)
    z[Jf[nz]] = r.x
    return z, r.fun


@pytest.mark.parametrize("seed", range(8))
def test_z_recover_is_the_minimiser(seed):
    rng = np.random.default_rng(600 + seed)
    p, k, M = 9, 4, 2.0
    perm = rng.permutation(p)
    nd = on.Node(p, k, J0=list(perm[:2]), J1=list(perm[2:3]))
    Jf = np.array(nd.Jf)
    beta = np.zeros(p)
    beta[Jf] = rng.standard_normal(Jf.size)
    beta[Jf] *= 0.9 * nd.kbar * M / np.sum(np.abs(beta[Jf]))   # budget binding, inside the domain
    beta = np.clip(beta, -M, M)
    beta[perm[2]] = 0.7
    z = on.z_recover(beta, nd, M)
    zs, gs = _z_by_slsqp(beta, nd, M)
    # the minimiser is unique on the nonzero coordinates (strictly convex in z_j there)
    nz = np.abs(beta) > 0
    free_nz = np.zeros(p, bool)
    free_nz[Jf] = True
    free_nz &= nz
    assert np.max(np.abs(z[free_nz] - zs[free_nz])) <= 2e-5
    assert abs(on.g_node(beta, nd, M) - 0.5 * beta[perm[2]] ** 2 - gs) <= 1e-8 * max(1.0, gs)


@pytest.mark.parametrize("bs,kbar", [([2.0, 1.0, 1.0], 2), ([3.0, 1.0, 1.0], 2), ([1.5, 1.5, 1.0, 0.5], 3),
                                     ([2.0, 2.0, 2.0, 1.0], 2), ([1.0, 1.0, 1.0, 1.0], 3)])
def test_theorem41_at_breakpoints(bs, kbar):
    """Magnitudes where tau equals a |beta|_(s) exactly (two choices of s give the
    same g): g and z from Theorem 4.1 against the direct minimisation over z."""
    p = len(bs)
    M = 4.0                                        # inside the box and the budget
    nd = on.Node(p, kbar)
    beta = np.array(bs) * np.array([1, -1] * (p // 2) + [1] * (p % 2))
    g = on.g_node(beta, nd, M)
    zs, gs = _z_by_slsqp(beta, nd, M)
    assert abs(g - gs) <= 1e-8 * max(1.0, gs), (g, gs)
    z = on.z_recover(beta, nd, M)
    assert abs(0.5 * float(np.sum(beta ** 2 / np.where(z > 0, z, 1.0))) - gs) <= 1e-8 * max(1.0, gs)
    assert np.sum(z) <= kbar + 1e-12 and np.all(z >= np.abs(beta) / M - 1e-12)
