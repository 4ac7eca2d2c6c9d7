"""One BnB node of the perspective relaxation, solved and certified in FP64.

Test infrastructure only (see ``oracle/__init__.py``).

A node N is given by its fixed-out set J0 (z_j = 0), fixed-in set J1
(z_j = 1) and free set Jf (z_j in [0, 1]), with reduced budget
kbar = k - |J1| (§3, definition of g_N below Eq. (node_composite)).

Readings of the paper (where it is silent) used here:

* step size eta = 1/L with L = 2||X||_2^2 (least squares) or ||X||_2^2/4
  (logistic), rho = 1/(2 eta lambda2) as in §3 Eq. (pgd_step_vector_form);
* the first-order method is FISTA with gradient restart (the footnote of §3
  allows acceleration and restart; App. E.2 says the paper's solver is an
  accelerated, restarted proximal gradient method);
* Algorithm 1 is stated for the root; at a node it runs on the free
  coordinates with budget kbar, J1 coordinates take the Huber prox with weight
  rho (z_j = 1), J0 coordinates are 0;
* ties in rounding and branching go to the smallest index.
"""

import numpy as np

from .losses import LSQ, LOGISTIC, loss, dloss, loss_conj, huber, prox_huber


class Node:
    """Fixing decisions of one BnB node (§3): J0, J1 and the free set Jf."""

    def __init__(self, p, k, J0=(), J1=()):
        self.p = int(p)
        self.k = int(k)
        self.J0 = sorted(set(int(j) for j in J0))
        self.J1 = sorted(set(int(j) for j in J1))
        if set(self.J0) & set(self.J1):
            raise ValueError("J0 and J1 overlap")
        if len(self.J1) > self.k:
            raise ValueError("|J1| > k")
        fixed = set(self.J0) | set(self.J1)
        self.Jf = [j for j in range(self.p) if j not in fixed]

    @property
    def kbar(self):
        """kbar(N) = k - |J1(N)| (§3 Eq. (prelim_node_conjugate))."""
        return self.k - len(self.J1)

    @property
    def pf(self):
        return len(self.Jf)

    def is_leaf(self):
        """No branching left: kbar = 0, or the free set fits in the budget."""
        return self.kbar == 0 or len(self.J1) + self.pf <= self.k

    def children(self, j):
        """The two children of a branch on free index j: z_j = 0 and z_j = 1 (App. A)."""
        if j not in self.Jf:
            raise ValueError("branch index must be free")
        return (Node(self.p, self.k, self.J0 + [j], self.J1),
                Node(self.p, self.k, self.J0, self.J1 + [j]))


def lipschitz(X, kind):
    """Lipschitz constant of grad F(X beta): 2||X||^2 (least squares) or ||X||^2/4 (logistic).

    ||X||_2 is the largest singular value (LAPACK SVD through numpy).
    """
    s = np.linalg.norm(np.asarray(X, dtype=np.float64), 2)
    return 2.0 * s * s if kind == LSQ else 0.25 * s * s


# --------------------------------------------------------------------------
# Algorithm 1 (App. B): prox of rho * g* on the free coordinates
# --------------------------------------------------------------------------

def alg1_prox_gconj(w, rho, kbar, M):
    """prox_{rho g*}(w) for the TopSum_kbar-of-H_M part of g* (Algorithm 1, App. B).

    Steps in the order of Algorithm 1:
      1. weights rho_j = rho for the kbar largest |w|, 0 for the others;
      2. sort |w| descending (permutation pi);
      3. v_j = prox_{rho_j H_M}(|w_pi(j)|);
      4. pool adjacent violators: while two adjacent blocks are out of
         non-increasing order, merge them; a merged block takes the common
         value prox_{rho_bar H_M}(xi_bar), rho_bar and xi_bar being the block
         means of rho_j and |w_pi(j)|;
      5. return sign(w) * pi^{-1}(v).
    The merging in step 4 is done with the usual stack (one left-to-right pass
    that merges a new block backwards while it violates the order); every
    merge order reaches the same, unique, isotonic solution.
    """
    w = np.asarray(w, dtype=np.float64)
    pf = w.size
    if pf == 0:
        return w.copy()
    a = np.abs(w)
    pi = np.argsort(-a, kind="stable")            # step 2
    a_sorted = a[pi]
    rho_j = np.where(np.arange(pf) < kbar, rho, 0.0)   # step 1 (in sorted order)
    v0 = np.array([float(prox_huber(a_sorted[j], rho_j[j], M)) for j in range(pf)])  # step 3

    # step 4: blocks as [start, end, sum_rho, sum_a, value]
    blocks = []
    for j in range(pf):
        blk = [j, j, rho_j[j], a_sorted[j], v0[j]]
        while blocks and blocks[-1][4] < blk[4]:
            prev = blocks.pop()
            start, end = prev[0], blk[1]
            s_rho = prev[2] + blk[2]
            s_a = prev[3] + blk[3]
            cnt = end - start + 1
            val = float(prox_huber(s_a / cnt, s_rho / cnt, M))
            blk = [start, end, s_rho, s_a, val]
        blocks.append(blk)
    v_sorted = np.empty(pf)
    for start, end, _, _, val in blocks:
        v_sorted[start:end + 1] = val

    v = np.empty(pf)                               # step 5
    v[pi] = v_sorted
    return np.sign(w) * v


def prox_node(u, node, rho, M):
    """beta = prox_{eta G_N}(u) = u - rho^{-1} prox_{rho g_N*}(rho u) (§3 Eq. (pgd_step_vector_form)).

    g_N* = sum_{J1} H_M + TopSum_kbar over Jf of H_M (§3 Eq. (prelim_node_conjugate)),
    so the prox of rho*g_N* splits into: identity on J0 (g* does not depend on
    those entries, so beta_J0 = 0), the Huber prox with weight rho on J1, and
    Algorithm 1 with budget kbar on Jf.
    """
    u = np.asarray(u, dtype=np.float64)
    w = rho * u
    v = w.copy()                                    # J0: identity
    if node.J1:
        J1 = np.array(node.J1)
        v[J1] = prox_huber(w[J1], rho, M)
    if node.Jf:
        Jf = np.array(node.Jf)
        v[Jf] = alg1_prox_gconj(w[Jf], rho, node.kbar, M)
    beta = u - v / rho
    if node.J0:
        beta[np.array(node.J0)] = 0.0              # u - (rho u)/rho, exactly
    return beta


# --------------------------------------------------------------------------
# g (Theorem 4.1) and g* (TopSum)
# --------------------------------------------------------------------------

FEAS_RTOL = 1e-12


def g_node(beta, node, M):
    """g_N(beta) = inf_z 1/2 sum beta_j^2 / z_j over the node polytope, via Theorem 4.1.

    Returns +inf when beta is outside the domain: beta_J0 != 0, |beta_j| > M,
    or sum_{Jf} |beta_j| / M > kbar (the existence argument in the proof of
    Theorem 4.1).  A relative slack of FEAS_RTOL absorbs FP64 rounding in the
    box and budget tests.
    """
    beta = np.asarray(beta, dtype=np.float64)
    if node.J0 and np.any(beta[np.array(node.J0)] != 0.0):
        return np.inf
    J1 = np.array(node.J1, dtype=int)
    Jf = np.array(node.Jf, dtype=int)
    if np.any(np.abs(beta[np.concatenate([J1, Jf])]) > M * (1.0 + FEAS_RTOL)):
        return np.inf
    g = 0.5 * float(np.sum(beta[J1] ** 2)) if J1.size else 0.0
    b = np.abs(beta[Jf]) if Jf.size else np.zeros(0)
    kbar = node.kbar
    if kbar == 0:
        return g if not np.any(b != 0.0) else np.inf
    if np.sum(b) / M > kbar * (1.0 + FEAS_RTOL):
        return np.inf
    if np.count_nonzero(b) <= kbar:                # non-binding budget: z_j = 1 on nonzeros
        return g + 0.5 * float(np.sum(b * b))
    bs = np.sort(b)[::-1]                          # |beta_pi(1)| >= ... >= |beta_pi(pf)|
    tail = np.cumsum(bs[::-1])[::-1]               # tail[r] = sum_{r' >= r} bs[r'] (0-based)
    s, tau = _capped_count(bs, tail, kbar)
    # z = 1 on the first s, z = |beta|/tau after: sum_{r>s} beta^2/z = tau * sum_{r>s} |beta|
    return g + 0.5 * (float(np.sum(bs[:s] ** 2)) + tau * float(tail[s]))


def _capped_count(bs, tail, kbar):
    """The s of Theorem 4.1 (coordinates with z_j = 1) and tau = tail[s] / (kbar - s).

    s is the smallest index in [0, kbar) with tau_s >= |beta|_(s+1); then also
    tau_s < |beta|_(s) (for s > 0, tau_{s-1} < |beta|_(s) is equivalent to
    tau_s < |beta|_(s)), so |beta|_(s) > tau >= |beta|_(s+1) as the theorem
    requires.  s = kbar - 1 always qualifies (tail[kbar-1] >= bs[kbar-1], also
    in floating point, where adding non-negative terms never decreases a sum),
    so the search needs no fallback.
    """
    for s in range(kbar):
        tau = tail[s] / (kbar - s)
        if tau >= bs[s]:
            return s, tau
    raise ArithmeticError("unreachable: tail[kbar-1] >= bs[kbar-1]")


def z_recover(beta, node, M):
    """The relaxed indicators z* of Theorem 4.1 (for tests and rounding checks)."""
    beta = np.asarray(beta, dtype=np.float64)
    p = beta.size
    z = np.zeros(p)
    for j in node.J1:
        z[j] = 1.0
    Jf = np.array(node.Jf, dtype=int)
    kbar = node.kbar
    if kbar == 0 or Jf.size == 0:
        return z
    b = np.abs(beta[Jf])
    if np.count_nonzero(b) <= kbar:
        z[Jf] = (b != 0.0).astype(float)
        return z
    order = np.argsort(-b, kind="stable")
    bs = b[order]
    tail = np.cumsum(bs[::-1])[::-1]
    s, tau = _capped_count(bs, tail, kbar)
    z[Jf[order]] = np.where(np.arange(bs.size) < s, 1.0, bs / tau)
    return z


def g_conj_node(q, node, M):
    """g_N*(q) = sum_{J1} H_M(q_j) + TopSum_kbar {H_M(q_j)}_{j in Jf} (§3 Eq. (prelim_node_conjugate))."""
    q = np.asarray(q, dtype=np.float64)
    val = float(np.sum(huber(q[np.array(node.J1, dtype=int)], M))) if node.J1 else 0.0
    if node.Jf and node.kbar > 0:
        h = np.sort(huber(q[np.array(node.Jf)], M))[::-1]
        val += float(np.sum(h[:node.kbar]))
    return val


# --------------------------------------------------------------------------
# objectives and the certificate
# --------------------------------------------------------------------------

def primal_value(X, y, beta, node, lam2, M, kind):
    """Phi_N(beta) = sum_i l((X beta)_i, y_i) + 2 lambda2 g_N(beta) (§4.4 Eq. (batched_primal_value_component))."""
    g = g_node(beta, node, M)
    if not np.isfinite(g):
        return np.inf
    s = np.asarray(X, dtype=np.float64) @ beta
    return float(np.sum(loss(s, y, kind))) + 2.0 * lam2 * g


def dual_value(X, y, zeta, node, lam2, M, kind):
    """Psi_N(zeta) = -sum_i l*(-zeta_i, y_i) - 2 lambda2 g_N*(X^T zeta / (2 lambda2)).

    §3 Eq. (prelim_fenchel_dual) with the conjugate scaling rule, written per
    node as in §4.4 Eq. (batched_dual_value_component).  A lower bound on
    min Phi_N for every zeta by weak duality.
    """
    zeta = np.asarray(zeta, dtype=np.float64)
    q = (np.asarray(X, dtype=np.float64).T @ zeta) / (2.0 * lam2)
    return -float(np.sum(loss_conj(-zeta, y, kind))) - 2.0 * lam2 * g_conj_node(q, node, M)


def dual_point(X, y, beta, kind):
    """zeta = -grad F(X beta) (§3 Eq. (dual_candidate_vector_form))."""
    s = np.asarray(X, dtype=np.float64) @ beta
    return -dloss(s, y, kind)


def certify(X, y, beta, node, lam2, M, kind):
    """(LB, Phi): the safe lower bound Psi_N(zeta(beta)) and the primal value at beta."""
    zeta = dual_point(X, y, beta, kind)
    return dual_value(X, y, zeta, node, lam2, M, kind), primal_value(X, y, beta, node, lam2, M, kind)


# --------------------------------------------------------------------------
# the node solver
# --------------------------------------------------------------------------

def solve_node(X, y, node, lam2, M, kind, L, T, beta0=None, restart=True,
               check_every=0, ub=np.inf, delta=0.0, gap_rtol=0.0):
    """T iterations of FISTA on Phi_N (§3 Eq. (node_composite)) from beta0.

    FISTA in the indexing of Beck and Teboulle (2009): y_1 = x_0 = beta0,
    t_1 = 1, and for k = 1, 2, ...
        x_k     = prox_node(y_k - eta * X^T dl(X y_k, y))   (§3 Eq. (pgd_step_vector_form))
        t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2
        y_{k+1} = x_k + ((t_k - 1) / t_{k+1}) (x_k - x_{k-1})
    so the first two proximal steps take no momentum.  Gradient restart
    (O'Donoghue and Candes 2015) with the proximal gradient mapping in place
    of the gradient: if <y_k - x_k, x_k - x_{k-1}> > 0 the method starts over
    from x_k, i.e. y_{k+1} = x_k and t_{k+1} = 1 (the step after it then takes
    no momentum either).
    With check_every > 0 the certificate is evaluated every check_every
    iterations; the loop stops once LB >= ub - delta or Phi - LB <=
    gap_rtol * max(1, |Phi|).  The returned LB is the best certificate seen
    (each one is valid, so the maximum is too), always including the last
    iterate.

    Returns dict(beta, lb, primal, iters).
    """
    X = np.asarray(X, dtype=np.float64)
    p = X.shape[1]
    eta = 1.0 / L
    rho = 1.0 / (2.0 * eta * lam2)
    beta = np.zeros(p) if beta0 is None else np.array(beta0, dtype=np.float64)
    if node.J0:
        beta[np.array(node.J0)] = 0.0
    beta_old = beta.copy()     # x_{k-1}
    yk = beta.copy()           # y_k
    t = 1.0                    # t_k
    best_lb = -np.inf
    primal = np.inf
    it = 0
    while it < T:
        grad = X.T @ dloss(X @ yk, y, kind)
        beta_new = prox_node(yk - eta * grad, node, rho, M)        # x_k
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        if restart and float(np.dot(yk - beta_new, beta_new - beta)) > 0.0:
            y_next, t_new = beta_new.copy(), 1.0
        else:
            y_next = beta_new + ((t - 1.0) / t_new) * (beta_new - beta)
        beta, yk, t = beta_new, y_next, t_new
        it += 1
        if check_every > 0 and it % check_every == 0 and it < T:
            lb, primal = certify(X, y, beta, node, lam2, M, kind)
            best_lb = max(best_lb, lb)
            if best_lb >= ub - delta or primal - best_lb <= gap_rtol * max(1.0, abs(primal)):
                return dict(beta=beta, lb=best_lb, primal=primal, iters=it)
    lb, primal = certify(X, y, beta, node, lam2, M, kind)
    best_lb = max(best_lb, lb)
    return dict(beta=beta, lb=best_lb, primal=primal, iters=it)


# --------------------------------------------------------------------------
# rounding and branching (§4.3)
# --------------------------------------------------------------------------

def round_support(beta, node):
    """S_N = J1 cup T_kbar, T_kbar the kbar largest |beta_j| over Jf, ties to the smaller index (§4.3)."""
    beta = np.asarray(beta, dtype=np.float64)
    Jf = np.array(node.Jf, dtype=int)
    take = []
    if node.kbar > 0 and Jf.size:
        order = sorted(range(Jf.size), key=lambda r: (-abs(beta[Jf[r]]), Jf[r]))
        take = [int(Jf[r]) for r in order[:node.kbar]]
    return sorted(node.J1 + take)


def branch_index(beta, node):
    """j* = argmax_{j in Jf} |beta_j|, ties to the smaller index (§4.3); -1 for a leaf."""
    if node.is_leaf() or not node.Jf:
        return -1
    beta = np.asarray(beta, dtype=np.float64)
    best = None
    for j in node.Jf:
        if best is None or abs(beta[j]) > abs(beta[best]):
            best = j
    return int(best)
