"""Re-optimization on a support and brute-force enumeration of supports (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

v(S) = min { F(X beta) + lambda2 ||beta||^2 : supp(beta) in S, ||beta||_inf <= M }
is the optimal objective on a support (§4.5, definition of v(S)); the optimum
of problem (intro_sparse_glm) is min over |S| <= k of v(S).
"""

import itertools

import numpy as np
from scipy.optimize import lsq_linear, minimize

from .losses import LSQ, LOGISTIC, loss, dloss
from .node import lipschitz


def objective(X, y, beta, lam2, kind):
    """F(X beta) + lambda2 ||beta||^2, the objective of problem (intro_sparse_glm)."""
    beta = np.asarray(beta, dtype=np.float64)
    return float(np.sum(loss(np.asarray(X, dtype=np.float64) @ beta, y, kind))) + lam2 * float(beta @ beta)


def reopt(X, y, S, lam2, M, kind, beta0=None, tol=1e-12, max_iter=200000):
    """Re-optimize on support S by projected FISTA (§4.3): the prox is the projection onto [-M, M].

    Step 1/L_S with L_S the Lipschitz constant of the gradient of
    F(X_S b) + lambda2 ||b||^2.  Stops when the gradient-mapping norm
    L_S * ||b - P(b - grad/L_S)|| <= tol * max(1, ||grad at the start||);
    FISTA indexing and gradient restart as in the node solver.  Returns
    (beta in R^p, v(S)).
    """
    X = np.asarray(X, dtype=np.float64)
    p = X.shape[1]
    S = np.array(sorted(S), dtype=int)
    beta_full = np.zeros(p)
    if S.size == 0:
        return beta_full, objective(X, y, beta_full, lam2, kind)
    XS = X[:, S]
    LS = lipschitz(XS, kind) + 2.0 * lam2
    b = np.zeros(S.size) if beta0 is None else np.clip(np.asarray(beta0, dtype=np.float64)[S], -M, M)

    def grad(v):
        return XS.T @ dloss(XS @ v, y, kind) + 2.0 * lam2 * v

    g0 = np.linalg.norm(grad(b))
    stop = tol * max(1.0, g0)
    v = b.copy()
    t = 1.0
    for _ in range(max_iter):
        b_new = np.clip(v - grad(v) / LS, -M, M)
        t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        if float(np.dot(v - b_new, b_new - b)) > 0.0:
            v, t_new = b_new.copy(), 1.0
        else:
            v = b_new + ((t - 1.0) / t_new) * (b_new - b)
        b, t = b_new, t_new
        gm = LS * np.linalg.norm(b - np.clip(b - grad(b) / LS, -M, M))
        if gm <= stop:
            break
    beta_full[S] = b
    return beta_full, objective(X, y, beta_full, lam2, kind)


# --------------------------------------------------------------------------
# brute force: the plain definition of the optimum
# --------------------------------------------------------------------------

def _v_lsq_exact(X, y, S, lam2, M):
    """v(S) for least squares by library routines: a LAPACK solve, or BVLS when the box binds."""
    XS = X[:, S]
    A = XS.T @ XS + lam2 * np.eye(len(S))
    b = np.linalg.solve(A, XS.T @ y)
    if np.max(np.abs(b)) > M:
        Aug = np.vstack([XS, np.sqrt(lam2) * np.eye(len(S))])
        rhs = np.concatenate([y, np.zeros(len(S))])
        b = lsq_linear(Aug, rhs, bounds=(-M, M), method="bvls", tol=1e-15).x
    r = XS @ b - y
    return float(r @ r) + lam2 * float(b @ b), b


def _v_logistic_exact(X, y, S, lam2, M):
    """v(S) for logistic loss by scipy's L-BFGS-B with the box as bounds."""
    XS = X[:, S]

    def fg(b):
        s = XS @ b
        f = float(np.sum(loss(s, y, LOGISTIC))) + lam2 * float(b @ b)
        g = XS.T @ dloss(s, y, LOGISTIC) + 2.0 * lam2 * b
        return f, g

    res = minimize(fg, np.zeros(len(S)), jac=True, method="L-BFGS-B",
                   bounds=[(-M, M)] * len(S),
                   options=dict(maxiter=10000, ftol=1e-16, gtol=1e-12, maxcor=30))
    return float(res.fun), res.x


def supports_of(p, k, J0=(), J1=()):
    """All supports consistent with a node: J1 in S, S in J1 cup Jf, |S| = min(k, |J1 cup Jf|).

    v(S) is non-increasing under inclusion, so supports of the largest size
    reach the node's optimum.
    """
    J0 = set(J0)
    J1 = sorted(set(J1))
    free = [j for j in range(p) if j not in J0 and j not in set(J1)]
    size = min(k, len(J1) + len(free)) - len(J1)
    for T in itertools.combinations(free, size):
        yield tuple(sorted(J1 + list(T)))


def brute_force(X, y, k, lam2, M, kind, J0=(), J1=(), top=2):
    """min over supports consistent with (J0, J1) of v(S), by enumeration.

    Least squares: every support is solved from the Gram matrix in one stacked
    LAPACK call; the best candidates are then re-solved exactly (residual
    form, BVLS if the box binds).  Logistic: L-BFGS-B per support.
    Returns a list of the ``top`` best (v, S) pairs, best first.
    """
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p = X.shape[1]
    sups = list(supports_of(p, k, J0, J1))
    if kind == LSQ:
        G = X.T @ X
        c = X.T @ y
        yy = float(y @ y)
        Sarr = np.array(sups, dtype=int)
        vals = np.empty(len(sups))
        chunk = 20000
        for lo in range(0, len(sups), chunk):
            idx = Sarr[lo:lo + chunk]
            A = G[idx[:, :, None], idx[:, None, :]] + lam2 * np.eye(idx.shape[1])[None]
            b = c[idx]
            beta = np.linalg.solve(A, b[..., None])[..., 0]
            vals[lo:lo + chunk] = yy - np.einsum("ij,ij->i", b, beta)
            # a binding box needs the exact solve; mark those supports
            bad = np.max(np.abs(beta), axis=1) > M
            for r in np.nonzero(bad)[0]:
                vals[lo + r] = _v_lsq_exact(X, y, list(idx[r]), lam2, M)[0]
        order = np.argsort(vals)[:max(top, 8)]
        exact = sorted((_v_lsq_exact(X, y, list(sups[r]), lam2, M)[0], sups[r]) for r in order)
        return exact[:top]
    out = sorted((_v_logistic_exact(X, y, list(S), lam2, M)[0], S) for S in sups)
    return out[:top]


def rashomon_set(X, y, k, lam2, M, kind, eps, N=None):
    """The support-level Rashomon set of §4.5 by its definition.

    R_eps = { S : |S| <= k, v(S) <= (1 + eps) Phi* } with v(S) from library
    routines (LAPACK / BVLS for least squares, L-BFGS-B for logistic) for every
    support of size 0..k, and Phi* = min over them.  With N, the N best members
    (the capped collection of §4.5).  Returns (Phi*, [(v, S)] ascending in v).
    """
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    p = X.shape[1]
    vals = []
    for size in range(0, k + 1):
        for S in itertools.combinations(range(p), size):
            if size == 0:
                v = objective(X, y, np.zeros(p), lam2, kind)
            elif kind == LSQ:
                v = _v_lsq_exact(X, y, list(S), lam2, M)[0]
            else:
                v = _v_logistic_exact(X, y, list(S), lam2, M)[0]
            vals.append((v, tuple(S)))
    vals.sort()
    phi = vals[0][0]
    R = [(v, S) for v, S in vals if v <= (1.0 + eps) * phi]
    if N is not None:
        R = R[:N]
    return phi, R
