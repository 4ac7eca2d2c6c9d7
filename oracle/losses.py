"""Scalar GLM losses, their derivatives and Fenchel conjugates, and H_M (FP64).

Test infrastructure only (see ``oracle/__init__.py``).

Readings of the paper used here:

* least squares: l(s, y) = (s - y)^2, no 1/2 and no 1/n, so that the ridge
  term is lambda2*||beta||^2 as in problem (intro_sparse_glm) of §1;
* logistic: y in {-1, +1}, l(s, y) = log(1 + exp(-y s)) (App. E.1 labels);
* H_M, only named in §3 Eq. (prelim_node_conjugate), is the Huber function
  with threshold M: the conjugate of 1/2 b^2 restricted to |b| <= M.
"""

import numpy as np
from scipy.special import expit, xlogy

LSQ = 0
LOGISTIC = 1


def loss(s, y, kind):
    """l(s_i, y_i) elementwise (§4.2: f(s, y) = sum_i l(s_i, y_i))."""
    s = np.asarray(s, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if kind == LSQ:
        return (s - y) ** 2
    if kind == LOGISTIC:
        return np.logaddexp(0.0, -y * s)
    raise ValueError(kind)


def dloss(s, y, kind):
    """d l / d s at (s_i, y_i): the entries R_{i,b} of §4.2 Eq. (gradient_matrix_form)."""
    s = np.asarray(s, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if kind == LSQ:
        return 2.0 * (s - y)
    if kind == LOGISTIC:
        return -y * expit(-y * s)
    raise ValueError(kind)


def loss_conj(w, y, kind):
    """l*(w, y) = sup_s  w*s - l(s, y), elementwise (§4.4 Eq. (batched_dual_value_component)).

    least squares: w*y + w^2/4.
    logistic:      a*ln(a) + (1-a)*ln(1-a) with a = -w*y in [0, 1] (0*ln 0 = 0),
                   +inf outside [0, 1].
    """
    w = np.asarray(w, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    if kind == LSQ:
        return w * y + 0.25 * w * w
    if kind == LOGISTIC:
        a = -w * y
        out = xlogy(a, a) + xlogy(1.0 - a, 1.0 - a)
        return np.where((a >= 0.0) & (a <= 1.0), out, np.inf)
    raise ValueError(kind)


def huber(q, M):
    """H_M(q) = q^2/2 for |q| <= M, M|q| - M^2/2 otherwise (§3 Eq. (prelim_node_conjugate))."""
    q = np.abs(np.asarray(q, dtype=np.float64))
    return np.where(q <= M, 0.5 * q * q, M * q - 0.5 * M * M)


def prox_huber(x, r, M):
    """prox_{r H_M}(x) = argmin_v 1/2 (v - x)^2 + r H_M(v), for r >= 0 (Algorithm 1, App. B).

    Inside the quadratic zone the minimiser is x/(1+r); once |x| > (1+r) M the
    linear zone applies and the minimiser is x - r*M*sign(x).
    """
    x = np.asarray(x, dtype=np.float64)
    ax = np.abs(x)
    inner = ax / (1.0 + r)
    outer = ax - r * M
    v = np.where(ax <= (1.0 + r) * M, inner, outer)
    return np.sign(x) * v
