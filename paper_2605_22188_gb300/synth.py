"""Seeded synthetic inputs shaped like the paper's workloads (App. E.1).

This module serves both the CUDA path and the oracle and therefore holds none
of the method's arithmetic: only the data model and random fixing masks.

Data model (readings of App. E.1 where it is silent or garbled):

* rows x_i ~ N(0, Sigma), Sigma_jl = rho^|j-l|, drawn by the AR(1) recursion
  x_1 = e_1, x_j = rho x_{j-1} + sqrt(1 - rho^2) e_j, which has exactly that
  covariance;
* columns are centred and scaled to unit sample variance (||col||^2 = n);
* beta* has k nonzeros at 0-based positions floor((i+1) p / k) - 1,
  i = 0..k-1, each +-1 with a random sign;
* least squares: y = X beta* + eps with eps = e ||X beta*|| / (SNR ||e||),
  e ~ N(0, I), so that ||X beta*|| / ||eps|| = SNR exactly;
* logistic: P(y_i = +1) = 1 / (1 + exp(-x_i^T beta*)), y_i in {-1, +1}.
"""

import math

import numpy as np

LSQ = 0
LOGISTIC = 1


def design(n, p, rho, rng):
    """n x p Toeplitz-correlated Gaussian design, columns standardized (FP64, row-major)."""
    e = rng.standard_normal((n, p))
    X = np.empty((n, p))
    X[:, 0] = e[:, 0]
    c = math.sqrt(1.0 - rho * rho)
    for j in range(1, p):
        X[:, j] = rho * X[:, j - 1] + c * e[:, j]
    X -= X.mean(axis=0, keepdims=True)
    X /= np.sqrt((X * X).mean(axis=0, keepdims=True))
    return np.ascontiguousarray(X)


def beta_star(p, k, rng, signed=True):
    b = np.zeros(p)
    idx = [(i + 1) * p // k - 1 for i in range(k)]
    signs = rng.choice([-1.0, 1.0], size=k) if signed else np.ones(k)
    b[idx] = signs
    return b


def instance(n, p, k, kind, rho=0.5, snr=5.0, seed=0, signed=True):
    """(X, y, beta*) for one synthetic instance; every draw comes from ``seed``."""
    rng = np.random.default_rng(seed)
    X = design(n, p, rho, rng)
    b = beta_star(p, k, rng, signed)
    s = X @ b
    if kind == LSQ:
        e = rng.standard_normal(n)
        y = s + e * (np.linalg.norm(s) / (snr * np.linalg.norm(e)))
    else:
        prob = 1.0 / (1.0 + np.exp(-s))
        y = np.where(rng.random(n) < prob, 1.0, -1.0)
    return X, np.ascontiguousarray(y), b


def random_nodes(m, p, k, rng, max_out=None, max_in=None):
    """m random fixing patterns (J0, J1): |J1| ~ U{0..max_in}, |J0| ~ U{0..max_out}, disjoint, uniform positions.

    Returns CSR arrays (in_ptr, in_idx, out_ptr, out_idx) as int32, indices
    sorted within each node.
    """
    max_in = k if max_in is None else max_in
    max_out = p // 2 if max_out is None else max_out
    in_ptr = [0]
    out_ptr = [0]
    in_idx = []
    out_idx = []
    for _ in range(m):
        n1 = int(rng.integers(0, max_in + 1))
        n0 = int(rng.integers(0, max_out + 1))
        n0 = min(n0, p - n1)
        perm = rng.permutation(p)
        J1 = np.sort(perm[:n1])
        J0 = np.sort(perm[n1:n1 + n0])
        in_idx.extend(J1.tolist())
        out_idx.extend(J0.tolist())
        in_ptr.append(len(in_idx))
        out_ptr.append(len(out_idx))
    as32 = lambda a: np.asarray(a, dtype=np.int32)
    return as32(in_ptr), as32(in_idx), as32(out_ptr), as32(out_idx)


def csr_to_sets(in_ptr, in_idx, out_ptr, out_idx):
    """Per-node (J0, J1) lists from CSR arrays."""
    m = len(in_ptr) - 1
    return [(list(map(int, out_idx[out_ptr[b]:out_ptr[b + 1]])),
             list(map(int, in_idx[in_ptr[b]:in_ptr[b + 1]]))) for b in range(m)]


def sets_to_csr(nodes):
    """CSR arrays from a list of (J0, J1)."""
    in_ptr, out_ptr, in_idx, out_idx = [0], [0], [], []
    for J0, J1 in nodes:
        in_idx.extend(sorted(J1))
        out_idx.extend(sorted(J0))
        in_ptr.append(len(in_idx))
        out_ptr.append(len(out_idx))
    as32 = lambda a: np.asarray(a, dtype=np.int32)
    return as32(in_ptr), as32(in_idx), as32(out_ptr), as32(out_idx)


# The five workloads, with the sizes and distributions of the paper's synthetic
# benchmark (App. E.1) at the shapes of the engine's configurations.
CONFIGS = {
    "c1_lsq_n200_p30_k5": dict(n=200, p=30, k=5, kind=LSQ, lam2=1e-3, M=2.0, rho=0.5, snr=5.0),
    "c2_logistic_n2000_p200_k10": dict(n=2000, p=200, k=10, kind=LOGISTIC, lam2=1e-2, M=2.0, rho=0.5, snr=5.0, m=1024),
    "c3_lsq_n5000_p1000_k15": dict(n=5000, p=1000, k=15, kind=LSQ, lam2=1e-3, M=2.0, rho=0.9, snr=3.0, m=4096),
    "c4_micro_n10000_p2000_k20": dict(n=10000, p=2000, k=20, kind=LSQ, lam2=1e-3, M=2.0, rho=0.5, snr=5.0, m=8192, T=50),
}


def config_instance(name, seed=0, kind=None):
    c = dict(CONFIGS[name])
    kind = c["kind"] if kind is None else kind
    X, y, b = instance(c["n"], c["p"], c["k"], kind, rho=c["rho"], snr=c["snr"], seed=seed)
    c["kind"] = kind
    return c, X, y, b


def serving_specs(count=64, seed=0):
    """Instance descriptions of the serving mix: loss uniform over {least squares,
    logistic}, p log-uniform on [100, 2000], n log-uniform on [5p, 10p], k uniform
    on {5..20}, Toeplitz rho in {0.5, 0.7, 0.9}, SNR in {3, 5}; lambda2 1e-3
    (least squares) or 1e-2 (logistic), M = 2.  Each spec carries its own data
    seed; instance(**spec) draws the data when the request is submitted."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kind = LSQ if rng.random() < 0.5 else LOGISTIC
        p = int(round(math.exp(rng.uniform(math.log(100), math.log(2000)))))
        n = int(round(math.exp(rng.uniform(math.log(5 * p), math.log(10 * p)))))
        k = int(rng.integers(5, 21))
        rho = float(rng.choice([0.5, 0.7, 0.9]))
        snr = float(rng.choice([3.0, 5.0]))
        out.append(dict(n=n, p=p, k=k, kind=kind, rho=rho, snr=snr, seed=int(seed * 1000 + i),
                        lam2=1e-3 if kind == LSQ else 1e-2, M=2.0))
    return out


def poisson_arrivals(count, rate, seed=0):
    """Arrival times (seconds from 0) of a Poisson stream with `rate` requests per second."""
    rng = np.random.default_rng(seed + 7919)
    return np.cumsum(rng.exponential(1.0 / rate, size=count)) if rate > 0 else np.zeros(count)
