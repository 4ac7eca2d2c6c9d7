"""ctypes binding of libkglm.so (include/kglm.h): argument marshalling only.

Every step of the node-bound path runs in the CUDA library; this module only
converts numpy arrays to pointers and status codes to exceptions.  There is no
CPU fallback: if the library is missing, ``lib()`` raises.
"""

import ctypes as C
import os

import numpy as np

from . import build as _build

KGLM_OK, KGLM_EINVAL, KGLM_ENOMEM, KGLM_ECUDA, KGLM_ETIMEOUT, KGLM_ESTATE, KGLM_ENUMERIC = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "ESTATE", -6: "ENUMERIC"}
LSQ, LOGISTIC = 0, 1
FP64, FP32, BF16, TF32, TF32X3 = 0, 1, 2, 3, 4
PREC = {"fp64": FP64, "fp32": FP32, "bf16": BF16, "tf32": TF32, "tf32x3": TF32X3}
MAX_K = 64


class kglm_desc(C.Structure):
    _fields_ = [
        ("n", C.c_int64), ("p", C.c_int64), ("k", C.c_int32), ("loss", C.c_int32),
        ("prec", C.c_int32), ("restart", C.c_int32), ("lambda2", C.c_double), ("M", C.c_double),
        ("lipschitz", C.c_double), ("gap_tol", C.c_double), ("max_batch", C.c_int32),
        ("pool_slots", C.c_int32), ("hbm_budget", C.c_int64), ("open_cap", C.c_int64),
    ]


class KglmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_LIB = None
P = C.c_void_p
D = C.POINTER(C.c_double)
I32 = C.POINTER(C.c_int32)
I64 = C.POINTER(C.c_int64)
U8 = C.POINTER(C.c_uint8)

_SIGS = {
    "kglm_create": (C.c_int, [C.POINTER(kglm_desc), D, D, P, C.POINTER(P)]),
    "kglm_push_nodes": (C.c_int, [P, C.c_int32, I32, I32, I32, I32, I32, D]),
    "kglm_evaluate": (C.c_int, [P, C.c_int32, C.c_int32, D, D, D, I32, D, I32, I32]),
    "kglm_read_batch": (C.c_int, [P, D, D]),
    "kglm_save_warm": (C.c_int, [P, C.c_int32, I32, I32]),
    "kglm_set_incumbent": (C.c_int, [P, C.c_double]),
    "kglm_prune": (C.c_int, [P, C.c_double, U8, I32]),
    "kglm_branch": (C.c_int, [P, C.c_double, I32, I32, I32]),
    "kglm_solve": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, C.c_double, D, I32, D, D, I64, I64]),
    "kglm_solve_device": (C.c_int, [P, C.c_int32, C.c_int32, C.c_int32, C.c_double, D, I32, D, D, I64, I64]),
    "kglm_last_error": (C.c_char_p, [P]),
    "kglm_destroy": (None, [P]),
    "kglm_version": (C.c_char_p, []),
    "kglm_push_nodes_dev": (C.c_int, [P, C.c_int32, P, P, P, P, C.c_int32, C.c_int32, P]),
    "kglm_stats_enable": (C.c_int, [P, C.c_int32]),
    "kglm_stats_read": (C.c_int, [P, D, I64, D]),
    "kglm_phase_name": (C.c_char_p, [C.c_int32]),
    "kglm_xtr": (C.c_int, [P, C.c_int32, P, P]),
    "kglm_xtz": (C.c_int, [P, C.c_int32, P, P, P]),
    "kglm_xtr_noalloc_f32": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, P, P, P, P]),
    "kglm_estimate_bytes": (C.c_int, [C.POINTER(kglm_desc), I64]),
    "kglm_device_bytes": (C.c_int, [P, I64]),
    "kglm_suggest_batch": (C.c_int, [C.POINTER(kglm_desc), C.c_int64, C.c_int32, C.POINTER(C.c_int32)]),
    "kglm_autotune": (C.c_int, [P, C.c_int32, C.c_uint64, C.c_void_p]),
    "kglm_configure": (C.c_int, [P, C.c_void_p]),
    "kglm_selftest_timeout": (C.c_int, [P, C.c_int32]),
    "kglm_checks_enabled": (C.c_int32, []),
    "kglm_selftest_checks": (C.c_int, [P]),
    "kglm_set_solve_limit": (C.c_int, [P, C.c_int64]),
    "kglm_solve_checkpoint": (C.c_int, [P, C.c_char_p]),
    "kglm_solve_resume": (C.c_int, [P, C.c_char_p, C.c_int32, C.c_int32, C.c_int32, C.c_double, D, I32, D, D, I64,
                                    I64]),
    "kglm_pool_create": (C.c_int, [C.c_int32, C.POINTER(P)]),
    "kglm_pool_insert": (C.c_int, [P, C.c_int32, I32, D, C.c_double, I64]),
    "kglm_pool_size": (C.c_int, [P, I64, I64, I64]),
    "kglm_pool_read": (C.c_int, [P, I64, D, D, I32, I32, I32]),
    "kglm_pool_support": (C.c_int, [P, C.c_int64, I32, I32]),
    "kglm_pool_filter": (C.c_int, [P, C.c_double, C.c_int64]),
    "kglm_pool_destroy": (None, [P]),
    "kglm_rashomon": (C.c_int, [P, C.c_double, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_double, P, D, I64,
                                C.POINTER(C.c_int32)]),
    "kglm_server_create": (C.c_int, [C.c_void_p, C.POINTER(P)]),
    "kglm_server_submit": (C.c_int, [P, C.POINTER(kglm_desc), D, D, I64]),
    "kglm_server_info": (C.c_int, [P, C.c_int64, C.c_void_p]),
    "kglm_server_wait": (C.c_int, [P, C.c_int64, C.c_double, C.c_void_p]),
    "kglm_server_drain": (C.c_int, [P, C.c_double]),
    "kglm_server_stats": (C.c_int, [P, C.c_void_p]),
    "kglm_server_last_error": (C.c_char_p, [P]),
    "kglm_server_destroy": (None, [P]),
}
class kglm_server_desc(C.Structure):
    _fields_ = [("hbm_budget", C.c_int64), ("max_active", C.c_int32), ("batch_cap", C.c_int32),
                ("iters", C.c_int32), ("check_every", C.c_int32), ("time_limit_s", C.c_double),
                ("open_cap", C.c_int64)]


class kglm_request_info(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("opt", C.c_double), ("gap", C.c_double),
                ("support", C.c_int32 * MAX_K), ("nodes", C.c_int64), ("batches", C.c_int64),
                ("device_bytes", C.c_int64), ("batch", C.c_int32), ("reserved", C.c_int32),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("message", C.c_char * 128)]


class kglm_server_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("finished", C.c_int64), ("queued", C.c_int64),
                ("active", C.c_int32), ("peak_active", C.c_int32), ("bytes_in_use", C.c_int64),
                ("peak_bytes", C.c_int64), ("budget", C.c_int64), ("elapsed_s", C.c_double),
                ("rounds", C.c_int64), ("round_batches", C.c_int64), ("shared_launches", C.c_int64)]


REQ_QUEUED, REQ_RUNNING, REQ_DONE, REQ_FAILED, REQ_CANCELLED = 0, 1, 2, 3, 4


class kglm_tune(C.Structure):
    _fields_ = [("batch", C.c_int32), ("link_tile_cols", C.c_int32), ("grad_tile_cols", C.c_int32),
                ("grad_split_cap", C.c_int32), ("timed", C.c_int32), ("pdl", C.c_int32),
                ("sub_batches", C.c_int32), ("prox_threads", C.c_int32), ("pair", C.c_int32),
                ("nodes_per_s", C.c_double), ("best_nodes_per_s", C.c_double)]
XTR_NOALLOC_MAX_TILES = 256
NPHASE = 11


def lib_path():
    """The normal library, or the bounds-checked one when KGLM_CHECKS=1 is set."""
    return _build.LIB_CHECKS if os.environ.get("KGLM_CHECKS") == "1" else _build.LIB


def lib():
    """The loaded libkglm.so; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            how = "build(checks=True)" if path == _build.LIB_CHECKS else "build()"
            raise RuntimeError("%s is not built; run paper_2605_22188_gb300.build.%s" % (path, how))
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def _ptr(a, t):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError("expected shape %s, got %s" % (shape, a.shape))
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _check(st, ctx):
    if st != KGLM_OK:
        raise KglmError(st, lib().kglm_last_error(ctx).decode())


# ------------------------------------------------------------------ C-named calls

def kglm_version():
    return lib().kglm_version().decode()


def make_desc(n, p, k, lambda2, M, loss, prec="fp64", max_batch=1024, lipschitz=0.0, gap_tol=0.0,
              restart=True, pool_slots=0, hbm_budget=0, open_cap=0):
    return kglm_desc(n=int(n), p=int(p), k=int(k), loss=int(loss), prec=PREC.get(prec, prec),
                     restart=int(bool(restart)), lambda2=float(lambda2), M=float(M), lipschitz=float(lipschitz),
                     gap_tol=float(gap_tol), max_batch=int(max_batch), pool_slots=int(pool_slots),
                     hbm_budget=int(hbm_budget), open_cap=int(open_cap))


def kglm_estimate_bytes(desc):
    """Device bytes kglm_create would allocate for a kglm_desc (host arithmetic only)."""
    b = C.c_int64()
    st = lib().kglm_estimate_bytes(C.byref(desc), C.byref(b))
    if st != KGLM_OK:
        raise KglmError(st, "kglm_estimate_bytes: desc rejected")
    return b.value


def kglm_device_bytes(ctx):
    b = C.c_int64()
    _check(lib().kglm_device_bytes(ctx, C.byref(b)), ctx)
    return b.value


def kglm_suggest_batch(desc, budget, cap=1 << 16):
    """Largest power-of-two batch <= cap whose instance fits in `budget` device bytes (App. E.4)."""
    m = C.c_int32()
    st = lib().kglm_suggest_batch(C.byref(desc), int(budget), int(cap), C.byref(m))
    if st != KGLM_OK:
        raise KglmError(st, "kglm_suggest_batch: no batch fits %d bytes" % budget if st == KGLM_ENOMEM
                        else "kglm_suggest_batch: bad arguments")
    return m.value


def kglm_create(X, y, k, lambda2, M, loss, prec="fp64", max_batch=1024, lipschitz=0.0, gap_tol=0.0,
                restart=True, pool_slots=0, hbm_budget=0, stream=None, open_cap=0):
    X = _f64(X)
    n, p = X.shape
    y = _f64(y, (n,))
    d = make_desc(n, p, k, lambda2, M, loss, prec, max_batch, lipschitz, gap_tol, restart, pool_slots, hbm_budget,
                  open_cap)
    out = P()
    st = lib().kglm_create(C.byref(d), _ptr(X, D), _ptr(y, D), P(stream) if stream else None, C.byref(out))
    _check(st, None)
    return out


def kglm_push_nodes(ctx, in_ptr, in_idx, out_ptr, out_idx, warm_slot=None, warm_B=None):
    in_ptr, in_idx, out_ptr, out_idx = map(_i32, (in_ptr, in_idx, out_ptr, out_idx))
    m = len(in_ptr) - 1
    ws = None if warm_slot is None else _i32(warm_slot)
    wb = None if warm_B is None else _f64(warm_B)
    st = lib().kglm_push_nodes(ctx, m, _ptr(in_ptr, I32), _ptr(in_idx, I32), _ptr(out_ptr, I32),
                               _ptr(out_idx, I32), _ptr(ws, I32), _ptr(wb, D))
    _check(st, ctx)
    return m


def kglm_push_nodes_dev(ctx, m, in_ptr, in_idx, out_ptr, out_idx, nnz_in, nnz_out, warm_slot=0):
    """Device-pointer variant: the arguments are integer device addresses (e.g. torch tensor.data_ptr())."""
    st = lib().kglm_push_nodes_dev(ctx, int(m), P(in_ptr), P(in_idx or None), P(out_ptr), P(out_idx or None),
                                   int(nnz_in), int(nnz_out), P(warm_slot or None))
    _check(st, ctx)
    return int(m)


def kglm_xtr(ctx, m, R_ptr, G_ptr):
    """G = R X for device buffers (integer addresses) of the context's working type."""
    _check(lib().kglm_xtr(ctx, int(m), P(R_ptr), P(G_ptr)), ctx)


def kglm_xtz(ctx, Z, p):
    """Certificate product Q = Z X (host FP64, Z: m x n) and its entrywise error bound."""
    Z = np.ascontiguousarray(Z, dtype=np.float64)
    m = Z.shape[0]
    Q = np.empty((m, p))
    E = np.empty((m, p))
    _check(lib().kglm_xtz(ctx, int(m), Z.ctypes.data, Q.ctypes.data, E.ctypes.data), ctx)
    return Q, E


def kglm_xtr_noalloc_f32(m, n, p, R_ptr, Xt_ptr, G_ptr, stream=None):
    """G = R X with no device allocation (device addresses; asynchronous on `stream`)."""
    st = lib().kglm_xtr_noalloc_f32(int(m), int(n), int(p), P(R_ptr), P(Xt_ptr), P(G_ptr),
                                    P(stream) if stream else None)
    if st != KGLM_OK:
        raise KglmError(st, "kglm_xtr_noalloc_f32 failed (m=%d, n=%d, p=%d)" % (m, n, p))


def kglm_stats_enable(ctx, enable=True):
    _check(lib().kglm_stats_enable(ctx, int(bool(enable))), ctx)


def kglm_stats_read(ctx):
    ms = np.zeros(NPHASE)
    n = np.zeros(NPHASE, dtype=np.int64)
    work = np.zeros(NPHASE)
    _check(lib().kglm_stats_read(ctx, _ptr(ms, D), _ptr(n, I64), _ptr(work, D)), ctx)
    names = [lib().kglm_phase_name(i).decode() for i in range(NPHASE)]
    return {names[i]: dict(ms=float(ms[i]), launches=int(n[i]), work=float(work[i])) for i in range(NPHASE)}


def kglm_evaluate(ctx, m, k, iters, check_every=0):
    lb, primal, ub = np.empty(m), np.empty(m), np.empty(m)
    support = np.empty((m, k), dtype=np.int32)
    beta_re = np.empty((m, k))
    bj = np.empty(m, dtype=np.int32)
    done = np.empty(m, dtype=np.int32)
    st = lib().kglm_evaluate(ctx, int(iters), int(check_every), _ptr(lb, D), _ptr(primal, D), _ptr(ub, D),
                             _ptr(support, I32), _ptr(beta_re, D), _ptr(bj, I32), _ptr(done, I32))
    _check(st, ctx)
    return dict(lb=lb, primal=primal, ub=ub, support=support, beta_re=beta_re, branch_j=bj, iters_done=done)


def kglm_read_batch(ctx, m, n, p, beta=True, zeta=True):
    B = np.empty((m, p)) if beta else None
    Z = np.empty((m, n)) if zeta else None
    _check(lib().kglm_read_batch(ctx, _ptr(B, D), _ptr(Z, D)), ctx)
    return B, Z


def kglm_save_warm(ctx, rows, slots):
    rows, slots = _i32(rows), _i32(slots)
    _check(lib().kglm_save_warm(ctx, len(rows), _ptr(rows, I32), _ptr(slots, I32)), ctx)


def kglm_set_incumbent(ctx, ub):
    _check(lib().kglm_set_incumbent(ctx, float(ub)), ctx)


def kglm_prune(ctx, m, ub):
    pruned = np.empty(m, dtype=np.uint8)
    ns = C.c_int32()
    _check(lib().kglm_prune(ctx, float(ub), _ptr(pruned, U8), C.byref(ns)), ctx)
    return pruned, ns.value


def kglm_branch(ctx, m, ub):
    parent = np.empty(m, dtype=np.int32)
    j = np.empty(m, dtype=np.int32)
    cnt = C.c_int32()
    _check(lib().kglm_branch(ctx, float(ub), _ptr(parent, I32), _ptr(j, I32), C.byref(cnt)), ctx)
    return parent[:cnt.value].copy(), j[:cnt.value].copy()


def kglm_solve(ctx, k, p, batch, iters, check_every=10, time_limit=0.0, device_queue=False):
    opt, gap = C.c_double(), C.c_double()
    nodes, batches = C.c_int64(), C.c_int64()
    sup = np.empty(k, dtype=np.int32)
    beta = np.empty(p)
    fn = lib().kglm_solve_device if device_queue else lib().kglm_solve
    st = fn(ctx, int(batch), int(iters), int(check_every), float(time_limit), C.byref(opt),
                          _ptr(sup, I32), _ptr(beta, D), C.byref(gap), C.byref(nodes), C.byref(batches))
    _check(st, ctx)
    return dict(opt=opt.value, support=[int(s) for s in sup if s >= 0], beta=beta, gap=gap.value,
                nodes=nodes.value, batches=batches.value)


def kglm_set_solve_limit(ctx, max_batches):
    _check(lib().kglm_set_solve_limit(ctx, int(max_batches)), ctx)


def kglm_solve_checkpoint(ctx, path):
    _check(lib().kglm_solve_checkpoint(ctx, os.fsencode(path)), ctx)


def kglm_solve_resume(ctx, path, k, p, batch, iters, check_every=10, time_limit=0.0):
    opt, gap = C.c_double(), C.c_double()
    nodes, batches = C.c_int64(), C.c_int64()
    sup = np.empty(k, dtype=np.int32)
    beta = np.empty(p)
    st = lib().kglm_solve_resume(ctx, os.fsencode(path), int(batch), int(iters), int(check_every), float(time_limit),
                                 C.byref(opt), _ptr(sup, I32), _ptr(beta, D), C.byref(gap), C.byref(nodes),
                                 C.byref(batches))
    _check(st, ctx)
    return dict(opt=opt.value, support=[int(s) for s in sup if s >= 0], beta=beta, gap=gap.value,
                nodes=nodes.value, batches=batches.value)


def kglm_autotune(ctx, iters=20, seed=1):
    """Tile shapes and batch size picked by timing (see kglm.h); returns the choice."""
    t = kglm_tune()
    _check(lib().kglm_autotune(ctx, int(iters), int(seed), C.byref(t)), ctx)
    return {f: getattr(t, f) for f, _ in t._fields_}


def kglm_configure(ctx, batch=0, link_tile_cols=0, grad_tile_cols=0, grad_split_cap=0, pdl=0, sub_batches=0,
                   prox_threads=0, pair=0):
    """Set tile shapes, split cap, batch, launch mode, sub-batches, prox threads and CTA pairs by hand."""
    t = kglm_tune(batch=batch, link_tile_cols=link_tile_cols, grad_tile_cols=grad_tile_cols,
                  grad_split_cap=grad_split_cap, pdl=pdl, sub_batches=sub_batches, prox_threads=prox_threads,
                  pair=pair)
    _check(lib().kglm_configure(ctx, C.byref(t)), ctx)


def kglm_selftest_timeout(ctx, rounds=10000):
    """Runs a bounded device wait that nothing ends; returns the status (KGLM_ETIMEOUT expected)."""
    return lib().kglm_selftest_timeout(ctx, int(rounds))


def checks_enabled():
    """True for the bounds-checked build (KGLM_CHECKS=1 in the environment selects it)."""
    return bool(lib().kglm_checks_enabled())


def kglm_selftest_checks(ctx):
    """A checked out-of-range write; returns the status (KGLM_EINVAL in the checked build)."""
    return lib().kglm_selftest_checks(ctx)


def kglm_destroy(ctx):
    if ctx:
        lib().kglm_destroy(ctx)


class Engine:
    """One instance (X, y, k, lambda2, M, loss) on the GPU; thin wrapper over the calls above."""

    def __init__(self, X, y, k, lambda2, M, loss, **kw):
        X = np.asarray(X)
        self.n, self.p = X.shape
        self.k = int(k)
        self.m = 0
        self.ctx = kglm_create(X, y, k, lambda2, M, loss, **kw)

    def push(self, in_ptr, in_idx, out_ptr, out_idx, warm_slot=None, warm_B=None):
        self.m = kglm_push_nodes(self.ctx, in_ptr, in_idx, out_ptr, out_idx, warm_slot, warm_B)
        return self.m

    def push_dev(self, m, in_ptr, in_idx, out_ptr, out_idx, nnz_in, nnz_out, warm_slot=0):
        self.m = kglm_push_nodes_dev(self.ctx, m, in_ptr, in_idx, out_ptr, out_idx, nnz_in, nnz_out, warm_slot)
        return self.m

    def stats_enable(self, enable=True):
        kglm_stats_enable(self.ctx, enable)

    def stats(self):
        return kglm_stats_read(self.ctx)

    def evaluate(self, iters, check_every=0):
        return kglm_evaluate(self.ctx, self.m, self.k, iters, check_every)

    def xtz(self, Z):
        return kglm_xtz(self.ctx, Z, self.p)

    def read_batch(self, beta=True, zeta=True):
        return kglm_read_batch(self.ctx, self.m, self.n, self.p, beta, zeta)

    def save_warm(self, rows, slots):
        kglm_save_warm(self.ctx, rows, slots)

    def set_incumbent(self, ub):
        kglm_set_incumbent(self.ctx, ub)

    def prune(self, ub):
        return kglm_prune(self.ctx, self.m, ub)

    def branch(self, ub):
        return kglm_branch(self.ctx, self.m, ub)

    def device_bytes(self):
        return kglm_device_bytes(self.ctx)

    def autotune(self, iters=20, seed=1):
        return kglm_autotune(self.ctx, iters, seed)

    def configure(self, **kw):
        kglm_configure(self.ctx, **kw)

    def rashomon(self, eps, max_models=0, batch=0, iters=200, check_every=10, time_limit=0.0):
        """The support-level Rashomon set (§4.5) as a Pool plus (opt, nodes, complete)."""
        pool = Pool(self.p)
        info = kglm_rashomon(self.ctx, pool, eps, max_models, batch, iters, check_every, time_limit)
        return pool, info

    def solve(self, batch, iters, check_every=10, time_limit=0.0):
        return kglm_solve(self.ctx, self.k, self.p, batch, iters, check_every, time_limit)

    def solve_device(self, batch, iters, check_every=10, time_limit=0.0):
        """kglm_solve_device: the open-node queue stays on the device (needs open_cap > 0)."""
        return kglm_solve(self.ctx, self.k, self.p, batch, iters, check_every, time_limit, device_queue=True)

    def set_solve_limit(self, max_batches):
        kglm_set_solve_limit(self.ctx, max_batches)

    def checkpoint(self, path):
        kglm_solve_checkpoint(self.ctx, path)

    def resume(self, path, batch, iters, check_every=10, time_limit=0.0):
        return kglm_solve_resume(self.ctx, path, self.k, self.p, batch, iters, check_every, time_limit)

    def close(self):
        if self.ctx:
            kglm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving loop

def _info_dict(i):
    return dict(state=i.state, status=i.status, opt=i.opt, gap=i.gap,
                support=[int(x) for x in i.support if x >= 0], nodes=i.nodes, batches=i.batches,
                device_bytes=i.device_bytes, batch=i.batch, t_submit=i.t_submit, t_admit=i.t_admit,
                t_done=i.t_done, message=i.message.decode(errors="replace"))


class Server:
    """kglm_server_*: certified solves of many instances admitted as they arrive."""

    def __init__(self, max_active=8, hbm_budget=0, iters=200, check_every=10, time_limit_s=0.0, batch_cap=0,
                 open_cap=0):
        d = kglm_server_desc(hbm_budget=int(hbm_budget), max_active=int(max_active), batch_cap=int(batch_cap),
                             iters=int(iters), check_every=int(check_every), time_limit_s=float(time_limit_s),
                             open_cap=int(open_cap))
        out = P()
        st = lib().kglm_server_create(C.byref(d), C.byref(out))
        if st != KGLM_OK:
            raise KglmError(st, "kglm_server_create failed")
        self.s = out

    def submit(self, X, y, k, lambda2, M, loss, prec="bf16", max_batch=0, lipschitz=0.0, gap_tol=0.0,
               restart=True, pool_slots=0):
        X = _f64(X)
        n, p = X.shape
        y = _f64(y, (n,))
        d = make_desc(n, p, k, lambda2, M, loss, prec, 1, lipschitz, gap_tol, restart, pool_slots, 0)
        d.max_batch = int(max_batch)
        rid = C.c_int64()
        st = lib().kglm_server_submit(self.s, C.byref(d), _ptr(X, D), _ptr(y, D), C.byref(rid))
        if st != KGLM_OK:
            raise KglmError(st, lib().kglm_server_last_error(self.s).decode())
        return rid.value

    def info(self, rid):
        i = kglm_request_info()
        st = lib().kglm_server_info(self.s, int(rid), C.byref(i))
        if st != KGLM_OK:
            raise KglmError(st, "unknown request %d" % rid)
        return _info_dict(i)

    def wait(self, rid, timeout=0.0):
        i = kglm_request_info()
        st = lib().kglm_server_wait(self.s, int(rid), float(timeout), C.byref(i))
        if st != KGLM_OK:
            raise KglmError(st, "wait for request %d" % rid)
        return _info_dict(i)

    def drain(self, timeout=0.0):
        st = lib().kglm_server_drain(self.s, float(timeout))
        if st != KGLM_OK:
            raise KglmError(st, "drain")

    def stats(self):
        t = kglm_server_stats_t()
        _check(lib().kglm_server_stats(self.s, C.byref(t)), None)
        return {f: getattr(t, f) for f, _ in t._fields_}

    def close(self):
        if self.s:
            lib().kglm_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ Rashomon pool (App. G layout)

class Pool:
    """kglm_pool_*: supports in a trie of included features, coefficients cut by offsets."""

    def __init__(self, p):
        out = P()
        st = lib().kglm_pool_create(int(p), C.byref(out))
        if st != KGLM_OK:
            raise KglmError(st, "kglm_pool_create")
        self.q = out
        self.p = int(p)

    def insert(self, seq, coef, objective):
        seq = _i32(seq)
        coef = _f64(coef)
        r = C.c_int64()
        st = lib().kglm_pool_insert(self.q, len(seq), _ptr(seq, I32), _ptr(coef, D), float(objective), C.byref(r))
        if st != KGLM_OK:
            raise KglmError(st, "kglm_pool_insert")
        return r.value

    def size(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        lib().kglm_pool_size(self.q, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def read(self):
        R, V, NC = self.size()
        off = np.empty(R + 1, dtype=np.int64)
        coef = np.empty(NC)
        obj = np.empty(R)
        leaf = np.empty(R, dtype=np.int32)
        parent = np.empty(V, dtype=np.int32)
        label = np.empty(V, dtype=np.int32)
        st = lib().kglm_pool_read(self.q, _ptr(off, I64), _ptr(coef, D), _ptr(obj, D), _ptr(leaf, I32),
                                  _ptr(parent, I32), _ptr(label, I32))
        if st != KGLM_OK:
            raise KglmError(st, "kglm_pool_read")
        return dict(offsets=off, coef=coef, objective=obj, leaf=leaf, parent=parent, label=label)

    def support(self, record):
        buf = np.empty(max(self.p, 1), dtype=np.int32)
        n = C.c_int32()
        st = lib().kglm_pool_support(self.q, int(record), _ptr(buf, I32), C.byref(n))
        if st != KGLM_OK:
            raise KglmError(st, "kglm_pool_support")
        return buf[:n.value].tolist()

    def filter(self, threshold, keep_best=0):
        st = lib().kglm_pool_filter(self.q, float(threshold), int(keep_best))
        if st != KGLM_OK:
            raise KglmError(st, "kglm_pool_filter")

    def records(self):
        """[(objective, support as a sorted tuple, coefficients in label order, labels)] in record order."""
        d = self.read()
        out = []
        for r in range(len(d["leaf"])):
            lab = self.support(r)
            out.append((float(d["objective"][r]), tuple(sorted(lab)),
                        d["coef"][d["offsets"][r]:d["offsets"][r + 1]].copy(), lab))
        return out

    def close(self):
        if self.q:
            lib().kglm_pool_destroy(self.q)
            self.q = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kglm_rashomon(ctx, pool, eps, max_models=0, batch=0, iters=200, check_every=10, time_limit=0.0):
    opt = C.c_double()
    nodes = C.c_int64()
    comp = C.c_int32()
    st = lib().kglm_rashomon(ctx, float(eps), int(max_models), int(batch), int(iters), int(check_every),
                             float(time_limit), pool.q, C.byref(opt), C.byref(nodes), C.byref(comp))
    _check(st, ctx)
    return dict(opt=opt.value, nodes=nodes.value, complete=bool(comp.value))
