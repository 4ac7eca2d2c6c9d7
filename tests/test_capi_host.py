"""Host-side checks of the C ABI: the library loads, exports every declared
entry point, and rejects bad arguments before touching the GPU."""

import os
import re

import numpy as np
import pytest

from paper_2605_22188_gb300 import build, kglm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(build.LIB):
        build.build()
    return kglm.lib()


def declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            text = open(os.path.join(ROOT, "include", f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(kglm_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert "kglm_evaluate" in names and len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_version(lib):
    assert "sm_103a" in kglm.kglm_version()


def test_normal_build_is_not_the_checked_one(lib):
    # kglm_checks_enabled needs no device; the checked build is a separate library
    if os.environ.get("KGLM_CHECKS") == "1":
        pytest.skip("the bounds-checked library is selected")
    assert kglm.checks_enabled() is False
    assert kglm.lib_path().endswith("libkglm.so")


def _inst(n=20, p=6):
    rng = np.random.default_rng(0)
    return rng.standard_normal((n, p)), rng.standard_normal(n)


@pytest.mark.parametrize("kw,needle", [
    (dict(k=0), "k must"),
    (dict(k=7), "k must"),
    (dict(lambda2=0.0), "lambda2"),
    (dict(M=-1.0), "M must"),
    (dict(loss=5), "unknown loss"),
    (dict(max_batch=0), "max_batch"),
    (dict(prec=5), "unknown precision"),
])
def test_create_rejects_bad_arguments(lib, kw, needle):
    X, y = _inst()
    args = dict(k=2, lambda2=0.1, M=2.0, loss=kglm.LSQ)
    args.update(kw)
    with pytest.raises(kglm.KglmError) as ei:
        kglm.kglm_create(X, y, **args)
    assert ei.value.status == kglm.KGLM_EINVAL and needle in str(ei.value)


def test_create_rejects_bad_labels_and_nan(lib):
    X, y = _inst()
    with pytest.raises(kglm.KglmError) as ei:
        kglm.kglm_create(X, y, 2, 0.1, 2.0, kglm.LOGISTIC)
    assert ei.value.status == kglm.KGLM_EINVAL
    X[3, 2] = np.nan
    with pytest.raises(kglm.KglmError) as ei:
        kglm.kglm_create(X, np.sign(y), 2, 0.1, 2.0, kglm.LOGISTIC)
    assert ei.value.status == kglm.KGLM_ENUMERIC


def test_null_context_calls(lib):
    assert lib.kglm_push_nodes(None, 1, None, None, None, None, None, None) == kglm.KGLM_EINVAL
    assert lib.kglm_evaluate(None, 1, 0, None, None, None, None, None, None, None) == kglm.KGLM_EINVAL
    lib.kglm_destroy(None)


def test_estimate_bytes_grows_with_the_batch_and_counts_the_instance(lib):
    """The footprint is host arithmetic: it needs no GPU.  It must grow with the
    batch capacity and cover at least the FP64 copies of X and X^T and the
    batch's m x n FP64 dual points."""
    n, p = 2000, 200
    prev = 0
    for m in (1, 64, 1024, 4096):
        for prec in ("fp64", "fp32", "bf16", "tf32"):
            b = kglm.kglm_estimate_bytes(kglm.make_desc(n, p, 10, 1e-2, 2.0, kglm.LOGISTIC, prec, m))
            assert b >= 2 * 8 * n * p + 8 * m * n
        b64 = kglm.kglm_estimate_bytes(kglm.make_desc(n, p, 10, 1e-2, 2.0, kglm.LOGISTIC, "fp64", m))
        assert b64 > prev
        prev = b64


def test_suggest_batch_is_the_largest_fitting_power_of_two(lib):
    """App. E.4: the batch is the largest power of two whose instance fits the budget."""
    d = kglm.make_desc(5000, 1000, 15, 1e-3, 2.0, kglm.LSQ, "bf16", 1)
    for budget in (1 << 30, 1 << 32, 1 << 34):
        m = kglm.kglm_suggest_batch(d, budget, cap=1 << 16)
        assert m >= 1 and (m & (m - 1)) == 0
        d.max_batch = m
        assert kglm.kglm_estimate_bytes(d) <= budget
        if m < (1 << 16):
            d.max_batch = 2 * m
            assert kglm.kglm_estimate_bytes(d) > budget
        d.max_batch = 1
    with pytest.raises(kglm.KglmError) as ei:
        kglm.kglm_suggest_batch(d, 1 << 20)          # X alone needs 80 MB
    assert ei.value.status == kglm.KGLM_ENOMEM
    bad = kglm.make_desc(5000, 1000, 0, 1e-3, 2.0, kglm.LSQ, "bf16", 1)
    with pytest.raises(kglm.KglmError) as ei:
        kglm.kglm_estimate_bytes(bad)
    assert ei.value.status == kglm.KGLM_EINVAL


def test_server_rejects_bad_descriptions_before_touching_the_gpu(lib):
    import ctypes as C
    for kw in (dict(max_active=0), dict(max_active=1000), dict(iters=0), dict(check_every=-1),
               dict(hbm_budget=-5), dict(batch_cap=-1)):
        base = dict(hbm_budget=0, max_active=2, batch_cap=0, iters=10, check_every=0, time_limit_s=0.0)
        base.update(kw)
        d = kglm.kglm_server_desc(**base)
        out = C.c_void_p()
        assert lib.kglm_server_create(C.byref(d), C.byref(out)) == kglm.KGLM_EINVAL, kw
        assert not out.value
    # calls on a null server
    assert lib.kglm_server_drain(None, 0.0) == kglm.KGLM_EINVAL
    assert lib.kglm_server_info(None, 1, None) == kglm.KGLM_EINVAL
    lib.kglm_server_destroy(None)


@pytest.mark.parametrize("loss", [kglm.LSQ, kglm.LOGISTIC])
def test_suggest_batch_rounds_a_capacity_near_two_to_the_sixteen(lib, loss):
    """App. E.4's example: a safe capacity slightly above 2^16 nodes gives a batch of
    65536, one slightly below gives 32768 (the largest power of two not above it)."""
    d = kglm.make_desc(1000, 500, 10, 1e-3, 2.0, loss, "bf16", 1 << 16)
    need = kglm.kglm_estimate_bytes(d)
    d.max_batch = 1
    assert kglm.kglm_suggest_batch(d, need + 4096, cap=1 << 20) == 1 << 16
    assert kglm.kglm_suggest_batch(d, need - 1, cap=1 << 20) == 1 << 15
