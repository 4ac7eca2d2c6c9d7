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
