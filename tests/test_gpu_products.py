"""GPU: the batched product G = R X (kglm_xtr) against an FP64 product of the same inputs."""

import numpy as np
import pytest

from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu


SHAPES = [(1024, 2000, 200), (37, 301, 150), (1, 5, 3), (300, 4000, 130), (129, 700, 300)]
# relative rounding of one operand: FP32 exact here; BF16 round-to-nearest 2^-8; TF32 (truncated) 2^-10;
# TF32 hi + lo split: each operand to 2^-22, the dropped lo*lo term 2^-22 of the product, and X taken
# from FP64 (2^-24 from the FP32 copy of the reference): (1 + 2^-21)^2 - 1 > 3 2^-22 + 2^-24
OPERAND_U = {"fp32": 0.0, "bf16": 2.0 ** -8, "tf32": 2.0 ** -10, "tf32x3": 2.0 ** -21}


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32", "tf32x3"])
@pytest.mark.parametrize("m,n,p", SHAPES)
def test_xtr_matches_fp64_product(prec, m, n, p):
    """|G - R X| <= ((1+u)^2 - 1 + n 2^-24) sum |r||x| with u the operand rounding of the mode."""
    import torch
    rng = np.random.default_rng(m + n + p)
    X, y, _ = synth.instance(n, p, min(3, p), synth.LSQ, seed=1)
    R = rng.standard_normal((m, n)).astype(np.float32)
    with kglm.Engine(X, y, min(3, p), 0.1, 2.0, synth.LSQ, prec=prec, max_batch=m) as eng:
        Rd = torch.from_numpy(R).cuda()
        Gd = torch.full((m, p), float("nan"), dtype=torch.float32, device="cuda")
        kglm.kglm_xtr(eng.ctx, m, Rd.data_ptr(), Gd.data_ptr())
        G = Gd.cpu().numpy().astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    ref = R.astype(np.float64) @ X32
    scale = np.abs(R.astype(np.float64)) @ np.abs(X32)
    u = OPERAND_U[prec]
    tol = ((1 + u) ** 2 - 1 + n * 2.0 ** -24) * scale * 1.01 + 1e-30
    assert np.all(np.isfinite(G))
    assert np.all(np.abs(G - ref) <= tol), float(np.max(np.abs(G - ref) / tol))


def _exact_products(Z, X, rows, cols):
    """sum_i Z[b, i] X[i, j] in exact rational arithmetic for the given (b, j)."""
    from fractions import Fraction
    out = {}
    for b in rows:
        zb = [Fraction(float(v)) for v in Z[b]]
        for j in cols:
            out[(b, j)] = sum((zi * Fraction(float(xi)) for zi, xi in zip(zb, X[:, j]) if zi != 0), Fraction(0))
    return out


def _dual_rows(n, rng):
    """Dual points of assorted scales and structure: Gaussian, tiny, huge, zero,
    logistic-like in [-1, 1], one nonzero, mixed magnitudes, integers."""
    Z = np.zeros((9, n))
    Z[0] = rng.standard_normal(n)
    Z[1] = 1e-8 * rng.standard_normal(n)
    Z[2] = 1e6 * rng.standard_normal(n)
    Z[4] = rng.uniform(-1, 1, n)
    Z[5, n // 3] = -0.7
    Z[6] = rng.standard_normal(n) * np.where(np.arange(n) % 2, 1e-9, 1e3)
    Z[7] = rng.integers(-5, 6, n)
    Z[8] = np.float32(rng.standard_normal(n)).astype(np.float64)   # FP32-valued, as in the engine
    return Z


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "tf32", "tf32x3"])
def test_certificate_product_is_within_its_bound(prec):
    """kglm_xtz: |Q - Z X| <= Qerr entrywise against exact rational sums, and the
    bound of the reduced modes' exact-splitting product is tiny: at most
    2^-38 n max|X_j| max|Z_b| (6-bit digits, 7 per value)."""
    n, p = 300, 24
    rng = np.random.default_rng(11)
    X, y, _ = synth.instance(n, p, 3, synth.LSQ, seed=2)
    Z = _dual_rows(n, rng)
    with kglm.Engine(X, y, 3, 0.1, 2.0, synth.LSQ, prec=prec, max_batch=16) as eng:
        Q, E = eng.xtz(Z)
    ex = _exact_products(Z, X, range(Z.shape[0]), range(p))
    for (b, j), v in ex.items():
        d = abs(Q[b, j] - float(v))
        if prec == "fp64":
            assert E[b, j] == 0.0
            assert d <= 1e-12 * (np.abs(Z[b]) @ np.abs(X[:, j])) + 1e-300
        else:
            assert d <= E[b, j], (b, j, d, E[b, j])
            assert E[b, j] <= 2.0 ** -38 * n * 2 * np.max(np.abs(X[:, j])) * 2 * np.max(np.abs(Z[b])) + 1e-300


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_certificate_product_exact_at_the_accumulator_limit(sign):
    """Constant X and Z whose leading digits are both 64: level 2 of the split
    sums n 64^2 = 2^24 per job at n = 8192 (two jobs of 4096 samples), the
    largest integer the planner lets an FP32 accumulation reach.  The result
    must equal the exact product to within the (tiny) bound: an accumulator
    that dropped a unit there would miss by 2^-12 relative."""
    n, p, m = 8192, 16, 4
    X = np.full((n, p), 0.99999 * sign)
    X[:, 1::2] = 0.999999999                     # other digit patterns in odd columns
    y = np.linspace(-1, 1, n)
    Z = np.full((m, n), -0.99999)
    Z[1] = 0.999999999
    Z[2, ::2] = 0.5
    with kglm.Engine(X, y, 2, 0.1, 2.0, synth.LSQ, prec="bf16", max_batch=m) as eng:
        Q, E = eng.xtz(Z)
    ex = _exact_products(Z, X, range(m), range(4))
    for (b, j), v in ex.items():
        d = abs(Q[b, j] - float(v))
        assert d <= E[b, j], (b, j, d, E[b, j])
        assert E[b, j] <= 1e-7, E[b, j]


@pytest.mark.parametrize("m,n,p", [(1024, 2000, 200), (300, 4000, 130)])
def test_fp32_accurate_split_is_as_close_to_fp64_as_fp32_products(m, n, p):
    """The TF32 hi + lo products have the accuracy of FP32 products: against the
    FP64 product of the same FP32 inputs, their worst relative error (scaled by
    sum |r||x|) is within a small factor of the CUDA-core FP32 product's, and
    far below the single TF32 product's."""
    import torch
    rng = np.random.default_rng(m + p)
    X, y, _ = synth.instance(n, p, 3, synth.LSQ, seed=2)
    X = X.astype(np.float32).astype(np.float64)           # exactly representable in FP32
    R = rng.standard_normal((m, n)).astype(np.float32)
    ref = R.astype(np.float64) @ X
    scale = np.abs(R.astype(np.float64)) @ np.abs(X)
    err = {}
    for prec in ("fp32", "tf32", "tf32x3"):
        with kglm.Engine(X, y, 3, 0.1, 2.0, synth.LSQ, prec=prec, max_batch=m) as eng:
            Rd = torch.from_numpy(R).cuda()
            Gd = torch.zeros((m, p), dtype=torch.float32, device="cuda")
            kglm.kglm_xtr(eng.ctx, m, Rd.data_ptr(), Gd.data_ptr())
            G = Gd.cpu().numpy().astype(np.float64)
        err[prec] = float(np.max(np.abs(G - ref) / scale))
    print("max |G - RX| / (|R||X|):", err)
    assert err["tf32x3"] <= 4.0 * err["fp32"] + 2.0 ** -22
    assert err["tf32x3"] * 100.0 <= err["tf32"]
