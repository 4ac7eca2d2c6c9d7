"""GPU: the batched product G = R X (kglm_xtr) against an FP64 product of the same inputs."""

import numpy as np
import pytest

from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu


SHAPES = [(1024, 2000, 200), (37, 301, 150), (1, 5, 3), (300, 4000, 130), (129, 700, 300)]
# relative rounding of one operand: FP32 exact here; BF16 round-to-nearest 2^-8; TF32 (truncated) 2^-10
OPERAND_U = {"fp32": 0.0, "bf16": 2.0 ** -8, "tf32": 2.0 ** -10}


@pytest.mark.parametrize("prec", ["fp32", "bf16", "tf32"])
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
