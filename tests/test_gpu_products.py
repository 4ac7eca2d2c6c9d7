"""GPU: the batched product G = R X (kglm_xtr) against an FP64 product of the same inputs."""

import numpy as np
import pytest

from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,p", [(1024, 2000, 200), (37, 301, 150), (1, 5, 3), (300, 4000, 130)])
def test_xtr_fp32_matches_fp64_product(m, n, p):
    import torch
    rng = np.random.default_rng(m + n + p)
    X, y, _ = synth.instance(n, p, min(3, p), synth.LSQ, seed=1)
    R = rng.standard_normal((m, n)).astype(np.float32)
    with kglm.Engine(X, y, min(3, p), 0.1, 2.0, synth.LSQ, prec="fp32", max_batch=m) as eng:
        Rd = torch.from_numpy(R).cuda()
        Gd = torch.empty((m, p), dtype=torch.float32, device="cuda")
        kglm.kglm_xtr(eng.ctx, m, Rd.data_ptr(), Gd.data_ptr())
        G = Gd.cpu().numpy().astype(np.float64)
    X32 = X.astype(np.float32).astype(np.float64)
    ref = R.astype(np.float64) @ X32
    scale = np.abs(R.astype(np.float64)) @ np.abs(X32)
    # FP32 accumulation over n terms: |error| <= n * 2^-24 * sum |r||x| (a loose bound)
    assert np.all(np.abs(G - ref) <= n * 2.0 ** -24 * scale + 1e-30)
