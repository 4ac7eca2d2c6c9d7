"""GPU: kglm_xtr_noalloc_f32, the product G = R X for callers that cannot
allocate device memory (inside graph capture, in a host application's own
pool, or in a process that must not grow once serving).  It must give what
the allocating entry point kglm_xtr gives, on two calls in a row (the shared
scratch keeps the previous call's partial tiles; its counters must be back at
zero).  This file is collected last so that a failure here comes after every
other test has run; it also passes on its own in a fresh process."""

import numpy as np
import pytest

from paper_2605_22188_gb300 import kglm, synth

pytestmark = pytest.mark.gpu


def _bound(R, X, n):
    # FP32 accumulation over n terms: |error| <= n * 2^-24 * sum |r||x|
    return n * 2.0 ** -24 * (np.abs(R.astype(np.float64)) @ np.abs(X.astype(np.float32).astype(np.float64)))


def test_noalloc_matches_kglm_xtr_on_two_calls():
    import torch
    m, n, p = 1024, 2000, 200
    X, y, _ = synth.instance(n, p, 5, synth.LOGISTIC, seed=3)
    Xt = torch.from_numpy(np.ascontiguousarray(X.T).astype(np.float32)).cuda()
    rng = np.random.default_rng(0)
    stream = torch.cuda.current_stream()
    with kglm.Engine(X, y, 5, 0.1, 2.0, synth.LOGISTIC, prec="fp32", max_batch=m) as eng:
        for call in range(2):
            R = rng.standard_normal((m, n)).astype(np.float32) * (1 + call)
            Rd = torch.from_numpy(R).cuda()
            G_ref = torch.empty((m, p), dtype=torch.float32, device="cuda")
            G_new = torch.full((m, p), float("nan"), dtype=torch.float32, device="cuda")
            kglm.kglm_xtr(eng.ctx, m, Rd.data_ptr(), G_ref.data_ptr())
            kglm.kglm_xtr_noalloc_f32(m, n, p, Rd.data_ptr(), Xt.data_ptr(), G_new.data_ptr(), stream.cuda_stream)
            stream.synchronize()
            a, b = G_ref.cpu().numpy().astype(np.float64), G_new.cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(b))
            assert np.all(np.abs(a - b) <= 2 * _bound(R, X, n)), "call %d" % call
        # nothing is allocated: device free memory is unchanged across further calls
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            kglm.kglm_xtr_noalloc_f32(m, n, p, Rd.data_ptr(), Xt.data_ptr(), G_new.data_ptr(), stream.cuda_stream)
        stream.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_ragged_sizes_and_limit():
    import torch
    m, n, p = 37, 301, 150
    X, y, _ = synth.instance(n, p, 3, synth.LSQ, seed=4)
    R = np.random.default_rng(1).standard_normal((m, n)).astype(np.float32)
    Rd = torch.from_numpy(R).cuda()
    Xt = torch.from_numpy(np.ascontiguousarray(X.T).astype(np.float32)).cuda()
    G = torch.empty((m, p), dtype=torch.float32, device="cuda")
    for _ in range(2):
        kglm.kglm_xtr_noalloc_f32(m, n, p, Rd.data_ptr(), Xt.data_ptr(), G.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        ref = R.astype(np.float64) @ X.astype(np.float32).astype(np.float64)
        assert np.all(np.abs(G.cpu().numpy() - ref) <= _bound(R, X, n) + 1e-30)
    # an output grid beyond the fixed scratch is refused before any launch
    with pytest.raises(kglm.KglmError) as ei:
        kglm.kglm_xtr_noalloc_f32(128 * 17, n, 128 * 16, Rd.data_ptr(), Xt.data_ptr(), G.data_ptr())
    assert ei.value.status == kglm.KGLM_EINVAL
