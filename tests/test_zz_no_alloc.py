"""GPU test of ssi_covariances_noalloc, the covariance entry point that allocates nothing.

Callers that cannot allocate device memory (inside a CUDA-graph capture, under a
framework that owns all device memory, under a fixed reservation) use this variant;
its scratch is a fixed 16 MiB device array inside the library.  The test calls it
through the C ABI on two different records in a row and checks each result against
the allocating entry point ssi_covariances (FP32 path) with the tolerance the
covariance tests use (2e-5 of max|R|).  It also checks the size limit is enforced.
This file is collected last so that a failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 2e-5


def _noalloc(P, Yd, max_lag):
    l, N = Yd.shape
    R = torch.empty((max_lag, l, l), dtype=torch.float64, device=Yd.device)
    st = P._lib.lib.ssi_covariances_noalloc(ctypes.c_void_p(Yd.data_ptr()), l, N, max_lag,
                                            ctypes.c_void_p(R.data_ptr()),
                                            ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    P._lib.check(st, "ssi_covariances_noalloc")
    return R


def test_noalloc_matches_allocating_entry_point_twice():
    import paper_2411_05510_gb300 as P
    ctx = P.Context(0)
    rng = np.random.default_rng(2024)
    cases = [(20, 30000, 24), (48, 12345, 33)]   # two different records, one after the other
    for l, N, max_lag in cases:
        Y = (rng.standard_normal((l, N)) * rng.uniform(0.5, 2.0, (l, 1))).astype(np.float32)
        Yd = torch.from_numpy(Y).cuda()
        Rn = _noalloc(P, Yd, max_lag)
        Ra = P.ssi_covariances(ctx, Yd, max_lag, "fp32")
        torch.cuda.synchronize()
        a, b = Rn.cpu().numpy(), Ra.cpu().numpy()
        err = np.abs(a - b).max() / np.abs(b).max()
        assert err < TOL, (l, N, max_lag, err)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_2411_05510_gb300 as P
    Yd = torch.zeros((186, 2000), dtype=torch.float32, device="cuda")
    # 119 lags x 192^2 floats > 4 Mi floats of scratch
    with pytest.raises(P._lib.SsiError, match="scratch"):
        _noalloc(P, Yd, 119)
