"""Parity of stage (a), the lag-covariance GEMMs, against the FP64 oracle.

Tolerance: both precisions accumulate FP32 partial sums over at most 8192
samples and add the partials in FP64.  Split BF16 represents every sample to
~2^-17 relative; with FP32 rounding on sums of <= 8192 terms the error of each
R_k entry stays below ~1e-5 of the largest |R| (errors scale with the variance,
not with the entry).  The bound used is 2e-5 * max|R|.
"""
import numpy as np
import pytest
import torch

import oracle as O
import ssi_synth as S

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def ctx():
    import paper_2411_05510_gb300 as P
    c = P.Context(0)
    yield c
    c.close()


def _gpu_R(ctx, Y, max_lag, prec):
    import paper_2411_05510_gb300 as P
    Yd = torch.from_numpy(np.ascontiguousarray(Y, dtype=np.float32)).cuda()
    R = P.ssi_covariances(ctx, Yd, max_lag, prec)
    torch.cuda.synchronize()
    return R.cpu().numpy()


def _check(Rg, Ro):
    scale = np.abs(Ro).max()
    err = np.abs(Rg - Ro).max() / scale
    assert err < TOL, f"max error {err:.3e} of max|R|"


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
@pytest.mark.parametrize("l,N,max_lag", [
    (4, 20000, 39),        # the 4-channel chain record
    (70, 5017, 9),         # two channel tiles with padding, ragged time, ragged last unit
    (1, 2, 1),             # degenerate: one channel, one product
    (300, 3000, 5),        # two N tiles of the tensor-core kernel
    (64, 9000, 64),        # exactly one channel atom, lags spanning many units
])
def test_covariances_match_oracle(ctx, prec, l, N, max_lag):
    rng = np.random.default_rng(l * 1000 + N)
    if l == 4 and N == 20000:
        Y, *_ = S.record(S.workload("chain4_tiny"))
    else:
        Y = rng.standard_normal((l, N)) * rng.uniform(0.5, 2.0, (l, 1))
    Y = Y.astype(np.float32)
    Ro = O.covariances(Y.astype(np.float64), max_lag)
    _check(_gpu_R(ctx, Y, max_lag, prec), Ro)


def test_covariances_precisions_agree_on_record(ctx):
    Y, *_ = S.record(S.workload("chain4_tiny"))
    a = _gpu_R(ctx, Y, 39, "split_bf16")
    b = _gpu_R(ctx, Y, 39, "fp32")
    assert np.abs(a - b).max() / np.abs(b).max() < TOL


def test_covariances_full_size_sampled(ctx):
    """186 channels, N = 360000, lags 1..119 (the bridge workload), checked on sampled entries."""
    w = S.workload("bridge186_i60")
    Y, *_ = S.record(w, np.float32)
    Rg = _gpu_R(ctx, Y, 119, "split_bf16")
    rng = np.random.default_rng(0)
    scale = max(abs(O.covariance_entry(Y, 1, a, a)) for a in range(0, 186, 5))
    worst = 0.0
    for _ in range(300):
        k = int(rng.integers(1, 120))
        a, b = (int(x) for x in rng.integers(0, 186, 2))
        worst = max(worst, abs(Rg[k - 1, a, b] - O.covariance_entry(Y, k, a, b)) / scale)
    assert worst < TOL, worst


def test_covariances_rejects_bad_shapes(ctx):
    import paper_2411_05510_gb300 as P
    Y = torch.zeros((4, 10), dtype=torch.float32, device="cuda")
    with pytest.raises(P._lib.SsiError):
        P.ssi_covariances(ctx, Y, 10)          # max_lag must be < N
    with pytest.raises(P._lib.SsiError):
        P.ssi_covariances(ctx, Y, 0)
