"""Sliding-window covariances (ssi_cov_stream_*) against whole-window computations.

After every push, R of the stream's window must equal ssi_covariances of the same
samples within the stage (a) tolerance, 2e-5 of max|R| (both accumulate FP32 partials over
time chunks and add them in FP64; the stream's sums are differences of segment sums, so
only the rounding differs).  The blocks are ragged, the window fills, slides and wraps
around the ring, and at the end the FP64 oracle's covariances of the final window are met
within the same bound.
"""
import numpy as np
import pytest
import torch

import oracle as O
import ssi_synth as S

pytestmark = pytest.mark.gpu

TOL = 2e-5


@pytest.fixture(scope="module")
def P():
    import paper_2411_05510_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def rec():
    w = S.workload("bridge186_3d", l=24, modes=6, f_lo=4.0, N=60000, lags=[20], k=32,
                   oversample=16, orders=list(range(2, 33, 2)))
    Y, *_ = S.record(w, np.float32)
    return np.ascontiguousarray(Y)


def _err(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def _run(P, ctx, Y, K, W, Bmax, blocks, prec, every=1):
    Yd = torch.from_numpy(Y).cuda()
    st = P.CovStream(ctx, Y.shape[0], K, W, Bmax, prec)
    worst, t, pushes = 0.0, 0, 0
    try:
        for B in blocks:
            if t + B > Y.shape[1]:
                break
            st.push(Yd[:, t:t + B].contiguous())
            t += B
            pushes += 1
            if pushes % every:
                continue
            R, n = st.covariances()
            assert n == min(t, W)
            ref = P.ssi_covariances(ctx, Yd[:, t - n:t].contiguous(), K, prec)
            worst = max(worst, _err(R.cpu().numpy(), ref.cpu().numpy()))
        R, n = st.covariances()
        torch.cuda.synchronize()
        return R.cpu().numpy(), t, n, worst, pushes
    finally:
        st.close()


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_stream_matches_whole_window_after_every_push(P, ctx, rec, prec):
    """l = 24, max_lag 39, window 20000, ragged blocks up to 6001 samples: the window fills,
    slides and wraps the ring (26001 columns) several times."""
    sizes = [4000, 2500, 777, 6001, 1234, 5000, 41, 3333]
    blocks = [sizes[j % len(sizes)] for j in range(40)]
    R, t, n, worst, pushes = _run(P, ctx, rec, 39, 20000, 6001, blocks, prec)
    assert pushes >= 20 and t > 2 * 26001 and n == 20000
    assert worst < TOL, worst
    Ro = O.covariances(rec[:, t - n:t].astype(np.float64), 39)
    assert _err(R, Ro) < TOL


def test_stream_smallest_window_and_long_drift(P, ctx, rec):
    """Window of max_lag + 1 samples slid by whole windows; then 300 pushes of 150 samples
    through a 3000-sample window (the sums are updated 300 times and rebuilt from the ring
    after every 3000 samples pushed)."""
    K = 39
    _, _, n, worst, _ = _run(P, ctx, rec, K, K + 1, K + 1, [K + 1] * 30, "split_bf16")
    assert n == K + 1 and worst < TOL, worst
    R, t, n, worst, pushes = _run(P, ctx, rec, K, 3000, 150, [150] * 300, "split_bf16",
                                  every=50)
    assert pushes == 300 and n == 3000 and worst < TOL, worst
    Ro = O.covariances(rec[:, t - n:t].astype(np.float64), K)
    assert _err(R, Ro) < TOL


def test_stream_thousands_of_pushes_with_rebuilds(P, ctx):
    """3000 pushes of 50 samples through a 4000-sample window (75 windows; the ring of
    4050 columns wraps at almost every push).  The sums are rebuilt from the ring every
    4000 samples and, in between, whenever ssi_cov_stream_refresh is called; after each
    refresh and every 250 pushes R must equal ssi_covariances of the window, and the final
    window the FP64 oracle's covariances, within the stage (a) bound."""
    w = S.workload("bridge186_3d", l=24, modes=6, f_lo=4.0, N=150000 + 64, seed=11)
    Y, *_ = S.record(w, np.float32)
    Yd = torch.from_numpy(np.ascontiguousarray(Y)).cuda()
    K, W, B = 39, 4000, 50
    st = P.CovStream(ctx, 24, K, W, B, "split_bf16")
    worst, t = 0.0, 0
    try:
        for j in range(3000):
            st.push(Yd[:, t:t + B].contiguous())
            t += B
            if j % 37 == 36:
                st.refresh()
            if j % 37 == 36 or j % 250 == 249:
                R, n = st.covariances()
                ref = P.ssi_covariances(ctx, Yd[:, t - n:t].contiguous(), K, "split_bf16")
                worst = max(worst, _err(R.cpu().numpy(), ref.cpu().numpy()))
        R, n = st.covariances()
        R = R.cpu().numpy()
    finally:
        st.close()
    assert n == W and worst < TOL, worst
    Ro = O.covariances(Y[:, t - n:t].astype(np.float64), K)
    assert _err(R, Ro) < TOL


def test_stream_rejects_bad_calls(P, ctx, rec):
    Yd = torch.from_numpy(rec[:, :100].copy()).cuda()
    with pytest.raises(P.SsiError):
        P.CovStream(ctx, 24, 39, 39, 100)            # window must exceed max_lag
    st = P.CovStream(ctx, 24, 39, 1000, 100)
    try:
        with pytest.raises(P.SsiError):
            st.push(Yd[:, :39].contiguous())          # first block too short
        with pytest.raises(P.SsiError):
            st.covariances()                          # nothing in the window yet
        st.push(Yd)
        with pytest.raises(P.SsiError):
            st.push(torch.from_numpy(rec[:, :101].copy()).cuda())   # above max_block
        R, n = st.covariances()
        assert n == 100
    finally:
        st.close()


def test_monitoring_chain_from_the_stream(P, ctx, rec):
    """Continuous monitoring: the window's covariances from the stream feed the stage calls
    (Toeplitz RSVD per lag, realisations, stability) and the clustering.  The reduced bridge
    record has 6 generating modes in 4-20 Hz; after the window (40000 samples) has slid by
    20000, every mode must come out of the 3D diagram of lags 14, 18, 22 within 1 %."""
    import ssi_synth as S2
    w = S2.workload("bridge186_3d", l=24, modes=6, f_lo=4.0, N=60000, lags=[14, 18, 22], k=32,
                    oversample=16, orders=list(range(2, 33, 2)))
    _, f_true, *_ = S2.record(w, np.float32)
    Yd = torch.from_numpy(rec).cuda()
    l, K = rec.shape[0], 2 * max(w["lags"]) - 1
    st = P.CovStream(ctx, l, K, 40000, 5000)
    try:
        for j in range(12):
            st.push(Yd[:, j * 5000:(j + 1) * 5000].contiguous())
        R, n = st.covariances()
    finally:
        st.close()
    assert n == 40000
    Us = []
    for i in w["lags"]:
        U, _ = P.ssi_toeplitz_rsvd(ctx, R, l, i, w["k"], w["oversample"], w["q"], seed=5)
        Us.append(U)
    poles, phi = P.ssi_realize_batch(ctx, w["lags"], Us, l, w["k"], w["orders"], 1.0 / w["fs"])
    P.ssi_stabilize(ctx, len(w["lags"]), w["orders"], l, poles, phi)
    modes, info, _ = P.ssi_cluster(ctx, len(w["lags"]), w["orders"], l, poles, phi,
                                   P.cluster_params(min_size=10))
    P.check_sync(ctx)
    for f0 in f_true:
        assert any(abs(m["f_hz"] - f0) / f0 < 1e-2 for m in modes), (f0, modes, info)
