"""The pair bookkeeping of the sliding-window covariances, on the host.

The GPU stream updates the window's unnormalised lag sums S_k with segment sums
F(seg) = (len - k) R_k(seg): F([e-T, e+B)) - F([e-T, e)) for the pairs that enter and
F([s, s+D+T)) - F([s+D, s+D+T)) for those that leave, with T = max_lag + 1.  Here the same
algebra runs on the oracle's FP64 covariances and must give the window's own lag sums to
rounding, for ragged blocks, a window that fills and slides, and the smallest window.
T = max_lag would already hold every pair (T = max_lag + 1 only keeps each segment longer
than max_lag, as the covariance call requires); a planted T = max_lag - 1 must break it.
"""
import numpy as np

import oracle as O


def _F(Y, a, n, K):
    """Lag sums of the segment [a, a + n): (n - k) R_k from the oracle, zero for lags the
    segment is too short to hold."""
    if n > K:
        return O.covariances(Y[:, a:a + n], K) * (n - np.arange(1, K + 1))[:, None, None]
    out = np.zeros((K, Y.shape[0], Y.shape[0]))
    if n > 1:
        out[:n - 1] = _F(Y, a, n, n - 1)
    return out


def _stream(Y, K, W, blocks, T):
    S, start, n, e = None, 0, 0, 0
    for B in blocks:
        e = start + n
        if n == 0:
            S = _F(Y, e, B, K)
        else:
            S = S + _F(Y, e - T, T + B, K) - _F(Y, e - T, T, K)
        n += B
        if n > W:
            D = n - W
            S = S - _F(Y, start, D + T, K) + _F(Y, start + D, T, K)
            start += D
            n = W
        yield S, start, n


def _check(Y, K, W, blocks, T, tol=1e-10):
    worst = 0.0
    for S, start, n in _stream(Y, K, W, blocks, T):
        ref = _F(Y, start, n, K)
        worst = max(worst, np.abs(S - ref).max() / np.abs(ref).max())
    return worst


def _record(l=3, N=3000, seed=2):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((l, N))
    for t in range(1, N):                      # some memory so the lags matter
        x[:, t] += 0.7 * x[:, t - 1]
    return x


def test_stream_bookkeeping_reproduces_window_sums():
    Y = _record()
    K = 7
    assert _check(Y, K, 400, [50, 13, 97, 8, 120, 61, 33, 200, 9, 77, 150, 31] * 2, K + 1) < 1e-12


def test_stream_bookkeeping_smallest_window():
    Y = _record(N=600)
    K = 5
    assert _check(Y, K, K + 1, [K + 1] * 40, K + 1) < 1e-12


def test_stream_bookkeeping_needs_the_full_lag_overlap():
    """With T = max_lag - 1 the pairs at the largest lag straddling a block edge are lost."""
    Y = _record()
    K = 7
    assert _check(Y, K, 400, [50, 13, 97, 8, 120, 61, 33, 200], K - 1) > 1e-3
