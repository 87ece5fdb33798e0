"""The FP32 MAC screen of the clustering kernels and its error bound, on the host.

The kernels compute MAC(a, b) = |a^H b|^2 / (|a|^2 |b|^2) in FP32 with lanes over channels
(channel c on lane c mod 32, each lane a chain of FMAs), a 5-level shuffle tree, and the
final products in FP32, and trust it to within eps(l) = 2 (5 gamma + 4 u), gamma =
(2 ceil(l/32) + 5) u, u = 2^-24, of the exact value.  Decisions closer than that are taken
again in FP64.  This emulates the same operation order in NumPy (an FMA as an exact FP64
product and sum rounded once to FP32, which can differ from a true FMA by one ulp on
rare ties, far inside the factor 2 of the bound) and checks the bound on random and
nearly parallel unit vectors.
"""
import numpy as np
import pytest

import oracle as O

f32 = np.float32


def _fma(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def _mac32(a, b):
    l = len(a)
    acc = np.zeros((32, 4), dtype=np.float32)
    for lane in range(32):
        dr = di = na = nb = f32(0)
        for c in range(lane, l, 32):
            xr, xi, yr, yi = f32(a[c].real), f32(a[c].imag), f32(b[c].real), f32(b[c].imag)
            dr = _fma(xr, yr, _fma(xi, yi, dr))
            di = _fma(xr, yi, _fma(-xi, yr, di))
            na = _fma(xr, xr, _fma(xi, xi, na))
            nb = _fma(yr, yr, _fma(yi, yi, nb))
        acc[lane] = (dr, di, na, nb)
    for o in (16, 8, 4, 2, 1):
        acc = (acc + acc[np.arange(32) ^ o]).astype(np.float32)
    dr, di, na, nb = acc[0]
    den = f32(na * nb)
    return float(f32(f32(dr * dr) + f32(di * di)) / den)


def _eps(l):
    u = 2.0 ** -24
    gamma = (2 * ((l + 31) // 32) + 5) * u
    return 2 * (5 * gamma + 4 * u)


def _unit(rng, l):
    v = rng.standard_normal(l) + 1j * rng.standard_normal(l)
    return (v / np.linalg.norm(v)).astype(np.complex64)


@pytest.mark.parametrize("l", [4, 24, 186, 512])
def test_fp32_mac_screen_within_its_bound(l):
    rng = np.random.Generator(np.random.PCG64(l))
    worst = 0.0
    for trial in range(12):
        a = _unit(rng, l)
        if trial % 3 == 0:
            b = _unit(rng, l)                                   # unrelated
        else:
            s = 10.0 ** -rng.uniform(1, 6)                      # nearly parallel
            b = (a * np.exp(1j * rng.uniform(0, 2 * np.pi)) + s * _unit(rng, l)).astype(np.complex64)
        exact = O.mac(a.astype(np.complex128), b.astype(np.complex128))
        worst = max(worst, abs(_mac32(a, b) - exact))
    assert worst <= _eps(l), (worst, _eps(l))
    # the bound is not vacuous: the screen's error is of the order of a few ulp
    assert worst < 1e-5
