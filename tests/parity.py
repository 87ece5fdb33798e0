"""Helpers shared by the GPU parity tests: GPU pole records -> per-realisation lists, and
the parity-set comparison against the oracle.

Parity set: for every true mode r and every model order n >= 2 * n_modes, take in each
result the pole of mode r: among the HC-passing poles within 5 % of f_r, the one whose
shape is closest (largest MAC) to the generating mode shape phi_r (nearest in frequency
when no shape is given).  When both results have one, gate relative frequency
(<= 1e-4), absolute damping (<= 2e-3) and MAC between the two shapes (>= 0.999).
Noise poles that happen to sit near f_r are thereby not mistaken for the mode.
"""
import numpy as np

import oracle as O

F_TOL, XI_TOL, MAC_MIN = 1e-4, 2e-3, 0.999


def gpu_cells(rec, phi, lags, orders, l):
    """Split flat GPU records into cells[t][m] = dict(f, xi, mu, Phi, mpc, mpd, flags)."""
    phi = np.asarray(phi, dtype=np.float32).reshape(-1, l, 2)
    slots = sum(n // 2 for n in orders)
    cells = []
    for t in range(len(lags)):
        row, off = [], t * slots
        for n in orders:
            sl = slice(off, off + n // 2)
            r = rec[sl]
            valid = (r["flags"] & 64) != 0
            ph = phi[sl][valid]
            row.append(dict(f=r["f_hz"][valid].astype(np.float64), xi=r["xi"][valid].astype(np.float64),
                            mu=(r["mu_re"] + 1j * r["mu_im"])[valid], mpc=r["mpc"][valid],
                            mpd=r["mpd"][valid], flags=r["flags"][valid],
                            Phi=(ph[..., 0] + 1j * ph[..., 1]).T))
            off += n // 2
        cells.append(row)
    return cells


def nearest(cell, f0, phi0=None, hc_only=True):
    f = cell["f"]
    ok = np.ones(len(f), bool)
    if hc_only and "flags" in cell:
        ok &= (np.asarray(cell["flags"]) & 8) != 0
    cand = np.where(ok & (np.abs(f - f0) < 0.05 * f0))[0]
    if len(cand) == 0:
        return None
    if phi0 is not None:
        macs = [O.mac(cell["Phi"][:, j], phi0) for j in cand]
        return int(cand[int(np.argmax(macs))])
    return int(cand[np.argmin(np.abs(f[cand] - f0))])


def separated_orders(orders, svals, ratio=2.0):
    """Orders n whose leading n-dimensional singular subspace is separated by a gap
    sigma_n / sigma_{n+1} >= ratio.  The poles of order n depend only on that subspace,
    so only these orders are reproducible between two computations of the SVD; beyond
    the physical rank the singular values of the estimation noise are nearly degenerate
    and each side may pick a different basis of the noise subspace."""
    return [n for n in orders if n < len(svals) and svals[n - 1] >= ratio * svals[n]]


def compare_parity_set(gpu, ora, f_true, orders, n_modes, min_matches=1, phi_true=None,
                       gate_orders=None):
    """Returns (n_compared, worst df, worst dxi, worst 1-MAC); asserts the gates."""
    worst = [0.0, 0.0, 0.0]
    where = [None, None, None]
    n_cmp = 0
    for t in range(len(gpu)):
        for m, n in enumerate(orders):
            if gate_orders is not None:
                if n not in gate_orders:
                    continue
            elif n < 2 * n_modes:
                continue
            for r, f0 in enumerate(f_true):
                phi0 = None if phi_true is None else phi_true[:, r]
                a = nearest(ora[t][m], f0, phi0)
                b = nearest(gpu[t][m], f0, phi0)
                if a is None or b is None:
                    continue
                fa, fb = ora[t][m]["f"][a], gpu[t][m]["f"][b]
                df = abs(fa - fb) / fa
                dxi = abs(ora[t][m]["xi"][a] - gpu[t][m]["xi"][b])
                mac = O.mac(ora[t][m]["Phi"][:, a], gpu[t][m]["Phi"][:, b])
                for q, v in enumerate((df, dxi, 1 - mac)):
                    if v > worst[q]:
                        worst[q], where[q] = v, (t, n, r, fa, fb)
                n_cmp += 1
    assert n_cmp >= min_matches, f"only {n_cmp} parity pairs"
    assert worst[0] <= F_TOL, f"frequency {worst[0]:.3e} at (lag, order, mode, f_ora, f_gpu) {where[0]}"
    assert worst[1] <= XI_TOL, f"damping {worst[1]:.3e} at {where[1]}"
    assert worst[2] <= 1 - MAC_MIN, f"1-MAC {worst[2]:.3e} at {where[2]}"
    return n_cmp, worst
