"""Helpers shared by the GPU parity tests: GPU pole records -> per-realisation lists, and
the parity-set comparison against the oracle.

Parity set: for every true mode r and every model order n >= 2 * n_modes, take in each
result the HC-passing pole nearest to f_r (within 5 % of f_r); when both exist, gate
relative frequency (<= 1e-4), absolute damping (<= 2e-3) and MAC (>= 0.999).
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


def nearest(cell, f0, hc_only=True):
    f = cell["f"]
    ok = np.ones(len(f), bool)
    if hc_only and "flags" in cell:
        ok &= (np.asarray(cell["flags"]) & 8) != 0
    cand = np.where(ok & (np.abs(f - f0) < 0.05 * f0))[0]
    if len(cand) == 0:
        return None
    return int(cand[np.argmin(np.abs(f[cand] - f0))])


def compare_parity_set(gpu, ora, f_true, orders, n_modes, min_matches=1):
    """Returns (n_compared, worst df, worst dxi, worst 1-MAC); asserts the gates."""
    worst = [0.0, 0.0, 0.0]
    n_cmp = 0
    for t in range(len(gpu)):
        for m, n in enumerate(orders):
            if n < 2 * n_modes:
                continue
            for f0 in f_true:
                a = nearest(ora[t][m], f0)
                b = nearest(gpu[t][m], f0)
                if a is None or b is None:
                    continue
                fa, fb = ora[t][m]["f"][a], gpu[t][m]["f"][b]
                df = abs(fa - fb) / fa
                dxi = abs(ora[t][m]["xi"][a] - gpu[t][m]["xi"][b])
                mac = O.mac(ora[t][m]["Phi"][:, a], gpu[t][m]["Phi"][:, b])
                worst = [max(worst[0], df), max(worst[1], dxi), max(worst[2], 1 - mac)]
                n_cmp += 1
    assert n_cmp >= min_matches, f"only {n_cmp} parity pairs"
    assert worst[0] <= F_TOL, f"frequency {worst[0]:.3e}"
    assert worst[1] <= XI_TOL, f"damping {worst[1]:.3e}"
    assert worst[2] <= 1 - MAC_MIN, f"1-MAC {worst[2]:.3e}"
    return n_cmp, worst
