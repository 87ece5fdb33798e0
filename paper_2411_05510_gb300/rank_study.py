"""Calibration of the minimum RSVD rank (Sec. 3.1, parametric analysis; Eq. empirical_formula).

Sec. 3.1 finds, for a given record and Toeplitz size T = l * j_b, the smallest rank k
(as a percentage of T) at which the modes identified with the RSVD agree with those
identified with the SVD; Eq. (empirical_formula) fits a line to those minima over T and
noise levels, and the paper notes that a structure may need its own calibration.  This
module runs that search on the GPU path for one record and one j_b:

  * reference: the identification with the SVD of T (the range finder at full width,
    K = T, no power iterations: Q spans the whole column space, so the K x K SVD of
    P = Q^T T is the SVD of T);
  * candidates: the RSVD with K = ceil(pct * T / 100) columns and q power iterations
    (default 1), for pct along an increasing grid, until the first one whose modes match
    the reference's.  Sec. 3.1 does not state q.  With q = 0 the damping of the clustered
    modes never settles within 1 % of the SVD's (on the 10-DOF frame at 20 dB and
    j_b = 100 it still differs by 5 % at K = T / 2), while one power iteration brings it
    within 0.4 % at 15 %; so the search runs with q = 1;
  * identification: the 2D stabilization diagram of the orders (hard and soft criteria),
    then the two-stage clustering of its stable poles into modes (ssi_cluster);
  * match: every reference mode of interest has a candidate mode within the matching
    tolerances (relative frequency, relative damping, 1 - MAC of the medoids' shapes;
    Sec. 3.1 uses 1 %, 1 % and 2 %; a tolerance of None leaves that quantity out).  The
    modes of interest are the reference modes nearest
    (within 5 %) to the frequencies the caller names -- the structure's modes, e.g. the
    generating model's in a synthetic study -- or, when none are named, every reference
    mode (the lists must then also have the same length).  Spurious clusters of the SVD's
    diagram come from its noise subspace, which no rank-k approximation reproduces, so a
    study over the structure's modes names them.

Every step runs in libssi's kernels; this module only chooses the calls and compares the
mode tables it gets back (a few numbers per mode).
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np
import torch

from . import api as A

__all__ = ["identify", "modes_match", "match_of", "modes_of_interest", "damping_differences",
           "minimum_rank", "rank_grid"]


def rank_grid(lo: float = 2.5, hi: float = 50.0, step: float = 2.5):
    """Percentages lo, lo + step, ..., hi."""
    n = int(round((hi - lo) / step)) + 1
    return [round(lo + j * step, 6) for j in range(n)]


def identify(ctx: A.Context, Y: torch.Tensor, fs: float, jb: int, orders: Sequence[int], K: int,
             stab=None, cluster=None, prec: str = "split_bf16", small: str = "fp32", seed: int = 1,
             q: int = 1):
    """Modes of the 2D diagram of `orders` at time-lag step jb from a range finder of K
    columns and q power iterations (none at K = T, where the range finder is exact).
    Returns a list of dicts f_hz, xi, size, phi (the medoid's shape)."""
    l = Y.shape[0]
    n_max = max(orders)
    stab = stab or A.stab_params(a_f=0.02, a_xi=0.02, a_mac=0.05, use_lag_axis=False)
    cluster = cluster or A.cluster_params(tau=0.05, min_size=max(3, len(orders) // 5))
    qq = 0 if K >= l * jb else q
    desc = A.job_desc(Y, fs, [jb], orders, k=n_max, oversample=K - n_max, q=qq, prec=prec, seed=seed,
                      stab=stab, small=small)
    poles, phi, _ = A.ssi_solve(ctx, desc, device=Y.device, with_s=False)
    modes, _, _ = A.ssi_cluster(ctx, 1, orders, l, poles, phi, cluster)
    A.check_sync(ctx, Y.device)
    ph = phi.view(-1, l, 2).cpu().numpy().astype(np.float64)
    out = []
    for m in modes:
        v = ph[m["medoid_slot"]]
        out.append(dict(f_hz=m["f_hz"], xi=m["xi"], size=m["size"], phi=v[:, 0] + 1j * v[:, 1]))
    return out


def _mac(a, b) -> float:
    den = np.vdot(a, a).real * np.vdot(b, b).real
    return float(abs(np.vdot(a, b)) ** 2 / den) if den > 0 else 0.0


def modes_of_interest(ref, f_names):
    """The reference modes nearest (within 5 %) to each named frequency, once each."""
    out = []
    for f0 in f_names:
        best = None
        for r in ref:
            d = abs(r["f_hz"] - f0) / f0
            if d < 0.05 and (best is None or d < best[0]):
                best = (d, r)
        if best is not None and all(best[1] is not o for o in out):
            out.append(best[1])
    return out


def modes_match(ref, cand, tol=(0.01, 0.01, 0.02), f_names=None) -> bool:
    """Every reference mode of interest (all of them, with equal counts, when f_names is
    None) has a candidate mode within the tolerances: |df| / f, |dxi| / xi (denominators
    the larger value) and 1 - MAC."""
    if f_names is None:
        if len(ref) != len(cand):
            return False
    else:
        ref = modes_of_interest(ref, f_names)
    if not ref:
        return False
    for r in ref:
        if match_of(r, cand, tol) is None:
            return False
    return True


def match_of(r, cand, tol=(0.01, 0.01, 0.02)):
    """The candidate mode matching reference mode r within tol (None entries are not
    compared), the nearest in frequency among several; None if none does."""
    best = None
    for c in cand:
        df = abs(r["f_hz"] - c["f_hz"]) / max(r["f_hz"], c["f_hz"])
        dxi = abs(r["xi"] - c["xi"]) / max(r["xi"], c["xi"])
        dm = 1.0 - _mac(r["phi"], c["phi"])
        if (tol[0] is None or df <= tol[0]) and (tol[1] is None or dxi <= tol[1]) and \
                (tol[2] is None or dm <= tol[2]):
            if best is None or df < best[0]:
                best = (df, dxi, dm, c)
    return best


def damping_differences(ref, cand, f_names, tol=(0.01, None, 0.02)):
    """Relative damping difference of each matched mode of interest (for the report)."""
    out = []
    for r in modes_of_interest(ref, f_names):
        m = match_of(r, cand, tol)
        if m is not None:
            out.append(m[1])
    return out


def minimum_rank(ctx: A.Context, Y: torch.Tensor, fs: float, jb: int, orders: Sequence[int],
                 grid: Sequence[float] | None = None, tol=(0.01, 0.01, 0.02), f_names=None, **kw):
    """Smallest percentage of T on `grid` whose RSVD identification matches the SVD's on
    the modes of interest (f_names, see modes_match).  Returns (kbar_pct or None,
    reference modes, trace of (pct, K, matched, n_modes, worst relative damping
    difference of the matched modes of interest))."""
    l = Y.shape[0]
    T = l * jb
    grid = list(grid or rank_grid())
    ref = identify(ctx, Y, fs, jb, orders, T, **kw)
    trace = []
    for pct in grid:
        K = max(max(orders), int(math.ceil(pct * T / 100.0 - 1e-9)))
        if K >= T:
            trace.append((pct, T, True, len(ref), 0.0))
            return pct, ref, trace
        cand = identify(ctx, Y, fs, jb, orders, K, **kw)
        ok = modes_match(ref, cand, tol, f_names)
        names = f_names if f_names is not None else [r["f_hz"] for r in ref]
        dxi = damping_differences(ref, cand, names, (tol[0], None, tol[2]))   # f and shape only
        trace.append((pct, K, ok, len(cand), round(max(dxi), 4) if dxi else None))
        if ok:
            return pct, ref, trace
    return None, ref, trace
