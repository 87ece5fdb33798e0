"""Calibration of the minimum RSVD rank (Sec. 3.1, parametric analysis; Eq. empirical_formula).

Sec. 3.1 finds, for a given record and Toeplitz size T = l * j_b, the smallest rank k
(as a percentage of T) at which the modes identified with the RSVD agree with those
identified with the SVD; Eq. (empirical_formula) fits a line to those minima over T and
noise levels, and the paper notes that a structure may need its own calibration.  This
module runs that search on the GPU path for one record and one j_b:

  * reference: the identification with the SVD of T (the range finder at full width,
    K = T, no power iterations: Q spans the whole column space, so the K x K SVD of
    P = Q^T T is the SVD of T);
  * candidates: the RSVD with K = ceil(pct * T / 100) columns, q = 0, for pct along an
    increasing grid, until the first one whose modes match the reference's;
  * identification: the 2D stabilization diagram of the orders (hard and soft criteria),
    then the two-stage clustering of its stable poles into modes (ssi_cluster);
  * match: the two mode lists have the same length and every reference mode has a mode
    within the matching tolerances (relative frequency, relative damping, 1 - MAC of the
    medoids' shapes; Sec. 3.1 uses 1 %, 1 % and 2 %).

Every step runs in libssi's kernels; this module only chooses the calls and compares the
mode tables it gets back (a few numbers per mode).
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np
import torch

from . import api as A

__all__ = ["identify", "modes_match", "minimum_rank", "rank_grid"]


def rank_grid(lo: float = 2.5, hi: float = 50.0, step: float = 2.5):
    """Percentages lo, lo + step, ..., hi."""
    n = int(round((hi - lo) / step)) + 1
    return [round(lo + j * step, 6) for j in range(n)]


def identify(ctx: A.Context, Y: torch.Tensor, fs: float, jb: int, orders: Sequence[int], K: int,
             stab=None, cluster=None, prec: str = "split_bf16", small: str = "fp32", seed: int = 1):
    """Modes of the 2D diagram of `orders` at time-lag step jb from a range finder of K
    columns (q = 0).  Returns a list of dicts f_hz, xi, size, phi (the medoid's shape)."""
    l = Y.shape[0]
    n_max = max(orders)
    stab = stab or A.stab_params(a_f=0.02, a_xi=0.02, a_mac=0.05, use_lag_axis=False)
    cluster = cluster or A.cluster_params(tau=0.05, min_size=max(3, len(orders) // 5))
    desc = A.job_desc(Y, fs, [jb], orders, k=n_max, oversample=K - n_max, q=0, prec=prec, seed=seed,
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


def modes_match(ref, cand, tol=(0.01, 0.01, 0.02)) -> bool:
    """Same number of modes, and every reference mode has a candidate mode within the
    tolerances: |df| / f, |dxi| / xi (denominators the larger value) and 1 - MAC."""
    if len(ref) != len(cand) or not ref:
        return False
    for r in ref:
        ok = False
        for c in cand:
            df = abs(r["f_hz"] - c["f_hz"]) / max(r["f_hz"], c["f_hz"])
            dxi = abs(r["xi"] - c["xi"]) / max(r["xi"], c["xi"])
            if df <= tol[0] and dxi <= tol[1] and 1.0 - _mac(r["phi"], c["phi"]) <= tol[2]:
                ok = True
                break
        if not ok:
            return False
    return True


def minimum_rank(ctx: A.Context, Y: torch.Tensor, fs: float, jb: int, orders: Sequence[int],
                 grid: Sequence[float] | None = None, tol=(0.01, 0.01, 0.02), **kw):
    """Smallest percentage of T on `grid` whose RSVD identification matches the SVD's.
    Returns (kbar_pct or None, reference modes, trace of (pct, K, matched, n_modes))."""
    l = Y.shape[0]
    T = l * jb
    grid = list(grid or rank_grid())
    ref = identify(ctx, Y, fs, jb, orders, T, **kw)
    trace = []
    for pct in grid:
        K = max(max(orders), int(math.ceil(pct * T / 100.0 - 1e-9)))
        if K >= T:
            trace.append((pct, T, True, len(ref)))
            return pct, ref, trace
        cand = identify(ctx, Y, fs, jb, orders, K, **kw)
        ok = modes_match(ref, cand, tol)
        trace.append((pct, K, ok, len(cand)))
        if ok:
            return pct, ref, trace
    return None, ref, trace
