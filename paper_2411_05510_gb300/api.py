"""Python entry points with the C ABI's names, on PyTorch device tensors.

Argument marshalling only: tensors are checked for device, dtype and layout,
their pointers and the current CUDA stream are passed to libssi, and outputs
are allocated with torch.  No step of the method runs here.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import numpy as np
import torch

from . import _lib
from ._lib import (SSI_PREC_FP32, SSI_PREC_SPLIT_BF16, SSI_SMALL_FP32, SSI_SMALL_FP64, SsiClusterInfo,
                   SsiClusterParams, SsiJobDesc, SsiMode, SsiStabParams, SsiTuning, check, lib)

__all__ = [
    "Context", "PREC", "ssi_covariances", "ssi_gaussian_omega", "ssi_toeplitz_rsvd",
    "ssi_realize_batch", "ssi_stabilize", "ssi_solve", "ssi_pole_slots", "poles_to_numpy",
    "stab_params", "job_desc", "ssi_rank_rule", "ssi_lag_rule", "ssi_time_lag", "check_sync",
    "ssi_job_sizes", "ssi_serve_config", "ssi_submit", "ssi_poll", "ssi_release",
    "cluster_params", "ssi_cluster", "CovStream", "ssi_autotune", "ssi_tuning_get",
    "ssi_tuning_set", "ssi_solve_batch",
]

PREC = {"fp32": SSI_PREC_FP32, "split_bf16": SSI_PREC_SPLIT_BF16}
SMALL = {"fp32": SSI_SMALL_FP32, "fp64": SSI_SMALL_FP64}


def _prec(p) -> int:
    return PREC[p] if isinstance(p, str) else int(p)


def _small(p) -> int:
    return SMALL[p] if isinstance(p, str) else int(p)


def _stream(device=None) -> ctypes.c_void_p:
    return ctypes.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _need(t: torch.Tensor, dtype, name: str):
    if not (t.is_cuda and t.dtype == dtype and t.is_contiguous()):
        raise ValueError(f"{name}: need a contiguous CUDA {dtype} tensor, got "
                         f"{t.dtype} on {t.device} contiguous={t.is_contiguous()}")


class Context:
    """An ssi_ctx bound to one CUDA device with an HBM budget (0 = half the free memory)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self.device = device
        self.ptr = ctypes.c_void_p()
        self._jobs = {}   # serving: job id -> descriptor kept alive until ssi_release
        check(lib.ssi_create(ctypes.byref(self.ptr), device, hbm_budget_bytes), "ssi_create")

    def close(self):
        if self.ptr:
            lib.ssi_destroy(self.ptr)
            self.ptr = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def memory_in_use(self) -> int:
        return int(lib.ssi_memory_in_use(self.ptr))

    def set_concurrency(self, solves_in_flight: int) -> None:
        """ssi_set_concurrency: how many solves share the device at once."""
        check(lib.ssi_set_concurrency(self.ptr, int(solves_in_flight)), "ssi_set_concurrency")

    STAGES = ["split", "lag_gemm", "lag_reduce", "sketch_gemm", "qr", "small_svd", "gram_factor",
              "eig", "stability", "other", "eig_vectors", "cluster"]

    def profile(self, enable: bool = True) -> None:
        check(lib.ssi_profile(self.ptr, 1 if enable else 0), "ssi_profile")

    def profile_read(self):
        """({stage: ms}, {stage: scopes}, kernel launches) since the previous read."""
        n = len(self.STAGES)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        launches = ctypes.c_int64()
        check(lib.ssi_profile_read(self.ptr, ms, cnt, n, ctypes.byref(launches)), "ssi_profile_read")
        return ({s: ms[i] for i, s in enumerate(self.STAGES)},
                {s: int(cnt[i]) for i, s in enumerate(self.STAGES)}, int(launches.value))


def ssi_covariances(ctx: Context, Y: torch.Tensor, max_lag: int, prec="split_bf16",
                    out: torch.Tensor | None = None) -> torch.Tensor:
    """R_k, k = 1..max_lag (float64, max_lag x l x l) from Y (l x N float32, channel-major)."""
    _need(Y, torch.float32, "Y")
    l, N = Y.shape
    R = out if out is not None else torch.empty((max_lag, l, l), dtype=torch.float64, device=Y.device)
    _need(R, torch.float64, "R")
    check(lib.ssi_covariances(ctx.ptr, ctypes.c_void_p(Y.data_ptr()), l, N, max_lag, _prec(prec),
                              ctypes.c_void_p(R.data_ptr()), _stream(Y.device)), "ssi_covariances")
    return R


def ssi_gaussian_omega(ctx: Context, rows: int, cols: int, seed: int, device="cuda") -> torch.Tensor:
    out = torch.empty((rows, cols), dtype=torch.float32, device=device)
    check(lib.ssi_gaussian_omega(ctx.ptr, rows, cols, seed, ctypes.c_void_p(out.data_ptr()),
                                 _stream(out.device)), "ssi_gaussian_omega")
    return out


def ssi_toeplitz_rsvd(ctx: Context, R: torch.Tensor, l: int, i: int, k: int, oversample: int = 0,
                      q: int = 0, seed: int = 0, prec="split_bf16", small="fp32"):
    """(U, S): U (l*i x k float64), S (k float64) of the block-Toeplitz T_{1|i} built from R;
    `small` is the arithmetic of the K x K SVD ("fp32" or "fp64")."""
    _need(R, torch.float64, "R")
    U = torch.empty((l * i, k), dtype=torch.float64, device=R.device)
    S = torch.empty((k,), dtype=torch.float64, device=R.device)
    check(lib.ssi_toeplitz_rsvd(ctx.ptr, ctypes.c_void_p(R.data_ptr()), l, i, k, oversample, q, seed,
                                _prec(prec), _small(small), ctypes.c_void_p(U.data_ptr()),
                                ctypes.c_void_p(S.data_ptr()), _stream(R.device)),
          "ssi_toeplitz_rsvd")
    return U, S


def _int_array(xs: Sequence[int]):
    arr = (ctypes.c_int * len(xs))(*[int(x) for x in xs])
    return arr


def ssi_pole_slots(orders: Sequence[int]) -> int:
    return int(lib.ssi_pole_slots(len(orders), _int_array(orders)))


def ssi_realize_batch(ctx: Context, lags: Sequence[int], Us: Sequence[torch.Tensor], l: int, k: int,
                      orders: Sequence[int], dt: float, small="fp32"):
    """Pole records (uint8 tensor, n_lags*slots x 40 bytes) and phi (float32, slots x l x 2)
    from float64 U (l*i x k) per lag; `small` is the arithmetic of A and eig(A)."""
    slots = ssi_pole_slots(orders) * len(lags)
    dev = Us[0].device
    poles = torch.zeros((slots, _lib.POLE_BYTES), dtype=torch.uint8, device=dev)
    phi = torch.zeros((slots, l, 2), dtype=torch.float32, device=dev)
    for U in Us:
        _need(U, torch.float64, "U")
    uptrs = (ctypes.c_void_p * len(Us))(*[U.data_ptr() for U in Us])
    check(lib.ssi_realize_batch(ctx.ptr, len(lags), _int_array(lags), uptrs, l, k, _int_array(orders),
                                len(orders), dt, _small(small), ctypes.c_void_p(poles.data_ptr()),
                                ctypes.c_void_p(phi.data_ptr()), _stream(dev)), "ssi_realize_batch")
    return poles, phi


def stab_params(xi_max=0.10, mpc_min=0.6, mpd_max=0.5, a_f=0.01, a_xi=0.03, a_mac=0.02,
                use_lag_axis=True) -> SsiStabParams:
    return SsiStabParams(xi_max, mpc_min, mpd_max, a_f, a_xi, a_mac, 1 if use_lag_axis else 0, 0)


def ssi_stabilize(ctx: Context, n_lags: int, orders: Sequence[int], l: int, poles: torch.Tensor,
                  phi: torch.Tensor, params: SsiStabParams | None = None):
    params = params or stab_params()
    check(lib.ssi_stabilize(ctx.ptr, n_lags, len(orders), _int_array(orders), l,
                            ctypes.c_void_p(poles.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                            ctypes.byref(params), _stream(poles.device)), "ssi_stabilize")
    return poles


class CovStream:
    """Sliding-window covariances (ssi_cov_stream_*): push channel-major blocks, read R of
    the last `window` samples."""

    def __init__(self, ctx: Context, l: int, max_lag: int, window: int, max_block: int,
                 prec="split_bf16"):
        self.ptr = ctypes.c_void_p()
        self.l, self.max_lag = l, max_lag
        self._ctx = ctx
        check(lib.ssi_cov_stream_create(ctx.ptr, l, max_lag, window, max_block, _prec(prec),
                                        ctypes.byref(self.ptr)), "ssi_cov_stream_create")

    def push(self, Y: torch.Tensor) -> None:
        _need(Y, torch.float32, "Y")
        check(lib.ssi_cov_stream_push(self.ptr, ctypes.c_void_p(Y.data_ptr()), Y.shape[1],
                                      _stream(Y.device)), "ssi_cov_stream_push")

    def covariances(self, R: torch.Tensor | None = None):
        """(R as a (max_lag, l, l) float64 device tensor, samples in the window)."""
        if R is None:
            R = torch.empty((self.max_lag, self.l, self.l), dtype=torch.float64, device="cuda")
        n = ctypes.c_int64()
        check(lib.ssi_cov_stream_covariances(self.ptr, ctypes.c_void_p(R.data_ptr()),
                                              ctypes.byref(n), _stream(R.device)),
              "ssi_cov_stream_covariances")
        return R, n.value

    def refresh(self) -> None:
        """Rebuild the window's lag sums from the samples held (ssi_cov_stream_refresh)."""
        check(lib.ssi_cov_stream_refresh(self.ptr, _stream()), "ssi_cov_stream_refresh")

    def close(self) -> None:
        """Free the stream's device memory (before its context is closed)."""
        if self.ptr:
            check(lib.ssi_cov_stream_destroy(self.ptr), "ssi_cov_stream_destroy")
            self.ptr = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc) -> None:
        self.close()


def cluster_params(tau=0.05, min_size=10, fcm_max_iter=500, fcm_m=2.0,
                   fcm_tol=1e-10) -> SsiClusterParams:
    return SsiClusterParams(tau, min_size, fcm_max_iter, fcm_m, fcm_tol)


def ssi_cluster(ctx: Context, n_lags: int, orders: Sequence[int], l: int, poles: torch.Tensor,
                phi: torch.Tensor, params: SsiClusterParams | None = None, max_modes: int = 1024,
                per_pole: bool = False):
    """Two-stage clustering of a flagged diagram.  Returns (modes, info, per_pole) where modes
    is a list of dicts (f_hz, xi, size, medoid_slot) sorted by frequency, info a dict of
    ssi_cluster_info, and per_pole (when asked) the device tensors features (slots x 5),
    membership and label."""
    params = params or cluster_params()
    n_slots = poles.numel() * poles.element_size() // _lib.POLE_BYTES
    feats = memb = lab = None
    if per_pole:
        feats = torch.empty((n_slots, 5), dtype=torch.float64, device=poles.device)
        memb = torch.empty(n_slots, dtype=torch.float64, device=poles.device)
        lab = torch.empty(n_slots, dtype=torch.int32, device=poles.device)
    buf = (SsiMode * max(1, max_modes))()
    n_modes = ctypes.c_int()
    info = SsiClusterInfo()
    ptr = (lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None)
    check(lib.ssi_cluster(ctx.ptr, n_lags, len(orders), _int_array(orders), l,
                          ctypes.c_void_p(poles.data_ptr()), ctypes.c_void_p(phi.data_ptr()),
                          ctypes.byref(params), buf, max_modes, ctypes.byref(n_modes), ptr(feats),
                          ptr(memb), ptr(lab), ctypes.byref(info), _stream(poles.device)),
          "ssi_cluster")
    modes = [dict(f_hz=buf[i].f_hz, xi=buf[i].xi, size=buf[i].size, medoid_slot=buf[i].medoid_slot)
             for i in range(min(n_modes.value, max_modes))]
    inf = {f: getattr(info, f) for f, _ in SsiClusterInfo._fields_ if f not in ("centroids", "reserved")}
    inf["centroids"] = np.array([[info.centroids[c][d] for d in range(5)] for c in range(2)])
    return modes, inf, (dict(features=feats, membership=memb, label=lab) if per_pole else None)


def job_desc(Y, fs: float, lags: Sequence[int], orders: Sequence[int], k: int, oversample: int = 0,
             q: int = 0, prec="split_bf16", seed: int = 0, stab: SsiStabParams | None = None,
             small="fp32"):
    """An ssi_job_desc for a device tensor or a (pinned) host tensor / numpy array Y (l x N)."""
    keep = []
    if isinstance(Y, torch.Tensor):
        if Y.dtype != torch.float32 or not Y.is_contiguous():
            raise ValueError("Y must be contiguous float32")
        ptr, on_host = Y.data_ptr(), 0 if Y.is_cuda else 1
    else:
        Y = np.ascontiguousarray(Y, dtype=np.float32)
        ptr, on_host = Y.ctypes.data, 1
    keep.append(Y)
    l, N = Y.shape
    lag_arr = (ctypes.c_int32 * len(lags))(*lags)
    ord_arr = (ctypes.c_int32 * len(orders))(*orders)
    keep += [lag_arr, ord_arr]
    d = SsiJobDesc(ptr, on_host, l, N, fs, len(lags), lag_arr, len(orders), ord_arr, k, oversample,
                   q, _prec(prec), seed, stab or stab_params(use_lag_axis=len(lags) > 1),
                   _small(small), 0)
    d._keep = keep
    return d


def check_sync(ctx: Context, device=None) -> None:
    """Synchronise the current stream and raise if a kernel reported a device-side status."""
    check(lib.ssi_sync_status(ctx.ptr, _stream(device)), "ssi_sync_status")


def ssi_job_sizes(desc: SsiJobDesc):
    n, p = ctypes.c_int64(), ctypes.c_int64()
    check(lib.ssi_job_sizes(ctypes.byref(desc), ctypes.byref(n), ctypes.byref(p)), "ssi_job_sizes")
    return n.value, p.value


def ssi_solve(ctx: Context, desc: SsiJobDesc, device="cuda", with_s: bool = True):
    """Full solve; returns (poles uint8 tensor, phi float32 tensor, S float64 tensor or None)."""
    n_slots, phi_floats = ssi_job_sizes(desc)
    poles = torch.zeros((n_slots, _lib.POLE_BYTES), dtype=torch.uint8, device=device)
    phi = torch.zeros((phi_floats,), dtype=torch.float32, device=device)
    S = torch.zeros((desc.n_lags, desc.k), dtype=torch.float64, device=device) if with_s else None
    check(lib.ssi_solve(ctx.ptr, ctypes.byref(desc), ctypes.c_void_p(poles.data_ptr()),
                        ctypes.c_void_p(phi.data_ptr()),
                        ctypes.c_void_p(S.data_ptr() if S is not None else 0),
                        _stream(torch.device(device))), "ssi_solve")
    return poles, phi, S


def ssi_solve_batch(ctx: Context, descs, device="cuda", with_s: bool = True):
    """Several jobs in one call, their eigen-decompositions in one launch; returns a list of
    (poles, phi, S) as ssi_solve does for each job."""
    n = len(descs)
    outs = []
    for d in descs:
        n_slots, phi_floats = ssi_job_sizes(d)
        poles = torch.zeros((n_slots, _lib.POLE_BYTES), dtype=torch.uint8, device=device)
        phi = torch.zeros((phi_floats,), dtype=torch.float32, device=device)
        S = torch.zeros((d.n_lags, d.k), dtype=torch.float64, device=device) if with_s else None
        outs.append((poles, phi, S))
    arr = (SsiJobDesc * n)(*descs)
    P = (ctypes.c_void_p * n)(*[o[0].data_ptr() for o in outs])
    F = (ctypes.c_void_p * n)(*[o[1].data_ptr() for o in outs])
    Sp = (ctypes.c_void_p * n)(*[o[2].data_ptr() for o in outs]) if with_s else None
    check(lib.ssi_solve_batch(ctx.ptr, n, arr, P, F, Sp, _stream(torch.device(device))),
          "ssi_solve_batch")
    return outs


def _tuning_dict(t: SsiTuning) -> dict:
    return {"cov_rows_per_split": t.cov_rows_per_split, "sketch_splits": t.sketch_splits,
            "jacobi_block": t.jacobi_block, "qr_chunks_per_cta": t.qr_chunks_per_cta,
            "stage_ms": [t.stage_ms[i] for i in range(4)]}


def ssi_autotune(ctx: Context, desc: SsiJobDesc) -> dict:
    """Time candidate plan choices on solves of the job and store the fastest in ctx."""
    t = SsiTuning()
    check(lib.ssi_autotune(ctx.ptr, ctypes.byref(desc), ctypes.byref(t)), "ssi_autotune")
    return _tuning_dict(t)


def ssi_tuning_get(ctx: Context, desc: SsiJobDesc) -> dict:
    t = SsiTuning()
    check(lib.ssi_tuning_get(ctx.ptr, ctypes.byref(desc), ctypes.byref(t)), "ssi_tuning_get")
    return _tuning_dict(t)


def ssi_tuning_set(ctx: Context, desc: SsiJobDesc, tuning: dict) -> None:
    t = SsiTuning(int(tuning.get("cov_rows_per_split", 0)), int(tuning.get("sketch_splits", 0)),
                  int(tuning.get("jacobi_block", 0)), int(tuning.get("qr_chunks_per_cta", 0)))
    check(lib.ssi_tuning_set(ctx.ptr, ctypes.byref(desc), ctypes.byref(t)), "ssi_tuning_set")


def ssi_serve_config(ctx: Context, max_slots: int = 2, max_queue: int = 64) -> None:
    check(lib.ssi_serve_config(ctx.ptr, max_slots, max_queue), "ssi_serve_config")


def ssi_submit(ctx: Context, desc: SsiJobDesc) -> int:
    """Queue a job; the descriptor (and a device record it points to) is kept alive by
    the context until ssi_release."""
    jid = ctypes.c_uint64()
    check(lib.ssi_submit(ctx.ptr, ctypes.byref(desc), ctypes.byref(jid)), "ssi_submit")
    ctx._jobs[jid.value] = desc
    return jid.value


def ssi_poll(ctx: Context, job_id: int, timeout_ms: int = -1):
    """Wait for a job; returns (pole records as a numpy structured array, phi float32
    array (slots x l x 2), latency in microseconds).  The arrays are copies."""
    pp, ff = ctypes.c_void_p(), ctypes.c_void_p()
    ns, lat = ctypes.c_int64(), ctypes.c_double()
    check(lib.ssi_poll(ctx.ptr, job_id, timeout_ms, ctypes.byref(pp), ctypes.byref(ff),
                       ctypes.byref(ns), ctypes.byref(lat)), "ssi_poll")
    desc = ctx._jobs[job_id]
    n = ns.value
    raw = ctypes.string_at(pp.value, n * _lib.POLE_BYTES) if n else b""
    rec = np.frombuffer(raw, dtype=_POLE_DTYPE).copy()
    nf = n * desc.l * 2
    phi = np.ctypeslib.as_array(ctypes.cast(ff.value, ctypes.POINTER(ctypes.c_float)),
                                shape=(nf,)).copy() if nf else np.zeros(0, np.float32)
    return rec, phi.reshape(n, desc.l, 2), lat.value


def ssi_release(ctx: Context, job_id: int) -> None:
    check(lib.ssi_release(ctx.ptr, job_id), "ssi_release")
    ctx._jobs.pop(job_id, None)


_POLE_DTYPE = np.dtype([("f_hz", "<f4"), ("xi", "<f4"), ("mu_re", "<f4"), ("mu_im", "<f4"),
                        ("mpc", "<f4"), ("mpd", "<f4"), ("lag", "<i4"), ("order", "<i4"),
                        ("flags", "<u4"), ("index", "<i4")])


def poles_to_numpy(poles) -> np.ndarray:
    """Pole records (uint8 tensor or bytes) -> numpy structured array."""
    if isinstance(poles, torch.Tensor):
        raw = poles.detach().cpu().contiguous().numpy().tobytes()
    else:
        raw = bytes(poles)
    return np.frombuffer(raw, dtype=_POLE_DTYPE).copy()


def ssi_rank_rule(T_size: int):
    kbar, k = ctypes.c_double(), ctypes.c_int64()
    check(lib.ssi_rank_rule(T_size, ctypes.byref(kbar), ctypes.byref(k)), "ssi_rank_rule")
    return kbar.value, k.value


def ssi_lag_rule(fs: float, f0: float, beta: float = 1.5):
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib.ssi_lag_rule(fs, f0, beta, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
          "ssi_lag_rule")
    return a.value, b.value, c.value


def ssi_time_lag(jb: int, fs: float) -> float:
    return float(lib.ssi_time_lag(jb, fs))
