#!/usr/bin/env python
"""Benchmark of the RSVD-CoV-SSI hot path: SSI solves/s on the 186-channel bridge record.

Workload (default "bridge186_i60"): l = 186 channels (62 triaxial stations), 20 modes
(1-20 Hz), fs = 100 Hz, N = 360000 samples (1 h), 5 % sensor noise; one solve =
covariances R_1..R_119, Toeplitz RSVD at i = 60 (T 11160 x 11160, k = 200 + 20, q = 2),
realisations of orders 2..200 step 2, hard and soft stability criteria.

Lines printed (one JSON line on rank 0):
  value      solves/s with the record resident in HBM: CUDA events around K solves dealt
             round robin to --inflight independent solvers (own context, record copy and
             stream each), so that one solve's latency-bound stages (the cluster Jacobi
             SVD, the tail of the per-order eigenproblems) overlap another's GEMMs
  serial     the same with one solve in flight (unloaded latency, per-stage times)
  e2e        the same through ssi_submit / ssi_poll with the record in pinned host memory
             (host->device copy and the read-back of poles and mode shapes inside)
  roofline   dominant kernel (the tcgen05 lag GEMM): algorithmic FP32-equivalent flops
             2 l^2 N K_lag per launch / its measured duration, against the measured BF16
             burst tensor peak divided by 3 (three BF16 products per split product); the
             fraction of the sustained peak is printed beside it
  fp32_path  the same pipeline with plain FP32 CUDA-core GEMMs (the plain FP32 GPU path)
  small_fp64 the same pipeline with the K x K SVD, the least squares for A and eig(A) in
             FP64 (the split-BF16 GEMMs unchanged)
  diagram_3d the 3D stabilization diagram (lags 20..100 step 10) of the same record
  batch      eight mixed-shape jobs in one ssi_solve_batch call (their eigen-decompositions
             in one launch) against one ssi_solve after another
  serving_mix  p50/p99 latency of a heterogeneous job stream through the serving API
  cpu_baseline  one complete FP64 oracle solve of the workload on the host cores, timed
             (oracle/reference_solve.py, which also stores its result)
  error_vs_oracle  the GPU results against that stored oracle result: leading singular
             values, poles at the separated orders of the two independent solves, and the
             realisation of every order from the oracle's own U (both small precisions)

--workload serving_mix runs the serving configuration instead: a seeded stream of
heterogeneous jobs through ssi_submit / ssi_poll under an HBM budget, capacity with all
jobs submitted at once and p50/p99 latency under Poisson arrivals at 0.5 / 0.8 / 1.0 of it.

--impl reference times the FP64 oracle (the CPU reference of the method) on the same
workload: the K timed steps together run one complete oracle solve, its units of work
(covariances, Toeplitz RSVD, the realisation of each order, stability) dealt in order over
the steps; the warm-up steps solve the 4-channel chain record.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import ssi_synth as S  # noqa: E402

PROFILES = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="bridge186_i60")
    ap.add_argument("--n-samples", type=int, default=0,
                    help="record length override (smaller cases for profiler captures)")
    ap.add_argument("--prec", default="split_bf16", choices=["split_bf16", "fp32"])
    ap.add_argument("--small", default="fp32", choices=["fp32", "fp64"],
                    help="arithmetic of the K x K SVD, A and eig(A) of the timed solves")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-cluster", action="store_true")
    ap.add_argument("--no-stream", action="store_true")
    ap.add_argument("--no-fp64-small", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--no-mix", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--rank-jb-max", type=int, default=500,
                    help="largest time-lag step of --workload rank_study")
    ap.add_argument("--inflight", type=int, default=4,
                    help="solves in flight at once, each on its own stream and context")
    return ap.parse_args()


# ----------------------------------------------------------------------------- helpers
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over the ranks of the default process group (x alone at N = 1).
    device: where the reduction tensor lives (a CUDA device under NCCL, CPU under gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, max_ms: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    # the profiling recipe's fallback: one earlier GB300 measurement (copy, cuBLAS burst)
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash():
    """Hash of the lag-GEMM kernel's own source (its template definition, the constants and
    parameter block above it, the time-split plan) and of the tcgen05/TMA helpers it uses:
    the stored DRAM traffic stays valid while these are unchanged."""
    csrc = os.path.join(ROOT, "paper_2411_05510_gb300", "csrc")
    with open(os.path.join(csrc, "covariance.cu")) as fh:
        src = fh.read()
    a = src.index("constexpr int BT = ")
    b = src.index("template <int NB, int STAGES>\n__global__ void __launch_bounds__(TC_THREADS, 1)")
    c = src.index("\n}\n", b) + 3
    d = src.index("CovPlan cov_plan(")
    e = src.index("\n}\n", d) + 3
    h = hashlib.sha256()
    h.update(src[a:src.index("// ------------------------------------------------------------------ split/transpose")].encode())
    h.update(src[b:c].encode())
    h.update(src[d:e].encode())   # the split plan sets the partial writes
    with open(os.path.join(csrc, "blackwell.cuh"), "rb") as fh:
        h.update(fh.read())
    return h.hexdigest()[:16]


def stored_traffic(workload):
    """DRAM bytes per launch of the lag GEMM from the committed ncu summary, if current."""
    path = os.path.join(PROFILES, f"lag_gemm_{workload}_traffic.json")
    if not os.path.exists(path):
        return None, None
    with open(path) as fh:
        d = json.load(fh)
    if d.get("source_hash") != kernel_source_hash():
        return None, "stale"
    return d.get("dram_bytes_per_launch"), d.get("note")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.th.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def pct(xs, q):
    xs = sorted(xs)
    if not xs:
        return None
    k = min(len(xs) - 1, max(0, int(round(q / 100.0 * (len(xs) - 1)))))
    return xs[k]


# ----------------------------------------------------------------------------- oracle sample
def oracle_sample_estimate(Y, w, log=None):
    """Seconds of one FP64-oracle solve of workload w, estimated stage by stage from a
    bounded sample: covariances on 1/50 of the record (x50); one Toeplitz product and
    one Householder QR (x(2+2q) each); one Jacobi sweep of P^T (x10 sweeps); full
    realisations of four orders scaled by sum(n^2); stability on those orders."""
    import oracle as O
    t = {}
    N = Y.shape[1]
    Ns = max(2 * max(w["lags"]) + 10, N // 50)
    t0 = time.perf_counter()
    R = O.covariances(Y[:, :Ns], 2 * max(w["lags"]) - 1)
    t["covariances"] = (time.perf_counter() - t0) * (N / Ns)
    i = w["lags"][0]
    t0 = time.perf_counter()
    T = O.block_toeplitz(R, i)
    t["toeplitz"] = time.perf_counter() - t0
    K = w["k"] + w["oversample"]
    om = O.gaussian_omega(T.shape[1], K, 1)
    t0 = time.perf_counter()
    Yk = T @ om
    t["products"] = (time.perf_counter() - t0) * (2 + 2 * w["q"])
    t0 = time.perf_counter()
    Q, _ = O.householder_qr(Yk)
    t["qr"] = (time.perf_counter() - t0) * (2 + 2 * w["q"])
    P = Q.T @ T
    t0 = time.perf_counter()
    O.jacobi_svd(P.T, max_sweeps=1)
    t["small_svd"] = (time.perf_counter() - t0) * 10
    U = Q[:, :w["k"]]
    Sv = np.linalg.norm(P[:w["k"]], axis=1)
    orders = w["orders"]
    sample = [orders[len(orders) // 5], orders[len(orders) // 2], orders[(4 * len(orders)) // 5],
              orders[-1]]
    l = Y.shape[0]
    t0 = time.perf_counter()
    cells = []
    for n in sample:
        mu, f, xi, Phi, _ = O.realize(U, Sv, l, i, n, 1.0 / w["fs"])
        cells.append(dict(mu=mu, f=f, xi=xi, Phi=Phi))
    ts = time.perf_counter() - t0
    t["realisation"] = ts * sum(n * n for n in orders) / sum(n * n for n in sample)
    t0 = time.perf_counter()
    O.stability([cells])
    t["stability"] = (time.perf_counter() - t0) * len(orders) / len(sample)
    return sum(t.values()), t


# ----------------------------------------------------------------------------- reference arm
def run_reference(args, world, rank):
    """The FP64 oracle on the host cores, on the workload of our arm.  The K timed steps
    together run ONE complete oracle solve: its units of work (covariances, the Toeplitz
    RSVD, the realisation of each order, stability) are dealt in order over the steps,
    unit u to step floor(u K / units).  value = 1 solve / the time of the K steps.  The
    warm-up steps solve the 4-channel chain record (untimed)."""
    if rank != 0:
        return
    from oracle import reference_solve as RS
    w = S.workload(args.workload, **({"N": args.n_samples} if args.n_samples else {}))
    w["name"] = args.workload
    Y, *_ = S.record(w, np.float32)
    Y = Y.astype(np.float64)
    wt = S.workload("chain4_tiny")
    Yt, *_ = S.record(wt)
    for _ in range(args.warmup):
        RS.run(Yt, wt, 1)
    _, units = RS.solve_units(Y, w, 12345)
    K = max(1, args.steps)
    step_s, stage_s = [], {}
    for st in range(K):
        t0 = time.perf_counter()
        for u in range(len(units)):
            if (u * K) // len(units) == st:
                name, fn = units[u]
                t1 = time.perf_counter()
                fn()
                stage_s[name] = stage_s.get(name, 0.0) + time.perf_counter() - t1
        step_s.append(time.perf_counter() - t0)
    total = sum(step_s)
    cores = os.cpu_count()
    value = 1.0 / total
    sample = (f"one complete solve of {args.workload}: its {len(units)} units of work in order, "
              f"dealt over the {K} timed steps")
    line = {"impl": "reference", "metric": "SSI solves/s", "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total * 1e3 / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, "fp64 oracle"),
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": sample, "threads": "numpy BLAS threads on every core; the "
                             "oracle's own loops run on one",
                             "stage_s": {k: round(v, 3) for k, v in stage_s.items()}},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- serving mix
def batch_measure(args, dev, n_jobs=8, reps=3):
    """Eight jobs of the serving mix's shapes (records resident in HBM), solved one
    ssi_solve after another on one stream, and in one ssi_solve_batch call (their front
    stages on four forked streams, one k_eig and one k_eig_vectors launch for all of
    them).  Device time per batch with CUDA events, best of `reps` after a warm-up."""
    import torch
    import paper_2411_05510_gb300 as P
    mix = S.serving_mix(n_jobs, seed=11)
    Ys = [torch.from_numpy(S.record(w, np.float32)[0]).to(dev) for w in mix]
    descs = [P.job_desc(Y, w["fs"], w["lags"], w["orders"], k=w["k"], oversample=w["oversample"],
                        q=w["q"], prec=args.prec, seed=12345) for w, Y in zip(mix, Ys)]
    ctx = P.Context(dev.index or 0)
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        best = None
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            P.check_sync(ctx, dev)
            if r > 0:
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
        return best

    ctx.profile_read()
    t_sep = timed(lambda: [P.ssi_solve(ctx, d, device=dev) for d in descs])
    n_sep = ctx.profile_read()[2]
    t_bat = timed(lambda: P.ssi_solve_batch(ctx, descs, device=dev))
    n_bat = ctx.profile_read()[2]
    ctx.close()
    return {"value": n_jobs / (t_bat / 1e3), "unit": "solves/s", "jobs": n_jobs,
            "ms_per_batch": t_bat, "separate_solves_per_s": n_jobs / (t_sep / 1e3),
            "ms_separate": t_sep, "launches_per_batch": n_bat / (reps + 1),
            "launches_separate": n_sep / (reps + 1),
            "shapes": [{"l": w["l"], "N": w["N"], "i": w["lags"][0], "k": w["k"]} for w in mix],
            "api": "ssi_solve_batch against one ssi_solve per job (CUDA events, best of 3)"}


def serving_mix_measure(args, world, rank, n_jobs):
    """The serving configuration: a seeded stream of heterogeneous jobs (16/48/96/186
    channels, N 30000-360000, i 20-80, 5-30 modes), records in pinned host memory, admitted
    by the serving loop under an HBM budget of half the free memory, J slots.  Capacity:
    all jobs submitted at once.  Then Poisson arrivals at 0.5, 0.8 and 1.0 of that capacity:
    achieved solves/s and each job's submit-to-result latency (p50/p99)."""
    import torch
    import torch.distributed as dist
    import paper_2411_05510_gb300 as P

    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    mix = S.serving_mix(n_jobs, seed=4 + rank)
    recs = []
    for w in mix:
        Y, *_ = S.record(w, np.float32)
        recs.append(torch.from_numpy(Y).pin_memory())
    free, _ = torch.cuda.mem_get_info(dev)
    ctx = P.Context(local, int(free * 0.5))
    J = max(1, args.inflight)
    P.ssi_serve_config(ctx, J, 4 * n_jobs)

    def desc_of(w, Yh):
        return P.job_desc(Yh, w["fs"], w["lags"], w["orders"], k=w["k"], oversample=w["oversample"],
                          q=w["q"], prec=args.prec, seed=12345)

    descs = [desc_of(w, Yh) for w, Yh in zip(mix, recs)]

    def run(arrivals):
        """Submit job j at arrivals[j] seconds (host clock); wait for all."""
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        ids = []
        for j, d in enumerate(descs):
            wait = arrivals[j] - (time.perf_counter() - t0)
            if wait > 0:
                time.sleep(wait)
            ids.append(P.ssi_submit(ctx, d))
        lat = []
        for jid in ids:
            _, _, lu = P.ssi_poll(ctx, jid, -1)
            P.ssi_release(ctx, jid)
            lat.append(lu / 1e3)
        t = max_over_ranks((time.perf_counter() - t0) * 1e3, dev)
        return t, lat

    n_warm = max(1, min(args.warmup, 2))
    for _ in range(n_warm):   # warm-up: slot buffers grow to the mix
        run([0.0] * n_jobs)
    t_cap, lat_cap = run([0.0] * n_jobs)
    capacity = whole_job_rate(n_jobs, world, t_cap)
    per_rank = capacity / world
    rng = np.random.Generator(np.random.PCG64(99 + rank))
    loads = {}
    for frac in (0.5, 0.8, 1.0):
        gaps = rng.exponential(1.0 / (frac * per_rank), size=n_jobs)
        arrivals = list(np.cumsum(gaps) - gaps[0])
        t, lat = run(arrivals)
        loads[str(frac)] = {"offered_solves_per_s": frac * capacity,
                            "achieved_solves_per_s": whole_job_rate(n_jobs, world, t),
                            "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99)}}
    ctx.close()
    return {"value": capacity, "unit": "solves/s", "jobs": n_jobs, "warmup": n_warm,
            "ms_per_job": t_cap / n_jobs,
            "config": {"workload": "serving_mix", "jobs": n_jobs, "slots": J,
                       "channels": [16, 48, 96, 186], "N": [30000, 360000], "i": [20, 80],
                       "modes": [5, 30], "hbm_budget_bytes": int(free * 0.5),
                       "prec": args.prec, "records": "pinned host memory"},
            "latency_ms": {"p50": pct(lat_cap, 50), "p99": pct(lat_cap, 99),
                           "kind": "submit to result, all jobs submitted at once"},
            "poisson": loads,
            "h2d_bytes_per_job": int(sum(w["l"] * w["N"] * 4 for w in mix) / n_jobs)}


def run_serving_mix(args, world, rank):
    """--workload serving_mix: the serving configuration as the benchmark's own line."""
    import torch
    import torch.distributed as dist
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    n_jobs = max(64, args.steps)
    r = serving_mix_measure(args, world, rank, n_jobs)
    if rank == 0:
        line = {"metric": "SSI solves/s", "value": r["value"], "unit": "solves/s", "n_gpus": world,
                "steps": n_jobs, "warmup": r["warmup"], "ms_per_step": r["ms_per_job"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16" if args.prec == "split_bf16" else "f32", "data": "synthetic",
                "config": r["config"], "latency_ms": r["latency_ms"], "poisson": r["poisson"],
                "e2e": {"value": r["value"], "unit": "solves/s",
                        "h2d_bytes_per_step": r["h2d_bytes_per_job"], "d2h_bytes_per_step": None,
                        "api": "ssi_submit/ssi_poll, host clock around all jobs"}}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- oracle result
def oracle_solve(args):
    """One complete FP64 oracle solve of the workload in a child process
    (oracle/reference_solve.py), which stores its result.  Returns (path of the stored
    result, seconds, seconds per stage, cores)."""
    cache = os.path.join(ROOT, ".oracle_cache")
    os.makedirs(cache, exist_ok=True)
    path = os.path.join(cache, f"{args.workload}_{args.n_samples or 'full'}_12345.npz")
    cmd = [sys.executable, "-m", "oracle.reference_solve", "--workload", args.workload,
           "--seed", "12345", "--out", path]
    if args.n_samples:
        cmd += ["--n-samples", str(args.n_samples)]
    subprocess.run(cmd, cwd=ROOT, check=True, stdout=subprocess.DEVNULL)
    d = np.load(path)
    parts = {str(k): float(v) for k, v in zip(d["stage_names"], d["stage_s"])}
    return path, sum(parts.values()), parts, int(d["cores"])


def oracle_cells(path):
    """The stored oracle diagram as cells[t][m] (mu, f, xi, Phi, flags), its singular
    values and U."""
    d = np.load(path)
    lags, orders = list(d["lags"]), list(d["orders"])
    cells, off, c = [], 0, 0
    for t in range(len(lags)):
        row = []
        for m in range(len(orders)):
            n = int(d["counts"][c])
            sl = slice(off, off + n)
            row.append(dict(mu=d["mu"][sl], f=d["f"][sl], xi=d["xi"][sl], Phi=d["phi"][sl].T,
                            flags=d["flags"][sl]))
            off += n
            c += 1
        cells.append(row)
    return cells, d["s"], d["U"]


def gpu_cells_of(P, poles, phi, lags, orders, l):
    rec = P.poles_to_numpy(poles)
    ph = phi.cpu().numpy().reshape(-1, l, 2)
    cells, off = [], 0
    for _ in lags:
        row = []
        for n in orders:
            r = rec[off:off + n // 2]
            v = (r["flags"] & 64) != 0
            p_ = ph[off:off + n // 2][v].astype(np.float64)
            row.append(dict(mu=(r["mu_re"] + 1j * r["mu_im"])[v].astype(np.complex128),
                            f=r["f_hz"][v].astype(np.float64), xi=r["xi"][v].astype(np.float64),
                            Phi=(p_[..., 0] + 1j * p_[..., 1]).T, flags=r["flags"][v]))
            off += n // 2
        cells.append(row)
    return cells


def _mac(a, b):
    den = np.vdot(a, a).real * np.vdot(b, b).real
    return float(abs(np.vdot(a, b)) ** 2 / den) if den > 0 else 0.0


def pole_errors(gpu, ora, f_true, phi_true, orders, n_modes, gate=None):
    """Parity set: per order n >= 2 m (and in `gate` when given) and generating mode r, the
    oracle's pole of mode r (HC-passing, within 5 % of f_r, largest MAC with the generating
    shape) against the GPU pole with the nearest discrete eigenvalue."""
    worst = {"df_rel": 0.0, "dxi_abs": 0.0, "mac_min": 1.0}
    pairs = missing = 0
    for t in range(len(ora)):
        for m, n in enumerate(orders):
            if n < 2 * n_modes or (gate is not None and n not in gate[t]):
                continue
            oc, gc = ora[t][m], gpu[t][m]
            for r, f0 in enumerate(f_true):
                cand = np.where(((oc["flags"] & 8) != 0) & (np.abs(oc["f"] - f0) < 0.05 * f0))[0]
                if len(cand) == 0 or len(gc["f"]) == 0:
                    missing += 1
                    continue
                a = int(cand[np.argmax([_mac(oc["Phi"][:, j], phi_true[:, r]) for j in cand])])
                b = int(np.argmin(np.abs(gc["mu"] - oc["mu"][a])))
                worst["df_rel"] = max(worst["df_rel"], abs(gc["f"][b] - oc["f"][a]) / oc["f"][a])
                worst["dxi_abs"] = max(worst["dxi_abs"], abs(gc["xi"][b] - oc["xi"][a]))
                worst["mac_min"] = min(worst["mac_min"], _mac(gc["Phi"][:, b], oc["Phi"][:, a]))
                pairs += 1
    worst.update(pairs=pairs, oracle_missing=missing)
    return worst


def error_vs_oracle(P, ctx, w, Y, f_true, phi_true, path, prec, dev):
    """The GPU results against the stored oracle result of the same record and Omega, in
    both small-problem precisions: the leading 2 m singular values of an independent solve,
    its poles at the orders whose leading subspace is separated (sigma_n/sigma_n+1 >= 2,
    reproducible between two SVDs), and the realisation of every order from the oracle's
    own U (ssi_realize_batch; the subspace shared, so every order n >= 2 m is comparable)."""
    import torch
    ora, s_ora, U_ora = oracle_cells(path)
    m = len(f_true)
    l = Y.shape[0]
    lags, orders = w["lags"], w["orders"]
    gate = [[n for n in orders if n < len(s) and s[n - 1] >= 2.0 * s[n]] for s in s_ora]
    out = {"tolerances": {"sigma_rel": 1e-4, "df_rel": 1e-4, "dxi_abs": 2e-3, "mac_min": 0.999},
           "separated_orders": gate}
    Yd = torch.from_numpy(Y).to(dev)
    for small in ("fp32", "fp64"):
        d = P.job_desc(Yd, w["fs"], lags, orders, k=w["k"], oversample=w["oversample"], q=w["q"],
                       prec=prec, seed=12345, small=small)
        poles, phi, Sg = P.ssi_solve(ctx, d, device=dev)
        P.check_sync(ctx, dev)
        sg = Sg.cpu().numpy()
        sig = float(max(np.max(np.abs(sg[t, :2 * m] / s_ora[t][:2 * m] - 1)) for t in range(len(lags))))
        gpu = gpu_cells_of(P, poles, phi, lags, orders, l)
        sep = pole_errors(gpu, ora, f_true, phi_true, orders, m, gate)
        res = {"sigma_rel_max": sig, "independent_solve_separated_orders": sep}
        if U_ora.size:
            Us = [torch.from_numpy(np.ascontiguousarray(U_ora[t])).to(dev) for t in range(len(lags))]
            pr, ph = P.ssi_realize_batch(ctx, lags, Us, l, w["k"], orders, 1.0 / w["fs"], small)
            P.ssi_stabilize(ctx, len(lags), orders, l, pr, ph, P.stab_params(use_lag_axis=len(lags) > 1))
            P.check_sync(ctx, dev)
            res["shared_U_every_order"] = pole_errors(gpu_cells_of(P, pr, ph, lags, orders, l), ora,
                                                      f_true, phi_true, orders, m)
        out[f"small_{small}"] = res
    return out


def run_frame10_table2(args, world, rank):
    """The 10-DOF frame of Sec. 3.1 identified by the 2D diagram (RSVD at j_b = 189) and by
    the 3D diagram (ten lags from 170 to 255) with the two-stage clustering, over seeds, in
    the form of Table 2 with the generating model's exact modal values as the reference:
    per mode, frequency and damping differences in percent and the MAC of the medoid's
    shape.  Runs on rank 0 of the job; other ranks exit."""
    import torch
    import paper_2411_05510_gb300 as P
    if rank != 0:
        return
    seeds = list(range(max(1, args.steps)))
    lags3 = [int(x) for x in np.linspace(170, 255, 10).round()]
    orders = list(range(2, 31, 2))
    ctx = P.Context(0)
    res = {"rsvd_2d": [], "rsvd_3d": []}
    t_3d = []
    for seed in seeds:
        w = S.workload("frame10", seed=100 + seed)
        Y, f_true, xi_true, phi_true = S.record(w, np.float32)
        Yd = torch.from_numpy(Y).cuda()
        for key, lags, min_size in (("rsvd_2d", [189], 5),
                                    ("rsvd_3d", lags3, len(lags3) * len(orders) // 4)):
            # Eq. (empirical_formula) at the largest Toeplitz size of the diagram: K columns
            # of the range finder (Algorithm 1, p = q = 0), the first 30 kept for the orders
            _, K = P.ssi_rank_rule(Y.shape[0] * max(lags))
            desc = P.job_desc(Yd, w["fs"], lags, orders, k=max(orders), oversample=K - max(orders),
                              q=0, prec="split_bf16", seed=seed)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            poles, phi, _ = P.ssi_solve(ctx, desc, with_s=False)
            modes, info, _ = P.ssi_cluster(ctx, len(lags), orders, Y.shape[0], poles, phi,
                                           P.cluster_params(tau=0.05, min_size=min_size))
            if key == "rsvd_3d":
                t_3d.append((time.perf_counter() - t0) * 1e3)
            P.check_sync(ctx)
            ph = phi.cpu().numpy().reshape(-1, Y.shape[0], 2)
            rows = []
            for r in range(len(f_true)):
                best = None
                for m in modes:
                    if abs(m["f_hz"] - f_true[r]) / f_true[r] > 0.02:
                        continue
                    v = ph[m["medoid_slot"]]
                    v = v[:, 0] + 1j * v[:, 1]
                    mac = abs(np.vdot(v, phi_true[:, r])) ** 2 / (
                        np.vdot(v, v).real * np.vdot(phi_true[:, r], phi_true[:, r]).real)
                    if best is None or mac > best[2]:
                        best = (m["f_hz"], m["xi"], float(mac))
                rows.append(None if best is None else
                            (abs(best[0] - f_true[r]) / f_true[r] * 100,
                             abs(best[1] - xi_true[r]) / xi_true[r] * 100, best[2]))
            res[key].append(rows)
    ctx.close()

    def table(runs):
        out = []
        for r in range(len(runs[0])):
            got = [run[r] for run in runs if run[r] is not None]
            out.append({"mode": r + 1, "found": len(got), "of": len(runs),
                        "df_pct_mean": float(np.mean([g[0] for g in got])) if got else None,
                        "df_pct_max": float(np.max([g[0] for g in got])) if got else None,
                        "dxi_pct_mean": float(np.mean([g[1] for g in got])) if got else None,
                        "dxi_pct_max": float(np.max([g[1] for g in got])) if got else None,
                        "mac_min": float(np.min([g[2] for g in got])) if got else None})
        return out

    line = {"metric": "modal identification error, 10-DOF frame (Sec. 3.1, Table 2 form)",
            "unit": "percent", "workload": "frame10_table2", "seeds": len(seeds),
            "reference": "generating model (exact ZOH modal values); the SVD arm of Table 2 "
                         "is the paper's comparison system and is not built",
            "config": {"fs": 200.0, "N": 60000, "noise": 0.1, "orders": "2..30",
                       "lags_2d": [189], "lags_3d": lags3,
                       "K": "Eq. (empirical_formula) at the largest T: 512 (2D), 664 (3D)", "q": 0,
                       "tau": 0.05, "min_size_2d": 5,
                       "min_size_3d": len(lags3) * len(orders) // 4},
            "rsvd_2d": table(res["rsvd_2d"]), "rsvd_3d": table(res["rsvd_3d"]),
            "ms_per_3d_solve_and_clustering": float(np.median(t_3d))}
    print(json.dumps(line), flush=True)


def run_rank_study(args, world, rank):
    """The parametric analysis of Sec. 3.1 on the 10-DOF frame: for SNR 10, 15, 20 and
    25 dB (5-minute records at 200 Hz) and j_b = 100, 200, ..., --rank-jb-max (T = 10 j_b),
    the minimum rank kbar (percent of T, on a 2.5 % grid) at which the RSVD identification
    (q = 1, orders 10..100) matches the SVD's (paper_2411_05510_gb300/rank_study.py).
    Beside the points: Eq. (empirical_formula) and the least-squares line through them,
    as the paper fits its line before shifting its intercept to 30 %.  Rank 0 only."""
    import torch
    import paper_2411_05510_gb300 as P
    from paper_2411_05510_gb300 import rank_study as RS
    if rank != 0:
        return
    ctx = P.Context(0)
    orders = list(range(10, 101, 2))
    grid = RS.rank_grid(2.5, 60.0, 2.5)
    jbs = list(range(100, args.rank_jb_max + 1, 100))
    points, t0 = [], time.perf_counter()
    for snr in (10, 15, 20, 25):
        w = S.workload("frame10", noise=10 ** (-snr / 20), seed=200 + snr)
        Y, f_true, *_ = S.record(w, np.float32)
        Yd = torch.from_numpy(Y).cuda()
        for jb in jbs:
            T = Y.shape[0] * jb
            ts = time.perf_counter()
            kbar, ref, trace = RS.minimum_rank(ctx, Yd, w["fs"], jb, orders, grid,
                                               f_names=f_true, seed=1, q=1)
            points.append({"snr_db": snr, "jb": jb, "T": T, "kbar_pct": kbar,
                           "modes_svd": len(ref), "trace": trace,
                           "seconds": round(time.perf_counter() - ts, 2)})
    ctx.close()
    xs = np.array([p["T"] for p in points if p["kbar_pct"] is not None], float)
    ys = np.array([p["kbar_pct"] for p in points if p["kbar_pct"] is not None], float)
    fit = None
    if len(xs) >= 2:
        b, a = np.polyfit(xs, ys, 1)
        fit = {"intercept_pct": float(a), "slope_pct_per_T": float(b)}
    line = {"metric": "minimum RSVD rank kbar (percent of T), 10-DOF frame (Sec. 3.1)",
            "unit": "percent", "workload": "rank_study",
            "config": {"fs": 200.0, "N": 60000, "snr_db": [10, 15, 20, 25], "jb": jbs,
                       "orders": "10..100 step 2", "grid_pct": [grid[0], grid[-1], 2.5],
                       "q": 1, "oversample": "K - 100 (k = 100, the largest order)",
                       "match_tol": [0.01, 0.01, 0.02],
                       "sc": [0.02, 0.02, 0.05], "hc": [0.10, 0.6, 0.5],
                       "modes_compared": "the SVD modes nearest the 10 generating frequencies",
                       "svd": "range finder at full width (K = T)"},
            "points": points, "least_squares_line": fit,
            "eq_empirical_formula": {str(p["T"]): max(30 - 0.00156 * p["T"], 25.0)
                                     for p in points},
            "total_s": round(time.perf_counter() - t0, 1)}
    print(json.dumps(line), flush=True)


def l2_note(w):
    mb = w.get("l", w.get("n_dof", 0)) * w["N"] * 4 / 1e6
    if mb > 129:
        return f"inputs larger than L2 (record {mb:.0f} MB fp32 > 129 MB)"
    return f"record {mb:.1f} MB fits in L2; no flush between steps"


def config_of(w, prec):
    cfg = {"workload": w.get("name", None) or "", "channels": w.get("l", w.get("n_dof")),
           "N": w["N"], "fs": w["fs"], "lags": w["lags"], "k": w["k"],
           "oversample": w["oversample"], "q": w["q"],
           "orders": f"{w['orders'][0]}..{w['orders'][-1]} step 2", "prec": prec,
           "l2": l2_note(w)}
    return cfg


# ----------------------------------------------------------------------------- our arm
def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, world, rank)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return

    if args.workload == "serving_mix":
        run_serving_mix(args, world, rank)
        return
    if args.workload == "frame10_table2":
        run_frame10_table2(args, world, rank)
        return
    if args.workload == "rank_study":
        run_rank_study(args, world, rank)
        return

    import torch
    import torch.distributed as dist
    import paper_2411_05510_gb300 as P

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    w = S.workload(args.workload, **({"N": args.n_samples} if args.n_samples else {}))
    w["name"] = args.workload
    Y, f_true, _, phi_true = S.record(w, np.float32)
    l, N = Y.shape
    J = max(1, args.inflight)

    def make_lanes(prec, small="fp32", wl=None, Ydev=None):
        """J independent solvers: own context (workspace), own copy of the record, own
        outputs and own stream."""
        wl = wl or w
        lanes = []
        for j in range(J):
            Yj = torch.from_numpy(Y).to(dev) if Ydev is None else Ydev[j]
            c = P.Context(local)
            c.set_concurrency(J)
            d = P.job_desc(Yj, wl["fs"], wl["lags"], wl["orders"], k=wl["k"],
                           oversample=wl["oversample"], q=wl["q"], prec=prec, seed=12345,
                           small=small)
            n_slots, phi_floats = P.ssi_job_sizes(d)
            lanes.append(dict(ctx=c, Y=Yj, desc=d,
                              poles=torch.zeros((n_slots, P._lib.POLE_BYTES), dtype=torch.uint8,
                                                device=dev),
                              phi=torch.zeros((phi_floats,), dtype=torch.float32, device=dev),
                              stream=torch.cuda.Stream(dev)))
        return lanes

    def solve_on(ln):
        P._lib.check(P._lib.lib.ssi_solve(ln["ctx"].ptr, P._lib.ctypes.byref(ln["desc"]),
                                          P._lib.ctypes.c_void_p(ln["poles"].data_ptr()),
                                          P._lib.ctypes.c_void_p(ln["phi"].data_ptr()), None,
                                          P._lib.ctypes.c_void_p(ln["stream"].cuda_stream)),
                     "ssi_solve")

    def warm(lanes):
        for ln in lanes:
            for _ in range(args.warmup):
                solve_on(ln)
        for ln in lanes:
            P.check_sync(ln["ctx"], dev)

    def run_inflight(lanes, K, sampler=None):
        """K solves dealt round robin over the lanes, each lane's solves in order on its
        stream, the lanes' solves overlapping on the device.  Returns the wall time from the
        first launch to the last completion (CUDA events) and each solve's own duration."""
        s0 = lanes[0]["stream"]
        st = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(K)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        with (sampler if sampler is not None else _Null()):
            e0.record(s0)
            for ln in lanes[1:]:
                ln["stream"].wait_event(e0)
            for s in range(K):
                ln = lanes[s % len(lanes)]
                st[s][0].record(ln["stream"])
                solve_on(ln)
                st[s][1].record(ln["stream"])
            for ln in lanes[1:]:
                ej = torch.cuda.Event()
                ej.record(ln["stream"])
                s0.wait_event(ej)
            e1.record(s0)
            torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        for ln in lanes:
            P.check_sync(ln["ctx"], dev)
        return e0.elapsed_time(e1), [a.elapsed_time(b2) for a, b2 in st]

    def autotune(ls):
        """The library's autotuner on lane 0, its choices copied to the other lanes."""
        if args.no_autotune:
            return None
        t = P.ssi_autotune(ls[0]["ctx"], ls[0]["desc"])
        for ln in ls[1:]:
            P.ssi_tuning_set(ln["ctx"], ln["desc"], t)
        return t

    lanes = make_lanes(args.prec, args.small)
    tuning = autotune(lanes)
    warm(lanes)
    for ln in lanes:
        ln["ctx"].profile_read()   # drop warm-up records
        ln["ctx"].profile(True)     # counts this context's launches (events only, no sync)
    clocks = ClockSampler(local)
    total_ms, step_ms = run_inflight(lanes, args.steps, None if args.no_clocks else clocks)
    launches = 0
    for ln in lanes:
        ln["ctx"].profile(False)
        launches += ln["ctx"].profile_read()[2]
    total_ms = max_over_ranks(total_ms, dev)
    value = whole_job_rate(args.steps, world, total_ms)

    # one solve at a time on lane 0: the latency of an unloaded solve and the per-stage
    # times (CUDA events around each stage on the solve's stream)
    ctx = lanes[0]["ctx"]
    n_ser = max(3, min(args.steps, 10))
    ctx.set_concurrency(1)
    solve_on(lanes[0])   # the first solve with the full-device QR grid, untimed
    ctx.profile(True)
    ser_total, ser_ms = run_inflight(lanes[:1], n_ser)
    ctx.profile(False)
    ctx.set_concurrency(J)
    stage_ms, stage_cnt, _ = ctx.profile_read()
    ser_total = max_over_ranks(ser_total, dev)

    # sanity: the record's modes are found
    rec = P.poles_to_numpy(lanes[0]["poles"])
    top = rec[-(w["orders"][-1] // 2):]
    hc = top[(top["flags"] & 8) != 0]
    found = int(sum(np.min(np.abs(hc["f_hz"] - f0) / f0) < 1e-2 for f0 in f_true)) if len(hc) else 0

    out = {}
    if rank == 0:
        peaks, peak_src = load_peaks()
        K_lag = 2 * max(w["lags"]) - 1
        flops = 2.0 * l * l * N * K_lag
        n_launch = max(1, stage_cnt["lag_gemm"])
        gemm_ms = stage_ms["lag_gemm"] / n_launch
        achieved = flops / (gemm_ms / 1e3) / 1e12
        frac_sus = None
        if args.prec == "split_bf16":
            peak = peaks["bf16_tflops"] / 3.0
            peak_note = (f"bf16_tflops/3 ({peak_src} burst peak, the kernel is timed alone for "
                         f"~4 ms): three BF16 MMAs per split product")
            if "bf16_tflops_sustained" in peaks:
                frac_sus = achieved / (peaks["bf16_tflops_sustained"] / 3.0)
        else:
            peak = 72.0
            peak_note = "FP32 FMA rate 72 TFLOP/s measured by a probe on this GB300"
        traffic, tnote = stored_traffic(args.workload)
        cfg = config_of(w, args.prec)
        cfg["inflight"] = J
        cfg["small"] = args.small
        out = {
            "metric": "SSI solves/s", "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16" if args.prec == "split_bf16" else "f32", "data": "synthetic",
            "config": cfg,
            "latency_ms": {"p50": pct(step_ms, 50), "p99": pct(step_ms, 99),
                           "kind": f"device, each solve from its first launch to its last "
                                   f"completion with {J} solves in flight"},
            "serial": {"value": whole_job_rate(n_ser, world, ser_total), "unit": "solves/s",
                       "solves": n_ser,
                       "latency_ms": {"p50": pct(ser_ms, 50), "p99": pct(ser_ms, 99),
                                      "kind": "device, one solve in flight"}},
            "roofline": {"bound": "tensor" if args.prec == "split_bf16" else "alu",
                         "kernel": "k_lag_gemm_tc" if args.prec == "split_bf16" else "k_lag_gemm_fp32",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "frac_of_sustained": frac_sus,
                         "traffic": traffic, "peak_note": peak_note,
                         "flops_per_launch": flops, "ms_per_launch": gemm_ms,
                         "timing": "CUDA events around the launch on its stream, serial solves",
                         "traffic_note": tnote},
            "stages_ms_per_step": {k: v / n_ser for k, v in stage_ms.items()},
            "gpu_launches": launches,
            "autotune": tuning,
            "modes_found": f"{found}/{len(f_true)}",
            # the same rate per realisation (one eig(A_n) per lag and order) and per pole
            # slot (n/2 per realisation of order n)
            "realisations_per_s": value * len(w["lags"]) * len(w["orders"]),
            "pole_slots_per_s": value * len(w["lags"]) * sum(o // 2 for o in w["orders"]),
        }
        if not args.no_clocks:
            out["clocks"] = clocks.summary()

    # e2e through the serving API, record in pinned host memory: latency with one job in
    # flight, throughput with the jobs submitted back to back (J serving slots, so the
    # host->device copies and the compute of the jobs overlap)
    if not args.no_e2e:
        Yh = torch.from_numpy(Y).pin_memory()
        P.ssi_serve_config(ctx, J, 64)
        desc_h = P.job_desc(Yh, w["fs"], w["lags"], w["orders"], k=w["k"],
                            oversample=w["oversample"], q=w["q"], prec=args.prec, seed=12345)
        n_slots, phi_floats = P.ssi_job_sizes(desc_h)
        n_e2e = max(3 * J, min(args.steps, 12))
        lat = []
        for s in range(2 + 3):
            jid = P.ssi_submit(ctx, desc_h)
            _, _, lu = P.ssi_poll(ctx, jid, -1)
            P.ssi_release(ctx, jid)
            if s >= 2:
                lat.append(lu / 1e3)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        ids = [P.ssi_submit(ctx, desc_h) for _ in range(n_e2e)]
        lat_q = []
        for jid in ids:
            _, _, lu = P.ssi_poll(ctx, jid, -1)
            P.ssi_release(ctx, jid)
            lat_q.append(lu / 1e3)
        t_run = max_over_ranks((time.perf_counter() - t0) * 1e3, dev)
        if rank == 0:
            out["e2e"] = {"value": whole_job_rate(n_e2e, world, t_run), "unit": "solves/s",
                          "h2d_bytes_per_step": int(l * N * 4),
                          "d2h_bytes_per_step": int(n_slots * P._lib.POLE_BYTES + phi_floats * 4),
                          "latency_ms": {"p50": pct(lat, 50), "p99": pct(lat, 99),
                                         "kind": "submit to completion, one job in flight"},
                          "queued_latency_ms": {"p50": pct(lat_q, 50), "p99": pct(lat_q, 99),
                                                "jobs": n_e2e},
                          "api": f"ssi_submit/ssi_poll ({J} slots), record in pinned host "
                                 f"memory, host clock around all jobs"}

    # the next stage of the method on the diagram of the solves above: two-stage clustering
    # of the stable poles into modes (Sec. 2.3, Sec. 3.1), one synchronous call at a time
    if not args.no_cluster:
        ln = lanes[0]
        ln["stream"].synchronize()
        prm = P.cluster_params(tau=0.05, min_size=10 if len(w["lags"]) == 1 else 50)
        n_cl = max(5, min(args.steps, 20))
        tc = []
        torch.cuda.nvtx.range_push("cluster")
        with torch.cuda.stream(ln["stream"]):
            for _ in range(3):
                P.ssi_cluster(ln["ctx"], len(w["lags"]), w["orders"], l, ln["poles"], ln["phi"], prm)
            ln["ctx"].profile(True)
            ln["ctx"].profile_read()
            for _ in range(n_cl):
                t0 = time.perf_counter()
                modes, info, _ = P.ssi_cluster(ln["ctx"], len(w["lags"]), w["orders"], l,
                                               ln["poles"], ln["phi"], prm)
                tc.append((time.perf_counter() - t0) * 1e3)
            st_ms, _, cl_launches = ln["ctx"].profile_read()
            ln["ctx"].profile(False)
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            found = sum(any(abs(m["f_hz"] - f0) / f0 < 1e-2 for m in modes) for f0 in f_true)
            out["cluster"] = {"ms_per_call": pct(tc, 50), "device_ms_per_call": st_ms["cluster"] / n_cl,
                              "kernel_launches_per_call": cl_launches / n_cl, "calls": n_cl,
                              "modes": len(modes), "generating_modes_within_1pct": int(found),
                              "candidates": info["n_candidates"], "kept": info["n_kept"],
                              "fcm_iterations": info["fcm_iterations"],
                              "params": {"tau": 0.05, "min_size": prm.min_size, "fcm_m": 2.0,
                                         "fcm_tol": 1e-10},
                              "api": "ssi_cluster on one solve's poles (synchronous, host clock)"}

    # continuous monitoring: sliding-window covariances of the record (window = the whole
    # record, one-minute blocks), a push against recomputing the window from scratch
    if not args.no_stream:
        ln = lanes[0]
        K = 2 * max(w["lags"]) - 1
        B = int(round(60 * w["fs"]))
        n_fill = N // B
        torch.cuda.nvtx.range_push("cov_stream")
        with torch.cuda.stream(ln["stream"]):
            blocks = [ln["Y"][:, j * B:(j + 1) * B].contiguous() for j in range(n_fill)]
            Yw = ln["Y"][:, :n_fill * B].contiguous()
            cs = P.CovStream(ln["ctx"], l, K, n_fill * B, B, args.prec)
            for j in range(n_fill):
                cs.push(blocks[j])
            n_t = 10
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(ln["stream"])
            for j in range(n_t):
                cs.push(blocks[j])
            ev[1].record(ln["stream"])
            Rw, n_win = cs.covariances()
            ev[2].record(ln["stream"])
            for _ in range(3):
                P.ssi_covariances(ln["ctx"], Yw, K, args.prec)
            ev[3].record(ln["stream"])
            ln["stream"].synchronize()
            cs.close()
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            push_ms = ev[0].elapsed_time(ev[1]) / n_t
            full_ms = ev[2].elapsed_time(ev[3]) / 3
            out["cov_stream"] = {"push_ms": push_ms, "window_recompute_ms": full_ms,
                                 "speedup": full_ms / push_ms, "block_samples": B,
                                 "window_samples": int(n_win), "max_lag": K, "pushes_timed": n_t,
                                 "api": "ssi_cov_stream_push against ssi_covariances of the "
                                        "window (CUDA events on the stream)"}

    def measure(prec, small="fp32", wl=None, n_solves=None, Ydev=None, stages=True):
        """solves/s with J in flight, p50/p99 latency, the serial latency and its stages."""
        ls = make_lanes(prec, small, wl, Ydev)
        tv = autotune(ls)
        saved_warmup = args.warmup
        args.warmup = 1
        warm(ls)
        args.warmup = saved_warmup
        Kx = n_solves or 2 * J
        tx, msx = run_inflight(ls, Kx)
        c0 = ls[0]["ctx"]
        c0.set_concurrency(1)
        solve_on(ls[0])
        c0.profile_read()
        c0.profile(True)
        sx, mss = run_inflight(ls[:1], 3)
        c0.profile(False)
        st_ms, _, _ = c0.profile_read()
        tx = max_over_ranks(tx, dev)
        res = {"value": whole_job_rate(Kx, world, tx), "unit": "solves/s",
               "latency_ms": {"p50": pct(msx, 50), "p99": pct(msx, 99),
                              "kind": f"{J} solves in flight"},
               "serial_latency_ms": pct(mss, 50)}
        if stages:
            res["stages_ms_per_step"] = {k: v / 3 for k, v in st_ms.items() if v > 0}
        if tv is not None:
            res["autotune"] = tv
        for ln in ls:
            ln["ctx"].close()
        return res

    # the plain FP32 path of the same pipeline on the same GPU, measured the same way
    if not args.no_fp32 and args.prec == "split_bf16":
        for ln in lanes[1:]:
            ln["ctx"].close()
        lanes = lanes[:1]
        r32 = measure("fp32", stages=False)
        if rank == 0:
            r32["split_bf16_speedup"] = value / r32["value"]
            out["fp32_path"] = r32

    # the same pipeline with the K x K SVD, A and eig(A) in FP64
    if not args.no_fp64_small and args.small == "fp32":
        for ln in lanes[1:]:
            ln["ctx"].close()
        lanes = lanes[:1]
        r64 = measure(args.prec, "fp64")
        if rank == 0:
            r64["note"] = ("FP64 small problems (one-sided Jacobi, Gram, Cholesky, A~_n, "
                           "Hessenberg and double-shift QR in FP64); GEMMs as the headline")
            out["small_fp64"] = r64

    # the 3D stabilization diagram of the same record: 9 lags x 100 orders per solve
    if not args.no_3d and args.workload == "bridge186_i60":
        w3 = S.workload("bridge186_3d")
        Yd = [ln["Y"] for ln in lanes] + [torch.from_numpy(Y).to(dev) for _ in range(J - len(lanes))]
        r3 = measure(args.prec, "fp32", w3, n_solves=2 * J, Ydev=Yd)
        if rank == 0:
            r3["config"] = {"lags": w3["lags"], "orders": "2..200 step 2", "k": w3["k"],
                            "oversample": w3["oversample"], "q": w3["q"], "realisations": 900}
            out["diagram_3d"] = r3

    # several jobs in one call: the mix's job shapes, their eig launches shared
    if not args.no_batch:
        rb = batch_measure(args, dev, n_jobs=8)
        if rank == 0:
            out["batch"] = rb

    # the serving configuration: a heterogeneous job stream through ssi_submit / ssi_poll
    if not args.no_mix:
        mx = serving_mix_measure(args, world, rank, n_jobs=32)
        if rank == 0:
            out["serving_mix"] = mx

    ora_path = None
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        ora_path, tot, parts, cores = oracle_solve(args)
        est, est_parts = oracle_sample_estimate(Y.astype(np.float64), w)
        out["cpu_baseline"] = {"value": 1.0 / tot, "unit": "solves/s", "cores": cores,
                               "kind": "oracle",
                               "sample": "one complete FP64 oracle solve of the workload, timed "
                                         "(oracle/reference_solve.py)",
                               "threads": "numpy BLAS threads on every core; the oracle's own "
                                          "loops run on one",
                               "stage_s": {k: round(v, 3) for k, v in parts.items()},
                               "sampled_estimate": {"value": 1.0 / est,
                                                    "stage_s": {k: round(v, 3) for k, v in
                                                                est_parts.items()},
                                                    "sample": "covariances on 1/50 of the record, "
                                                              "one Toeplitz product, one QR, one "
                                                              "Jacobi sweep, four realisations, "
                                                              "scaled to one solve"}}
    if rank == 0 and ora_path is not None:
        out["error_vs_oracle"] = error_vs_oracle(P, lanes[0]["ctx"], w, Y, f_true, phi_true,
                                                 ora_path, args.prec, dev)

    if rank == 0:
        print(json.dumps(out), flush=True)
    for ln in lanes:
        ln["ctx"].close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


if __name__ == "__main__":
    main()
