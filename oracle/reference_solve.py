"""One complete FP64 oracle solve of a named workload, stage by stage, timed, and saved.

TEST INFRASTRUCTURE ONLY: used by the benchmark's CPU-baseline and reference arms, which
time the oracle on the host cores and compare the CUDA path's results against the stored
oracle result.  It calls only the oracle and the seeded input generators.

The solve follows Sec. 2.1-2.2 in the oracle's own steps: covariances R_1..R_{2i-1}; per
lag the explicit block Toeplitz T and its randomized SVD with the Philox Omega of the
given seed (Algorithm 1 with oversampling and power iterations); the realisation of
every order from a fresh Householder QR of O^to (numpy eig); the hard and soft
criteria.  ``solve_units`` lists the solve as units of work run in order, so a caller can
spread one solve over several timed steps.

    python -m oracle.reference_solve --workload bridge186_i60 --seed 12345 --out FILE.npz
"""
from __future__ import annotations

import argparse
import os
import sys
import time

import numpy as np

if __package__ in (None, ""):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle as O  # noqa: E402
else:
    from . import ssi_oracle as O  # noqa: E402


def solve_units(Y, w, seed):
    """(state, units): units is a list of (stage name, callable) that, run in order, leave
    in state: R, per lag U and s, the diagram (per lag, per order: mu, f, xi, Phi and,
    after the stability unit, mpc, mpd, flags)."""
    state = {"U": [], "s": [], "diagram": []}
    lags, orders = list(w["lags"]), list(w["orders"])
    l, dt = Y.shape[0], 1.0 / w["fs"]
    K_lag = 2 * max(lags) - 1
    units = [("covariances", lambda: state.__setitem__("R", O.covariances(Y, K_lag)))]

    def rsvd(i):
        U, s = O.rsvd(O.block_toeplitz(state["R"], i), w["k"], w["oversample"], w["q"], seed)
        state["U"].append(U)
        state["s"].append(s)
        state["diagram"].append([])

    def realize(t, i, n):
        mu, f, xi, Phi, _ = O.realize(state["U"][t], state["s"][t], l, i, n, dt)
        state["diagram"][t].append(dict(mu=mu, f=f, xi=xi, Phi=Phi))

    for t, i in enumerate(lags):
        units.append(("toeplitz_rsvd", lambda i=i: rsvd(i)))
        for n in orders:
            units.append(("realisation", lambda t=t, i=i, n=n: realize(t, i, n)))
    units.append(("stability", lambda: O.stability(state["diagram"], use_lag_axis=len(lags) > 1)))
    return state, units


def run(Y, w, seed):
    """Run every unit in order; returns (state, seconds per stage)."""
    state, units = solve_units(Y, w, seed)
    stage_s = {}
    for name, fn in units:
        t0 = time.perf_counter()
        fn()
        stage_s[name] = stage_s.get(name, 0.0) + time.perf_counter() - t0
    return state, stage_s


def save(path, w, seed, state, stage_s, cores):
    """Flatten the diagram: per (lag, order) the pole count, then the poles' mu, f, xi,
    mpc, mpd, flags and Phi in that order."""
    counts, mu, f, xi, mpc, mpd, flags, phi = [], [], [], [], [], [], [], []
    for row in state["diagram"]:
        for c in row:
            counts.append(len(c["f"]))
            mu.append(c["mu"]); f.append(c["f"]); xi.append(c["xi"])
            mpc.append(c["mpc"]); mpd.append(c["mpd"]); flags.append(c["flags"])
            phi.append(c["Phi"].T)
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)  # noqa: E731
    l = state["U"][0].shape[0] // w["lags"][0] if state["U"] else 0
    np.savez(path, workload=str(w.get("name", "")), seed=seed, lags=np.array(w["lags"]),
             orders=np.array(w["orders"]), counts=np.array(counts, np.int64),
             mu=cat(mu, np.complex128), f=cat(f, np.float64), xi=cat(xi, np.float64),
             mpc=cat(mpc, np.float64), mpd=cat(mpd, np.float64), flags=cat(flags, np.int64),
             phi=np.concatenate(phi).astype(np.complex128) if phi else np.zeros((0, l), np.complex128),
             s=np.stack(state["s"]), U=np.stack(state["U"]) if len(set(u.shape for u in state["U"])) == 1
             else np.zeros(0), stage_names=np.array(list(stage_s.keys())),
             stage_s=np.array(list(stage_s.values())), cores=cores)


def main():
    import ssi_synth as S
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="bridge186_i60")
    ap.add_argument("--seed", type=int, default=12345)
    ap.add_argument("--n-samples", type=int, default=0)
    ap.add_argument("--out", required=True)
    a = ap.parse_args()
    w = S.workload(a.workload, **({"N": a.n_samples} if a.n_samples else {}))
    w["name"] = a.workload
    Y, *_ = S.record(w, np.float32)
    Y = Y.astype(np.float64)
    state, stage_s = run(Y, w, a.seed)
    save(a.out, w, a.seed, state, stage_s, os.cpu_count())
    print(f"oracle solve of {a.workload}: {sum(stage_s.values()):.1f} s "
          + " ".join(f"{k} {v:.1f}" for k, v in stage_s.items()), flush=True)


if __name__ == "__main__":
    main()
