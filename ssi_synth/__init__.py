"""Seeded synthetic structures and output records for covariance-driven SSI.

This module holds only the generating models (structural dynamics, sampling,
sensor noise) and the named workloads.  It contains none of the identification
method's arithmetic: no covariance estimation, no Toeplitz assembly, no SVD and
no realisation.  Both the FP64 oracle (``oracle/``) and the CUDA path's tests and
benchmark draw their inputs from here, so the two sides see identical records.

Models
------
* ``shear_chain``: fixed-base lumped shear chain (the 10-DOF frame of Sec. 3.1,
  storey mass 100 kg and storey stiffness 5000 kN/m, and the small 4-DOF chain).
* ``rayleigh_damping`` / ``modal_damping``: the two damping models used.
* ``chain_state_space``: continuous model -> exact zero-order-hold discrete
  stochastic state-space model x_{h+1} = A x_h + B u_h, y_h = C x_h + D u_h
  (the discrete model of Sec. 2.1), with unit white Gaussian input u_h.
* ``bridge_record``: modal superposition on a 3-span deck with triaxial
  stations; each modal coordinate is an exact ZOH-discretised second-order
  filter driven by unit white noise.

Every random draw comes from ``numpy.random.Generator(PCG64(seed))``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.linalg
import scipy.signal

__all__ = [
    "shear_chain", "rayleigh_damping", "modal_damping", "DiscreteModel",
    "chain_state_space", "simulate", "stationary_state_cov", "model_covariances",
    "BridgeRecord", "bridge_record", "WORKLOADS", "workload", "serving_mix",
]


# ----------------------------------------------------------------------------
# structural matrices
# ----------------------------------------------------------------------------
def shear_chain(n: int, mass: float, stiffness: float):
    """Mass and stiffness matrices of a fixed-base shear chain of ``n`` storeys.

    Storey j (0 = bottom) has mass ``mass``; the spring below storey j has
    stiffness ``stiffness`` (the bottom spring ties storey 0 to the ground).
    """
    M = np.eye(n) * float(mass)
    K = np.zeros((n, n))
    for j in range(n):
        K[j, j] += stiffness
        if j + 1 < n:
            K[j, j] += stiffness
            K[j, j + 1] -= stiffness
            K[j + 1, j] -= stiffness
    return M, K


def _undamped_modes(M, K):
    w2, phi = scipy.linalg.eigh(K, M)
    return np.sqrt(w2), phi


def rayleigh_damping(M, K, mode_a: int, mode_b: int, xi: float):
    """C = a M + b K with damping ratio ``xi`` at modes ``mode_a``/``mode_b`` (1-based)."""
    w, _ = _undamped_modes(M, K)
    wa, wb = w[mode_a - 1], w[mode_b - 1]
    # xi = a/(2w) + b w/2 at both frequencies
    lhs = np.array([[1.0 / (2 * wa), wa / 2.0], [1.0 / (2 * wb), wb / 2.0]])
    a, b = np.linalg.solve(lhs, np.array([xi, xi]))
    return a * M + b * K


def modal_damping(M, K, xi: float):
    """Classical damping with the same ratio ``xi`` in every mode."""
    w, phi = _undamped_modes(M, K)          # phi^T M phi = I
    Mphi = M @ phi
    return Mphi @ np.diag(2.0 * xi * w) @ Mphi.T


# ----------------------------------------------------------------------------
# discrete stochastic state-space model
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class DiscreteModel:
    A: np.ndarray      # (2n, 2n)
    B: np.ndarray      # (2n, m)
    C: np.ndarray      # (l, 2n)
    D: np.ndarray      # (l, m)
    dt: float
    f_true: np.ndarray     # (n,) natural frequencies of the damped system [Hz]
    xi_true: np.ndarray    # (n,) damping ratios
    phi_true: np.ndarray   # (l, n) complex mode shapes at the outputs


def _zoh(Ac, Bc, dt):
    """Exact zero-order-hold discretisation via the augmented exponential."""
    ns, m = Bc.shape
    big = np.zeros((ns + m, ns + m))
    big[:ns, :ns] = Ac
    big[:ns, ns:] = Bc
    e = scipy.linalg.expm(big * dt)
    return e[:ns, :ns], e[:ns, ns:]


def _continuous_modes(Ac, Cc):
    lam, psi = np.linalg.eig(Ac)
    keep = lam.imag > 0
    lam, psi = lam[keep], psi[:, keep]
    order = np.argsort(np.abs(lam))
    lam, psi = lam[order], psi[:, order]
    f = np.abs(lam) / (2 * np.pi)
    xi = -lam.real / np.abs(lam)
    return f, xi, Cc @ psi


def chain_state_space(M, K, Cdamp, dt: float, excitation: str):
    """Discrete model of a chain measured by absolute floor accelerations.

    ``excitation='base'``: white ground acceleration a_g (one input);
    the absolute accelerations are -M^{-1}(C v + K u), so D = 0.
    ``excitation='floors'``: an independent white force at every floor;
    the accelerations are M^{-1}(f - C v - K u), so D = M^{-1}.
    """
    n = M.shape[0]
    Minv = np.linalg.inv(M)
    Ac = np.zeros((2 * n, 2 * n))
    Ac[:n, n:] = np.eye(n)
    Ac[n:, :n] = -Minv @ K
    Ac[n:, n:] = -Minv @ Cdamp
    Cc = np.hstack([-Minv @ K, -Minv @ Cdamp])
    if excitation == "base":
        Bc = np.zeros((2 * n, 1))
        Bc[n:, 0] = -1.0
        Dc = np.zeros((n, 1))
    elif excitation == "floors":
        Bc = np.zeros((2 * n, n))
        Bc[n:, :] = Minv
        Dc = Minv.copy()
    else:
        raise ValueError(excitation)
    Ad, Bd = _zoh(Ac, Bc, dt)
    f, xi, phi = _continuous_modes(Ac, Cc)
    return DiscreteModel(Ad, Bd, Cc, Dc, dt, f, xi, phi)


def stationary_state_cov(model: DiscreteModel):
    """Sigma = A Sigma A^T + B B^T (unit-variance white input)."""
    return scipy.linalg.solve_discrete_lyapunov(model.A, model.B @ model.B.T)


def model_covariances(model: DiscreteModel, max_lag: int):
    """Exact output covariances of the model, lags 0..max_lag.

    R_0 = C Sigma C^T + D D^T, and for j >= 1 R_j = C A^{j-1} G with
    G = A Sigma C^T + B D^T (the factorisation quoted in Sec. 2.1).
    Returns an array of shape (max_lag + 1, l, l).
    """
    S = stationary_state_cov(model)
    A, C, B, D = model.A, model.C, model.B, model.D
    G = A @ S @ C.T + B @ D.T
    out = np.empty((max_lag + 1, C.shape[0], C.shape[0]))
    out[0] = C @ S @ C.T + D @ D.T
    Ak = np.eye(A.shape[0])
    for j in range(1, max_lag + 1):
        out[j] = C @ Ak @ G
        Ak = Ak @ A
    return out


def simulate(model: DiscreteModel, N: int, seed: int, noise_frac: float):
    """Stationary simulation of ``model`` for N samples plus sensor noise.

    The initial state is drawn from the stationary distribution, so every
    sample of the record is stationary.  Sensor noise is white Gaussian with a
    standard deviation of ``noise_frac`` times each channel's exact standard
    deviation.  Returns Y with shape (l, N), float64.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    S = stationary_state_cov(model)
    ns = model.A.shape[0]
    x = np.linalg.cholesky(S + 1e-300 * np.eye(ns)) @ rng.standard_normal(ns)
    u = rng.standard_normal((N, model.B.shape[1]))
    X = np.empty((N, ns))
    A, B = model.A, model.B
    for h in range(N):
        X[h] = x
        x = A @ x + B @ u[h]
    Y = X @ model.C.T + u @ model.D.T
    R0 = model.C @ S @ model.C.T + model.D @ model.D.T
    std = np.sqrt(np.diag(R0))
    Y += rng.standard_normal(Y.shape) * (noise_frac * std)[None, :]
    return np.ascontiguousarray(Y.T)


# ----------------------------------------------------------------------------
# bridge-scale modal superposition records
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class BridgeRecord:
    Y: np.ndarray          # (l, N) float64
    fs: float
    f_true: np.ndarray     # (m,)
    xi_true: np.ndarray    # (m,)
    phi_true: np.ndarray   # (l, m) real mode shapes


def _station_layout(n_channels: int):
    """(position along the deck in [0,1), axis) for every channel.

    Channels come in triaxial stations at s_j = (j + 0.5)/n_st; when the count
    is not a multiple of three the last station keeps only its first axes.
    """
    n_st = -(-n_channels // 3)
    pos, axis = [], []
    for c in range(n_channels):
        j, a = divmod(c, 3)
        pos.append((j + 0.5) / n_st)
        axis.append(a)
    return np.asarray(pos), np.asarray(axis)


def _modal_filter(f_hz: float, xi: float, dt: float):
    """Exact ZOH discretisation of q'' + 2 xi w q' + w^2 q = u as (b, a), scaled to
    unit stationary variance of q."""
    w = 2 * np.pi * f_hz
    Ac = np.array([[0.0, 1.0], [-w * w, -2 * xi * w]])
    Bc = np.array([[0.0], [1.0]])
    Ad, Bd = _zoh(Ac, Bc, dt)
    S = scipy.linalg.solve_discrete_lyapunov(Ad, Bd @ Bd.T)
    gain = 1.0 / math.sqrt(S[0, 0])
    # q_h = c (zI - Ad)^{-1} Bd u: numerator from the adjugate, denominator det(zI - Ad)
    a1 = -np.trace(Ad)
    a2 = np.linalg.det(Ad)
    b1 = Bd[0, 0]
    b2 = Ad[0, 1] * Bd[1, 0] - Ad[1, 1] * Bd[0, 0]
    return np.array([0.0, b1, b2]) * gain, np.array([1.0, a1, a2]), Ad


def bridge_record(n_channels: int, n_modes: int, f_lo: float, f_hi: float, fs: float,
                  N: int, noise_frac: float, seed: int, dtype=np.float64) -> BridgeRecord:
    """Synthetic ambient-vibration record of a 3-span deck (modal superposition).

    * frequencies log-uniform in [f_lo, f_hi], damping uniform in [0.5 %, 3 %];
    * shape of mode r on axis a: w_{r,a} sin(3 pi h_r s + theta_{r,a}) with
      h_r = 1 + (r mod 6) half-waves per span, w ~ U[0.2, 1], theta ~ U[0, 2 pi);
    * each modal coordinate is an exact ZOH-discretised second-order filter
      driven by unit white noise, scaled to unit stationary variance, started
      from its stationary distribution (a burn-in of ten decay times);
    * sensor noise: white, ``noise_frac`` times each channel's standard deviation.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    f = np.sort(np.exp(rng.uniform(np.log(f_lo), np.log(f_hi), n_modes)))
    xi = rng.uniform(0.005, 0.03, n_modes)
    w_amp = rng.uniform(0.2, 1.0, (n_modes, 3))
    theta = rng.uniform(0.0, 2 * np.pi, (n_modes, 3))
    s, axis = _station_layout(n_channels)
    phi = np.empty((n_channels, n_modes))
    for r in range(n_modes):
        h = 1 + (r % 6)
        phi[:, r] = w_amp[r, axis] * np.sin(3 * np.pi * h * s + theta[r, axis])
    dt = 1.0 / fs
    q = np.empty((n_modes, N))
    for r in range(n_modes):
        b, a, _ = _modal_filter(f[r], xi[r], dt)
        burn = int(min(200000, 10.0 / (xi[r] * 2 * np.pi * f[r]) * fs)) + 16
        u = rng.standard_normal(N + burn)
        q[r] = scipy.signal.lfilter(b, a, u)[burn:]
    Y = phi @ q
    std = np.sqrt(np.sum(phi * phi, axis=1))       # unit-variance, independent modes
    Y += rng.standard_normal(Y.shape) * (noise_frac * std)[:, None]
    return BridgeRecord(np.ascontiguousarray(Y.astype(dtype)), fs, f, xi, phi)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
WORKLOADS = {
    # 4-DOF chain, masses 1, springs 1e3, 2 % modal damping, base excitation
    "chain4_tiny": dict(kind="chain", n_dof=4, mass=1.0, stiffness=1e3, damping=("modal", 0.02),
                        excitation="base", fs=100.0, N=20000, noise=0.01, seed=0,
                        lags=[20], k=80, oversample=0, q=0, orders=list(range(2, 41, 2)),
                        full_svd=True),
    # 186 channels, 20 modes, one lag i=60, RSVD k=200 p=20 q=2, orders 2..200
    "bridge186_i60": dict(kind="bridge", l=186, modes=20, f_lo=1.0, f_hi=20.0, fs=100.0,
                          N=360000, noise=0.05, seed=1, lags=[60], k=200, oversample=20, q=2,
                          orders=list(range(2, 201, 2))),
    # same record, 3D diagram over 9 lags
    "bridge186_3d": dict(kind="bridge", l=186, modes=20, f_lo=1.0, f_hi=20.0, fs=100.0,
                         N=360000, noise=0.05, seed=1, lags=list(range(20, 101, 10)), k=200,
                         oversample=20, q=2, orders=list(range(2, 201, 2))),
    # 512 channels, 40 modes, i=100, k=400 p=40 q=3, orders 2..400
    "bridge512_i100": dict(kind="bridge", l=512, modes=40, f_lo=0.5, f_hi=30.0, fs=100.0,
                           N=1080000, noise=0.05, seed=5, lags=[100], k=400, oversample=40, q=3,
                           orders=list(range(2, 401, 2))),
    # 10-DOF frame of Sec. 3.1 (Rayleigh 1 % at modes 1 and 4), floor forces, fs 200 Hz
    "frame10": dict(kind="chain", n_dof=10, mass=100.0, stiffness=5e6, damping=("rayleigh", 0.01),
                    excitation="floors", fs=200.0, N=60000, noise=0.1, seed=7,
                    lags=[189], k=512, oversample=0, q=0, orders=list(range(2, 31, 2))),
}


def workload(name: str, **overrides):
    """Parameters of a named workload, with optional overrides."""
    w = dict(WORKLOADS[name])
    w.update(overrides)
    return w


def chain_model(w: dict) -> DiscreteModel:
    M, K = shear_chain(w["n_dof"], w["mass"], w["stiffness"])
    kind, xi = w["damping"]
    Cd = modal_damping(M, K, xi) if kind == "modal" else rayleigh_damping(M, K, 1, 4, xi)
    return chain_state_space(M, K, Cd, 1.0 / w["fs"], w["excitation"])


def record(w: dict, dtype=np.float64):
    """Y (l, N) for a workload dict, and the true modal values (f, xi, phi)."""
    if w["kind"] == "chain":
        model = chain_model(w)
        Y = simulate(model, w["N"], w["seed"], w["noise"]).astype(dtype)
        return Y, model.f_true, model.xi_true, model.phi_true
    rec = bridge_record(w["l"], w["modes"], w["f_lo"], w["f_hi"], w["fs"], w["N"], w["noise"],
                        w["seed"], dtype)
    return rec.Y, rec.f_true, rec.xi_true, rec.phi_true


def serving_mix(n_jobs: int, seed: int = 4, channels=(16, 48, 96, 186), N_range=(30000, 360000),
                i_range=(20, 80), modes_range=(5, 30)):
    """Workload dicts of a heterogeneous job stream (bridge records of uneven size).

    Per job: l uniform over ``channels``; N, i and the number of modes uniform
    integers in their ranges; frequencies and damping as in ``bridge_record``;
    orders 2..2m+40 step 2 with k = the largest order, oversampling 20, q = 2.
    Each job has its own record seed.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for j in range(n_jobs):
        l = int(rng.choice(channels))
        N = int(rng.integers(N_range[0], N_range[1] + 1))
        i = int(rng.integers(i_range[0], i_range[1] + 1))
        m = int(rng.integers(modes_range[0], modes_range[1] + 1))
        n_max = 2 * m + 40
        jobs.append(dict(kind="bridge", l=l, modes=m, f_lo=1.0, f_hi=20.0, fs=100.0, N=N,
                         noise=0.05, seed=1000 * seed + j, lags=[i], k=n_max, oversample=20, q=2,
                         orders=list(range(2, n_max + 1, 2))))
    return jobs
