"""Plain FP64 oracle of RSVD-based covariance-driven SSI (arXiv 2411.05510).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline arm, never by the product path.  It shares no code,
table or constant generator with the CUDA library.

Everything is float64 NumPy, written step by step in the paper's order and
notation.  Library routines appear only as single steps: a matrix product
(``@``), ``numpy.linalg.eig`` for the eigen-decomposition of A, ``numpy.log`` of
a complex number.  The SVD is a one-sided (Hestenes) Jacobi SVD written out
here; the QR factorisations are Householder QR written out here.

Readings of the paper where it is silent, garbled or ambiguous (each is listed
again in the design notes):

* Eq. for f and xi (Sec. 2.1): the printed f = Re(lambda)/(2 pi xi) and
  xi = Re(mu)/|mu| are garbled.  Read with lambda = -xi w + i w sqrt(1-xi^2):
  lambda = ln(mu)/dt, f = |lambda|/(2 pi), xi = -Re(lambda)/|lambda|.
* The eigen-decomposition printed as A = Psi M Psi^T is read A = Psi M Psi^{-1},
  Psi in C^{n x n}, Phi = C Psi.
* O^to / O^bo are the first / last l(j_b - 1) rows of O.
* Covariances R_1..R_{2 j_b - 1} with normalisation 1/(N - k), no mean removal.
* Omega has as many rows as T has columns (Algorithm 1 writes randn(m, k)).
* Oversampling p and q power iterations, re-orthonormalised by QR after every
  product; with p = q = 0 the range finder is Algorithm 1 exactly.
* Soft criteria: "m-1" is the previous analysed order, "t-1" the previous lag
  of the grid; a pole is stable along an axis if SOME pole at the neighbouring
  order (lag) passes all three thresholds; stable = HC and (order or lag).
  The MAC criterion is 1 - MAC <= alpha_MAC.  Neighbour poles must pass HC.
* MPC / MPD: from X = [Re phi, Im phi] (uncentred).  MPC = ((s1^2 - s2^2)/
  (s1^2 + s2^2))^2; MPD = |phi_j|-weighted mean angle between (Re phi_j, Im phi_j)
  and the principal line of X, divided by 90 degrees.
* Only eigenvalues with Im(mu) > 0 become poles (one per conjugate pair).
* "int(.)" in the time-lag rules is the ceiling (reproduces 189, 170, 76, 69,
  104 and 512 quoted in Sec. 3).
* Two-stage clustering (Sec. 2.3 "3D clustering", Sec. 3.1):
  * Stage I features of a stable pole: (d_f, d_xi, 1 - MAC) to its nearest HC-passing
    neighbour (previous order of the same lag or same order of the previous lag),
    nearest in d_f + d_xi + (1 - MAC), then 1 - MPC and MPD of the pole.
  * Fuzzy C-means with two clusters and fuzzifier 2, started from the feature-wise
    minimum and maximum.  The cluster whose centroid is nearer the origin is the
    possibly physical one; poles with membership >= 0.5 in it are kept.  A cluster whose
    memberships are all zero (every pole on the other centroid, e.g. a single pole)
    keeps its centroid instead of the undefined 0/0 update.
  * Stage II: single linkage in d_f + d_xi + (1 - MAC), cut at a distance tau;
    clusters of at least min_size poles are modes (mean f and xi, medoid pole).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "philox4x32_10", "gaussian_omega",
    "covariances", "covariance_entry", "block_toeplitz",
    "householder_qr", "jacobi_svd", "full_svd", "rsvd",
    "realize", "poles_from_eig", "mpc", "mpd", "mac", "normalize_shape",
    "hard_criteria", "stability", "rank_rule", "lag_rule", "time_lag",
    "ssi_solve", "HC_XI", "HC_MPC", "HC_MPD", "ST_HC", "ST_ORDER", "ST_LAG",
    "rel_diff", "pole_distance", "stage1_features", "fuzzy_c_means", "stage1",
    "single_linkage_labels", "stage2", "cluster_modes",
]

# ---------------------------------------------------------------------------
# Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11)
# ---------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds on uint32 counter words (arrays) with a 64-bit key.

    Round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); key bumped by (W0, W1).
    """
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & _MASK32 for x in (c0, c1, c2, c3))
    k0 = np.uint64(k0) & _MASK32
    k1 = np.uint64(k1) & _MASK32
    for _ in range(10):
        p0 = _PHILOX_M0 * c0
        p1 = _PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK32, lo1, (hi0 ^ c3 ^ k1) & _MASK32, lo0
        k0 = (k0 + _PHILOX_W0) & _MASK32
        k1 = (k1 + _PHILOX_W1) & _MASK32
    return c0, c1, c2, c3


def gaussian_omega(rows: int, cols: int, seed: int):
    """Gaussian test matrix Omega (Sec. 2.2, Eq. for Y = A Omega), rows x cols.

    Entry (r, c) uses the Philox counter (r, c, 0, 0) with key (seed low 32
    bits, seed high 32 bits).  Outputs x0, x1 become uniforms
    u = (x + 0.5) / 2^32 and one Box-Muller normal
    z = sqrt(-2 ln u0) cos(2 pi u1).
    """
    r = np.repeat(np.arange(rows, dtype=np.uint64), cols)
    c = np.tile(np.arange(cols, dtype=np.uint64), rows)
    x0, x1, _, _ = philox4x32_10(r, c, 0, 0, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)
    u0 = (x0.astype(np.float64) + 0.5) / 4294967296.0
    u1 = (x1.astype(np.float64) + 0.5) / 4294967296.0
    z = np.sqrt(-2.0 * np.log(u0)) * np.cos(2.0 * np.pi * u1)
    return z.reshape(rows, cols)


# ---------------------------------------------------------------------------
# Sec. 2.1: output covariances and the block-Toeplitz matrix
# ---------------------------------------------------------------------------
def covariances(Y, max_lag: int):
    """R_k = 1/(N-k) sum_{t=0}^{N-k-1} y_{t+k} y_t^T for k = 1..max_lag (Sec. 2.1).

    Y is (l, N).  Returns (max_lag, l, l) float64 with R_k at index k-1.  Each
    lag is one matrix product of the shifted records.
    """
    Y = np.asarray(Y, dtype=np.float64)
    l, N = Y.shape
    R = np.empty((max_lag, l, l))
    for k in range(1, max_lag + 1):
        R[k - 1] = (Y[:, k:] @ Y[:, :N - k].T) / (N - k)
    return R


def covariance_entry(Y, k: int, a: int, b: int) -> float:
    """One entry R_k[a, b] as a plain dot product (for sampled checks at any size)."""
    Y = np.asarray(Y)
    N = Y.shape[1]
    return float(np.dot(Y[a, k:].astype(np.float64), Y[b, :N - k].astype(np.float64)) / (N - k))


def block_toeplitz(R, i: int):
    """T_{1|i} of Eq. (Toeplitz): block (a, b) = R_{i + a - b}, a, b = 0..i-1.

    R holds R_1.. at indices 0.., so block (a, b) is R[i + a - b - 1].
    """
    l = R.shape[1]
    T = np.empty((i * l, i * l))
    for a in range(i):
        for b in range(i):
            T[a * l:(a + 1) * l, b * l:(b + 1) * l] = R[i + a - b - 1]
    return T


# ---------------------------------------------------------------------------
# Householder QR and one-sided Jacobi SVD
# ---------------------------------------------------------------------------
def householder_qr(A):
    """Economy QR, A = Q R with Q (m x n) orthonormal, R (n x n) upper triangular.

    Column j: reflector H = I - 2 v v^T / (v^T v) maps A[j:, j] to alpha e_1 with
    alpha = -sign(A[j, j]) ||A[j:, j]||.  Q is formed by applying the reflectors
    in reverse order to the first n columns of the identity.
    """
    R = np.array(A, dtype=np.float64, copy=True)
    m, n = R.shape
    if m < n:
        raise ValueError("householder_qr expects m >= n")
    vs = []
    for j in range(n):
        x = R[j:, j]
        nx = math.sqrt(float(x @ x))
        if nx == 0.0:
            vs.append(None)
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        vv = float(v @ v)
        R[j:, j:] -= np.outer(v, (2.0 / vv) * (v @ R[j:, j:]))
        vs.append((v, vv))
    Q = np.zeros((m, n))
    Q[:n, :n] = np.eye(n)
    for j in range(n - 1, -1, -1):
        if vs[j] is None:
            continue
        v, vv = vs[j]
        Q[j:, :] -= np.outer(v, (2.0 / vv) * (v @ Q[j:, :]))
    return Q, np.triu(R[:n, :])


def _round_robin(n_pad):
    """Pairings of the circle method: n_pad - 1 rounds of n_pad/2 disjoint pairs."""
    players = list(range(n_pad))
    rounds = []
    for _ in range(n_pad - 1):
        half = n_pad // 2
        rounds.append([(players[i], players[n_pad - 1 - i]) for i in range(half)])
        players = [players[0]] + [players[-1]] + players[1:-1]
    return rounds


def jacobi_svd(A, tol: float = 1e-15, max_sweeps: int = 30):
    """One-sided (Hestenes) Jacobi SVD of A (m x n, m >= n): A = U diag(s) V^T.

    Column pairs (p, q) are rotated until every pair is orthogonal to
    |a_p^T a_q| <= tol ||a_p|| ||a_q||.  Rotation: zeta = (b - a)/(2 g),
    t = sign(zeta)/(|zeta| + sqrt(1 + zeta^2)), c = 1/sqrt(1 + t^2), s = c t,
    a = ||a_p||^2, b = ||a_q||^2, g = a_p^T a_q.  Each round of the circle
    ordering rotates disjoint pairs (vectorised).  Returns U (m x n), s
    (descending), V (n x n) and the number of sweeps used.
    """
    W = np.array(A, dtype=np.float64, copy=True)
    m, n = W.shape
    if m < n:
        raise ValueError("jacobi_svd expects m >= n")
    V = np.eye(n)
    n_pad = n + (n % 2)
    rounds = []
    for rnd in _round_robin(n_pad):
        pq = np.array([(p, q) for p, q in rnd if p < n and q < n], dtype=np.int64).reshape(-1, 2)
        rounds.append((pq[:, 0], pq[:, 1]))
    sweeps = 0
    for sweep in range(max_sweeps):
        sweeps = sweep + 1
        rotated = False
        for p, q in rounds:
            if p.size == 0:
                continue
            ap, aq = W[:, p], W[:, q]
            a = np.einsum("ij,ij->j", ap, ap)
            b = np.einsum("ij,ij->j", aq, aq)
            g = np.einsum("ij,ij->j", ap, aq)
            act = np.abs(g) > tol * np.sqrt(a * b)
            if not act.any():
                continue
            rotated = True
            p, q, a, b, g = p[act], q[act], a[act], b[act], g[act]
            zeta = (b - a) / (2.0 * g)
            t = np.where(zeta >= 0, 1.0, -1.0) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
            c = 1.0 / np.sqrt(1.0 + t * t)
            s = c * t
            wp, wq = W[:, p], W[:, q]
            W[:, p], W[:, q] = c * wp - s * wq, s * wp + c * wq
            vp, vq = V[:, p], V[:, q]
            V[:, p], V[:, q] = c * vp - s * vq, s * vp + c * vq
        if not rotated:
            break
    sv = np.sqrt(np.einsum("ij,ij->j", W, W))
    order = np.argsort(-sv, kind="stable")
    sv, W, V = sv[order], W[:, order], V[:, order]
    U = np.zeros_like(W)
    nz = sv > 0
    U[:, nz] = W[:, nz] / sv[nz]
    return U, sv, V, sweeps


def full_svd(T):
    """Eq. (SVD) of a square T by the one-sided Jacobi SVD: returns U, s."""
    U, s, _, _ = jacobi_svd(T)
    return U, s


# ---------------------------------------------------------------------------
# Sec. 2.2, Algorithm 1: randomized SVD with oversampling and power iterations
# ---------------------------------------------------------------------------
def rsvd(T, k: int, oversample: int = 0, q: int = 0, seed: int = 0, omega=None):
    """Randomized SVD of T (Algorithm 1), returning U (rows x k) and S (k,).

    Omega = randn(cols, k + p) (Philox, ``gaussian_omega``); Y = T Omega;
    (Q, R) = qr(Y); q times: Q = qr(T Q_z) with Q_z = qr(T^T Q); P = Q^T T;
    (U~, S, V) = svd(P, econ) via Jacobi on P^T; U = Q U~.
    """
    T = np.asarray(T, dtype=np.float64)
    K = k + oversample
    if omega is None:
        omega = gaussian_omega(T.shape[1], K, seed)
    Y = T @ omega
    Q, _ = householder_qr(Y)
    for _ in range(q):
        Z = T.T @ Q
        Qz, _ = householder_qr(Z)
        Y = T @ Qz
        Q, _ = householder_qr(Y)
    P = Q.T @ T
    # P^T = W diag(s) V^T  =>  P = V diag(s) W^T, so U~ = V
    _, s, V, _ = jacobi_svd(P.T)
    U = Q @ V[:, :k]
    return U, s[:k]


# ---------------------------------------------------------------------------
# Sec. 2.1: realisation, eigen-decomposition and modal parameters
# ---------------------------------------------------------------------------
def normalize_shape(phi):
    """Unit 2-norm, largest-modulus component real and positive (output only)."""
    phi = np.asarray(phi, dtype=np.complex128)
    j = int(np.argmax(np.abs(phi)))
    phase = phi[j] / abs(phi[j]) if abs(phi[j]) > 0 else 1.0
    out = phi / phase
    nrm = np.linalg.norm(out)
    return out / nrm if nrm > 0 else out


def mac(a, b) -> float:
    """MAC(a, b) = |a^H b|^2 / ((a^H a)(b^H b))."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    num = abs(np.vdot(a, b)) ** 2
    den = np.vdot(a, a).real * np.vdot(b, b).real
    return float(num / den) if den > 0 else 0.0


def _xtx(phi):
    X = np.stack([np.real(phi), np.imag(phi)], axis=1)
    return X, X.T @ X


def mpc(phi) -> float:
    """Modal phase collinearity: ((s1^2 - s2^2)/(s1^2 + s2^2))^2, s from X = [Re, Im]."""
    _, S = _xtx(phi)
    tr = S[0, 0] + S[1, 1]
    if tr <= 0:
        return 0.0
    # eigenvalues of the symmetric 2x2 X^T X
    d = math.sqrt(max((S[0, 0] - S[1, 1]) ** 2 + 4 * S[0, 1] ** 2, 0.0))
    e1, e2 = (tr + d) / 2, (tr - d) / 2
    return float(((e1 - e2) / (e1 + e2)) ** 2)


def mpd(phi) -> float:
    """Mean phase deviation in [0, 1]: |phi_j|-weighted mean angle (degrees) between
    (Re phi_j, Im phi_j) and the principal line of X = [Re phi, Im phi], / 90."""
    X, S = _xtx(phi)
    w, v = np.linalg.eigh(S)
    v1 = v[:, int(np.argmax(w))]
    nrm = np.sqrt(np.sum(X * X, axis=1))
    nz = nrm > 0
    if not nz.any():
        return 0.0
    cosang = np.clip(np.abs(X[nz] @ v1) / nrm[nz], 0.0, 1.0)
    ang = np.degrees(np.arccos(cosang))
    return float(np.sum(nrm[nz] * ang) / np.sum(nrm[nz]) / 90.0)


def poles_from_eig(mu, Psi, C, dt):
    """Modal parameters from eig(A) (Sec. 2.1): lambda = ln(mu)/dt, f = |lambda|/(2 pi),
    xi = -Re(lambda)/|lambda|, Phi = C Psi; one pole per conjugate pair (Im mu > 0)."""
    keep = np.imag(mu) > 0
    mu, Psi = mu[keep], Psi[:, keep]
    lam = np.log(mu) / dt
    f = np.abs(lam) / (2 * np.pi)
    xi = -np.real(lam) / np.abs(lam)
    Phi = C @ Psi
    order = np.argsort(f, kind="stable")
    return mu[order], f[order], xi[order], Phi[:, order]


def realize(U, S, l: int, i: int, n: int, dt: float):
    """One model order n of Sec. 2.1: O = U S^{1/2}, C = first l rows, A = O^to+ O^bo.

    The pseudo-inverse is applied through a fresh Householder QR of O^to:
    A = R^{-1} Q^T O^bo (back substitution).  Returns (mu, f, xi, Phi, A).
    """
    O = U[:, :n] * np.sqrt(S[:n])[None, :]
    C = O[:l, :]
    O_to = O[:l * (i - 1), :]
    O_bo = O[l:l * i, :]
    Qo, Ro = householder_qr(O_to)
    rhs = Qo.T @ O_bo
    A = np.zeros((n, n))
    for r in range(n - 1, -1, -1):
        A[r] = (rhs[r] - Ro[r, r + 1:] @ A[r + 1:]) / Ro[r, r]
    mu, Psi = np.linalg.eig(A)
    mu, f, xi, Phi = poles_from_eig(mu, Psi, C, dt)
    return mu, f, xi, Phi, A


# ---------------------------------------------------------------------------
# Sec. 2.1 and 2.3: hard and soft criteria (2D and 3D stabilization)
# ---------------------------------------------------------------------------
HC_XI, HC_MPC, HC_MPD = 1, 2, 4          # failure bits
ST_HC, ST_ORDER, ST_LAG = 8, 16, 32       # pass bits


def hard_criteria(mu, f, xi, Phi, xi_max=0.10, mpc_min=0.6, mpd_max=0.5):
    """HC: discard xi > xi_max (and xi <= 0 or |mu| >= 1), MPC <= mpc_min, MPD >= mpd_max.

    Returns (mpc values, mpd values, fail bit masks).
    """
    n = len(f)
    mpcs = np.array([mpc(Phi[:, j]) for j in range(n)])
    mpds = np.array([mpd(Phi[:, j]) for j in range(n)])
    fail = np.zeros(n, dtype=np.int64)
    fail |= np.where((xi > xi_max) | (xi <= 0) | (np.abs(mu) >= 1), HC_XI, 0)
    fail |= np.where(mpcs <= mpc_min, HC_MPC, 0)
    fail |= np.where(mpds >= mpd_max, HC_MPD, 0)
    return mpcs, mpds, fail


def _pair_ok(f1, xi1, p1, f2, xi2, p2, a_f, a_xi, a_mac):
    df = abs(f1 - f2) / max(f1, f2)
    dxi = abs(xi1 - xi2) / max(xi1, xi2)
    return df <= a_f and dxi <= a_xi and (1.0 - mac(p1, p2)) <= a_mac


def stability(diagram, a_f=0.01, a_xi=0.03, a_mac=0.02, use_lag_axis=True, **hc):
    """Soft criteria of Eq. (stabcriteria3D) over a diagram.

    ``diagram[t][m]`` is a dict with keys mu, f, xi, Phi for lag index t and
    order index m (orders ascending).  Adds 'mpc', 'mpd', 'flags' to each entry.
    A pole passes HC (bit 8) when none of the HC fail bits is set; it is stable
    along orders (bit 16) if some HC-passing pole at order index m-1 of the same
    lag meets all three thresholds, along lags (bit 32) likewise at lag index
    t-1 and the same order.  Returns the diagram.
    """
    for row in diagram:
        for cell in row:
            mpcs, mpds, fail = hard_criteria(cell["mu"], cell["f"], cell["xi"], cell["Phi"], **hc)
            cell["mpc"], cell["mpd"] = mpcs, mpds
            cell["flags"] = fail | np.where(fail == 0, ST_HC, 0)
    for t, row in enumerate(diagram):
        for m, cell in enumerate(row):
            for i in range(len(cell["f"])):
                if not cell["flags"][i] & ST_HC:
                    continue
                nbrs = []
                if m > 0:
                    nbrs.append((row[m - 1], ST_ORDER))
                if use_lag_axis and t > 0:
                    nbrs.append((diagram[t - 1][m], ST_LAG))
                for nb, bit in nbrs:
                    for j in range(len(nb["f"])):
                        if not nb["flags"][j] & ST_HC:
                            continue
                        if _pair_ok(cell["f"][i], cell["xi"][i], cell["Phi"][:, i],
                                    nb["f"][j], nb["xi"][j], nb["Phi"][:, j], a_f, a_xi, a_mac):
                            cell["flags"][i] |= bit
                            break
    return diagram


# ---------------------------------------------------------------------------
# Sec. 2.3 ("3D clustering") and Sec. 3.1: two-stage clustering of the stable poles
# ---------------------------------------------------------------------------
def rel_diff(a: float, b: float) -> float:
    """d = |a - b| / max(a, b): the relative differences d_f, d_xi of Sec. 3.1."""
    return abs(a - b) / max(a, b)


def pole_distance(f1, xi1, p1, f2, xi2, p2) -> float:
    """Stage II metric (Sec. 2.3): the sum of the relative differences in frequency and
    damping and of 1 - MAC between two poles."""
    return rel_diff(f1, f2) + rel_diff(xi1, xi2) + (1.0 - mac(p1, p2))


def stage1_features(diagram):
    """Stage I inputs (Sec. 2.3, Sec. 3.1).  For every pole that passes HC and is stable
    along orders or lags (bits 16/32, as set by ``stability``), the feature vector
        x = (d_f, d_xi, 1 - MAC, 1 - MPC, MPD),
    where the first three are taken against the pole's nearest HC-passing neighbour in the
    sense of ``pole_distance``, among the poles of the previous order of the same lag and
    of the same order of the previous lag (the neighbourhoods of Eq. (stabcriteria3D)).
    MPC enters as 1 - MPC so that every feature is 0 for an ideal physical pole.
    Returns X (n, 5) and the list of (t, m, i) of those poles, in diagram order."""
    X, idx = [], []
    for t, row in enumerate(diagram):
        for m, cell in enumerate(row):
            for i in range(len(cell["f"])):
                fl = cell["flags"][i]
                if not (fl & ST_HC) or not (fl & (ST_ORDER | ST_LAG)):
                    continue
                best = None
                nbrs = []
                if m > 0:
                    nbrs.append(row[m - 1])
                if t > 0:
                    nbrs.append(diagram[t - 1][m])
                for nb in nbrs:
                    for j in range(len(nb["f"])):
                        if not nb["flags"][j] & ST_HC:
                            continue
                        df = rel_diff(cell["f"][i], nb["f"][j])
                        dxi = rel_diff(cell["xi"][i], nb["xi"][j])
                        dmac = 1.0 - mac(cell["Phi"][:, i], nb["Phi"][:, j])
                        if best is None or df + dxi + dmac < best[0]:
                            best = (df + dxi + dmac, df, dxi, dmac)
                if best is None:
                    continue
                X.append([best[1], best[2], best[3], 1.0 - cell["mpc"][i], cell["mpd"][i]])
                idx.append((t, m, i))
    return np.array(X, dtype=np.float64).reshape(-1, 5), idx


def fuzzy_c_means(X, m: float = 2.0, tol: float = 1e-10, max_iter: int = 500):
    """Fuzzy C-means with two clusters (Bezdek): alternate
        u_ck = 1 / sum_j (||x_k - v_c|| / ||x_k - v_j||)^(2 / (m - 1)),
        v_c  = sum_k u_ck^m x_k / sum_k u_ck^m,
    from v_1 = the feature-wise minimum and v_2 = the feature-wise maximum of X, until
    the largest change of a membership is below tol.  A point on a centroid belongs to it
    alone; a cluster whose memberships are all zero keeps its centroid.  Returns U (n, 2),
    V (2, d) and the number of iterations."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    V = np.stack([X.min(axis=0), X.max(axis=0)])
    U = np.full((n, 2), 0.5)
    it = 0
    for it in range(1, max_iter + 1):
        D = np.sqrt(((X[:, None, :] - V[None, :, :]) ** 2).sum(axis=2))
        Un = np.empty_like(U)
        for k in range(n):
            zero = np.nonzero(D[k] == 0.0)[0]
            if len(zero):
                Un[k] = 0.0
                Un[k, zero[0]] = 1.0
            else:
                for c in range(2):
                    Un[k, c] = 1.0 / sum((D[k, c] / D[k, j]) ** (2.0 / (m - 1.0)) for j in range(2))
        Wm = Un ** m
        W = Wm.sum(axis=0)
        # a cluster whose memberships are all zero keeps its centroid (the update is 0/0)
        V = np.where((W > 0)[:, None], (Wm.T @ X) / np.where(W > 0, W, 1.0)[:, None], V)
        delta = np.abs(Un - U).max() if n else 0.0
        U = Un
        if delta < tol:
            break
    return U, V, it


def stage1(X, **fcm):
    """Stage I (Sec. 2.3, Sec. 3.1): the possibly physical cluster is the one whose centroid
    lies nearer the origin; a pole is kept when its membership P of that cluster is
    >= 0.5.  Returns (keep mask, P, V, index of the physical cluster, iterations)."""
    U, V, it = fuzzy_c_means(X, **fcm)
    phys = int(np.argmin(np.linalg.norm(V, axis=1)))
    P = U[:, phys]
    return P >= 0.5, P, V, phys, it


def single_linkage_labels(D, tau: float):
    """Clusters of the single-linkage dendrogram cut at distance tau: the connected
    components of the graph joining i and j whenever D[i, j] <= tau.  Each pole is
    labelled with the smallest index of its component."""
    n = D.shape[0]
    label = np.full(n, -1, dtype=np.int64)
    for s in range(n):
        if label[s] >= 0:
            continue
        label[s] = s
        stack = [s]
        while stack:
            a = stack.pop()
            for b in np.nonzero(D[a] <= tau)[0]:
                if label[b] < 0:
                    label[b] = s
                    stack.append(b)
    return label


def stage2(f, xi, Phi, tau: float, min_size: int):
    """Stage II (Sec. 2.3): single-linkage hierarchical clustering of the kept poles in
    ``pole_distance``, cut at tau; clusters of at least min_size poles are modes.
    A mode reports the mean frequency and damping of its poles, its size and its medoid
    (the member with the smallest sum of distances to the others; ties to the smaller
    index).  Returns (modes sorted by frequency, labels, D)."""
    n = len(f)
    D = np.zeros((n, n))
    for a in range(n):
        for b in range(a + 1, n):
            D[a, b] = D[b, a] = pole_distance(f[a], xi[a], Phi[:, a], f[b], xi[b], Phi[:, b])
    labels = single_linkage_labels(D, tau)
    modes = []
    for lab in np.unique(labels):
        mem = np.nonzero(labels == lab)[0]
        if len(mem) < min_size:
            continue
        sums = D[np.ix_(mem, mem)].sum(axis=1)
        medoid = int(mem[int(np.argmin(sums))])
        modes.append(dict(f=float(np.mean(np.asarray(f, dtype=np.float64)[mem])),
                          xi=float(np.mean(np.asarray(xi, dtype=np.float64)[mem])),
                          size=int(len(mem)), medoid=medoid, members=mem))
    modes.sort(key=lambda d: d["f"])
    return modes, labels, D


def cluster_modes(diagram, tau: float = 0.05, min_size: int = 10, **fcm):
    """Both stages on a stabilization diagram whose flags come from ``stability``.
    Returns (modes, stage I keep mask, P, the (t, m, i) of the stage I poles)."""
    X, idx = stage1_features(diagram)
    if len(idx) == 0:
        return [], np.zeros(0, bool), np.zeros(0), idx
    keep, P, V, phys, it = stage1(X, **fcm)
    kept = [idx[q] for q in np.nonzero(keep)[0]]
    f = np.array([diagram[t][m]["f"][i] for t, m, i in kept])
    xi = np.array([diagram[t][m]["xi"][i] for t, m, i in kept])
    l = diagram[0][0]["Phi"].shape[0]
    Phi = np.stack([diagram[t][m]["Phi"][:, i] for t, m, i in kept], axis=1) if kept else \
        np.zeros((l, 0), complex)
    modes, labels, D = stage2(f, xi, Phi, tau, min_size)
    for md in modes:
        md["medoid"] = kept[md["medoid"]]
        md["members"] = [kept[q] for q in md["members"]]
    return modes, keep, P, idx


# ---------------------------------------------------------------------------
# Sec. 3 parameter rules
# ---------------------------------------------------------------------------
def rank_rule(T_size: int):
    """Eq. (empirical_formula): kbar(T) = max(30 - 0.00156 T, 25) percent; k = ceil(kbar T/100)."""
    kbar = max(30.0 - 0.00156 * T_size, 25.0)
    return kbar, int(math.ceil(kbar * T_size / 100.0 - 1e-9))


def lag_rule(fs: float, f0: float, beta: float = 1.5):
    """Eq. (jb) and Eq. (jb_3D) with int() read as ceiling: (jb, jb_min, jb_max)."""
    jb = int(math.ceil(10.0 * fs / (2.0 * f0) - 1e-9))
    jb_min = int(math.ceil(9.0 * fs / (2.0 * f0) - 1e-9))
    jb_max = int(math.ceil(beta * jb_min - 1e-9))
    return jb, jb_min, jb_max


def time_lag(jb: int, fs: float) -> float:
    """Eq. (tlag): tau = (2 jb - 1)/fs."""
    return (2 * jb - 1) / fs


# ---------------------------------------------------------------------------
# one complete solve
# ---------------------------------------------------------------------------
def ssi_solve(Y, fs, lags, orders, k=None, oversample=0, q=0, seed=0, full_svd_=False,
              stab=None, R=None):
    """Covariances -> per lag (Toeplitz, (R)SVD, realisation for every order) -> stability.

    Returns (diagram, svals) where svals[t] are the singular values used at lag t.
    """
    dt = 1.0 / fs
    l = Y.shape[0] if R is None else R.shape[1]
    if R is None:
        R = covariances(Y, 2 * max(lags) - 1)
    diagram, svals = [], []
    for i in lags:
        T = block_toeplitz(R, i)
        if full_svd_:
            U, S = full_svd(T)
        else:
            U, S = rsvd(T, k, oversample, q, seed)
        svals.append(S)
        row = []
        for n in orders:
            mu, f, xi, Phi, _ = realize(U, S, l, i, n, dt)
            row.append(dict(mu=mu, f=f, xi=xi, Phi=Phi))
        diagram.append(row)
    stability(diagram, **(stab or {}))
    return diagram, svals
