"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test ties an oracle function to something other than itself: values the
paper prints (tests/golden), closed forms of the generating models, invariants,
published known-answer vectors, or an independent library routine on a special
case.  The mutation tests at the end plant plausible mistakes in the oracle and
check that a pin catches them.
"""
import math

import numpy as np
import pytest

import oracle as O
import ssi_synth as S
from conftest import golden_rows


# --------------------------------------------------------------------------- Philox
def test_philox_known_answers():
    for row in golden_rows("philox4x32_10_kat.txt"):
        v = [int(x, 16) for x in row]
        out = O.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_omega_is_shape_independent_and_standard_normal():
    a = O.gaussian_omega(300, 40, seed=123)
    b = O.gaussian_omega(200, 64, seed=123)
    assert np.array_equal(a[:200, :40], b[:, :40])
    z = O.gaussian_omega(500, 200, seed=9).ravel()
    assert abs(z.mean()) < 5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
    # fourth moment of a standard normal is 3
    assert abs(np.mean(z ** 4) - 3) < 0.1
    assert not np.array_equal(O.gaussian_omega(10, 10, 1), O.gaussian_omega(10, 10, 2))


# --------------------------------------------------------------------------- covariances
def test_covariance_closed_forms():
    N = 101
    t = np.arange(N)
    Y = np.stack([(-1.0) ** t, np.ones(N)])
    R = O.covariances(Y, 7)
    for k in range(1, 8):
        # alternating channel: y_{t+k} y_t = (-1)^k for every t
        assert R[k - 1, 0, 0] == pytest.approx((-1) ** k, abs=1e-15)
        # R_k[0, 1] = (-1)^k (sum_{t<N-k} (-1)^t)/(N-k) = (-1)^k [N-k odd]/(N-k)
        expect = (-1) ** k * ((N - k) % 2) / (N - k)
        assert R[k - 1, 0, 1] == pytest.approx(expect, abs=1e-15)
        # R_k[1, 0] = sum_t y_{t}... constant first factor: sum_{t<N-k} (-1)^t/(N-k)
        assert R[k - 1, 1, 0] == pytest.approx(((N - k) % 2) / (N - k), abs=1e-15)
        assert R[k - 1, 1, 1] == pytest.approx(1.0, abs=1e-15)


def test_covariance_linear_ramp_closed_form():
    # y_t = t: R_k = sum_{t=0}^{N-k-1} (t+k) t / (N-k), with closed-form power sums
    N, k = 57, 5
    Y = np.arange(N, dtype=float)[None, :]
    M = N - k
    s1 = (M - 1) * M / 2
    s2 = (M - 1) * M * (2 * M - 1) / 6
    assert O.covariances(Y, k)[k - 1, 0, 0] == pytest.approx((s2 + k * s1) / M, rel=1e-14)
    assert O.covariance_entry(Y, k, 0, 0) == pytest.approx((s2 + k * s1) / M, rel=1e-14)


def test_sample_covariances_converge_to_model_covariances():
    w = S.workload("chain4_tiny")
    model = S.chain_model(w)
    Ra = S.model_covariances(model, 39)[1:]
    errs = []
    for N in (20000, 320000):
        Y = S.simulate(model, N, seed=3, noise_frac=0.0)
        R = O.covariances(Y, 39)
        errs.append(np.linalg.norm(R - Ra) / np.linalg.norm(Ra))
    # CLT: error falls like N^-1/2 (factor 4 for 16x the samples); allow slack
    assert errs[1] < 0.1
    assert errs[1] < errs[0] / 2.0


# --------------------------------------------------------------------------- Toeplitz
def test_block_toeplitz_matches_printed_layout():
    layout = np.array(golden_rows("toeplitz_layout.txt"), dtype=int)
    jb = layout.shape[0]
    l = 2
    R = np.stack([np.full((l, l), float(k)) for k in range(1, 2 * jb)])
    T = O.block_toeplitz(R, jb)
    for a in range(jb):
        for b in range(jb):
            assert np.all(T[a * l:(a + 1) * l, b * l:(b + 1) * l] == layout[a, b])


def test_toeplitz_of_model_covariances_has_rank_2n():
    w = S.workload("chain4_tiny")
    model = S.chain_model(w)
    Ra = S.model_covariances(model, 39)[1:]
    T = O.block_toeplitz(Ra, 20)
    _, s = O.full_svd(T)
    assert s[7] / s[0] > 1e-3
    assert s[8] / s[0] < 1e-12


# --------------------------------------------------------------------------- QR / SVD
def test_householder_qr_invariants():
    rng = np.random.default_rng(0)
    A = rng.standard_normal((70, 12)) @ np.diag(10.0 ** -np.arange(12))
    Q, R = O.householder_qr(A)
    assert np.allclose(Q.T @ Q, np.eye(12), atol=1e-14)
    assert np.allclose(Q @ R, A, atol=1e-14)
    assert np.allclose(np.tril(R, -1), 0)
    _, Rl = np.linalg.qr(A)
    assert np.allclose(np.abs(np.diag(R)), np.abs(np.diag(Rl)), rtol=1e-10)


def test_jacobi_svd_invariants_and_known_spectrum():
    rng = np.random.default_rng(1)
    m, n = 40, 25
    Q1, _ = np.linalg.qr(rng.standard_normal((m, n)))
    Q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s_true = np.logspace(0, -9, n)
    A = Q1 @ np.diag(s_true) @ Q2.T
    U, s, V, sweeps = O.jacobi_svd(A)
    assert sweeps < 30
    assert np.allclose(s, s_true, rtol=1e-6, atol=1e-15)
    assert np.allclose(U.T @ U, np.eye(n), atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-13)
    assert np.allclose((U * s) @ V.T, A, atol=1e-14)
    B = rng.standard_normal((30, 30))
    assert np.allclose(O.jacobi_svd(B)[1], np.linalg.svd(B, compute_uv=False), rtol=1e-12)
    D = np.diag([3.0, -5.0, 1.0])
    assert np.allclose(O.jacobi_svd(D)[1], [5.0, 3.0, 1.0])


# --------------------------------------------------------------------------- RSVD
def _chain_T():
    w = S.workload("chain4_tiny")
    Y, *_ = S.record(w)
    return O.block_toeplitz(O.covariances(Y, 39), 20), S.chain_model(w)


def test_rsvd_full_width_equals_svd():
    T, _ = _chain_T()
    _, s_full = O.full_svd(T)
    U, s = O.rsvd(T, T.shape[0], 0, 0, seed=5)
    assert np.allclose(s, s_full, rtol=1e-10, atol=1e-14 * s_full[0])
    assert np.allclose(U.T @ U, np.eye(T.shape[0]), atol=1e-10)


def test_rsvd_exact_on_rank_deficient_model_toeplitz():
    model = S.chain_model(S.workload("chain4_tiny"))
    T = O.block_toeplitz(S.model_covariances(model, 39)[1:], 20)
    _, s_full = O.full_svd(T)
    _, s = O.rsvd(T, 8, 0, 0, seed=2)           # Algorithm 1 with k = rank(T)
    assert np.allclose(s, s_full[:8], rtol=1e-9)


def test_rsvd_leading_values_with_power_iterations():
    T, _ = _chain_T()
    _, s_full = O.full_svd(T)
    _, s = O.rsvd(T, 20, 10, 2, seed=4)
    assert np.allclose(s[:8], s_full[:8], rtol=1e-6)


# --------------------------------------------------------------------------- realisation
def test_realisation_recovers_model_modes_exactly():
    model = S.chain_model(S.workload("chain4_tiny"))
    T = O.block_toeplitz(S.model_covariances(model, 39)[1:], 20)
    U, s = O.full_svd(T)
    mu, f, xi, Phi, _ = O.realize(U, s, 4, 20, 8, model.dt)
    assert np.allclose(f, model.f_true, rtol=1e-9)
    assert np.allclose(xi, model.xi_true, atol=1e-9)
    for j in range(4):
        assert O.mac(Phi[:, j], model.phi_true[:, j]) > 1 - 1e-9


def test_realisation_reproduces_table1_of_the_paper():
    """10-DOF frame (Sec. 3.1): exact covariances -> Table 1's f and xi to the printed digits."""
    w = S.workload("frame10")
    model = S.chain_model(w)
    i = 12
    T = O.block_toeplitz(S.model_covariances(model, 2 * i - 1)[1:], i)
    U, s = O.full_svd(T)
    _, f, xi, _, _ = O.realize(U, s, 10, i, 20, model.dt)
    table = np.array(golden_rows("table1_frame10.txt"), dtype=float)
    assert np.allclose(f, table[:, 1], atol=5.01e-4)
    assert np.allclose(100 * xi, table[:, 2], atol=5.01e-4)


def test_chain_closed_form_frequencies_match_table1():
    n, m, k = 10, 100.0, 5e6
    j = np.arange(1, n + 1)
    w = 2 * math.sqrt(k / m) * np.sin((2 * j - 1) * math.pi / (2 * (2 * n + 1)))
    table = np.array(golden_rows("table1_frame10.txt"), dtype=float)
    assert np.allclose(w / (2 * math.pi), table[:, 1], atol=5.01e-4)


def test_pole_formulas_invert_the_continuous_eigenvalue():
    dt = 0.01
    for f0, xi0 in [(1.0, 0.005), (7.3, 0.03), (20.0, 0.2)]:
        w0 = 2 * math.pi * f0
        lam = complex(-xi0 * w0, w0 * math.sqrt(1 - xi0 ** 2))
        mu = np.array([np.exp(lam * dt), np.exp(np.conj(lam) * dt), 0.5])
        Psi = np.eye(3, dtype=complex)
        m, f, xi, Phi = O.poles_from_eig(mu, Psi, np.eye(3), dt)
        assert len(f) == 1
        assert f[0] == pytest.approx(f0, rel=1e-12)
        assert xi[0] == pytest.approx(xi0, rel=1e-10)


# --------------------------------------------------------------------------- MPC / MPD / MAC
def test_mpc_mpd_mac_hand_values():
    real = np.array([1.0, -2.0, 0.5]) + 0j
    assert O.mpc(real) == pytest.approx(1.0)
    assert O.mpd(real) == pytest.approx(0.0, abs=1e-12)
    # Re and Im orthogonal with equal norms: no collinearity
    circ = np.array([1.0, 1j])
    assert O.mpc(circ) == pytest.approx(0.0, abs=1e-15)
    # phases 0, 0, 90 deg, unit moduli: X^T X = diag(2, 1)
    phi = np.array([1.0, 1.0, 1j])
    assert O.mpc(phi) == pytest.approx(1.0 / 9.0)
    assert O.mpd(phi) == pytest.approx(1.0 / 3.0)
    a = np.array([1 + 2j, 3 - 1j, 0.5j])
    assert O.mac(a, (2 - 3j) * a) == pytest.approx(1.0)
    assert O.mac(np.array([1.0, 0.0]), np.array([0.0, 1.0])) == 0.0
    # |a^H b|^2 / (|a|^2 |b|^2) for a = (1, 1), b = (1, 0): 1/2
    assert O.mac(np.array([1.0, 1.0]), np.array([1.0, 0.0])) == pytest.approx(0.5)


# --------------------------------------------------------------------------- stability
def _cell(f, xi, phis):
    f = np.asarray(f, float)
    return dict(mu=np.exp((-np.asarray(xi) * 2 * np.pi * f + 2j * np.pi * f) * 0.01),
                f=f, xi=np.asarray(xi, float), Phi=np.stack(phis, axis=1))


def test_stability_hand_built_diagram():
    p = np.array([1.0, 0.5, -0.2]) + 0j
    q = np.array([0.2, -1.0, 0.9]) + 0j
    # lag 0: order 2 -> one pole at 2.00 Hz; order 4 -> 2.02 Hz (1 % off: exactly at a_f), 5 Hz
    # lag 1: order 2 -> 2.0 Hz with xi 10 % off (fails a_xi = 3 %), order 4 -> 5.0 Hz
    d = [[_cell([2.0], [0.02], [p]), _cell([2.0 * 1.01, 5.0], [0.02, 0.01], [p, q])],
         [_cell([2.0], [0.022], [p]), _cell([5.0], [0.012], [q])]]
    O.stability(d, a_f=0.01, a_xi=0.03, a_mac=0.02)
    assert d[0][0]["flags"][0] == O.ST_HC                      # first order, first lag
    # |2.02 - 2|/2.02 < 1 %: stable along orders
    assert d[0][1]["flags"][0] & O.ST_ORDER
    assert not d[0][1]["flags"][1] & O.ST_ORDER                # 5 Hz has no neighbour
    assert not d[1][0]["flags"][0] & O.ST_LAG                  # xi differs by 9 %
    f_lag = d[1][1]["flags"][0]
    assert not f_lag & O.ST_ORDER                              # no 5 Hz at lag 1 order 2
    assert not f_lag & O.ST_LAG                                # xi 0.012 vs 0.01: 16.7 %
    d2 = [[_cell([5.0], [0.01], [q])], [_cell([5.0 * 1.0099], [0.0101], [q])]]
    O.stability(d2, a_f=0.01, a_xi=0.03, a_mac=0.02)
    assert d2[1][0]["flags"][0] & O.ST_LAG
    # HC: damping above 10 % fails and is never a neighbour
    d3 = [[_cell([3.0], [0.2], [p]), _cell([3.0], [0.2], [p])]]
    O.stability(d3)
    assert d3[0][1]["flags"][0] & O.HC_XI
    assert not d3[0][1]["flags"][0] & (O.ST_HC | O.ST_ORDER)


# --------------------------------------------------------------------------- rules
def test_parameter_rules_reproduce_worked_values():
    for row in golden_rows("parameter_rules.txt"):
        if row[0] == "rank":
            kbar, k = O.rank_rule(int(row[1]))
            assert kbar == pytest.approx(float(row[2]), abs=1e-9)
            assert k == int(row[3])
        elif row[0] == "lag":
            assert O.lag_rule(float(row[1]), float(row[2])) == tuple(int(x) for x in row[3:6])
        elif row[0] == "tau":
            assert O.time_lag(int(row[1]), float(row[2])) == pytest.approx(float(row[3]), abs=1e-12)


# --------------------------------------------------------------------------- planted mistakes
def test_pins_catch_a_transposed_toeplitz(monkeypatch):
    model = S.chain_model(S.workload("chain4_tiny"))
    Ra = S.model_covariances(model, 39)[1:]

    def wrong(R, i):   # block (a, b) = R_{i - a + b}: the transpose of Eq. (Toeplitz)
        l = R.shape[1]
        T = np.empty((i * l, i * l))
        for a in range(i):
            for b in range(i):
                T[a * l:(a + 1) * l, b * l:(b + 1) * l] = R[i - a + b - 1]
        return T

    U, s = O.full_svd(wrong(Ra, 20))
    _, f, xi, _, _ = O.realize(U, s, 4, 20, 8, model.dt)
    assert not (len(f) == 4 and np.allclose(xi, model.xi_true, atol=1e-3))


def test_pins_catch_a_wrong_damping_sign(monkeypatch):
    orig = O.ssi_oracle.poles_from_eig

    def wrong(mu, Psi, C, dt):
        m, f, xi, Phi = orig(mu, Psi, C, dt)
        return m, f, -xi, Phi

    monkeypatch.setattr(O.ssi_oracle, "poles_from_eig", wrong)
    model = S.chain_model(S.workload("chain4_tiny"))
    T = O.block_toeplitz(S.model_covariances(model, 39)[1:], 20)
    U, s = O.full_svd(T)
    _, f, xi, _, _ = O.ssi_oracle.realize(U, s, 4, 20, 8, model.dt)
    assert not np.allclose(xi, model.xi_true, atol=1e-9)
