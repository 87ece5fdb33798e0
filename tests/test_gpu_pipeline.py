"""Parity of stages (b)-(d) and of a complete solve against the FP64 oracle.

Tolerances (fixed by the gates of the method's parity set): leading singular values
<= 1e-4 relative; pole frequency <= 1e-4 relative, damping <= 2e-3 absolute,
MAC >= 0.999.  Omega: the GPU and the oracle evaluate the same Philox4x32-10 counters;
the Box-Muller transform runs in FP32 on the GPU and FP64 in the oracle, so entries
agree to ~1e-6 absolute (bound 2e-5).
"""
import ctypes
import functools

import numpy as np
import pytest
import torch

import oracle as O
import ssi_synth as S
from parity import compare_parity_set, gpu_cells, nearest, separated_orders

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2411_05510_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()


def test_omega_matches_oracle_philox(P, ctx):
    for rows, cols, seed in [(300, 37, 0), (1000, 220, 11), (5, 5, (7 << 32) | 9)]:
        g = P.ssi_gaussian_omega(ctx, rows, cols, seed).cpu().numpy()
        o = O.gaussian_omega(rows, cols, seed)
        assert np.abs(g - o).max() < 2e-5


def _rsvd_case(P, ctx, R, l, i, k, p, q, seed, prec, small="fp32"):
    Rd = torch.from_numpy(np.ascontiguousarray(R)).cuda()
    U, Sv = P.ssi_toeplitz_rsvd(ctx, Rd, l, i, k, p, q, seed, prec, small)
    P.check_sync(ctx)
    return U.cpu().numpy(), Sv.cpu().numpy()


@pytest.mark.parametrize("prec", ["split_bf16", "fp32"])
def test_rsvd_full_width_equals_full_svd_on_chain(P, ctx, prec):
    """4-channel chain, i = 20: k = L = 80 with no sketching reduces RSVD to the SVD."""
    Y, *_ = S.record(S.workload("chain4_tiny"))
    R = O.covariances(Y, 39)
    T = O.block_toeplitz(R, 20)
    _, s_ref = O.full_svd(T)
    U, s = _rsvd_case(P, ctx, R, 4, 20, 80, 0, 0, 3, prec)
    assert np.allclose(s[:8], s_ref[:8], rtol=1e-4)
    assert np.abs(U[:, :8].T @ U[:, :8] - np.eye(8)).max() < 1e-4


@functools.lru_cache(maxsize=None)
def _oracle_rsvd_case(l, i, k, p, q):
    rec = S.bridge_record(l, 8, 1.0, 12.0, 50.0, 40000, 0.05, seed=l + i)
    R = O.covariances(rec.Y, 2 * i - 1)
    _, s_ref = O.rsvd(O.block_toeplitz(R, i), k, p, q, seed=5)
    return R, s_ref


@pytest.mark.parametrize("prec,small", [("split_bf16", "fp32"), ("fp32", "fp32"),
                                        ("split_bf16", "fp64")])
@pytest.mark.parametrize("l,i,k,p,q", [(24, 10, 40, 10, 2), (70, 7, 60, 20, 1), (9, 30, 30, 6, 3),
                                       (64, 10, 300, 20, 1)])
def test_rsvd_matches_oracle_rsvd(P, ctx, prec, small, l, i, k, p, q):
    """Same Omega (Philox) on both sides: leading singular values agree to 1e-4, in both
    small-problem precisions (the K x K Jacobi SVD in FP32 or FP64)."""
    R, s_ref = _oracle_rsvd_case(l, i, k, p, q)
    U, s = _rsvd_case(P, ctx, R, l, i, k, p, q, 5, prec, small)
    lead = 16
    assert np.allclose(s[:lead], s_ref[:lead], rtol=1e-4), np.abs(s[:lead] / s_ref[:lead] - 1).max()
    G = U.T @ U
    assert np.abs(G - np.eye(k)).max() < 2e-4


@functools.lru_cache(maxsize=None)
def _wide_case(l, i):
    rec = S.bridge_record(l, 10, 1.0, 12.0, 50.0, 60000, 0.05, seed=3 * l + i)
    R = O.covariances(rec.Y, 2 * i - 1)
    # leading singular values of T by the oracle's RSVD with three power iterations
    _, s_ref = O.rsvd(O.block_toeplitz(R, i), 48, 16, 3, seed=9)
    return R, s_ref


@pytest.mark.parametrize("l,i,small", [(32, 32, "fp32"), (64, 32, "fp32"), (32, 32, "fp64")])
def test_rsvd_full_width_above_512(P, ctx, l, i, small):
    """The range finder at full width K = L = 1024 and 2048 (no sketching error): the
    K x K Jacobi runs on the cooperative grid with 74 (FP32, 1024), 147 (FP32, 2048) or
    152 (FP64) CTAs.  The leading 16 singular values match the oracle's converged RSVD of
    the same T to 1e-4 and U has orthonormal columns."""
    R, s_ref = _wide_case(l, i)
    L = l * i
    U, s = _rsvd_case(P, ctx, R, l, i, L, 0, 0, 7, "split_bf16", small)
    assert np.allclose(s[:16], s_ref[:16], rtol=1e-4), np.abs(s[:16] / s_ref[:16] - 1).max()
    assert np.all(np.diff(s) <= 0)
    G = U[:, :64].T @ U[:, :64]
    assert np.abs(G - np.eye(64)).max() < 2e-4


def _realize(P, ctx, Us, lags, l, k, orders, dt, small="fp32"):
    Ud = [torch.from_numpy(np.ascontiguousarray(U, dtype=np.float64)).cuda() for U in Us]
    poles, phi = P.ssi_realize_batch(ctx, lags, Ud, l, k, orders, dt, small)
    P.check_sync(ctx)
    return P.poles_to_numpy(poles), phi.cpu().numpy()


@pytest.mark.parametrize("small", ["fp32", "fp64"])
def test_realize_recovers_exact_modes_from_model_covariances(P, ctx, small):
    model = S.chain_model(S.workload("chain4_tiny"))
    T = O.block_toeplitz(S.model_covariances(model, 39)[1:], 20)
    U, s = O.full_svd(T)
    rec, phi = _realize(P, ctx, [U[:, :8]], [20], 4, 8, [2, 4, 6, 8], model.dt, small)
    cells = gpu_cells(rec, phi, [20], [2, 4, 6, 8], 4)
    c8 = cells[0][3]
    assert len(c8["f"]) == 4
    # FP64: the modes of the model to the precision of the output records (FP32)
    rtol, atol = (2e-5, 2e-4) if small == "fp32" else (1e-6, 1e-6)
    assert np.allclose(c8["f"], model.f_true, rtol=rtol)
    assert np.allclose(c8["xi"], model.xi_true, atol=atol)
    for j in range(4):
        assert O.mac(c8["Phi"][:, j], model.phi_true[:, j]) > 0.9999


@pytest.mark.parametrize("small", ["fp32", "fp64"])
def test_realize_matches_oracle_on_noisy_chain(P, ctx, small):
    w = S.workload("chain4_tiny")
    Y, f_true, _, phi_true = S.record(w)
    T = O.block_toeplitz(O.covariances(Y, 39), 20)
    U, s = O.full_svd(T)
    orders = list(range(2, 41, 2))
    rec, phi = _realize(P, ctx, [U[:, :40]], [20], 4, 40, orders, 0.01, small)
    gpu = gpu_cells(rec, phi, [20], orders, 4)
    ora = [[]]
    for n in orders:
        mu, f, xi, Phi, _ = O.realize(U, s, 4, 20, n, 0.01)
        cell = dict(mu=mu, f=f, xi=xi, Phi=Phi)
        mpcs, mpds, fail = O.hard_criteria(mu, f, xi, Phi)
        cell["flags"] = np.where(fail == 0, 8, 0)
        ora[0].append(cell)
    # GPU cells carry HC bits only after ssi_stabilize: apply the same HC to their values
    for row in gpu:
        for c in row:
            ok = (c["xi"] > 0) & (c["xi"] <= 0.1) & (c["mpc"] > 0.6) & (c["mpd"] < 0.5) & (np.abs(c["mu"]) < 1)
            c["flags"] = np.where(ok, 8, 0)
    n, worst = compare_parity_set(gpu, ora, f_true, orders, 4, min_matches=40, phi_true=phi_true)


def test_stabilize_flags_match_oracle_on_shared_poles(P, ctx):
    """Identical pole sets on both sides (oracle poles uploaded): flags must agree."""
    w = S.workload("chain4_tiny")
    Y, *_ = S.record(w)
    T = O.block_toeplitz(O.covariances(Y, 39), 20)
    U, s = O.full_svd(T)
    orders = list(range(2, 21, 2))
    lags = [20, 21]
    diag = []
    for _ in lags:
        row = []
        for n in orders:
            mu, f, xi, Phi, _ = O.realize(U, s, 4, 20, n, 0.01)
            row.append(dict(mu=mu, f=f, xi=xi, Phi=np.stack([O.normalize_shape(Phi[:, j]) for j in
                                                            range(Phi.shape[1])], 1) if len(f) else Phi))
        diag.append(row)
    # perturb the second lag slightly so the lag axis has non-trivial decisions
    for c in diag[1]:
        c["f"] = c["f"] * 1.004
        c["xi"] = c["xi"] * 1.02
    l = 4
    slots = sum(n // 2 for n in orders)
    rec = np.zeros(slots * len(lags), dtype=P.api._POLE_DTYPE)
    phi = np.zeros((slots * len(lags), l, 2), np.float32)
    off = 0
    for t, row in enumerate(diag):
        for m, n in enumerate(orders):
            c = row[m]
            for j in range(len(c["f"])):
                e = rec[off + j]
                e["f_hz"], e["xi"] = c["f"][j], c["xi"][j]
                e["mu_re"], e["mu_im"] = c["mu"][j].real, c["mu"][j].imag
                e["mpc"], e["mpd"] = O.mpc(c["Phi"][:, j]), O.mpd(c["Phi"][:, j])
                e["lag"], e["order"], e["flags"], e["index"] = lags[t], n, 64, j
                phi[off + j, :, 0] = c["Phi"][:, j].real
                phi[off + j, :, 1] = c["Phi"][:, j].imag
                rec[off + j] = e
            off += n // 2
    pd = torch.from_numpy(np.frombuffer(rec.tobytes(), np.uint8).reshape(len(rec), -1).copy()).cuda()
    fd = torch.from_numpy(phi).cuda()
    P.ssi_stabilize(ctx, len(lags), orders, l, pd, fd, P.stab_params())
    torch.cuda.synchronize()
    g = P.poles_to_numpy(pd)
    O.stability(diag)
    off = 0
    n_checked = 0
    for t, row in enumerate(diag):
        for m, n in enumerate(orders):
            for j in range(len(row[m]["f"])):
                assert int(g["flags"][off + j]) & 63 == int(row[m]["flags"][j]) & 63, (t, n, j)
                n_checked += 1
            off += n // 2
    assert n_checked > 50


@pytest.mark.parametrize("prec,small", [("split_bf16", "fp32"), ("fp32", "fp32"),
                                        ("split_bf16", "fp64")])
def test_full_solve_chain_matches_oracle(P, ctx, prec, small):
    """Complete solve of the 4-channel chain record (i = 20, full width k = 80, orders 2..40)."""
    w = S.workload("chain4_tiny")
    Y, f_true, _, phi_true = S.record(w, np.float32)
    orders = w["orders"]
    desc = P.job_desc(torch.from_numpy(Y).cuda(), w["fs"], w["lags"], orders, k=40, oversample=40,
                      q=0, prec=prec, seed=1, small=small)
    poles, phi, Sg = P.ssi_solve(ctx, desc)
    P.check_sync(ctx)
    rec = P.poles_to_numpy(poles)
    gpu = gpu_cells(rec, phi.cpu().numpy(), w["lags"], orders, 4)
    ora, sv = O.ssi_solve(Y.astype(np.float64), w["fs"], w["lags"], orders, full_svd_=True)
    assert np.allclose(Sg.cpu().numpy()[0, :8], sv[0][:8], rtol=1e-4)
    gate = separated_orders(orders, sv[0])
    assert 8 in gate
    compare_parity_set(gpu, ora, f_true, orders, 4, min_matches=4, phi_true=phi_true,
                       gate_orders=gate)
    # at every order from 2m on, every mode is identified by an HC-passing pole within 1 %
    for m, n in enumerate(orders):
        if n < 8:
            continue
        cell = dict(gpu[0][m])
        cell["flags"] = rec_flags = cell["flags"]
        for r, f0 in enumerate(f_true):
            j = nearest(cell, f0, phi_true[:, r])
            assert j is not None and abs(cell["f"][j] - f0) / f0 < 1e-2, (n, r)


def test_3d_diagram_matches_oracle(P, ctx):
    """3D stabilization diagram of a reduced bridge record (24 channels, 6 modes in
    4-20 Hz, N = 60000, lags 14, 18, 22, RSVD k = 32 + 16 with q = 2, orders 2..32, one
    solve): each lag against the oracle's FP64 RSVD with the same Omega at its separated
    orders, and the stability flags of the matched true-mode poles."""
    w = S.workload("bridge186_3d", l=24, modes=6, f_lo=4.0, N=60000, lags=[14, 18, 22], k=32,
                   oversample=16, orders=list(range(2, 33, 2)))
    Y, f_true, _, phi_true = S.record(w, np.float32)
    desc = P.job_desc(torch.from_numpy(Y).cuda(), w["fs"], w["lags"], w["orders"], k=w["k"],
                      oversample=w["oversample"], q=w["q"], prec="split_bf16", seed=5)
    poles, phi, Sg = P.ssi_solve(ctx, desc)
    P.check_sync(ctx)
    rec = P.poles_to_numpy(poles)
    gpu = gpu_cells(rec, phi.cpu().numpy(), w["lags"], w["orders"], w["l"])
    ora, sv = O.ssi_solve(Y.astype(np.float64), w["fs"], w["lags"], w["orders"], k=w["k"],
                          oversample=w["oversample"], q=w["q"], seed=5)
    n_cmp_total, n_flag = 0, 0
    gates = [separated_orders(w["orders"], sv[t]) for t in range(len(w["lags"]))]
    for t in range(len(w["lags"])):
        s_gpu = Sg.cpu().numpy()[t].astype(np.float64)
        assert np.allclose(s_gpu[:12], sv[t][:12], rtol=1e-4), t
        gate = gates[t]
        assert 12 in gate, (t, gate)
        n_cmp, _ = compare_parity_set([gpu[t]], [ora[t]], f_true, w["orders"], 6, min_matches=6,
                                      phi_true=phi_true, gate_orders=gate)
        n_cmp_total += n_cmp
        # stability flags of the matched true-mode poles: HC always; stable-along-orders
        # when the previous order is separated too, stable-along-lags when the same order
        # of the previous lag is (then every pole those neighbour cells hold is
        # reproducible); the first lag has no lag neighbour on either side
        for m, n in enumerate(w["orders"]):
            if n not in gate:
                continue
            for r, f0 in enumerate(f_true):
                a = nearest(ora[t][m], f0, phi_true[:, r])
                b = nearest(gpu[t][m], f0, phi_true[:, r])
                if a is None or b is None:
                    continue
                fa, fb = int(ora[t][m]["flags"][a]), int(gpu[t][m]["flags"][b])
                bits = O.ST_HC
                if (n - 2) in gate:
                    bits |= O.ST_ORDER
                if t == 0 or n in gates[t - 1]:
                    bits |= O.ST_LAG
                assert fa & bits == fb & bits, (t, n, r, fa, fb)
                n_flag += 1 + (t > 0 and n in gates[t - 1])
    assert n_cmp_total >= 18
    assert n_flag >= 24


@pytest.mark.parametrize("small", ["fp32", "fp64"])
def test_realize_orders_above_shared_memory_recover_model_modes(P, ctx, small):
    """Orders above 224 run with A in global scratch, and k = 240 factors each lag in
    global scratch too.  From the exact covariances of a 240-state model (120-storey shear
    chain, 2 % modal damping, white forces at every storey, accelerations of every storey)
    the realisation of order 240 must return the model's 120 poles.  Order 230 (also the
    global-scratch path) and order 200 (shared memory, same launch) must run without
    failure flags."""
    M, K = S.shear_chain(120, 1.0, 1e3)
    model = S.chain_state_space(M, K, S.modal_damping(M, K, 0.02), 1.0 / 40.0, "floors")
    i = 4
    T = O.block_toeplitz(S.model_covariances(model, 2 * i - 1)[1:], i)
    U, s = O.full_svd(T)
    assert s[239] > 1e-9 * s[0] and s[240] < 1e-9 * s[0]   # rank 240 = 2 x 120 modes
    orders = [200, 230, 240]
    rec, phi = _realize(P, ctx, [U[:, :240]], [i], 120, 240, orders, model.dt, small)
    cells = gpu_cells(rec, phi, [i], orders, 120)
    c240 = cells[0][2]
    assert len(c240["f"]) == 120
    order = np.argsort(c240["f"])
    f_gpu, xi_gpu, mu_gpu = c240["f"][order], c240["xi"][order], c240["mu"][order]
    # the discrete poles themselves: FP32 eigenvalues of a 240 x 240 matrix, |d mu| ~ 1e-5
    w_true = 2 * np.pi * model.f_true
    lam = -model.xi_true * w_true + 1j * w_true * np.sqrt(1 - model.xi_true ** 2)
    mu_true = np.exp(lam * model.dt)
    assert np.abs(mu_gpu - mu_true).max() < 1e-4, np.abs(mu_gpu - mu_true).max()
    if small == "fp64":   # FP64 eigenvalues, rounded once to the FP32 records
        assert np.abs(mu_gpu - mu_true).max() < 2e-7, np.abs(mu_gpu - mu_true).max()
    # f and xi amplify d mu by 1 / (omega dt): the lowest modes (mu within 0.01 of 1) get
    # looser gates, the modes above 1 Hz the parity gates
    hi = model.f_true >= 1.0
    assert np.allclose(f_gpu[hi], model.f_true[hi], rtol=1e-4), np.abs(f_gpu / model.f_true - 1)[hi].max()
    assert np.allclose(f_gpu, model.f_true, rtol=5e-3)
    assert np.allclose(xi_gpu[hi], model.xi_true[hi], atol=2e-3)
    assert np.allclose(xi_gpu, model.xi_true, atol=1e-2)
    macs = np.array([O.mac(c240["Phi"][:, order[j]], model.phi_true[:, j]) for j in range(120)])
    assert macs[hi].min() > 0.999 and macs.min() > 0.99, (macs[hi].min(), macs.min())
    for c in (cells[0][0], cells[0][1]):
        assert len(c["f"]) >= 90
