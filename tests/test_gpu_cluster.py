"""Two-stage clustering (Sec. 2.3 "3D clustering", Sec. 3.1) on the GPU against the oracle.

The GPU solve's own poles, mode shapes and stability flags are the input of both sides:
the oracle receives them as FP64 cells (frequency, damping, MPC, MPD, complex128 shapes),
so the two compute the same definition on the same numbers.  Checked pole by pole:
  * the Stage I candidates are the same slots, and their features agree to 1e-12
    (both take the neighbour decisions on FP64 distances; the sums differ only in order);
  * memberships of the physical C-means cluster agree to 1e-9 (the two reductions run in
    different orders, the fixed point is the same) and the keep decisions are equal
    (no membership lies within 1e-6 of 1/2 here);
  * Stage II: no kept pair lies within 1e-9 of tau, so the components are unique; every
    oracle mode is a GPU mode with the same members, size and medoid, and mean frequency
    and damping to 1e-12 relative.
On the bridge records of the benchmark (one lag, and the 9-lag 3D diagram) the modes are
checked against the generating modes instead: every generating mode is found within 1 %
in frequency with a medoid shape of MAC >= 0.99.
"""
import numpy as np
import pytest
import torch

import oracle as O
import ssi_synth as S
from parity import gpu_cells

pytestmark = pytest.mark.gpu

TAU, MIN_SIZE = 0.05, 10


@pytest.fixture(scope="module")
def P():
    import paper_2411_05510_gb300 as P
    return P


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()


def _solve(P, ctx, w, seed=5):
    Y, f_true, _, phi_true = S.record(w, np.float32)
    desc = P.job_desc(torch.from_numpy(Y).cuda(), w["fs"], w["lags"], w["orders"], k=w["k"],
                      oversample=w["oversample"], q=w["q"], prec="split_bf16", seed=seed)
    poles, phi, _ = P.ssi_solve(ctx, desc)
    P.check_sync(ctx)
    return poles, phi, f_true, phi_true


def _fp64_cells(rec, phi, w):
    cells = gpu_cells(rec, phi, w["lags"], w["orders"], w["l"])
    for row in cells:
        for c in row:
            c["mpc"] = np.asarray(c["mpc"], dtype=np.float64)
            c["mpd"] = np.asarray(c["mpd"], dtype=np.float64)
            c["Phi"] = np.asarray(c["Phi"], dtype=np.complex128)
    return cells


def _slot_map(rec, w):
    """(t, m, i) of the oracle cells -> slot; valid poles form a prefix of their cell."""
    offs = np.concatenate([[0], np.cumsum([n // 2 for n in w["orders"]])])
    spl = offs[-1]
    for t in range(len(w["lags"])):
        for m, n in enumerate(w["orders"]):
            v = (rec["flags"][t * spl + offs[m]: t * spl + offs[m] + n // 2] & 64) != 0
            assert not np.any(v[np.argmin(v):]) or v.all(), (t, m)
    return lambda tmi: int(tmi[0] * spl + offs[tmi[1]] + tmi[2])


@pytest.fixture(scope="module")
def diag3(P, ctx):
    """Reduced bridge record (24 channels, 6 modes in 4-20 Hz, N = 60000), 3D diagram over
    lags 14, 18, 22, RSVD k = 32 + 16 with q = 2, orders 2..32."""
    w = S.workload("bridge186_3d", l=24, modes=6, f_lo=4.0, N=60000, lags=[14, 18, 22], k=32,
                   oversample=16, orders=list(range(2, 33, 2)))
    poles, phi, f_true, phi_true = _solve(P, ctx, w)
    return w, poles, phi, f_true, phi_true


def test_cluster_matches_oracle_pole_by_pole(P, ctx, diag3):
    w, poles, phi, f_true, phi_true = diag3
    modes, info, pp = P.ssi_cluster(ctx, len(w["lags"]), w["orders"], w["l"], poles, phi,
                                    P.cluster_params(tau=TAU, min_size=MIN_SIZE), per_pole=True)
    rec = P.poles_to_numpy(poles)
    slot = _slot_map(rec, w)
    cells = _fp64_cells(rec, phi.cpu().numpy(), w)
    feats = pp["features"].cpu().numpy()
    memb = pp["membership"].cpu().numpy()
    lab = pp["label"].cpu().numpy()

    # Stage I: candidates and features
    X, idx = O.stage1_features(cells)
    slots = np.array([slot(q) for q in idx])
    assert info["n_candidates"] == len(idx) > 50
    assert np.array_equal(np.nonzero(memb >= 0)[0], slots)
    assert np.abs(feats[slots] - X).max() <= 1e-12

    # Stage I: C-means
    keep, Pm, V, phys, it = O.stage1(X)
    assert info["physical"] == phys and info["fcm_converged"] == 1
    assert abs(info["fcm_iterations"] - it) <= 1, (info["fcm_iterations"], it)
    assert np.abs(info["centroids"] - V).max() <= 1e-9
    assert np.abs(memb[slots] - Pm).max() <= 1e-9
    assert np.abs(Pm - 0.5).min() > 1e-6
    assert np.array_equal(memb[slots] >= 0.5, keep)
    assert info["n_kept"] == int(keep.sum()) > 20

    # Stage II
    kept = [idx[q] for q in np.nonzero(keep)[0]]
    kslots = np.array([slot(q) for q in kept])
    f = np.array([cells[t][m]["f"][i] for t, m, i in kept])
    xi = np.array([cells[t][m]["xi"][i] for t, m, i in kept])
    Phi = np.stack([cells[t][m]["Phi"][:, i] for t, m, i in kept], axis=1)
    omodes, olab, D = O.stage2(f, xi, Phi, TAU, MIN_SIZE)
    iu = np.triu_indices(len(kept), 1)
    assert np.abs(D[iu] - TAU).min() > 1e-9
    assert np.array_equal(np.nonzero(lab >= 0)[0], kslots)
    # the same partition: GPU labels are the first slot of each component
    assert np.array_equal(lab[kslots], kslots[olab])
    assert info["n_components"] == len(np.unique(olab))
    assert info["n_modes"] == len(omodes) == len(modes) >= 4
    for om, gm in zip(omodes, modes):
        assert gm["size"] == om["size"]
        assert abs(gm["f_hz"] - om["f"]) <= 1e-12 * om["f"]
        assert abs(gm["xi"] - om["xi"]) <= 1e-12 * om["xi"]
        mem = kslots[om["members"]]
        assert np.array_equal(np.sort(np.nonzero(lab == lab[mem[0]])[0]), mem)
        sums = D[np.ix_(om["members"], om["members"])].sum(axis=1)
        if gm["medoid_slot"] != kslots[om["medoid"]]:
            j = int(np.nonzero(mem == gm["medoid_slot"])[0][0])
            assert sums[j] - sums.min() <= 1e-12 * sums.min()
    # and the modes are the generating ones
    for r, f0 in enumerate(f_true):
        near = [m for m in modes if abs(m["f_hz"] - f0) / f0 < 1e-2]
        assert near, (r, f0)


def test_cluster_is_deterministic_and_grid_independent(P, diag3):
    """Two calls, and a call with the C-means grid cut to a quarter of the SMs
    (set_concurrency(4)), give the same bytes: the reductions run over fixed chunks in a
    fixed order, and the components do not depend on the order of the links."""
    w, poles, phi, *_ = diag3
    out = []
    for conc in (1, 1, 4):
        c = P.Context(0)
        try:
            c.set_concurrency(conc)
            modes, info, pp = P.ssi_cluster(c, len(w["lags"]), w["orders"], w["l"], poles, phi,
                                            per_pole=True)
            out.append((modes, {k: v for k, v in info.items() if k != "centroids"},
                        info["centroids"].tobytes(),
                        [pp[k].cpu().numpy().tobytes() for k in ("features", "membership", "label")]))
        finally:
            c.close()
    for o in out[1:]:
        assert o[0] == out[0][0]
        assert o[1] == out[0][1]
        assert o[2] == out[0][2]
        assert o[3] == out[0][3]


def test_cluster_edge_cases(P, ctx, diag3):
    w, poles, phi, *_ = diag3
    n_lags, orders, l = len(w["lags"]), w["orders"], w["l"]
    base, info0, _ = P.ssi_cluster(ctx, n_lags, orders, l, poles, phi)
    # a mode table shorter than the number of modes: the first ones, the full count
    short, info, _ = P.ssi_cluster(ctx, n_lags, orders, l, poles, phi, max_modes=2)
    assert short == base[:2] and info["n_modes"] == len(base) > 2
    # min_size above every component: no modes, the same Stage I
    none, info, _ = P.ssi_cluster(ctx, n_lags, orders, l, poles, phi,
                                  P.cluster_params(min_size=10 ** 6))
    assert none == [] and info["n_kept"] == info0["n_kept"]
    # tau = 0 with min_size 1: (almost) every kept pole is its own mode
    _, info, pp = P.ssi_cluster(ctx, n_lags, orders, l, poles, phi,
                                P.cluster_params(tau=0.0, min_size=1), max_modes=0, per_pole=True)
    lab = pp["label"].cpu().numpy()
    kept = np.nonzero(lab >= 0)[0]
    assert info["n_components"] == info["n_modes"] == len(np.unique(lab[kept]))
    assert info["n_components"] >= info["n_kept"] - 2
    # no stable pole at all (zero soft-criteria thresholds): nothing enters Stage I
    p2 = poles.clone()
    P.ssi_stabilize(ctx, n_lags, orders, l, p2, phi,
                    P.stab_params(a_f=0.0, a_xi=0.0, a_mac=0.0))
    torch.cuda.synchronize()
    rec = P.poles_to_numpy(p2)
    assert not np.any(rec["flags"] & 48)
    modes, info, pp = P.ssi_cluster(ctx, n_lags, orders, l, p2, phi, per_pole=True)
    assert modes == [] and info["n_candidates"] == 0 and info["n_kept"] == 0
    assert np.all(pp["membership"].cpu().numpy() == -1.0)
    assert np.all(pp["label"].cpu().numpy() == -1)
    # bad parameters are refused
    for bad in (P.cluster_params(tau=-1.0), P.cluster_params(min_size=0),
                P.cluster_params(fcm_m=1.0), P.cluster_params(fcm_tol=0.0)):
        with pytest.raises(P.SsiError):
            P.ssi_cluster(ctx, n_lags, orders, l, poles, phi, bad)


def _identified(modes, rec_phi, f_true, phi_true):
    """Generating modes matched one to one by a mode within 1 % in frequency whose
    medoid shape has MAC >= 0.99 with the generating shape."""
    used = set()
    for r, f0 in enumerate(f_true):
        for k, m in enumerate(modes):
            if k in used or abs(m["f_hz"] - f0) / f0 >= 1e-2:
                continue
            v = rec_phi[m["medoid_slot"]]
            if O.mac(v[:, 0] + 1j * v[:, 1], phi_true[:, r]) >= 0.99:
                used.add(k)
                break
    return len(used)


@pytest.mark.slow
@pytest.mark.parametrize("name", ["bridge186_i60", "bridge186_3d"])
def test_cluster_identifies_bridge_modes(P, ctx, name):
    """The benchmark's bridge record (186 channels, 20 modes in 1-20 Hz): one lag i = 60,
    and the 3D diagram over lags 20..100; orders 2..200, min_size 10 (1 lag) or 50 (9 lags)."""
    w = S.workload(name)
    poles, phi, f_true, phi_true = _solve(P, ctx, w, seed=12345)
    min_size = 10 if len(w["lags"]) == 1 else 50
    modes, info, _ = P.ssi_cluster(ctx, len(w["lags"]), w["orders"], w["l"], poles, phi,
                                   P.cluster_params(tau=TAU, min_size=min_size))
    rec_phi = phi.cpu().numpy().reshape(-1, w["l"], 2)
    assert _identified(modes, rec_phi, f_true, phi_true) == w["modes"] == len(modes), (info, modes)


@pytest.mark.slow
def test_cluster_identifies_frame10_modes_from_the_3d_diagram(P, ctx):
    """The 10-DOF frame of Sec. 3.1 (fs 200 Hz, 10 % noise, N = 60000): 3D diagram over ten
    lags from 170 to 255, RSVD k = 512 with p = q = 0 (Algorithm 1), orders 2..30, then the
    clustering.  Every generating mode is matched by a mode within 0.5 % in frequency whose
    medoid's shape has MAC >= 0.99 with the model's and whose damping is within 40 % (a
    300 s record); a mode may also come out twice (a second component of the same poles
    above min_size), so at most two extra modes are allowed."""
    w = S.workload("frame10", seed=100)
    Y, f_true, xi_true, phi_true = S.record(w, np.float32)
    lags = [int(x) for x in np.linspace(170, 255, 10).round()]
    orders = list(range(2, 31, 2))
    desc = P.job_desc(torch.from_numpy(Y).cuda(), w["fs"], lags, orders, k=512, oversample=0, q=0,
                      prec="split_bf16", seed=0)
    poles, phi, _ = P.ssi_solve(ctx, desc, with_s=False)
    modes, info, _ = P.ssi_cluster(ctx, len(lags), orders, Y.shape[0], poles, phi,
                                   P.cluster_params(tau=TAU, min_size=len(lags) * len(orders) // 4))
    ph = phi.cpu().numpy().reshape(-1, Y.shape[0], 2)
    assert len(f_true) <= len(modes) <= len(f_true) + 2, (info, modes)

    def mac_of(m, r):
        v = ph[m["medoid_slot"]]
        return O.mac(v[:, 0] + 1j * v[:, 1], phi_true[:, r])

    for r, f0 in enumerate(f_true):
        near = [m for m in modes if abs(m["f_hz"] - f0) / f0 < 5e-3]
        assert near, (r, f0, modes)
        m = max(near, key=lambda m: mac_of(m, r))
        assert mac_of(m, r) >= 0.99, (r, m)
        assert abs(m["xi"] - xi_true[r]) / xi_true[r] < 0.4, (r, m, xi_true[r])


def test_cluster_single_stable_pole(P, ctx, diag3):
    """One stable pole in the whole diagram (the stability bits of all others cleared): it is
    the only Stage I candidate, C-means puts it on the first centroid (the second cluster,
    without weight, keeps its start centroid), it is kept, and with min_size 1 it is a mode
    of its own and its own medoid; the oracle agrees."""
    w, poles, phi, *_ = diag3
    rec = P.poles_to_numpy(poles)
    stable = np.nonzero((rec["flags"] & 48) != 0)[0]
    one = int(stable[len(stable) // 2])
    raw = poles.cpu().numpy().copy()
    words = raw.view(np.uint32).reshape(len(raw), 10)    # flags are word 8 of a record
    keep_bits = words[one, 8]
    words[:, 8] &= ~np.uint32(48)
    words[one, 8] = keep_bits
    p1 = torch.from_numpy(raw).cuda()
    modes, info, pp = P.ssi_cluster(ctx, len(w["lags"]), w["orders"], w["l"], p1, phi,
                                    P.cluster_params(min_size=1), per_pole=True)
    assert info["n_candidates"] == 1 and info["n_kept"] == 1 and info["n_modes"] == 1, info
    assert info["fcm_converged"] == 1 and info["physical"] == 0
    assert np.all(np.isfinite(info["centroids"]))
    assert modes[0]["medoid_slot"] == one and modes[0]["size"] == 1
    assert modes[0]["f_hz"] == float(rec["f_hz"][one])
    memb = pp["membership"].cpu().numpy()
    lab = pp["label"].cpu().numpy()
    assert memb[one] == 1.0 and np.count_nonzero(memb >= 0) == 1
    assert lab[one] == one and np.count_nonzero(lab >= 0) == 1
    cells = _fp64_cells(P.poles_to_numpy(p1), phi.cpu().numpy(), w)
    omodes, keep, _, idx = O.cluster_modes(cells, tau=TAU, min_size=1)
    assert len(idx) == 1 and keep.all() and len(omodes) == 1
