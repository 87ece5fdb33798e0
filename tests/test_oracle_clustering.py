"""Pins of the oracle's two-stage clustering (Sec. 2.3 "3D clustering", Sec. 3.1).

Fuzzy C-means is tied to a brute-force minimisation of its own objective on a small
case; single linkage to an independent library routine; Stage II to a hand-built pole
set with known groups; the features of Stage I to values worked out by hand; the whole
procedure to the exact modes of a generating model.
"""
import numpy as np
import pytest

import oracle as O
import ssi_synth as S


def _cell(f, xi, phis, mpc=None, mpd=None, flags=None):
    f = np.asarray(f, float)
    n = len(f)
    return dict(mu=np.exp((-np.asarray(xi) * 2 * np.pi * f + 2j * np.pi * f) * 0.01),
                f=f, xi=np.asarray(xi, float), Phi=np.stack(phis, axis=1) if n else np.zeros((3, 0)),
                mpc=np.ones(n) if mpc is None else np.asarray(mpc, float),
                mpd=np.zeros(n) if mpd is None else np.asarray(mpd, float),
                flags=np.full(n, O.ST_HC, dtype=np.int64) if flags is None else np.asarray(flags))


def _fcm_objective(X, V, m=2.0):
    """J(V) = sum_k sum_c u_ck^m |x_k - v_c|^2 with the memberships that minimise J for
    these centroids (the reduced objective of fuzzy C-means)."""
    D2 = ((X[:, None, :] - V[None, :, :]) ** 2).sum(axis=2)
    D2 = np.maximum(D2, 1e-300)
    U = 1.0 / (D2[:, :, None] / D2[:, None, :]).sum(axis=2) ** (1.0 / (m - 1.0))
    return float(((U ** m) * D2).sum())


def test_fcm_fixed_point_minimises_the_objective():
    X = np.array([[0.0], [0.05], [0.2], [0.8], [0.9], [1.0]])
    U, V, it = O.fuzzy_c_means(X)
    assert np.allclose(U.sum(axis=1), 1.0)
    # brute force: the minimum of the reduced objective over a grid of centroid pairs
    g = np.linspace(-0.1, 1.1, 601)
    best = min((_fcm_objective(X, np.array([[a], [b]])), a, b) for a in g for b in g if a < b)
    assert V[0, 0] == pytest.approx(best[1], abs=3e-3)
    assert V[1, 0] == pytest.approx(best[2], abs=3e-3)
    assert _fcm_objective(X, V) <= best[0] + 1e-9


def test_fcm_points_on_centroids_are_crisp_and_separated_blobs_converge_to_their_means():
    X = np.array([[0.0, 0.0], [1.0, 2.0]])
    U, V, _ = O.fuzzy_c_means(X)
    assert np.array_equal(U, np.eye(2)) and np.allclose(V, X)
    rng = np.random.default_rng(3)
    a = rng.normal([0.01, 0.02], 1e-4, size=(50, 2))
    b = rng.normal([0.6, 0.4], 1e-4, size=(50, 2))
    U, V, _ = O.fuzzy_c_means(np.vstack([a, b]))
    assert np.allclose(V[0], a.mean(axis=0), atol=1e-4) and np.allclose(V[1], b.mean(axis=0), atol=1e-4)
    assert (U[:50, 0] > 0.99).all() and (U[50:, 1] > 0.99).all()


def test_single_linkage_cut_matches_the_library_dendrogram():
    hier = pytest.importorskip("scipy.cluster.hierarchy")
    from scipy.spatial.distance import squareform
    rng = np.random.default_rng(7)
    P = np.vstack([rng.normal(c, 0.05, size=(20, 2)) for c in ([0, 0], [1, 0], [0.55, 0.1])])
    D = np.sqrt(((P[:, None] - P[None]) ** 2).sum(-1))
    for tau in (0.05, 0.12, 0.3):
        ours = O.single_linkage_labels(D, tau)
        ref = hier.fcluster(hier.linkage(squareform(D, checks=False), "single"), tau, "distance")
        # the same partition: i, j together in one exactly when together in the other
        assert np.array_equal(ours[:, None] == ours[None], ref[:, None] == ref[None])


def test_stage2_recovers_hand_built_groups():
    rng = np.random.default_rng(11)
    shapes = np.eye(4)[:, :3] + 0j
    f0, xi0 = [2.0, 5.0, 9.0], [0.02, 0.015, 0.03]
    f, xi, Phi = [], [], []
    for r in range(3):
        for _ in range(12):
            f.append(f0[r] * (1 + rng.normal(0, 1e-3)))
            xi.append(xi0[r] * (1 + rng.normal(0, 1e-2)))
            Phi.append(shapes[:, r] + rng.normal(0, 1e-3, 4))
    for q in range(5):   # isolated poles
        f.append(3.0 + q)
        xi.append(0.05)
        Phi.append(np.array([1, 1, 1, 1.0]) + 0j)
    modes, labels, D = O.stage2(np.array(f), np.array(xi), np.stack(Phi, 1), tau=0.05, min_size=5)
    assert [m["size"] for m in modes] == [12, 12, 12]
    for md, fr, xr in zip(modes, f0, xi0):
        assert md["f"] == pytest.approx(fr, rel=2e-3) and md["xi"] == pytest.approx(xr, rel=2e-2)
    # the medoid minimises the sum of distances within its group
    md = modes[0]
    sums = D[np.ix_(md["members"], md["members"])].sum(axis=1)
    assert md["medoid"] == md["members"][int(np.argmin(sums))]


def test_stage1_features_by_hand():
    p = np.array([1.0, 0.0, 0.0]) + 0j
    q = np.array([1.0, 0.1, 0.0]) + 0j
    mac_pq = O.mac(p, q)
    # lag 0: order 2 -> 2.0 Hz; order 4 -> 2.02 Hz (stable, shape q), 7 Hz (not stable)
    d = [[_cell([2.0], [0.020], [p]),
          _cell([2.02, 7.0], [0.021, 0.01], [q, p], mpc=[0.9, 1.0], mpd=[0.05, 0.0],
                flags=[O.ST_HC | O.ST_ORDER, O.ST_HC])]]
    X, idx = O.stage1_features(d)
    assert idx == [(0, 1, 0)]
    assert np.allclose(X[0], [0.02 / 2.02, 0.001 / 0.021, 1 - mac_pq, 0.1, 0.05])


def test_two_stage_clustering_separates_model_poles_from_spurious_ones():
    """A 3D diagram (3 lags x 5 orders) holding the 4 poles of the chain model in every
    cell (perturbed by ~1e-4) plus 3 spurious stable poles per cell at random frequencies,
    damping and shapes.  Stage I must keep exactly the model poles (their features are
    near the origin), and Stage II must return the 4 model modes, each with 14 poles (the
    first cell has no neighbour, so its poles are never Stage I candidates)."""
    model = S.chain_model(S.workload("chain4_tiny"))
    rng = np.random.default_rng(5)
    diagram = []
    for t in range(3):
        row = []
        for m in range(5):
            f = list(model.f_true * (1 + rng.normal(0, 1e-4, 4)))
            xi = list(model.xi_true * (1 + rng.normal(0, 1e-3, 4)))
            phis = [model.phi_true[:, r] * (1 + rng.normal(0, 1e-5, 4)) for r in range(4)]
            mpc = [1.0] * 4
            mpd = [0.0] * 4
            for _ in range(3):
                f.append(rng.uniform(1.0, 10.0))
                xi.append(rng.uniform(0.01, 0.09))
                phis.append(rng.normal(size=4) + 1j * rng.normal(size=4))
                mpc.append(rng.uniform(0.61, 0.8))
                mpd.append(rng.uniform(0.2, 0.49))
            row.append(_cell(f, xi, phis, mpc=mpc, mpd=mpd,
                             flags=np.full(7, O.ST_HC | O.ST_ORDER, dtype=np.int64)))
        diagram.append(row)
    modes, keep, P, idx = O.cluster_modes(diagram, tau=0.05, min_size=5)
    is_model = np.array([i < 4 for t, m, i in idx])
    assert np.array_equal(keep, is_model)
    assert [md["size"] for md in modes] == [14, 14, 14, 14]
    assert np.allclose([md["f"] for md in modes], model.f_true, rtol=1e-4)
    assert np.allclose([md["xi"] for md in modes], model.xi_true, rtol=1e-3)


def test_pin_catches_a_wrong_fcm_exponent(monkeypatch):
    """Plant u = 1 / sum (d_c/d_j)^(1/(m-1)) (the exponent 2/(m-1) halved) in the oracle's
    membership update: the fixed point no longer minimises the objective, and the
    brute-force pin fails."""
    real_sum = sum

    def fcm_wrong(X, m=2.0, tol=1e-10, max_iter=500):
        X = np.asarray(X, dtype=np.float64)
        V = np.stack([X.min(axis=0), X.max(axis=0)])
        U = np.full((X.shape[0], 2), 0.5)
        for it in range(1, max_iter + 1):
            D = np.sqrt(((X[:, None, :] - V[None, :, :]) ** 2).sum(axis=2))
            D = np.maximum(D, 1e-300)
            Un = np.array([[1.0 / real_sum((D[k, c] / D[k, j]) ** (1.0 / (m - 1.0)) for j in range(2))
                            for c in range(2)] for k in range(X.shape[0])])
            W = Un ** m
            V = (W.T @ X) / W.sum(axis=0)[:, None]
            done = np.abs(Un - U).max() < tol
            U = Un
            if done:
                break
        return U, V, it

    monkeypatch.setattr(O, "fuzzy_c_means", fcm_wrong)
    with pytest.raises(AssertionError):
        test_fcm_fixed_point_minimises_the_objective()


def test_fcm_cluster_without_weight_keeps_its_centroid():
    """Reading: a C-means cluster whose memberships are all zero keeps its centroid (the
    update would be 0/0).  One pole, or two equal poles (their mean is exact), sit on the
    first centroid: they belong to it alone, the second keeps the start value, and nothing
    becomes NaN; the poles are kept (the physical cluster is the first of two equally near
    centroids)."""
    import warnings
    for X in (np.array([[0.01, 0.02, 0.001, 0.05, 0.1]]),
              np.repeat([[0.01, 0.02, 0.001, 0.05, 0.1]], 2, axis=0)):
        with warnings.catch_warnings():
            warnings.simplefilter("error")
            U, V, it = O.fuzzy_c_means(X)
            keep, P, V2, phys, _ = O.stage1(X)
        assert np.all(U == [1.0, 0.0]) and np.all(V == X[0]) and it == 2
        assert phys == 0 and np.all(keep) and np.all(P == 1.0)
