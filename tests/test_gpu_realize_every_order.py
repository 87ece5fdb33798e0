"""Realisation parity at every model order, at the full bridge size.

Both sides realise the SAME left singular vectors: the oracle's FP64 RSVD of the record's
FP64 covariances (186 channels, N = 360000, same Omega seed as the benchmark), handed to
the GPU in FP64 (its FP32 mode rounds them once to FP32; its FP64 mode keeps them).  The
oracle realises every order n = 2..200 from them by its own route (Sec. 2.1: O = U S^{1/2}, a fresh Householder QR of O^to per
order, numpy eig, Phi = C Psi); the GPU by its nested-order factorisation and its
eigensolver.  With the subspace shared, the degeneracy of the noise singular values
(which makes orders above the physical rank irreproducible between two SVDs) plays no
part, so every order n >= 2 m is gated, not only the separated ones.

Parity set, per order n >= 2 m and generating mode r: the oracle's pole of mode r (HC-
passing, within 5 % of f_r, largest MAC with the generating shape) and the GPU pole with
the nearest discrete eigenvalue mu: frequency <= 1e-4 relative, damping <= 2e-3 absolute,
MAC >= 0.999.  Every oracle pole of the parity set must have its GPU counterpart.  The
FP64 mode must in addition meet 100 times tighter bounds (frequency 1e-6, damping 2e-5,
1 - MAC 1e-5; its pole records and mode shapes are rounded once to FP32).

Two Toeplitz sizes: i = 60 (T 11160 x 11160, the benchmark) and i = 100 (T 18600 x
18600, the largest lag of the 3D diagram), k = 200 + 20, q = 2.  The oracle leg takes a
few minutes of host time; its realisations run in a spawned process pool.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest
import torch

import oracle as O
import ssi_synth as S
from parity import F_TOL, MAC_MIN, XI_TOL, gpu_cells, nearest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SEED = 12345
LAGS = (60, 100)

_U = None


def _init(U, s):
    global _U
    _U = (U, s)


def _realize(args):
    l, i, n, dt = args
    U, s = _U
    mu, f, xi, Phi, _ = O.realize(U, s, l, i, n, dt)
    mpcs, mpds, fail = O.hard_criteria(mu, f, xi, Phi)
    return dict(mu=mu, f=f, xi=xi, Phi=Phi, mpc=mpcs, mpd=mpds,
                flags=fail | np.where(fail == 0, O.ST_HC, 0))


@pytest.fixture(scope="module")
def oracle_side():
    w = S.workload("bridge186_i60")
    Y, f_true, _, phi_true = S.record(w, np.float32)
    R = O.covariances(Y.astype(np.float64), 2 * max(LAGS) - 1)
    out = {}
    ctx = mp.get_context("spawn")
    for i in LAGS:
        U, s = O.rsvd(O.block_toeplitz(R, i), w["k"], w["oversample"], w["q"], SEED)
        with cf.ProcessPoolExecutor(8, mp_context=ctx, initializer=_init, initargs=(U, s)) as ex:
            cells = list(ex.map(_realize, [(w["l"], i, n, 1.0 / w["fs"]) for n in w["orders"]]))
        out[i] = dict(U=U, s=s, cells=cells)
    return dict(w=w, f_true=f_true, phi_true=phi_true, lags=out)


def _gpu_realize(w, i, U64, small):
    import paper_2411_05510_gb300 as P
    ctx = P.Context(0)
    U = torch.from_numpy(U64).cuda()
    poles, phi = P.ssi_realize_batch(ctx, [i], [U], w["l"], w["k"], w["orders"], 1.0 / w["fs"],
                                     small)
    P.ssi_stabilize(ctx, 1, w["orders"], w["l"], poles, phi, P.stab_params(use_lag_axis=False))
    P.check_sync(ctx)
    rec = P.poles_to_numpy(poles)
    cells = gpu_cells(rec, phi.cpu().numpy(), [i], w["orders"], w["l"])[0]
    ctx.close()
    return cells


def _compare(gpu, ora, f_true, phi_true, orders, n_modes):
    worst = [0.0, 0.0, 0.0]
    where = [None, None, None]
    n_cmp = missing = 0
    for m, n in enumerate(orders):
        if n < 2 * n_modes:
            continue
        for r, f0 in enumerate(f_true):
            a = nearest(ora[m], f0, phi_true[:, r])
            if a is None:
                missing += 1
                continue
            mu_a = ora[m]["mu"][a]
            assert len(gpu[m]["mu"]) > 0, (n, r)
            b = int(np.argmin(np.abs(gpu[m]["mu"] - mu_a)))
            fa, fb = ora[m]["f"][a], gpu[m]["f"][b]
            v = (abs(fa - fb) / fa, abs(ora[m]["xi"][a] - gpu[m]["xi"][b]),
                 1.0 - O.mac(ora[m]["Phi"][:, a], gpu[m]["Phi"][:, b]))
            for q in range(3):
                if v[q] > worst[q]:
                    worst[q], where[q] = v[q], (n, r, fa, fb)
            n_cmp += 1
    return n_cmp, missing, worst, where


@pytest.mark.parametrize("small", ["fp32", "fp64"])
@pytest.mark.parametrize("i", LAGS)
def test_every_order_matches_oracle_on_shared_subspace(oracle_side, i, small):
    w = oracle_side["w"]
    side = oracle_side["lags"][i]
    gpu = _gpu_realize(w, i, side["U"], small)
    m = w["modes"]
    n_cmp, missing, worst, where = _compare(gpu, side["cells"], oracle_side["f_true"],
                                            oracle_side["phi_true"], w["orders"], m)
    n_gated_orders = sum(1 for n in w["orders"] if n >= 2 * m)
    print(f"i={i} {small}: {n_cmp} pole pairs over {n_gated_orders} orders ({missing} mode-orders "
          f"without an oracle pole); worst df {worst[0]:.2e} dxi {worst[1]:.2e} "
          f"1-MAC {worst[2]:.2e}")
    # the oracle finds (nearly) every mode at every order, and each of its poles has a GPU twin
    assert missing <= n_gated_orders, missing
    assert n_cmp == m * n_gated_orders - missing
    assert worst[0] <= F_TOL, ("frequency", worst[0], where[0])
    assert worst[1] <= XI_TOL, ("damping", worst[1], where[1])
    assert worst[2] <= 1 - MAC_MIN, ("MAC", worst[2], where[2])
    if small == "fp64":
        assert worst[0] <= 1e-6 and worst[1] <= 2e-5 and worst[2] <= 1e-5, (worst, where)
