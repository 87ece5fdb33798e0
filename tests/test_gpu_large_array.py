"""Parity on the large-array configuration (512 channels, 40 modes 0.5-30 Hz, i = 100,
k = 400 + 40, q = 3, orders 2..400), on its decimated instance: the first 128 channels
of the same kind of record (40 modes, fs = 100 Hz, N = 1.08 M, 5 % noise, seed 5) at
i = 40 (T 5120 x 5120).  The oracle's full Jacobi SVD of the 512-channel T (51200 x
51200, about 8e15 flops) is out of reach, so the decimated instance stands in for it.

  * Range finder: the GPU's split-BF16 RSVD with q = 3 (as configured) against the
    oracle's FP64 RSVD of the same T with q = 6 and the same Omega: the leading 2 m = 80
    singular values agree to 1e-4 relative, in both small-problem precisions; and against
    the full SVD of T from LAPACK, the same 80 to 1e-4.
  * Realisation: from the oracle's own U (shared subspace) every order n >= 2 m up to 400
    is realised by both sides; the parity set (the oracle's HC-passing pole of each
    generating mode against the GPU pole with the nearest eigenvalue) meets frequency
    1e-4, damping 2e-3 and MAC 0.999.  With FP64 small problems: all three gates at every
    order.  With FP32 ones: frequency and damping at the orders up to 224, shapes at the
    orders up to 152.  Above 152 a generating mode's shape can sit beside a second
    eigenvalue within ~1e-6 of it (order 154 onwards, the 0.61 Hz mode), where the
    eigenvector of the pair is ill-conditioned and FP32 rounding rotates it inside the
    pair's invariant subspace; above 224 the 0.5 Hz mode's frequency misses 1e-4 (df/f =
    |d mu| / (omega dt) amplifies the FP32 eigenvalue error 32-fold there).  So the large
    array needs SSI_SMALL_FP64.  Orders above 224 run with A in global scratch (in both
    precisions), and k = 400 factors in global scratch.
The oracle leg takes a few minutes of host time.
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
L_CH, I_LAG = 128, 40

_U = None


def _init(U, s):
    global _U
    _U = (U, s)


def _realize(args):
    l, i, n, dt = args
    U, s = _U
    mu, f, xi, Phi, _ = O.realize(U, s, l, i, n, dt)
    mpcs, mpds, fail = O.hard_criteria(mu, f, xi, Phi)
    return dict(mu=mu, f=f, xi=xi, Phi=Phi, flags=fail | np.where(fail == 0, O.ST_HC, 0))


@pytest.fixture(scope="module")
def case():
    w = S.workload("bridge512_i100", l=L_CH, lags=[I_LAG])
    Y, f_true, _, phi_true = S.record(w, np.float32)
    R = O.covariances(Y.astype(np.float64), 2 * I_LAG - 1)
    U, s = O.rsvd(O.block_toeplitz(R, I_LAG), w["k"], w["oversample"], 6, SEED)
    with cf.ProcessPoolExecutor(8, mp_context=mp.get_context("spawn"), initializer=_init,
                                initargs=(U, s)) as ex:
        cells = list(ex.map(_realize, [(L_CH, I_LAG, n, 1.0 / w["fs"]) for n in w["orders"]]))
    return dict(w=w, R=R, U=U, s=s, cells=cells, f_true=f_true, phi_true=phi_true)


@pytest.mark.parametrize("small", ["fp32", "fp64"])
def test_large_array_leading_singular_values(case, small):
    import paper_2411_05510_gb300 as P
    w = case["w"]
    ctx = P.Context(0)
    Rd = torch.from_numpy(case["R"]).cuda()
    U, Sg = P.ssi_toeplitz_rsvd(ctx, Rd, L_CH, I_LAG, w["k"], w["oversample"], w["q"], SEED,
                                "split_bf16", small)
    P.check_sync(ctx)
    s = Sg.cpu().numpy()
    ctx.close()
    m2 = 2 * w["modes"]
    rel = np.abs(s[:m2] / case["s"][:m2] - 1)
    print(f"{small}: leading {m2} singular values, worst relative error {rel.max():.2e}")
    assert rel.max() <= 1e-4, (int(rel.argmax()), rel.max())


def test_large_array_singular_values_against_lapack_svd(case):
    """The full SVD of the decimated T (5120 x 5120) from LAPACK: the GPU's leading 2 m = 80
    singular values (split-BF16 range finder, q = 3, as configured) within 1e-4."""
    import paper_2411_05510_gb300 as P
    w = case["w"]
    s_full = np.linalg.svd(O.block_toeplitz(case["R"], I_LAG), compute_uv=False)
    ctx = P.Context(0)
    Rd = torch.from_numpy(case["R"]).cuda()
    _, Sg = P.ssi_toeplitz_rsvd(ctx, Rd, L_CH, I_LAG, w["k"], w["oversample"], w["q"], SEED,
                                "split_bf16")
    P.check_sync(ctx)
    s = Sg.cpu().numpy()
    ctx.close()
    m2 = 2 * w["modes"]
    rel = np.abs(s[:m2] / s_full[:m2] - 1)
    print(f"leading {m2} singular values against LAPACK's full SVD: worst relative error {rel.max():.2e}")
    assert rel.max() <= 1e-4, (int(rel.argmax()), rel.max())


@pytest.mark.parametrize("small", ["fp32", "fp64"])
def test_large_array_every_order_on_shared_subspace(case, small):
    import paper_2411_05510_gb300 as P
    w = case["w"]
    ctx = P.Context(0)
    Ud = torch.from_numpy(np.ascontiguousarray(case["U"])).cuda()
    poles, phi = P.ssi_realize_batch(ctx, [I_LAG], [Ud], L_CH, w["k"], w["orders"], 1.0 / w["fs"],
                                     small)
    P.ssi_stabilize(ctx, 1, w["orders"], L_CH, poles, phi, P.stab_params(use_lag_axis=False))
    P.check_sync(ctx)
    gpu = gpu_cells(P.poles_to_numpy(poles), phi.cpu().numpy(), [I_LAG], w["orders"], L_CH)[0]
    ctx.close()
    m = w["modes"]
    worst, where, n_cmp, missing = [0.0, 0.0, 0.0], [None] * 3, 0, 0
    notconv = [n for mi, n in enumerate(w["orders"])
               if np.any(P.poles_to_numpy(poles)["flags"][sum(o // 2 for o in w["orders"][:mi]):
                                                          sum(o // 2 for o in w["orders"][:mi + 1])]
                         & 128)]
    n_top = 400 if small == "fp64" else 224          # frequency and damping gates
    n_top_mac = 400 if small == "fp64" else 152      # shape gate
    first_fail = None
    for mi, n in enumerate(w["orders"]):
        if n < 2 * m:
            continue
        ora = case["cells"][mi]
        for r, f0 in enumerate(case["f_true"]):
            a = nearest(ora, f0, case["phi_true"][:, r])
            if a is None:
                missing += n <= n_top
                continue
            b = int(np.argmin(np.abs(gpu[mi]["mu"] - ora["mu"][a])))
            v = (abs(gpu[mi]["f"][b] - ora["f"][a]) / ora["f"][a], abs(gpu[mi]["xi"][b] - ora["xi"][a]),
                 1.0 - O.mac(gpu[mi]["Phi"][:, b], ora["Phi"][:, a]))
            if first_fail is None and (v[0] > F_TOL or v[1] > XI_TOL or v[2] > 1 - MAC_MIN):
                first_fail = (n, r)
            if n > n_top:
                continue
            for q_ in range(3):
                if q_ == 2 and n > n_top_mac:
                    continue
                if v[q_] > worst[q_]:
                    worst[q_], where[q_] = v[q_], (n, r, float(ora["f"][a]), float(gpu[mi]["f"][b]),
                                                   complex(ora["mu"][a]), complex(gpu[mi]["mu"][b]))
            n_cmp += 1
    n_orders = sum(1 for n in w["orders"] if 2 * m <= n <= n_top)
    print(f"{small}: {n_cmp} pole pairs over {n_orders} orders up to {n_top} ({missing} without an "
          f"oracle pole); worst df {worst[0]:.2e} dxi {worst[1]:.2e} 1-MAC {worst[2]:.2e} "
          f"(shapes up to order {n_top_mac})")
    print(f"{small}: worst at (order, mode, f_oracle, f_gpu, mu_oracle, mu_gpu): {where}; "
          f"first (order, mode) outside the gates at any order: {first_fail}; "
          f"orders with a non-converged eig: {notconv}")
    assert missing <= n_orders and n_cmp >= (m - 1) * n_orders
    assert worst[0] <= F_TOL and worst[1] <= XI_TOL and worst[2] <= 1 - MAC_MIN, (worst, where)
