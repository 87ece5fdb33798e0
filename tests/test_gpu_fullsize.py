"""Parity at the full bridge size, in the configuration the benchmark times.

Record: 186 channels, 20 modes (1-20 Hz), N = 360000, 5 % noise; i = 60 (T 11160 x
11160), RSVD k = 200 + 20 with q = 2, orders 2..200, split-BF16 lag and sketch GEMMs,
seed 12345 (the benchmark's).  The oracle computes the FP64 covariances of the whole
record, its own FP64 RSVD of the explicit T with the same Omega, and realisations at
the orders whose leading singular subspace is separated by a gap >= 2 (here n = 40 =
2 m).  Checked:
  * leading 2 m singular values <= 1e-4 relative;
  * the parity set at those orders (frequency <= 1e-4 relative, damping <= 2e-3,
    MAC >= 0.999 between the two results);
  * identification quality, a property of the record independent of both
    implementations: every generating mode found at the separated orders, and at least
    m - 1 of them at every order from 2 m on.
The oracle leg takes about 1.5 minutes of host time.
"""
import numpy as np
import pytest
import torch

import oracle as O
import ssi_synth as S
from parity import compare_parity_set, gpu_cells, nearest, separated_orders

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

SEED = 12345


@pytest.fixture(scope="module")
def case():
    import paper_2411_05510_gb300 as P
    w = S.workload("bridge186_i60")
    Y, f_true, _, phi_true = S.record(w, np.float32)
    ctx = P.Context(0)
    desc = P.job_desc(torch.from_numpy(Y).cuda(), w["fs"], w["lags"], w["orders"], k=w["k"],
                      oversample=w["oversample"], q=w["q"], prec="split_bf16", seed=SEED)
    poles, phi, Sg = P.ssi_solve(ctx, desc)
    P.check_sync(ctx)
    rec = P.poles_to_numpy(poles)
    gpu = gpu_cells(rec, phi.cpu().numpy(), w["lags"], w["orders"], w["l"])
    s_gpu = Sg.cpu().numpy()[0].astype(np.float64)
    ctx.close()
    # oracle: FP64 covariances of the whole record, FP64 RSVD with the same Omega
    i = w["lags"][0]
    R = O.covariances(Y.astype(np.float64), 2 * i - 1)
    U, s = O.rsvd(O.block_toeplitz(R, i), w["k"], w["oversample"], w["q"], SEED)
    gate = separated_orders(w["orders"], s)
    ora_row = []
    for n in w["orders"]:
        if n in gate:
            mu, f, xi, Phi, _ = O.realize(U, s, w["l"], i, n, 1.0 / w["fs"])
            ora_row.append(dict(mu=mu, f=f, xi=xi, Phi=Phi))
        else:
            ora_row.append(dict(mu=np.zeros(0), f=np.zeros(0), xi=np.zeros(0),
                                Phi=np.zeros((w["l"], 0))))
    return dict(w=w, f_true=f_true, phi_true=phi_true, gpu=gpu, s_gpu=s_gpu, s=s, gate=gate,
                ora=[ora_row])


def test_leading_singular_values(case):
    m2 = 2 * case["w"]["modes"]
    rel = np.abs(case["s_gpu"][:m2] - case["s"][:m2]) / case["s"][:m2]
    assert rel.max() <= 1e-4, (rel.argmax(), rel.max())


def test_parity_set_at_separated_orders(case):
    w = case["w"]
    assert 2 * w["modes"] in case["gate"]
    n_cmp, worst = compare_parity_set(case["gpu"], case["ora"], case["f_true"], w["orders"],
                                      w["modes"], min_matches=w["modes"],
                                      phi_true=case["phi_true"], gate_orders=case["gate"])
    assert n_cmp >= w["modes"]


def test_modes_identified_at_every_order(case):
    """Identification quality, a property of the record: at the separated orders every
    generating mode is found (within 1 % in frequency, MAC >= 0.99 with its generating
    shape); at every order from 2 m on at least m - 1 modes are, each with MAC >= 0.85.
    The FP64 oracle itself, on the same record and Omega, reaches worst MACs of 0.90 and
    misses one mode at one order, so these bounds are the record's, not the GPU's."""
    w = case["w"]
    for m_i, n in enumerate(w["orders"]):
        if n < 2 * w["modes"]:
            continue
        cell = case["gpu"][0][m_i]
        found, worst = 0, 1.0
        for r, f0 in enumerate(case["f_true"]):
            phi0 = case["phi_true"][:, r]
            j = nearest(cell, f0, phi0)
            if j is None or abs(cell["f"][j] - f0) / f0 >= 1e-2:
                continue
            found += 1
            worst = min(worst, O.mac(cell["Phi"][:, j], phi0))
        if n in case["gate"]:
            assert found == w["modes"] and worst >= 0.99, (n, found, worst)
        else:
            assert found >= w["modes"] - 1 and worst >= 0.85, (n, found, worst)
