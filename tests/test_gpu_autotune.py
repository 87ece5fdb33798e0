"""The autotuner of a job shape's plan choices (lag-GEMM time split, Toeplitz GEMM splits,
Jacobi block width, QR chunks per CTA): ssi_autotune stores its choices in the context, ssi_tuning_get and
ssi_tuning_set read and copy them, and a solve planned with the tuned choices still meets
the parity gates against the oracle (leading singular values 1e-4, and the same poles as
the untuned solve at the separated orders within the parity tolerances)."""
import numpy as np
import pytest
import torch

import oracle as O
import ssi_synth as S
from parity import compare_parity_set, gpu_cells, separated_orders

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("small", ["fp32", "fp64"])
def test_autotune_choices_are_stored_and_keep_parity(small):
    import paper_2411_05510_gb300 as P
    w = S.workload("bridge186_3d", l=24, modes=6, f_lo=4.0, N=60000, lags=[14], k=32,
                   oversample=16, orders=list(range(2, 33, 2)))
    Y, f_true, _, phi_true = S.record(w, np.float32)
    Yd = torch.from_numpy(Y).cuda()
    ctx, ctx2 = P.Context(0), P.Context(0)
    desc = P.job_desc(Yd, w["fs"], w["lags"], w["orders"], k=w["k"], oversample=w["oversample"],
                      q=w["q"], prec="split_bf16", seed=5, small=small)
    with pytest.raises(P.SsiError):
        P.ssi_tuning_get(ctx, desc)
    poles0, phi0, S0 = P.ssi_solve(ctx, desc)
    t = P.ssi_autotune(ctx, desc)
    assert t["cov_rows_per_split"] >= 512 and t["sketch_splits"] >= 1 and t["jacobi_block"] >= 1, t
    assert t["qr_chunks_per_cta"] == 1, t   # one solve at a time: the whole-device QR grid
    assert all(x > 0 for x in t["stage_ms"]), t
    keys = ("cov_rows_per_split", "sketch_splits", "jacobi_block", "qr_chunks_per_cta")
    g = P.ssi_tuning_get(ctx, desc)
    assert [g[k] for k in keys] == [t[k] for k in keys]
    P.ssi_tuning_set(ctx2, desc, t)
    assert P.ssi_tuning_get(ctx2, desc)["jacobi_block"] == t["jacobi_block"]
    poles1, phi1, S1 = P.ssi_solve(ctx2, desc)
    P.check_sync(ctx)
    P.check_sync(ctx2)
    ora, sv = O.ssi_solve(Y.astype(np.float64), w["fs"], w["lags"], w["orders"], k=w["k"],
                          oversample=w["oversample"], q=w["q"], seed=5)
    s1 = S1.cpu().numpy()[0]
    assert np.allclose(s1[:12], sv[0][:12], rtol=1e-4), np.abs(s1[:12] / sv[0][:12] - 1).max()
    gate = separated_orders(w["orders"], sv[0])
    for poles, phi in ((poles0, phi0), (poles1, phi1)):
        gpu = gpu_cells(P.poles_to_numpy(poles), phi.cpu().numpy(), w["lags"], w["orders"], w["l"])
        compare_parity_set(gpu, ora, f_true, w["orders"], 6, min_matches=6, phi_true=phi_true,
                           gate_orders=gate)
    ctx.close()
    ctx2.close()
