"""Several jobs in one call (ssi_solve_batch): the eigen-decompositions of every job's
(lag, order) realisations run in one k_eig launch (plus one for orders above 224) and one
k_eig_vectors launch.  Each job's poles, mode shapes and singular values must be
bit-identical to its own ssi_solve: the same kernels compute every item in the same
arithmetic, only the launches are shared.  The jobs differ in channels, record length,
lags, k, orders (one of them above the shared-memory limit of 224) and GEMM precision."""
import numpy as np
import pytest
import torch

import ssi_synth as S

pytestmark = pytest.mark.gpu


def _jobs(P):
    specs = [
        # (workload overrides, k, oversample, orders, prec)
        (dict(l=24, modes=6, f_lo=4.0, N=60000, lags=[14]), 32, 16, list(range(2, 33, 2)), "split_bf16"),
        (dict(l=48, modes=8, f_lo=2.0, N=80000, lags=[16, 20]), 40, 8, list(range(2, 41, 2)), "split_bf16"),
        (dict(l=24, modes=10, f_lo=2.0, N=90000, lags=[14]), 240, 16, list(range(2, 241, 2)), "split_bf16"),
        (dict(l=32, modes=5, f_lo=3.0, N=50000, lags=[12]), 30, 10, list(range(2, 31, 2)), "fp32"),
    ]
    out = []
    for ov, k, p, orders, prec in specs:
        w = S.workload("bridge186_3d", **ov)
        Y, *_ = S.record(w, np.float32)
        Yd = torch.from_numpy(Y).cuda()
        d = P.job_desc(Yd, w["fs"], w["lags"], orders, k=k, oversample=p, q=2, prec=prec, seed=7)
        out.append((Yd, d))
    return out


def test_batch_equals_separate_solves():
    import paper_2411_05510_gb300 as P
    ctx = P.Context(0)
    jobs = _jobs(P)
    descs = [d for _, d in jobs]
    ref = [P.ssi_solve(ctx, d) for d in descs]
    P.check_sync(ctx)
    for rep in range(2):   # twice: the second call reuses the context's batch buffers
        got = P.ssi_solve_batch(ctx, descs)
        P.check_sync(ctx)
        for j, ((p0, f0, s0), (p1, f1, s1)) in enumerate(zip(ref, got)):
            assert torch.equal(p0, p1), f"job {j}: pole records differ"
            assert torch.equal(f0, f1), f"job {j}: mode shapes differ"
            assert torch.equal(s0, s1), f"job {j}: singular values differ"
    # the batch found the poles at all: every job has poles that pass the hard criteria
    for j, (p1, _, _) in enumerate(got):
        rec = P.poles_to_numpy(p1)
        assert np.count_nonzero(rec["flags"] & 8) > 0, j
    ctx.close()


def test_batch_rejects_fp64_small_problems():
    import paper_2411_05510_gb300 as P
    ctx = P.Context(0)
    w = S.workload("bridge186_3d", l=16, modes=4, f_lo=4.0, N=30000, lags=[10])
    Y, *_ = S.record(w, np.float32)
    Yd = torch.from_numpy(Y).cuda()
    d32 = P.job_desc(Yd, w["fs"], w["lags"], list(range(2, 17, 2)), k=16, oversample=8, q=1,
                     prec="split_bf16", seed=3)
    d64 = P.job_desc(Yd, w["fs"], w["lags"], list(range(2, 17, 2)), k=16, oversample=8, q=1,
                     prec="split_bf16", seed=3, small="fp64")
    with pytest.raises(P.SsiError):
        P.ssi_solve_batch(ctx, [d32, d64])
    # a batch of one is a solve
    (p1, f1, s1), = P.ssi_solve_batch(ctx, [d32])
    p0, f0, s0 = P.ssi_solve(ctx, d32)
    P.check_sync(ctx)
    assert torch.equal(p0, p1) and torch.equal(f0, f1) and torch.equal(s0, s1)
    ctx.close()
