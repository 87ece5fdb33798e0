"""Serving: continuous batching gives each job the result it gets alone.

A stream of uneven bridge records (16/48/96 channels, N 30000-60000, i 20-40, 5-10
modes, orders up to 2m+40) is solved job by job through ssi_solve with the record on
the device, then submitted all at once to the serving loop with the record in host
memory.  With three slots the jobs overlap on the device and later jobs wait for a
slot; with an HBM budget that holds about one job, admission serialises them.  Every
job's poles must agree with its solo solve within the parity gates (frequency <= 1e-4
relative, damping <= 2e-3 absolute, MAC >= 0.999) and carry the same flags.
"""
import numpy as np
import pytest
import torch

import oracle as O
import ssi_synth as S
from parity import F_TOL, MAC_MIN, XI_TOL

pytestmark = pytest.mark.gpu

MIX = dict(channels=(16, 48, 96), N_range=(30000, 60000), i_range=(20, 40), modes_range=(5, 10))


@pytest.fixture(scope="module")
def P():
    import paper_2411_05510_gb300 as P
    return P


@pytest.fixture(scope="module")
def jobs():
    out = []
    for w in S.serving_mix(6, seed=4, **MIX):
        Y, f_true, *_ = S.record(w, np.float32)
        out.append((w, Y, f_true))
    return out


def _desc(P, w, Y):
    return P.job_desc(Y, w["fs"], w["lags"], w["orders"], k=w["k"], oversample=w["oversample"],
                      q=w["q"], prec="split_bf16", seed=7)


@pytest.fixture(scope="module")
def solo(P, jobs):
    ctx = P.Context(0)
    res = []
    for w, Y, _ in jobs:
        poles, phi, _ = P.ssi_solve(ctx, _desc(P, w, torch.from_numpy(Y).cuda()))
        P.check_sync(ctx)
        res.append((P.poles_to_numpy(poles), phi.cpu().numpy().reshape(-1, w["l"], 2)))
    peak = ctx.memory_in_use()
    ctx.close()
    return res, peak


def _same(a, b, l):
    rec_a, phi_a = a
    rec_b, phi_b = b
    assert len(rec_a) == len(rec_b)
    assert np.array_equal(rec_a["flags"], rec_b["flags"])
    v = (rec_a["flags"] & 64) != 0
    assert v.sum() > 0
    fa, fb = rec_a["f_hz"][v].astype(np.float64), rec_b["f_hz"][v].astype(np.float64)
    assert np.max(np.abs(fa - fb) / fa) <= F_TOL
    assert np.max(np.abs(rec_a["xi"][v].astype(np.float64) - rec_b["xi"][v])) <= XI_TOL
    pa = phi_a[v, :, 0] + 1j * phi_a[v, :, 1]
    pb = phi_b[v, :, 0] + 1j * phi_b[v, :, 1]
    macs = [O.mac(pa[j], pb[j]) for j in range(len(pa))]
    assert min(macs) >= MAC_MIN


def _serve(P, ctx, jobs, slots):
    P.ssi_serve_config(ctx, slots, 64)
    ids = [P.ssi_submit(ctx, _desc(P, w, Y)) for w, Y, _ in jobs]
    out = []
    for jid in ids:
        rec, phi, lat = P.ssi_poll(ctx, jid, 120000)
        out.append((rec, phi))
        P.ssi_release(ctx, jid)
    return out


def test_solo_solves_find_the_modes(jobs, solo):
    res, _ = solo
    for (w, _, f_true), (rec, _) in zip(jobs, res):
        top = rec[-(w["orders"][-1] // 2):]
        hc = top[(top["flags"] & 8) != 0]
        found = sum(np.min(np.abs(hc["f_hz"] - f0) / f0) < 1e-2 for f0 in f_true)
        assert found >= len(f_true) - 1, (w["l"], w["N"], w["lags"], found, len(f_true))


def test_mix_matches_solo_with_overlap(P, jobs, solo):
    ctx = P.Context(0)
    try:
        mixed = _serve(P, ctx, jobs, slots=3)
    finally:
        ctx.close()
    for (w, _, _), a, b in zip(jobs, solo[0], mixed):
        _same(a, b, w["l"])


def test_mix_matches_solo_under_a_tight_budget(P, jobs, solo):
    """Budget for about one job at a time: admission waits for memory, results unchanged."""
    ctx = P.Context(0, int(solo[1] * 1.3) + (64 << 20))
    try:
        mixed = _serve(P, ctx, jobs, slots=3)
        assert ctx.memory_in_use() <= int(solo[1] * 1.3) + (64 << 20)
    finally:
        ctx.close()
    for (w, _, _), a, b in zip(jobs, solo[0], mixed):
        _same(a, b, w["l"])


def test_job_larger_than_budget_fails_cleanly(P, jobs):
    ctx = P.Context(0, 8 << 20)
    try:
        P.ssi_serve_config(ctx, 1, 4)
        w, Y, _ = jobs[0]
        jid = P.ssi_submit(ctx, _desc(P, w, Y))
        with pytest.raises(P.SsiError) as e:
            P.ssi_poll(ctx, jid, 60000)
        assert e.value.status == 2   # SSI_E_NOMEM
        P.ssi_release(ctx, jid)
    finally:
        ctx.close()


def test_concurrency_hint_leaves_results_bit_identical(P, jobs):
    """ssi_set_concurrency changes the QR grid (every SM, or half of them with two row
    chunks per CTA); the reductions run over the same chunks in the same order, so the
    poles and mode shapes must be the same bit for bit."""
    w, Y, _ = max(jobs, key=lambda j: j[0]["l"] * j[0]["N"])
    out = []
    for n in (1, 3):
        ctx = P.Context(0)
        try:
            ctx.set_concurrency(n)
            poles, phi, S = P.ssi_solve(ctx, _desc(P, w, torch.from_numpy(Y).cuda()))
            P.check_sync(ctx)
            out.append((poles.cpu().numpy().tobytes(), phi.cpu().numpy().tobytes(),
                        S.cpu().numpy().tobytes()))
        finally:
            ctx.close()
    assert out[0][2] == out[1][2]
    assert out[0][0] == out[1][0]
    assert out[0][1] == out[1][1]


def test_concurrency_hint_rejects_bad_values(P):
    ctx = P.Context(0)
    try:
        with pytest.raises(P.SsiError):
            ctx.set_concurrency(0)
    finally:
        ctx.close()
