"""The unit-by-unit oracle solve that the benchmark times on the host cores
(oracle/reference_solve.py) computes exactly the oracle's one-call solve: run in order,
its units (covariances, each lag's Toeplitz RSVD, each realisation, stability) leave the
same diagram, bit for bit, as oracle.ssi_solve on the same record, Omega seed and
settings, for one lag and for several.  The saved file holds that diagram."""
import numpy as np
import pytest

import oracle as O
import ssi_synth as S
from oracle import reference_solve as RS


def _case(lags):
    w = S.workload("chain4_tiny", N=6000, lags=lags, k=24, oversample=8, q=1,
                   orders=list(range(2, 25, 2)))
    Y, *_ = S.record(w, np.float32)
    return w, Y.astype(np.float64)


@pytest.mark.parametrize("lags", [[12], [8, 12]])
def test_units_reproduce_the_one_call_solve(lags):
    w, Y = _case(lags)
    state, units = RS.solve_units(Y, w, seed=3)
    names = [n for n, _ in units]
    assert names.count("covariances") == 1 and names.count("stability") == 1
    assert names.count("toeplitz_rsvd") == len(lags)
    assert names.count("realisation") == len(lags) * len(w["orders"])
    assert names[0] == "covariances" and names[-1] == "stability"
    for _, fn in units:
        fn()
    ref, svals = O.ssi_solve(Y, w["fs"], lags, w["orders"], k=w["k"], oversample=w["oversample"],
                             q=w["q"], seed=3, stab=dict(use_lag_axis=len(lags) > 1))
    for t in range(len(lags)):
        assert np.array_equal(state["s"][t], svals[t])
        for m, n in enumerate(w["orders"]):
            a, b = state["diagram"][t][m], ref[t][m]
            for key in ("mu", "f", "xi", "Phi", "flags", "mpc", "mpd"):
                assert np.array_equal(a[key], b[key]), (t, n, key)


def test_saved_file_holds_the_diagram(tmp_path):
    w, Y = _case([12])
    state, stage_s = RS.run(Y, w, seed=3)
    path = tmp_path / "oracle.npz"
    RS.save(str(path), w, 3, state, stage_s, cores=1)
    z = np.load(path)
    cells = state["diagram"][0]
    assert list(z["counts"]) == [len(c["f"]) for c in cells]
    assert np.array_equal(z["f"], np.concatenate([c["f"] for c in cells]))
    assert np.array_equal(z["flags"], np.concatenate([c["flags"] for c in cells]))
    assert z["phi"].shape == (sum(len(c["f"]) for c in cells), Y.shape[0])
    assert np.array_equal(z["s"][0], state["s"][0])
    assert set(z["stage_names"]) == {"covariances", "toeplitz_rsvd", "realisation", "stability"}
