"""Host logic of the rank calibration (Sec. 3.1): the grid, the selection of the modes of
interest and the match decision on hand-built mode tables (no GPU)."""
import numpy as np

from paper_2411_05510_gb300 import rank_study as RS


def _modes(fs, xis, phis):
    return [dict(f_hz=f, xi=x, size=20, phi=p) for f, x, p in zip(fs, xis, phis)]


def _shapes(n, l=10, seed=0):
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(l) + 1j * rng.standard_normal(l) for _ in range(n)]


def test_rank_grid():
    assert RS.rank_grid(2.5, 10.0, 2.5) == [2.5, 5.0, 7.5, 10.0]
    assert len(RS.rank_grid()) == 20


def test_match_follows_each_tolerance():
    ph = _shapes(3)
    ref = _modes([1.0, 2.0, 3.0], [0.01, 0.02, 0.03], ph)
    names = np.array([1.0, 2.0, 3.0])
    tol = (0.01, 0.01, 0.02)
    # inside every tolerance
    ok = _modes([1.005, 2.0, 3.0], [0.01005, 0.02, 0.03], ph)
    assert RS.modes_match(ref, ok, tol, names)
    # frequency 1.5 % off on one mode
    bad_f = _modes([1.0, 2.03, 3.0], [0.01, 0.02, 0.03], ph)
    assert not RS.modes_match(ref, bad_f, tol, names)
    # damping 3 % off (relative to the larger value)
    bad_x = _modes([1.0, 2.0, 3.0], [0.01, 0.02, 0.0309], ph)
    assert not RS.modes_match(ref, bad_x, tol, names)
    assert RS.modes_match(ref, bad_x, (0.01, None, 0.02), names)   # damping not compared
    # a different shape
    other = _shapes(3, seed=7)
    bad_s = _modes([1.0, 2.0, 3.0], [0.01, 0.02, 0.03], [ph[0], other[1], ph[2]])
    assert not RS.modes_match(ref, bad_s, tol, names)
    # a missing mode
    assert not RS.modes_match(ref, ok[:2], tol, names)


def test_modes_of_interest_and_extra_clusters():
    ph = _shapes(4)
    # the reference has an extra (noise) cluster at 5 Hz that no name points to
    ref = _modes([1.0, 2.0, 3.0, 5.0], [0.01] * 4, ph)
    names = [1.01, 2.0, 2.98]
    moi = RS.modes_of_interest(ref, names)
    assert [m["f_hz"] for m in moi] == [1.0, 2.0, 3.0]
    cand = _modes([1.0, 2.0, 3.0], [0.01] * 3, ph[:3])
    assert RS.modes_match(ref, cand, (0.01, 0.01, 0.02), names)
    # without names every reference mode counts, and the counts must agree
    assert not RS.modes_match(ref, cand, (0.01, 0.01, 0.02), None)
    # a name more than 5 % from every mode selects nothing
    assert RS.modes_of_interest(ref, [10.0]) == []


def test_damping_differences_report_matched_modes():
    ph = _shapes(2)
    ref = _modes([1.0, 2.0], [0.010, 0.020], ph)
    cand = _modes([1.0, 2.0], [0.011, 0.020], ph)
    d = RS.damping_differences(ref, cand, np.array([1.0, 2.0]))
    assert np.allclose(d, [0.001 / 0.011, 0.0])


def test_minimum_rank_search_bookkeeping(monkeypatch):
    """The search over the grid with a stand-in identification: K = ceil(pct T / 100)
    (at least the largest order), the first matching percentage is returned, the reference
    is identified at K = T, and the trace records each step."""
    ph = _shapes(2)
    ref = _modes([1.0, 2.0], [0.01, 0.02], ph)
    calls = []

    def fake_identify(ctx, Y, fs, jb, orders, K, **kw):
        calls.append(K)
        if K >= 10 * jb:                 # the reference (full width)
            return ref
        xi = 0.0201 if K >= 300 else 0.03   # damping within 1 % from K = 300 on
        return _modes([1.0, 2.0], [0.01, xi], ph)

    monkeypatch.setattr(RS, "identify", fake_identify)

    class _Y:
        shape = (10, 1000)

    kbar, r, trace = RS.minimum_rank(None, _Y(), 200.0, 100, list(range(10, 101, 2)),
                                     RS.rank_grid(2.5, 50.0, 2.5), f_names=[1.0, 2.0])
    assert r is ref and calls[0] == 1000
    assert kbar == 30.0                          # ceil(30 % of 1000) = 300
    assert [t[1] for t in trace] == [100, 100, 100, 100, 125, 150, 175, 200, 225, 250, 275, 300]
    assert [t[2] for t in trace] == [False] * 11 + [True]
    # an identification that matches only at full width: K reaching T stops the search
    # there (the reference matches itself), before the grid's end
    monkeypatch.setattr(RS, "identify", lambda ctx, Y, fs, jb, orders, K, **kw:
                        ref if K >= 10 * jb else _modes([1.0, 2.0], [0.01, 0.03], ph))
    kbar, _, trace = RS.minimum_rank(None, _Y(), 200.0, 100, [10, 20], [50.0, 100.0, 150.0],
                                     f_names=[1.0, 2.0])
    assert kbar == 100.0 and len(trace) == 2
    assert trace[-1][1] == 1000 and trace[-1][2]
