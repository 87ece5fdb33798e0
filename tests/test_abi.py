"""The C-ABI library loads on any machine and exports every function include/ssi.h declares;
the host-only parameter rules reproduce the worked values of the paper (no GPU needed)."""
import os
import re

import pytest

from conftest import ROOT, golden_rows


def _declared():
    with open(os.path.join(ROOT, "include", "ssi.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ssi_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_function():
    import paper_2411_05510_gb300._lib as L
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L.lib, n)]
    assert not missing, missing
    assert not L.MISSING
    assert set(names) == set(L.PROTOTYPES), set(names) ^ set(L.PROTOTYPES)


def test_host_rules_match_paper_worked_values():
    import paper_2411_05510_gb300 as P
    for row in golden_rows("parameter_rules.txt"):
        if row[0] == "rank":
            kbar, k = P.ssi_rank_rule(int(row[1]))
            assert kbar == pytest.approx(float(row[2]), abs=1e-9)
            assert k == int(row[3])
        elif row[0] == "lag":
            assert P.ssi_lag_rule(float(row[1]), float(row[2])) == tuple(int(x) for x in row[3:6])
        elif row[0] == "tau":
            assert P.ssi_time_lag(int(row[1]), float(row[2])) == pytest.approx(float(row[3]), abs=1e-12)


def test_pole_slot_layout():
    import paper_2411_05510_gb300 as P
    assert P.ssi_pole_slots([2, 4, 6]) == 6
    assert P.ssi_pole_slots(list(range(2, 201, 2))) == 5050
    assert P._lib.POLE_BYTES == 40


def test_invalid_arguments_fail_before_any_device_work():
    import paper_2411_05510_gb300 as P
    with pytest.raises(P._lib.SsiError):
        P.ssi_rank_rule(0)
    with pytest.raises(P._lib.SsiError):
        P.ssi_lag_rule(100.0, -1.0)


def test_cluster_abi_layout_and_argument_checks():
    import ctypes

    import paper_2411_05510_gb300 as P
    L = P._lib
    assert ctypes.sizeof(L.SsiClusterParams) == 32
    assert ctypes.sizeof(L.SsiMode) == 24
    assert ctypes.sizeof(L.SsiClusterInfo) == 32 + 80
    orders = (ctypes.c_int * 2)(2, 4)
    n_modes = ctypes.c_int(-1)
    params = P.cluster_params()
    # a null context, poles or phi is refused before any device work
    st = L.lib.ssi_cluster(None, 1, 2, orders, 4, None, None, ctypes.byref(params), None, 0,
                           ctypes.byref(n_modes), None, None, None, None, None)
    assert st == 1


def test_cov_stream_argument_checks_without_a_device():
    import ctypes

    import paper_2411_05510_gb300 as P
    L = P._lib
    out = ctypes.c_void_p(1)
    # a null context is refused before any device work, and the handle is cleared
    assert L.lib.ssi_cov_stream_create(None, 4, 3, 100, 10, 1, ctypes.byref(out)) == 1
    assert not out.value
    assert L.lib.ssi_cov_stream_push(None, None, 10, None) == 1
    n = ctypes.c_int64()
    assert L.lib.ssi_cov_stream_covariances(None, None, ctypes.byref(n), None) == 1
    assert L.lib.ssi_cov_stream_destroy(None) == 0
