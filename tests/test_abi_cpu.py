"""The C ABI library builds, loads and exports every entry point of include/qw.h,
and rejects bad arguments before touching the GPU (runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def qwlib():
    from paper_1003_3779_gb300 import _build
    _build.build()
    import paper_1003_3779_gb300.qw as qw
    return qw


def header_functions():
    src = open(os.path.join(ROOT, "include", "qw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qw_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = header_functions()
    for must in ["qw_create", "qw_set_coin", "qw_set_state", "qw_step", "qw_probabilities",
                 "qw_batch_step", "qw_backward", "qw_destroy", "qw_status_string"]:
        assert must in names


def test_library_exports_every_declared_symbol(qwlib):
    out = subprocess.run(["nm", "-D", "--defined-only", qwlib.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (qw_[a-z0-9_]+)", out))
    missing = [n for n in header_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    # the binding knows every declared call too
    L = qwlib.lib()
    for n in header_functions():
        assert getattr(L, n).argtypes is not None or n in ("qw_version",)


def test_version_and_status_strings(qwlib):
    assert "sm_103a" in qwlib.qw_version()
    L = qwlib.lib()
    assert L.qw_status_string(0) == b"ok"
    assert L.qw_status_string(qwlib.QW_ETIMEOUT) == b"device wait timed out"


@pytest.mark.parametrize("args", [
    dict(ndim=3, dims=[4, 4, 4], coin_dim=6),
    dict(ndim=1, dims=[0], coin_dim=2),
    dict(ndim=1, dims=[16], coin_dim=4),
    dict(ndim=2, dims=[4, -1], coin_dim=4),
    dict(ndim=1, dims=[16], coin_dim=2, bc=7),
    dict(ndim=1, dims=[16], coin_dim=2, prec=9),
    dict(ndim=2, dims=[1 << 21, 1 << 21], coin_dim=4),
])
def test_create_rejects_bad_arguments_without_a_gpu(qwlib, args):
    L = qwlib.lib()
    h = ctypes.c_void_p(123)
    dims = np.array(args["dims"], dtype=np.int64)
    st = L.qw_create(args["ndim"], dims.ctypes.data_as(ctypes.c_void_p), args["coin_dim"],
                     args.get("bc", 0), args.get("shift", 0), args.get("prec", 1), None,
                     ctypes.byref(h))
    assert st == qwlib.QW_EINVAL
    assert h.value is None


def test_null_handles_are_rejected(qwlib):
    L = qwlib.lib()
    assert L.qw_step(None, 5) == qwlib.QW_EINVAL
    assert L.qw_set_coin(None, None, 0, 0) == qwlib.QW_EINVAL
    assert L.qw_probabilities(None, None, 0, 0, None) == qwlib.QW_EINVAL
    assert L.qw_destroy(None) == qwlib.QW_OK
    assert L.qw_create(1, None, 2, 0, 0, 1, None, None) == qwlib.QW_EINVAL
    assert L.qw_last_error(None) == b"null handle"


def test_graph_arcs_match_the_oracle_bitwise(qwlib):
    """qw_graph_arcs (host code of the library) and the oracle's own arc builder
    give the same arc form: integer work, compared exactly."""
    import oracle
    from paper_1003_3779_gb300 import inputs
    for nvert, edges in [(3, [(0, 1), (1, 1), (2, 0)]),
                         (7, [(i, (i * 3 + 1) % 7) for i in range(7)] + [(2, 2), (5, 6), (5, 6)]),
                         (2000, inputs.chung_lu_edges(2000, 5, 2.3, seed=9)),
                         (4, np.zeros((0, 2), dtype=np.int64))]:
        off, partner = qwlib.graph_arcs(nvert, edges)
        off_o, partner_o = oracle.graph_arcs(nvert, edges)
        assert np.array_equal(off, off_o) and np.array_equal(partner, partner_o)
    with pytest.raises(qwlib.QWError):
        qwlib.graph_arcs(3, [(0, 3)])


def test_graph_walk_create_rejects_bad_graphs_without_a_gpu(qwlib):
    L = qwlib.lib()

    def create(off, partner, prec=1):
        off = np.asarray(off, dtype=np.int64)
        partner = np.asarray(partner, dtype=np.int64)
        h = ctypes.c_void_p(123)
        st = L.qw_gwalk_create(len(off) - 1, off.ctypes.data_as(ctypes.c_void_p),
                               partner.ctypes.data_as(ctypes.c_void_p), prec, None, ctypes.byref(h))
        return st, h.value

    assert create([0, 2, 4], [1, 2, 3, 0]) == (qwlib.QW_EINVAL, None)      # not an involution
    assert create([0, 2, 4], [1, 0, 3, 4]) == (qwlib.QW_EINVAL, None)      # out of range
    assert create([0, 3, 2], [1, 0]) == (qwlib.QW_EINVAL, None)            # off decreasing
    assert create([1, 3], [1, 0]) == (qwlib.QW_EINVAL, None)               # off[0] != 0
    assert create([0, 2], [1, 0], prec=2) == (qwlib.QW_EUNSUPPORTED, None)  # bf16 storage
    assert L.qw_gwalk_step(None, 1) == qwlib.QW_EINVAL
    assert L.qw_gwalk_destroy(None) == qwlib.QW_OK
    assert L.qw_gwalk_narcs(None) == -1
