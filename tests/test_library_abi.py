"""The C-ABI library builds, loads and exports every symbol the header declares (CPU only)."""
import os
import re

import pytest

from paper_2410_01657_gb300 import _build
from paper_2410_01657_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return B.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(gnn_[a-z0-9_]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert "gnn_mp_forward" in declared and "gnn_halo_exchange" in declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared <= set(B.exported_symbols()) | {"gnn_graph_destroy", "gnn_partition_destroy"}


def test_version_and_error_reporting(lib):
    assert B.load().gnn_version() >= 10000
    with pytest.raises(B.GnnError) as ei:
        from paper_2410_01657_gb300.graph import MeshGraph
        MeshGraph((0, 1, 1), 1)
    assert ei.value.code == B.GNN_EINVAL
    assert "nel" in B.last_error()


def test_compute_entry_points_reject_bad_arguments(lib):
    import ctypes as C
    cfg = B.gnn_mp_config()
    cfg.hidden, cfg.precision, cfg.ln_eps = 64, 7, 1e-5
    G = B.gnn_graph_dev()
    W = B.gnn_mp_params()
    rc = lib.gnn_mp_forward(C.byref(G), C.byref(cfg), C.byref(W), None, None, None, None, None, None, 0, None)
    assert rc == B.GNN_EDTYPE
    cfg.precision = B.GNN_PREC_BF16
    cfg.hidden = 48
    rc = lib.gnn_mp_forward(C.byref(G), C.byref(cfg), C.byref(W), None, None, None, None, None, None, 0, None)
    assert rc == B.GNN_ESHAPE
    assert lib.gnn_mp_forward(None, C.byref(cfg), C.byref(W), None, None, None, None, None, None, 0, None) \
        == B.GNN_EINVAL
