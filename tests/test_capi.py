"""The C-ABI library loads and exports every symbol include/bfc.h declares (no GPU work)."""
import ctypes

import pytest

from paper_1801_00338_gb300 import bfc
from paper_1801_00338_gb300 import build as B


@pytest.fixture(scope="module")
def lib():
    B.build()
    return bfc.load()


def test_header_declares_the_boundary():
    syms = bfc.header_symbols()
    for name in ("bfc_graph_from_edges", "bfc_graph_free", "bfc_exact", "bfc_per_vertex", "bfc_per_edge",
                 "bfc_espar", "bfc_clrspar", "bfc_vsamp", "bfc_proposal_from_weights", "bfc_strerror"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(bfc.LIB_PATH)
    for name in bfc.header_symbols():
        assert hasattr(raw, name), name


def test_strerror_and_argument_checks_without_gpu(lib):
    assert bfc.strerror(0) == "ok"
    assert "duplicate" in bfc.strerror(-3)
    # null handles are rejected before any device work
    assert lib.bfc_exact(None, 0, None, None, None) == -1
    assert lib.bfc_graph_free(None) == -1
    out = ctypes.c_void_p()
    assert lib.bfc_graph_from_edges(None, None, 5, 3, 3, 0, None, ctypes.byref(out)) == -1   # m > 0, null arrays
    assert lib.bfc_graph_from_edges(None, None, 0, 0, 3, 0, None, ctypes.byref(out)) == -1   # nU == 0
    assert lib.bfc_graph_from_edges(None, None, 1 << 32, 3, 3, 0, None, ctypes.byref(out)) in (-1, -2)
