"""bfc_exact_csr_noalloc: the exact count for callers that cannot allocate
device memory (under a fixed memory budget, on a path that must not wait on
the allocator).  Its only working memory is a
scratch array inside the library.  Checked against bfc_exact on the same
edges, on two calls in a row, so that the shared scratch array is seen to be
reset between calls.

This file is collected last on purpose: it must pass both on its own in a
fresh process and after every other test has run.
"""
import numpy as np
import pytest

from paper_1801_00338_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bfc():
    import torch
    assert torch.cuda.is_available()
    from paper_1801_00338_gb300 import build as B
    B.build()
    from paper_1801_00338_gb300 import bfc as mod
    mod.load()
    return mod


def _device_csr(rows, cols, n):
    """Row offsets (uint64 bits in int64) and neighbours (int32) on the device."""
    import torch
    order = np.lexsort((cols, rows))
    counts = np.bincount(rows, minlength=n).astype(np.int64)
    off = np.zeros(n + 1, np.int64)
    np.cumsum(counts, out=off[1:])
    nbr = cols[order].astype(np.int32)
    return torch.from_numpy(off).cuda(), torch.from_numpy(nbr if nbr.size else np.zeros(1, np.int32)).cuda()


@pytest.mark.parametrize("make", [
    lambda: synth.uniform_small(1),
    lambda: synth.chung_lu_scaled(3000, 9000, 40_000, 2.1, 2.4, 5),
    lambda: synth.Graph(*synth.complete_bipartite(40, 7), 40, 7),
])
def test_noalloc_matches_bfc_exact_twice(bfc, make):
    import torch
    g = make()
    offU, nbrU = _device_csr(g.u, g.v, g.nU)
    offV, nbrV = _device_csr(g.v, g.u, g.nV)
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        for side, flags in ((None, 0), ("U", bfc.BFC_SIDE_U), ("V", bfc.BFC_SIDE_V)):
            want, _ = G.exact(side)
            for _ in range(2):
                out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
                rc = bfc.bfc_exact_csr_noalloc(offU, nbrU, g.nU, offV, nbrV, g.nV, out, flags)
                assert rc == 0, bfc.strerror(rc)
                torch.cuda.synchronize()
                assert int(out.item()) == want


def test_noalloc_rejects_sizes_beyond_the_scratch(bfc):
    import torch
    z = torch.zeros(2, dtype=torch.int64, device="cuda")
    too_big = bfc.load().bfc_exact_csr_noalloc(z.data_ptr(), z.data_ptr(), 1 << 31, z.data_ptr(), z.data_ptr(), 3, 0,
                                               z.data_ptr(), None)
    assert too_big == -2  # BFC_ERANGE, before any pointer is touched
    assert bfc.bfc_exact_csr_noalloc(z, z, 3, z, z, 3, z, flags=0x30) == -1  # both sides forced: BFC_EINVAL


def test_noalloc_makes_no_library_allocation(bfc):
    """With the library's next device allocation set to fail, the call still
    succeeds (it never asks the library's allocator for memory) and gives
    bfc_exact's count."""
    import torch
    g = synth.chung_lu_scaled(3000, 9000, 40_000, 2.1, 2.4, 5)
    offU, nbrU = _device_csr(g.u, g.v, g.nU)
    offV, nbrV = _device_csr(g.v, g.u, g.nV)
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        want, _ = G.exact()
    out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    try:
        bfc.bfc_fail_alloc_after(0)
        rc = bfc.bfc_exact_csr_noalloc(offU, nbrU, g.nU, offV, nbrV, g.nV, out, 0)
    finally:
        bfc.bfc_fail_alloc_after(-1)
    assert rc == 0, bfc.strerror(rc)
    torch.cuda.synchronize()
    assert int(out.item()) == want
