"""A small case of the benchmark's counting kernels, for profilers.

    python -m paper_1801_00338_gb300.profile_case [--scale S]

The benchmark graph shrunk by S (default 4): a seeded Chung-Lu bipartite graph
with |U| = 10^6 / S, |V| = 5 x 10^6 / S, 5 x 10^7 / S distinct edges and the
same exponents (2.1 on U, 2.5 on V).  It builds the graph, runs
bfc_exact(BFC_HUB_MMA) and bfc_local_counts once as a warm-up and once more,
and prints B.  At S = 4 the device holds a few hundred MB, and each window
kernel launch takes a few milliseconds, so a profiler capture of one launch
ends quickly.
"""
from __future__ import annotations

import argparse
import ctypes

import numpy as np

from . import bfc, synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=4)
    args = ap.parse_args()
    import torch
    S = args.scale
    g = synth.chung_lu_scaled(1_000_000 // S, 5_000_000 // S, 50_000_000 // S, 2.1, 2.5, 2)
    du = torch.from_numpy(g.u.astype(np.int32)).cuda()
    dv = torch.from_numpy(g.v.astype(np.int32)).cuda()
    bU = torch.empty(g.nU, dtype=torch.int64, device="cuda")
    bV = torch.empty(g.nV, dtype=torch.int64, device="cuda")
    be = torch.empty(g.m, dtype=torch.int64, device="cuda")
    L = bfc.load()
    sp = torch.cuda.current_stream().cuda_stream
    B, B2, side = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()
    for _ in range(2):
        h = bfc.bfc_graph_from_edges(du, dv, g.nU, g.nV, 0, sp)
        try:
            bfc._check(L.bfc_exact(h, bfc.BFC_HUB_MMA, ctypes.byref(B), ctypes.byref(side), sp), "bfc_exact")
            bfc._check(L.bfc_local_counts(h, 0, bU.data_ptr(), bV.data_ptr(), be.data_ptr(), ctypes.byref(B2), sp),
                       "bfc_local_counts")
        finally:
            bfc.bfc_graph_free(h)
    torch.cuda.synchronize()
    assert B.value == B2.value
    print(f"profile case 1/{S}: |U|={g.nU} |V|={g.nV} m={g.m} B={B.value}")


if __name__ == "__main__":
    main()
