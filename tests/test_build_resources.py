"""The hot kernels compile for sm_103a without register spills (ptxas resource
report, no GPU needed).  A spill in the window or hub kernels would put
local-memory traffic on the counting path."""
import os
import re
import shutil
import subprocess

import pytest

from paper_1801_00338_gb300 import build as B

NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"


def ptxas_report(src: str, tmp_path) -> dict:
    """{kernel symbol: (registers, spill store bytes, spill load bytes)} from ptxas -v."""
    out = os.path.join(str(tmp_path), os.path.basename(src) + ".o")
    cmd = [NVCC, *B.ARCH, "-O3", "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(B.ROOT, "include"),
           "-Xptxas", "-v", "-c", os.path.join(B.CSRC, src), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    rep, cur = {}, None
    spill = (0, 0)
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '([^']+)'", line)
        if m:
            cur = m.group(1)
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m and cur:
            spill = (int(m.group(1)), int(m.group(2)))
            continue
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            rep[cur] = (int(m.group(1)), *spill)
            cur, spill = None, (0, 0)
    return rep


@pytest.mark.skipif(not os.path.exists(NVCC), reason="needs nvcc")
def test_window_and_warp_kernels_do_not_spill(tmp_path):
    rep = ptxas_report("wedge.cu", tmp_path)
    hot = {k: v for k, v in rep.items() if re.search(r"k_cta_win|k_cta_big|k_warp_class", k)}
    assert len(hot) >= 40, sorted(rep)
    for k, (regs, st, ld) in hot.items():
        assert st == 0 and ld == 0, (k, regs, st, ld)
    # eleven 128-thread CTAs per SM for the ordered sweeps (modes 0, 1): at most
    # 46 registers a thread; nine for the whole-row ones (at most 56)
    small = [v[0] for k, v in hot.items() if re.search(r"k_cta_winILi[01]ELi\d+ELi4E", k)]
    assert small and max(small) <= 46
    full = [v[0] for k, v in hot.items() if re.search(r"k_cta_winILi[23]ELi\d+ELi4E", k)]
    assert full and max(full) <= 56


@pytest.mark.skipif(not os.path.exists(NVCC), reason="needs nvcc")
def test_hub_tile_kernel_local_memory_stays_small(tmp_path):
    """The tcgen05 tile kernel spills a few words in its issuing thread's
    pipeline loop (36 bytes of stores at 32 registers); the tensor work is
    asynchronous, so this is off the MMA path.  The bound keeps it from growing."""
    rep = ptxas_report("hub.cu", tmp_path)
    mma = {k: v for k, v in rep.items() if "k_hub_mma" in k}
    assert mma
    for k, (regs, st, ld) in mma.items():
        assert st <= 64 and ld <= 64, (k, regs, st, ld)
