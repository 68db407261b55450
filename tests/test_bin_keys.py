"""Host check of the row-bin key functions (no GPU): for every threshold the
tuning accepts and every row size up to 2^40 products, the symbolic and
numeric keys stay inside the key arrays (0 <= key < NKEYS), the heavy keys
order rows largest first, and rows below the bitmap threshold never reach a
heavy key.  The heavy keys once went one past the arrays for rows of fewer
than 4096 products when the bitmap threshold was lowered; this compiles the
library's own key functions for the host and walks them."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include "internal.h"
using namespace hs;
int main() {
  long long bad = 0, order = 0, below = 0;
  int maxk = -1;
  for (int vb : {0, 4, 8})
    for (int shf : {2048, 3072, 4096, 6144, 8192})
      for (int nhf : {2048, 4096, 8192}) {
        BinCfg b = bin_config(vb);
        b.sym_heavy_from = shf < b.cap_large ? shf : b.cap_large;
        b.num_heavy_from = nhf < b.cap_large ? nhf : b.cap_large;
        int prev = NKEYS;
        for (long long f = 1; f < (1LL << 40); f = f < 70000 ? f + 1 : f + f / 97) {
          const int k = sym_key(f, b);
          if (k < 0 || k >= NKEYS) ++bad;
          if (k > maxk) maxk = k;
          if (f <= b.sym_heavy_from && k >= KEY_HEAVY) ++below;
          if (k >= KEY_HEAVY) {  // heavy keys never grow with f (largest rows first)
            if (k > prev) ++order;
            prev = k;
          }
          for (long long c : {1LL, f / 3 + 1, f}) {
            const int k2 = num_key(f, c, b);
            if (k2 < 0 || k2 >= NKEYS) ++bad;
            if (k2 > maxk) maxk = k2;
          }
        }
      }
  printf("bad %lld order %lld below %lld maxkey %d nkeys %d\n", bad, order, below, maxk, NKEYS);
  return (bad || order || below) ? 1 : 0;
}
"""


def test_bin_keys_stay_inside_the_key_arrays(tmp_path):
    from paper_1109_3739_gb300 import build
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    lib = build.build()
    src = tmp_path / "keys.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "keys"
    libdir = os.path.dirname(lib)
    cmd = [nvcc, "-std=c++17", "-O1", *build.ARCH, "-I", os.path.join(ROOT, "paper_1109_3739_gb300", "csrc"),
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lhspgemm",
           "-Xlinker", f"-rpath={libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "bad 0 order 0 below 0" in out.stdout
