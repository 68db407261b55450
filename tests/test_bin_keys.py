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


PAIRS_PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include "hspgemm.h"
#include "internal.h"
using namespace hs;
// argv: warp_s_max mid_s_max large_s_max sym_mid_s_max sym_heavy_from sort_max sort_pct num_heavy_from;
// stdin: "f c" pairs; stdout: the key constants, then "sym_key num_key" per pair
int main(int argc, char **argv) {
  if (argc != 9) return 2;
  hs_tuning t;
  hs_get_tuning(&t);
  t.warp_s_max = atoi(argv[1]); t.mid_s_max = atoi(argv[2]); t.large_s_max = atoi(argv[3]);
  t.sym_mid_s_max = atoi(argv[4]); t.sym_heavy_from = atoi(argv[5]); t.sort_max = atoi(argv[6]);
  t.sort_pct = atoi(argv[7]); t.num_heavy_from = atoi(argv[8]);
  hs_set_tuning(&t);
  const BinCfg b = bin_config(4);
  const BinCfg bs = product_bins(b, 1 << 20, 4), bn = numeric_bins(bs, 1 << 20);
  printf("%d %d %d %d %d %d %d %d %d %d %d %d\n", KEY_TINY, KEY_WARP_S, KEY_WARP, KEY_MID_S, KEY_MID, KEY_LARGE_S,
         KEY_LARGE, KEY_SORT_XS, KEY_SORT_S, KEY_SORT_M, KEY_SORT, KEY_HEAVY);
  long long f, c;
  while (scanf("%lld %lld", &f, &c) == 2) printf("%d %d\n", sym_key(f, bs), num_key(f, c, bn));
  return 0;
}
"""

SETTINGS = [
    (128, 1024, 4096, 1024, 0, 1024, 50, 0),       # the library's defaults
    (32, 0, 2048, 512, 2048, 256, 75, 2048),
    (64, 768, 3072, 768, 3072, 512, 101, 4096),
    (128, 512, 4096, 1024, 6144, 1024, 0, 8192),
    (100000, -5, 1 << 30, 0, 1, 1 << 20, -3, 0),  # out of range: clamped
]


def test_bench_bins_follow_the_library(tmp_path):
    """bench.py rebuilds in Python which rows each bin holds, to count the
    dominant kernel's algorithmic bytes; it must bin every row as the library
    does, for any tuning."""
    import numpy as np
    import bench
    from paper_1109_3739_gb300 import build
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    lib = build.build()
    src = tmp_path / "pairs.cu"
    src.write_text(PAIRS_PROGRAM)
    exe = tmp_path / "pairs"
    libdir = os.path.dirname(lib)
    cmd = [nvcc, "-std=c++17", "-O1", *build.ARCH, "-I", os.path.join(ROOT, "paper_1109_3739_gb300", "csrc"),
           "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe), "-L", libdir, "-lhspgemm",
           "-Xlinker", f"-rpath={libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    # row sizes around every threshold, output counts from 1 to f
    edges = [1, 32, 128, 256, 512, 768, 1024, 2048, 3072, 4096, 6144, 8192, 16384, 1 << 20]
    fs = sorted({max(1, e + d) for e in edges for d in (-1, 0, 1)} | {5000, 20000, 100000})
    pairs = []
    for fv in fs:
        for cv in sorted({1, fv // 3 + 1, fv // 2, fv // 2 + 1, fv, *[e + d for e in edges for d in (-1, 0, 1)]}):
            if 1 <= cv <= fv:
                pairs.append((fv, cv))
    f = np.array([p[0] for p in pairs], dtype=np.int64)
    c = np.array([p[1] for p in pairs], dtype=np.int64)
    stdin = "".join(f"{a} {b}\n" for a, b in pairs)
    names = ["warp_s_max", "mid_s_max", "large_s_max", "sym_mid_s_max", "sym_heavy_from", "sort_max", "sort_pct",
             "num_heavy_from"]
    for st in SETTINGS:
        out = subprocess.run([str(exe), *map(str, st)], input=stdin, capture_output=True, text=True, timeout=120)
        assert out.returncode == 0, out.stderr
        lines = out.stdout.split("\n")
        (kt, kws, kw, kms, km, kls, kl, ksx, kss, ksm, ks, kh) = map(int, lines[0].split())
        keys = np.array([list(map(int, ln.split())) for ln in lines[1:] if ln.strip()])
        assert len(keys) == len(pairs)
        sym, num = keys[:, 0], keys[:, 1]
        t = dict(zip(names, st))
        got = bench.bin_rows(t, f, c)
        want = {"symbolic_tiny": sym == kt, "symbolic_warp": sym == kw, "symbolic_mid_s": sym == kms,
                "symbolic_mid": sym == km, "symbolic_large": sym == kl, "symbolic_heavy": sym >= kh,
                "numeric_tiny": num == kt, "numeric_warp_s": num == kws, "numeric_warp": num == kw,
                "numeric_mid_s": num == kms, "numeric_mid": num == km, "numeric_large_s": num == kls,
                "numeric_large": num == kl, "numeric_sort_xs": num == ksx, "numeric_sort_s": num == kss,
                "numeric_sort_m": num == ksm, "numeric_sort": num == ks, "numeric_heavy": num >= kh}
        for name, mask in want.items():
            bad = np.nonzero(got[name] != mask)[0]
            assert bad.size == 0, (st, name, [pairs[i] for i in bad[:5]])
        # every row in exactly one symbolic and one numeric bin
        for side in ("symbolic_", "numeric_"):
            k = sum(v.astype(int) for name, v in got.items() if name.startswith(side))
            assert (k == 1).all(), (st, side)


def test_code_hash_ignores_comments_only():
    """The traffic record is tied to the device code by a hash that skips
    comments and blank lines but not code, nor text inside literals."""
    import bench
    a = 'int a = 1;  // one\n\n/* two\n   lines */\nconst char *s = "// kept /* kept */";\n'
    b = 'int a = 1;\nconst char *s = "// kept /* kept */";   \n'
    assert bench.strip_comments(a) == bench.strip_comments(b)
    assert bench.strip_comments('x = "a\\"//b"; // c') == 'x = "a\\"//b";'
    assert bench.strip_comments("int a = 2;") != bench.strip_comments("int a = 1;")
    srcs = {fn: "int k = 0;\n" for fn in bench.KERNEL_SOURCES}
    h0 = bench.csrc_hash(srcs.__getitem__)
    srcs[bench.KERNEL_SOURCES[0]] = "int k = 0;  // a note\n"
    assert bench.csrc_hash(srcs.__getitem__) == h0
    srcs[bench.KERNEL_SOURCES[0]] = "int k = 1;\n"
    assert bench.csrc_hash(srcs.__getitem__) != h0
