"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/hspgemm.h (no compute call: this runs without a GPU)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hspgemm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(hs_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_operations():
    names = declared_functions()
    for must in ("hs_spgemm", "hs_spref", "hs_spasgn", "hs_mat_free", "hs_strerror"):
        assert must in names


def test_library_builds_and_exports_every_symbol():
    from paper_1109_3739_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in hspgemm.h but not exported"


def test_status_strings_without_gpu():
    from paper_1109_3739_gb300 import hspgemm as H
    L = H.library()
    for code in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert L.hs_strerror(code)
    assert L.hs_version() >= 100


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1109_3739_gb300 import hspgemm as H
    monkeypatch.setattr(H, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(H, "_L", None)
    with pytest.raises(RuntimeError):
        H.library()


def test_tuning_round_trip_without_gpu():
    from paper_1109_3739_gb300 import hspgemm as H
    H.set_tuning(None)
    d = H.get_tuning()
    assert d == {"warp_s_max": 128, "mid_s_max": 1024, "large_s_max": 4096, "sym_mid_s_max": 1024,
                 "sym_heavy_from": 0}
    H.set_tuning({"mid_s_max": 512, "sym_heavy_from": 6144})
    d2 = H.get_tuning()
    assert d2["mid_s_max"] == 512 and d2["sym_heavy_from"] == 6144 and d2["warp_s_max"] == 128
    H.set_tuning(None)
    assert H.get_tuning() == d
