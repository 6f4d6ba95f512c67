"""The C-ABI library builds, loads and exports every symbol its headers declare
(no GPU needed: no compute calls)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2508_11443_b300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fks_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


def test_headers_declare_the_boundary():
    names = declared_functions()
    for want in ("fks_build_u64", "fks_build_bytes", "fks_lookup_u64", "fks_lookup_bytes",
                 "fks_build_batched", "fks_lookup_batched", "fks_map_info", "fks_map_export",
                 "fks_map_destroy", "fks_status_str"):
        assert want in names


def test_library_exports_every_declared_symbol():
    path = B.build()
    L = ctypes.CDLL(path)
    missing = [n for n in sorted(declared_functions()) if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings_need_no_gpu():
    from paper_2508_11443_b300 import fks
    assert fks.fks_status_str(fks.FKS_OK) == "ok"
    assert "duplicate" in fks.fks_status_str(fks.FKS_ERR_DUPLICATE_KEY)


def test_build_targets_sm103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_product_path_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2508_11443_b300")
    for f in glob.glob(os.path.join(pkg, "**", "*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
            src = open(f).read()
            assert "oracle" not in src.replace("no oracle", "").lower() or f.endswith("workloads.py"), f
