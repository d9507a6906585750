"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/*.h declares (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

import paper_2203_14927_b300 as gz
import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(gz\w*)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    names = declared_symbols()
    assert "gz_create" in names and "gz_edge_update" in names and len(names) >= 15
    L = ctypes.CDLL(gz.LIB_PATH)
    missing = [n for n in sorted(names) if not hasattr(L, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert declared_symbols() <= set(gz._SIGNATURES)


def test_geometry_agrees_with_oracle():
    for V in [2, 3, 5, 1000, 1024, 4097, 1 << 13, 1 << 17, 1 << 20]:
        assert gz.geometry(V) == oracle.geometry(V)
    with pytest.raises(ValueError):
        gz.geometry(1)


def test_version_string():
    assert b"sm_103a" in gz.lib().gz_version()


def test_memory_estimate():
    n = ctypes.c_size_t()
    assert gz.lib().gz_memory_bytes(1 << 17, None, ctypes.byref(n)) == 0
    K, R = gz.geometry(1 << 17)
    assert n.value >= (1 << 17) * K * 7 * R * 12
