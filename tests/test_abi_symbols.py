"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function include/sz3g.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_2111_02925_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sz3g.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sz3g_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("sz3g_compress", "sz3g_decompress", "sz3g_compress_bound", "sz3g_read_header",
                 "sz3g_workspace_size", "sz3g_strerror", "sz3g_predict_quantize", "sz3g_recover",
                 "sz3g_huffman_build", "sz3g_huffman_encode", "sz3g_huffman_decode"):
        assert must in names


def test_library_loads_and_exports_every_declared_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls_without_gpu():
    from paper_2111_02925_gb300 import sz3g as G

    G.load()
    p = G.make_params((512, 512, 512), 1e-3, eb_mode=G.REL, interp=G.CUBIC)
    assert G.sz3g_compress_bound(p) > 512 ** 3 * 4
    assert G.sz3g_workspace_size(p, 0) > 512 ** 3 * 2
    assert G.sz3g_workspace_size(p, 1) > 512 ** 3 * 2
    assert G.strerror(G.E_CORRUPT).startswith("stream")
    bad = G.make_params((4, 4), 1e-3, order=(0, 0))
    with pytest.raises(G.SZ3GError):
        G.sz3g_compress_bound(bad)
