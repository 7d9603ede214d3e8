"""CPU-side checks of the boundary: the library loads, exports every entry point
include/tkc.h declares, and the binding's struct layouts match the header."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tkc.h")


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|uint64_t|const char \*)\s*\*?\s*(tkc_\w+)\s*\(", text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1704_01077_gb300 import build

    build.build()
    return ctypes.CDLL(build.LIB)


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1704_01077_gb300 import tkc

    assert sorted(tkc.EXPORTED) == _declared()
    for name in tkc.EXPORTED:
        assert callable(getattr(tkc, name))


def test_struct_layouts_match_header():
    from paper_1704_01077_gb300 import tkc

    # int + pad + pointer + 6 x uint32 + uint64 + 4 x uint32
    assert ctypes.sizeof(tkc.tkc_options) == 64
    assert tkc.tkc_options.timeout_cycles.offset == 40
    assert tkc.tkc_options.large_blocks.offset == 56
    # 5 pointers, 3 x uint32 (+pad), 6 x uint64, 2 x uint32, 2 x double
    assert ctypes.sizeof(tkc.tkc_result) == 144
    assert tkc.tkc_result.edges_visited.offset == 56
    assert tkc.tkc_result.ms_bfs.offset == 120


def test_error_strings(lib):
    lib.tkc_strerror.restype = ctypes.c_char_p
    for code in (0, -1, -2, -3, -5, -6):
        assert lib.tkc_strerror(code)
    assert lib.tkc_strerror(-99) == b"unknown error"


def test_constants_match_header():
    from paper_1704_01077_gb300 import tkc

    text = open(HEADER).read()
    for name in ("TKC_OK", "TKC_EINVAL", "TKC_EGRAPH", "TKC_ENOMEM", "TKC_ECUDA", "TKC_ETIMEOUT",
                 "TKC_EOVERFLOW", "TKC_ORDER_DEG", "TKC_ORDER_GIVEN", "TKC_ORDER_LEARNED", "TKC_ORDER_NB", "TKC_MAX_K",
                 "TKC_NOALLOC_MAX_N", "TKC_MLP_FEATURES", "TKC_MLP_HIDDEN", "TKC_MLP_PARAMS"):
        m = re.search(rf"#define {name} (-?\d+)", text)
        assert m and int(m.group(1)) == getattr(tkc, name), name
