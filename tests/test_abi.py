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

    # int + pad + pointer + 6 x uint32 + uint64 + 5 x uint32 (+ pad)
    assert ctypes.sizeof(tkc.tkc_options) == 72
    assert tkc.tkc_options.timeout_cycles.offset == 40
    assert tkc.tkc_options.large_blocks.offset == 56
    # 5 pointers, 3 x uint32 (+pad), 6 x uint64, 2 x uint32, 2 x double
    assert ctypes.sizeof(tkc.tkc_result) == 144
    assert tkc.tkc_result.edges_visited.offset == 56
    assert tkc.tkc_result.ms_bfs.offset == 120
    assert tkc.tkc_options.deterministic.offset == 60
    assert tkc.tkc_options.relabel.offset == 64
    # 6 x uint32, 17 x uint64, 1 double
    assert ctypes.sizeof(tkc.tkc_run_stats) == 168
    assert tkc.tkc_run_stats.ms_kernel.offset == 160


def test_struct_layouts_match_a_c_compiler(tmp_path):
    """Every field offset the binding uses, against what gcc makes of the header."""
    import subprocess

    from paper_1704_01077_gb300 import tkc

    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "tkc.h"', "int main(void) {"]
    for cname, cls in (("tkc_options", tkc.tkc_options), ("tkc_result", tkc.tkc_result),
                       ("tkc_run_stats", tkc.tkc_run_stats)):
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = subprocess.check_output([str(exe)]).decode().split("\n")
    classes = {"tkc_options": tkc.tkc_options, "tkc_result": tkc.tkc_result, "tkc_run_stats": tkc.tkc_run_stats}
    for line in filter(None, got):
        cname, what, value = line.split()
        cls = classes[cname]
        want = ctypes.sizeof(cls) if what == "size" else getattr(cls, what).offset
        assert int(value) == want, line


def test_error_strings(lib):
    lib.tkc_strerror.restype = ctypes.c_char_p
    for code in (0, -1, -2, -3, -5, -6):
        assert lib.tkc_strerror(code)
    assert lib.tkc_strerror(-99) == b"unknown error"


def test_constants_match_header():
    from paper_1704_01077_gb300 import tkc

    text = open(HEADER).read()
    for name in ("TKC_OK", "TKC_EINVAL", "TKC_EGRAPH", "TKC_ENOMEM", "TKC_ECUDA", "TKC_ETIMEOUT",
                 "TKC_EOVERFLOW", "TKC_ORDER_DEG", "TKC_ORDER_GIVEN", "TKC_ORDER_LEARNED", "TKC_ORDER_NB", "TKC_ORDER_LEARNED_NB", "TKC_MAX_K",
                 "TKC_NOALLOC_MAX_N", "TKC_MLP_FEATURES", "TKC_MLP_HIDDEN", "TKC_MLP_PARAMS"):
        m = re.search(rf"#define {name} (-?\d+)", text)
        assert m and int(m.group(1)) == getattr(tkc, name), name


def test_argument_errors_before_any_device_call(lib):
    """Errors include/tkc.h documents for bad arguments, returned before the
    library touches a device (so they hold on a machine without a GPU)."""
    from paper_1704_01077_gb300 import tkc

    EINVAL, EOVERFLOW = tkc.TKC_EINVAL, tkc.TKC_EOVERFLOW
    vp, u32, u64 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64
    lib.tkc_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(tkc.tkc_options)]
    good = tkc.Options().to_c()
    assert lib.tkc_create(None, ctypes.byref(good)) == EINVAL
    for bad in (dict(batch_bits=96), dict(batch_bits=1024), dict(order=5), dict(nb_levels=65536),
                dict(large_blocks=3), dict(deterministic=2), dict(relabel=3)):
        out = vp(1234)
        assert lib.tkc_create(ctypes.byref(out), ctypes.byref(tkc.Options(**bad).to_c())) == EINVAL, bad
        assert out.value is None, bad
    lib.tkc_set_options.argtypes = [vp, ctypes.POINTER(tkc.tkc_options)]
    assert lib.tkc_set_options(None, ctypes.byref(good)) == EINVAL
    lib.tkc_load_csr.argtypes = [vp, u32, u64, vp, vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(vp)]
    g = vp(1234)
    assert lib.tkc_load_csr(None, 4, 0, None, None, 1, 0, ctypes.byref(g)) == EINVAL
    lib.tkc_load_csr_many.argtypes = [vp, u32, vp, vp, vp, vp, vp, ctypes.c_int, vp, ctypes.POINTER(u32)]
    bad = u32(7)
    assert lib.tkc_load_csr_many(None, 0, None, None, None, None, None, 0, None, ctypes.byref(bad)) == EINVAL
    assert lib.tkc_load_csr_many(vp(1234), 2, None, None, None, None, None, 0, None, ctypes.byref(bad)) == EINVAL
    res = tkc.tkc_result()
    for name in ("tkc_topk_closeness", "tkc_topk_harmonic", "tkc_topk_closeness_bound"):
        fn = getattr(lib, name)
        fn.argtypes = [vp, u32, ctypes.POINTER(tkc.tkc_result)]
        assert fn(None, 10, ctypes.byref(res)) == EINVAL, name
    for name in ("tkc_topk_closeness_multi", "tkc_topk_harmonic_multi"):
        fn = getattr(lib, name)
        fn.argtypes = [vp, vp, u32, u32, ctypes.POINTER(tkc.tkc_result)]
        assert fn(None, None, 1, 10, ctypes.byref(res)) == EINVAL, name
    lib.tkc_distance_sums.argtypes = [vp, u32, vp, vp, vp]
    assert lib.tkc_distance_sums(None, 1, None, None, None) == EINVAL
    lib.tkc_source_order.argtypes = [vp, vp]
    assert lib.tkc_source_order(None, None) == EINVAL
    lib.tkc_nb_bounds.argtypes = [vp, u32, vp, vp, vp, vp, vp, vp]
    assert lib.tkc_nb_bounds(None, 0, None, None, None, None, None, None) == EINVAL
    lib.tkc_distance_sums_noalloc.argtypes = [vp, vp, u32, u64, u32, vp, vp, vp, vp]
    assert lib.tkc_distance_sums_noalloc(None, None, tkc.TKC_NOALLOC_MAX_N + 1, 0, 1, None, None, None,
                                         None) == EINVAL
    assert lib.tkc_distance_sums_noalloc(None, None, 10, 1 << 32, 1, None, None, None, None) == EOVERFLOW
    assert lib.tkc_distance_sums_noalloc(None, None, 10, 0, 0, None, None, None, None) == tkc.TKC_OK
    assert lib.tkc_distance_sums_noalloc(None, None, 10, 0, 1, None, None, None, None) == EINVAL
    lib.tkc_destroy.argtypes = [vp]
    lib.tkc_free_graph.argtypes = [vp]
    lib.tkc_destroy(None)
    lib.tkc_free_graph(None)


def test_plain_c_client_compiles_and_links(lib, tmp_path):
    """include/tkc.h is valid C99 (no C++ needed) and a C program links against
    libtkc.so with every call it makes resolved (built, not run: no GPU here)."""
    import subprocess

    from paper_1704_01077_gb300 import build

    src = os.path.join(ROOT, "tests", "c", "abi_client.c")
    exe = tmp_path / "abi_client"
    libdir = os.path.dirname(build.LIB)
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           src, "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(build.LIB),
                           "-Wl,-rpath," + libdir, "-Wl,--no-undefined", "-Wl,--unresolved-symbols=ignore-in-shared-libs"])
    assert exe.exists()
