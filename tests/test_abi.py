"""Host-side checks of the C-ABI boundary (no GPU needed): the library builds,
loads and exports every function include/linprim.h declares, and the product
path is independent of the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "linprim.h")
PKG = os.path.join(ROOT, "paper_2501_16312_gb300")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lp_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def built_lib():
    from paper_2501_16312_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lp_create", "lp_destroy", "lp_render_forward", "lp_render_backward"):
        assert required in names


def test_library_exports_every_declared_symbol(built_lib):
    lib = ctypes.CDLL(built_lib)
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_lists_every_declared_symbol():
    from paper_2501_16312_gb300 import _native
    assert sorted(_native.EXPORTS) == declared_functions()


def test_status_strings_without_gpu(built_lib):
    from paper_2501_16312_gb300 import _native
    L = _native.load(built_lib)
    assert L.lp_status_string(0) == b"LP_OK"
    assert L.lp_status_string(2) == b"LP_ERR_CAPACITY"
    # no device here: lp_create reports a CUDA error instead of crashing
    h = ctypes.c_void_p()
    import torch
    if not torch.cuda.is_available():
        assert L.lp_create(ctypes.byref(h), 0) == _native.LP_ERR_CUDA


def test_product_path_never_touches_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"\boracle\b", text), f"{f} mentions the oracle"
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert not re.search(r"^\s*(import|from)\s+paper_2501_16312_gb300", text, re.M)
            assert "#include" not in text or "linprim.h" not in text


def test_missing_library_fails_loudly(tmp_path):
    from paper_2501_16312_gb300 import _native
    saved = _native._lib
    _native._lib = None
    try:
        with pytest.raises(ImportError):
            _native.load(str(tmp_path / "nope.so"))
    finally:
        _native._lib = saved


STRUCTS = ("lp_camera", "lp_prims", "lp_tuning", "lp_stats", "lp_adam_group", "lp_population_rules",
           "lp_param_arrays")
CONSTANTS = ("LP_OK", "LP_ERR_INVALID", "LP_ERR_CAPACITY", "LP_ERR_CUDA", "LP_ERR_TIMEOUT",
             "LP_ERR_UNSUPPORTED", "LP_ERR_STATE", "LP_TETRAHEDRON", "LP_OCTAHEDRON", "LP_MAX_CAMERAS",
             "LP_ADAM_MAX_GROUPS", "LP_POP_PRUNE", "LP_POP_KEEP", "LP_POP_CLONE", "LP_POP_SPLIT")


def test_struct_layouts_and_constants_match_the_header(tmp_path):
    """The binding's ctypes structures have the header's size and field
    offsets, and its constants the header's values: a C program compiled
    against include/linprim.h prints them (host compiler only)."""
    import shutil
    import subprocess
    from paper_2501_16312_gb300 import _native
    header = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    assert sorted(re.findall(r"}\s*(lp_[a-z_]+)\s*;", header)) == sorted(STRUCTS + ("lp_status",))
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "linprim.h"', "int main(void) {"]
    for s in STRUCTS:
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for name, _ in getattr(_native, s)._fields_:
            lines.append(f'  printf("{s} {name} %zu\\n", offsetof({s}, {name}));')
    for k in CONSTANTS:
        lines.append(f'  printf("{k} const %lld\\n", (long long)({k}));')
    lines.append('  printf("stages const %d\\n", (int)LP_NUM_STAGES);')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.check_output([str(exe)], text=True).splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for s in STRUCTS:
        cls = getattr(_native, s)
        assert got[(s, "size")] == ctypes.sizeof(cls), s
        for name, _ in cls._fields_:
            assert got[(s, name)] == getattr(cls, name).offset, (s, name)
    for k in CONSTANTS:
        assert got[(k, "const")] == getattr(_native, k), k
    assert got[("stages", "const")] == len(_native.STAGES)
