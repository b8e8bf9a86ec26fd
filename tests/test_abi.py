"""The C ABI library builds, loads without a GPU, and exports every entry
point include/cqr2.h declares; the Python binding covers the same set."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions() -> list[str]:
    names = []
    for f in sorted(os.listdir(HEADER_DIR)):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(HEADER_DIR, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(cqr2_[a-z0-9_]+)\s*\(", src):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1710_08471_gb300 import build

    return build.build()


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("cqr2_plan_create", "cqr2_factor", "cqr2_lstsq", "cqr2_plan_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_match_header(lib_path):
    from paper_1710_08471_gb300 import _native

    assert sorted(_native.SIGNATURES) == declared_functions()


def test_status_strings_without_gpu(lib_path):
    from paper_1710_08471_gb300 import _native

    lib = _native.load(lib_path)
    assert lib.cqr2_status_string(0) == b"CQR2_OK"
    assert lib.cqr2_status_string(2) == b"CQR2_ERR_NOT_SPD"
    assert b"sm_103a" in lib.cqr2_version()


def test_plan_create_rejects_bad_shapes_without_touching_gpu(lib_path):
    from paper_1710_08471_gb300 import _native

    lib = _native.load(lib_path)
    h = ctypes.c_void_p()
    # argument checks come before any CUDA call
    assert lib.cqr2_plan_create(ctypes.byref(h), 3, 5, 0, 0, None) == _native.CQR2_ERR_INVALID_ARG
    assert lib.cqr2_plan_create(ctypes.byref(h), 10, 0, 0, 0, None) == _native.CQR2_ERR_INVALID_ARG
    assert lib.cqr2_plan_create(None, 10, 5, 0, 0, None) == _native.CQR2_ERR_INVALID_ARG
    assert lib.cqr2_plan_create(ctypes.byref(h), 10, 5, 0, 0x80, None) == _native.CQR2_ERR_INVALID_ARG
    assert h.value is None


def test_product_package_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1710_08471_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, flags=re.M), f
                assert "oracle/" not in src, f


def test_header_constants_match_binding():
    """The Python binding's flag, precision and status values are the ones
    the C header defines."""
    from paper_1710_08471_gb300 import _native

    hdr = open(os.path.join(ROOT, "include", "cqr2.h")).read()
    vals = {k: int(v, 0) for k, v in re.findall(r"#define\s+(CQR2_[A-Z_]+)\s+(0x[0-9a-fA-F]+)u", hdr)}
    vals.update({k: int(v) for k, v in re.findall(r"\b(CQR2_[A-Z0-9_]+)\s*=\s*(\d+)", hdr)})
    for name in ("CQR2_FUSED", "CQR2_GRAPH", "CQR2_SHIFTED", "CQR2_INPLACE", "CQR2_FP64", "CQR2_OZAKI_BF16",
                 "CQR2_OZAKI_BF16_S6", "CQR2_OK", "CQR2_ERR_INVALID_ARG", "CQR2_ERR_NOT_SPD", "CQR2_ERR_OOM",
                 "CQR2_ERR_TIMEOUT", "CQR2_ERR_UNSUPPORTED"):
        assert getattr(_native, name) == vals[name], name


def test_header_is_plain_c():
    """include/cqr2.h compiles as C99 (no C++ in the ABI), and a C program
    that calls every group of entry points links against the library."""
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = (
        '#include "cqr2.h"\n'
        "int main(void) {\n"
        "  cqr2_problem_t p = {0}; cqr2_info_t i = {0}; cqr2_batch_config_t c = {0}; cqr2_tune_result_t t = {0};\n"
        "  (void)p; (void)i; (void)c; (void)t;\n"
        "  return cqr2_status_string(CQR2_OK)[0] == 'C' ? 0 : 1;\n"
        "}\n"
    )
    out = subprocess.run([cc, "-x", "c", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", "-I", HEADER_DIR, "-"],
                         input=src, capture_output=True, text=True)
    assert out.returncode == 0, out.stderr
