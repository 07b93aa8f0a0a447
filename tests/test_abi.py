"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/hkgeneo.h (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

from paper_2406_06283_gb300 import build, hk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "hkgeneo.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hk_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def library():
    if not os.path.exists(hk.LIB_PATH):
        build.build()
    return ctypes.CDLL(hk.LIB_PATH)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("hk_setup", "hk_solve", "hk_solve_device", "hk_info", "hk_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(library):
    missing = [n for n in declared_functions() if not hasattr(library, n)]
    assert not missing, missing


def test_status_strings_without_gpu(library):
    library.hk_status_string.restype = ctypes.c_char_p
    assert library.hk_status_string(0) == b"HK_OK"
    assert library.hk_status_string(2) == b"HK_SINGULAR_LOCAL"
    # every status the header declares has its own name
    text = open(os.path.join(ROOT, "include", "hkgeneo.h")).read()
    for name, code in re.findall(r"\b(HK_[A-Z_]+) = (\d+),?\s", text[:text.index("} hk_status;")]):
        assert library.hk_status_string(int(code)) == name.encode(), name


def test_setup_rejects_bad_arguments_before_touching_the_device(library):
    out = ctypes.c_void_p()
    # NULL mesh: argument checks run before any CUDA call
    assert library.hk_setup(None, None, ctypes.c_double(1.0), None, None, ctypes.byref(out)) == hk.HK_BAD_ARG
    assert not out.value


def test_binding_fails_loudly_when_library_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(hk, "_lib", None)
    monkeypatch.setattr(hk, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(hk.HKLibraryMissing):
        hk.lib()


def test_info_struct_layout_matches_the_header(tmp_path):
    """hk.hk_info_t (ctypes) has the size and field offsets of the C struct in include/hkgeneo.h."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in hk.hk_info_t._fields_]
    src = tmp_path / "layout.c"
    body = "\n".join(f'  printf("{f} %zu\\n", offsetof(hk_info_t, {f}));' for f in fields)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "hkgeneo.h"\nint main(void) {\n'
                   f'  printf("size %zu\\n", sizeof(hk_info_t));\n{body}\n  return 0;\n}}\n')
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    assert int(out["size"]) == ctypes.sizeof(hk.hk_info_t)
    for f in fields:
        assert int(out[f]) == getattr(hk.hk_info_t, f).offset, f
