"""The C ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/mgar.h declares (no compute calls here)."""
import ctypes
import os
import re

from paper_2210_00947_gb300 import build, mgar

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(mgar_\w+)\s*\(", src)
    return sorted(set(names))


def test_library_builds_and_exports_header():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) <= set(mgar.EXPORTS) | {"mgar_default_params"}


def test_params_layout_and_defaults():
    p = mgar.default_params()
    assert ctypes.sizeof(mgar.Params) == 152
    assert (p.k0, p.kmin, p.penal, p.rmin, p.nl, p.m) == (1.0, 1e-3, 3.0, 1.5, 4, 2)
    assert (p.eps1, p.eps2, p.cg_max, p.omega) == (0.5, 1e-8, 200, 0.9)


def test_create_rejects_bad_arguments_without_touching_the_gpu():
    lib = mgar.load()
    h = ctypes.c_void_p()
    # null pointers are refused before any CUDA call
    assert lib.mgar_create(ctypes.byref(h), None, None, None, None) == mgar.MGAR_ERR_ARG
    assert b"null" in lib.mgar_last_error(None)


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of mgar_params and mgar_step_info against the C
    compiler's layout of include/mgar.h (sizes and every field offset)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no C compiler")
    fields = {"mgar_params": mgar.Params, "mgar_step_info": mgar.StepInfo}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mgar.h"', 'int main(void) {']
    for cname, cls in fields.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            cf = "lambda" if fname == "lambda_" else fname
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l}
    for cname, cls in fields.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)
