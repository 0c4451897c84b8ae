"""CPU checks of the C ABI: the library builds, loads and exports every
function declared in include/tomo.h; the Python binding mirrors the names.
No compute call is made (there may be no GPU)."""
import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "tomo.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tomo_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1806_07938_gb300 import _build
    path = _build.library_path()
    if not os.path.exists(path):
        if os.environ.get("TOMO_SKIP_BUILD"):
            pytest.skip("library not built")
        _build.build_library()
    return path


def test_header_declares_the_boundary():
    names = declared()
    for fn in ["tomo_create", "tomo_layout", "tomo_apply_css", "tomo_apply_css_f64", "tomo_apply_cos",
               "tomo_solve", "tomo_solve_host", "tomo_destroy", "tomo_strerror"]:
        assert fn in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for fn in declared():
        assert hasattr(lib, fn), fn


def test_binding_mirrors_the_names(libpath):
    from paper_1806_07938_gb300 import tomo
    for fn in declared():
        assert callable(getattr(tomo, fn)), fn
    assert set(tomo.EXPORTS) == set(declared())


def test_strerror_needs_no_gpu(libpath):
    from paper_1806_07938_gb300 import tomo
    tomo.lib(libpath)
    assert tomo.tomo_strerror(0) == "ok"
    assert "invalid" in tomo.tomo_strerror(1)


def test_missing_library_fails_loudly(tmp_path):
    from paper_1806_07938_gb300 import tomo
    saved = tomo._lib
    tomo._lib = None
    try:
        with pytest.raises(RuntimeError):
            tomo.lib(str(tmp_path / "nope.so"))
    finally:
        tomo._lib = saved


def test_binding_structs_match_the_header_layout(tmp_path):
    # the ctypes mirrors must have the C layout field by field: a C program
    # built from the header prints every offset and size, compared here
    import shutil
    import subprocess

    from paper_1806_07938_gb300 import tomo
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {name: getattr(tomo, name) for name in
               ("tomo_gs", "tomo_config", "tomo_layout_info", "tomo_solve_opts", "tomo_frame_info")}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "tomo.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "sizeof")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)
