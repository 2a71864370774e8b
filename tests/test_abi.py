"""The C ABI library loads and exports every entry point the header declares (CPU only)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsw.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsw_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2404_17754_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("gsw_create", "gsw_model_upload", "gsw_set_time", "gsw_set_input", "gsw_step",
                     "gsw_run", "gsw_read_waveforms", "gsw_misfit"):
        assert required in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), "libgsw.so does not export %s" % name
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (gsw_[a-z_0-9]+)", out))
    assert set(declared_symbols()) <= exported


def test_binding_declares_signatures_for_every_symbol(lib_path):
    from paper_2404_17754_gb300 import gsw

    assert set(gsw.SIGNATURES) == set(declared_symbols())
    gsw.load(lib_path)


def test_binding_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the option and statistics structs have the header's size and field offsets."""
    import shutil

    from paper_2404_17754_gb300 import gsw

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"gsw_solver_opts": gsw.SolverOpts, "gsw_stats": gsw.Stats, "gsw_learn_opts": gsw.LearnOpts}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gsw.h"', "int main(void) {"]
    for cname, py in mirrors.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in py._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    seen = {}
    for line in filter(None, out):
        cname, field, value = line.split()
        seen[(cname, field)] = int(value)
    for cname, py in mirrors.items():
        assert seen[(cname, "size")] == ctypes.sizeof(py), cname
        for fname, _ in py._fields_:
            assert seen[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
