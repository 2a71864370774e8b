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
