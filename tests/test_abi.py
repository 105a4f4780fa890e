"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/nglod.h declares (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_2101_10994_gb300 import build as B
from paper_2101_10994_gb300 import nglod

HEADER = os.path.join(B.INCLUDE, "nglod.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_five_calls():
    names = declared_functions()
    for n in ("svo_build", "svo_trace_rays", "sdf_query", "sphere_trace"):
        assert n in names


def test_every_declared_symbol_is_exported(libpath):
    lib = ctypes.CDLL(libpath)
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(nglod.EXPORTS) == sorted(n for n in names if n in nglod.EXPORTS)
    assert set(names) <= set(nglod.EXPORTS) | {"sdf_backward"}


def test_built_for_sm103a_only():
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_binding_has_no_cpu_fallback(monkeypatch, tmp_path):
    monkeypatch.setattr(nglod, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(nglod, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        nglod.lib()
