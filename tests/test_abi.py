"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point the headers under include/ declare (no compute call is
made here)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2101_10994_gb300 import build as B
from paper_2101_10994_gb300 import nglod

HEADERS = sorted(glob.glob(os.path.join(B.INCLUDE, "*.h")))


def declared_functions():
    names = []
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while")))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def test_header_declares_the_five_calls():
    assert any(h.endswith("nglod.h") for h in HEADERS) and any(h.endswith("nglod_probe.h") for h in HEADERS)
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


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures of the binding have the header's sizes and field
    offsets (a host C compiler lays the header's structs out; no GPU)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    structs = {"nglod_features": nglod._Features, "nglod_decoder": nglod._Decoder,
               "nglod_trace_params": nglod._TraceParams, "nglod_trace_job": nglod._TraceJob}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "nglod.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", B.INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line}
    for cname, cls in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_staged_traversal_rejects_bad_arguments_on_the_host(libpath):
    """svo_trace_rays_staged_async checks its arguments before any device
    work: a width outside 0..4, a NULL output pointer or a NULL octree each
    return NGLOD_ERR_INVALID_ARG and name the call (no GPU touched)."""
    lib = ctypes.CDLL(libpath)
    f = lib.svo_trace_rays_staged_async
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    f.argtypes = [P, P, P, i64, i32, P, sz, i64, i32, P, P, P, P]
    lib.nglod_last_error.restype = ctypes.c_char_p
    outs = [ctypes.c_void_p() for _ in range(3)]
    refs = [ctypes.byref(x) for x in outs]
    assert f(None, None, None, 16, 3, None, 0, 64, 5, *refs, None) == nglod.ERR_INVALID_ARG
    assert b"ctas_per_sm" in lib.nglod_last_error()
    assert f(None, None, None, 16, 3, None, 0, 64, 0, refs[0], None, refs[2], None) == nglod.ERR_INVALID_ARG
    assert b"NULL output" in lib.nglod_last_error()
    assert f(None, None, None, 16, 3, None, 0, 64, 0, *refs, None) == nglod.ERR_INVALID_ARG
    assert b"svo_trace_rays_staged_async" in lib.nglod_last_error()
