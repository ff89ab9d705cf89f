"""The Python binding's view of the C ABI matches the headers: every struct the binding
marshals has the size and field offsets the C compiler gives it, and every HELM_* /
UNET_* constant the binding names has the header's value.  A C probe is compiled from
include/unet.h (which includes helm.h) with the host compiler; no GPU is needed."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = ["helm_desc", "unet_cfg", "fgmres_opts", "fgmres_result"]


def _binding():
    from paper_2203_11025_gb300 import lib
    return lib


def _constants(lib):
    return {k: v for k, v in vars(lib).items() if re.fullmatch(r"(HELM|UNET)_[A-Z0-9_]+", k) and isinstance(v, int)}


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lib = _binding()
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "unet.h"', "int main(void) {"]
    for name in sorted(_constants(lib)):
        lines.append(f'  printf("%s %lld\\n", "{name}", (long long)({name}));')
    for s in STRUCTS:
        lines.append(f'  printf("sizeof.{s} %zu\\n", sizeof({s}));')
        for fname, *_ in getattr(lib, s)._fields_:
            lines.append(f'  printf("{s}.{fname} %zu\\n", offsetof({s}, {fname}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "probe.c", d / "probe"
    src.write_text("\n".join(lines) + "\n")
    r = subprocess.run([cc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    return dict(line.rsplit(" ", 1) for line in out.splitlines())


def test_headers_compile_as_c_and_constants_match(probe):
    lib = _binding()
    consts = _constants(lib)
    assert {"HELM_BC_REFLECT", "HELM_STENCIL_COMPACT4", "HELM_OP_RHS", "HELM_PREC_VU"} <= set(consts)
    for name, value in consts.items():
        assert int(probe[name]) == value, name


@pytest.mark.parametrize("struct", STRUCTS)
def test_struct_layout_matches(probe, struct):
    cls = getattr(_binding(), struct)
    assert int(probe[f"sizeof.{struct}"]) == ctypes.sizeof(cls)
    for fname, *_ in cls._fields_:
        assert int(probe[f"{struct}.{fname}"]) == getattr(cls, fname).offset, f"{struct}.{fname}"


def test_named_desc_values():
    lib = _binding()
    assert lib.desc_value("bc", "reflect") == lib.HELM_BC_REFLECT
    assert lib.desc_value("stencil", "compact4") == lib.HELM_STENCIL_COMPACT4
    assert lib.desc_value("levels", 4) == 4
    with pytest.raises(ValueError):
        lib.desc_value("bc", "periodic")
    with pytest.raises(ValueError):
        lib.desc_value("levels", "three")


def test_headers_compile_as_cpp(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "probe.cpp"
    src.write_text('#include "unet.h"\nint main() { helm_desc d{}; unet_cfg c{}; return d.nx + c.levels; }\n')
    r = subprocess.run([cxx, "-std=c++17", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-I",
                        os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
