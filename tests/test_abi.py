"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/*.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\([^;{]*\)\s*;", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def built_lib():
    from paper_2203_11025_gb300 import build
    return build.build()


def test_library_builds_and_loads(built_lib):
    assert os.path.exists(built_lib)
    ctypes.CDLL(built_lib)


def test_every_declared_symbol_is_exported(built_lib):
    from paper_2203_11025_gb300 import lib
    declared = _declared_functions()
    assert declared, "no declarations parsed"
    assert set(lib.ABI_SYMBOLS) == declared
    so = ctypes.CDLL(built_lib)
    for name in declared:
        assert hasattr(so, name), name


def test_binding_signatures_load(built_lib):
    from paper_2203_11025_gb300 import lib
    L = lib.load()
    for name in lib.ABI_SYMBOLS:
        assert getattr(L, name).argtypes is not None or name == "helm_last_error"


def test_null_arguments_fail_with_einval(built_lib):
    """Entry points reject null handles and pointers with HELM_EINVAL and a message before
    touching the GPU (so this runs without one)."""
    from paper_2203_11025_gb300 import lib
    L = lib.load()
    opts = lib.fgmres_opts(10, 1e-7, 100, 0)
    res = lib.fgmres_result(0, 0, 0.0, 0, None, None, 0)
    calls = {
        "fgmres_solve": lambda: L.fgmres_solve(None, lib.HELM_PREC_V, None, None, None, 1, ctypes.byref(opts),
                                               ctypes.byref(res), None),
        "bfgmres_solve": lambda: L.bfgmres_solve(None, lib.HELM_PREC_V, None, None, None, 1, ctypes.byref(opts),
                                                 ctypes.byref(res), None),
        "unet_residual_loss": lambda: L.unet_residual_loss(None, None, None, 1, None, None, None),
        "unet_mse": lambda: L.unet_mse(None, None, 0, 1, None, None, None),
        "unet_forward": lambda: L.unet_forward(None, None, None, 1, 16, 16, 0, None),
        "unet_precond": lambda: L.unet_precond(None, None, lib.HELM_PREC_VU, None, None, 1, 0, None),
        "unet_train_step": lambda: L.unet_train_step(None, None, None, None, 1, None, None, None),
        "unet_save": lambda: L.unet_save(None, b"x.ckpt", None),
        "unet_load": lambda: L.unet_load(None, b"x.ckpt"),
        "unet_wait_probe": lambda: L.unet_wait_probe(None, 10, 0, None),
    }
    for name, call in calls.items():
        assert call() == lib.HELM_EINVAL, name
        assert L.helm_last_error(), name
