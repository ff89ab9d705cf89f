"""Network checkpoint files on the CPU: the library's own writer and reader
(unet_save / unet_load in csrc/checkpoint.cu, compiled with the host compiler over a
stand-in network of host arrays) against the Python description of the same layout
(checkpoint.encode / decode): round trips, files written by either side read by the
other, configuration checks and the detection of damaged files."""
import ctypes
import json
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2203_11025_gb300 import checkpoint as C
from paper_2203_11025_gb300 import lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    if cxx is None or not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no host C++ compiler or CUDA headers")
    out = str(tmp_path_factory.mktemp("ckpt") / "libckpt.so")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-shared", "-fPIC",
                        "-I", os.path.join(ROOT, "paper_2203_11025_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
                        "-I", cuda_inc, os.path.join(ROOT, "tests", "cpp", "checkpoint_shim.cpp"), "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    so = ctypes.CDLL(out)
    P = ctypes.c_void_p
    so.shim_new.restype = P
    so.shim_new.argtypes = [ctypes.POINTER(lib.unet_cfg), P, ctypes.c_longlong, P, ctypes.c_longlong]
    so.shim_free.argtypes = [P]
    so.shim_error.restype = ctypes.c_char_p
    so.unet_save.argtypes = [P, ctypes.c_char_p, ctypes.c_char_p]
    so.unet_load.argtypes = [P, ctypes.c_char_p]
    so.unet_get_params.argtypes = [P, P, ctypes.c_longlong]
    so.unet_get_bn_stats.argtypes = [P, P, ctypes.c_longlong]
    return so


class Net:
    """A stand-in network inside the shim (weights and BN statistics on the host)."""

    def __init__(self, so, cfg, n_params=1000, n_bn=64, seed=0):
        rng = np.random.default_rng(seed)
        self.so, self.cfg = so, cfg
        p = rng.standard_normal(n_params).astype(np.float32)
        b = rng.standard_normal(n_bn).astype(np.float32)
        self.h = so.shim_new(ctypes.byref(cfg), p.ctypes.data, p.size, b.ctypes.data, b.size)
        self.n_params, self.n_bn = n_params, n_bn

    def params(self):
        a = np.empty(self.n_params, np.float32)
        assert self.so.unet_get_params(self.h, a.ctypes.data, a.size) == 0
        return a

    def bn(self):
        a = np.empty(self.n_bn, np.float32)
        assert self.so.unet_get_bn_stats(self.h, a.ctypes.data, a.size) == 0
        return a

    def save(self, path, meta=None):
        m = json.dumps(meta).encode() if meta is not None else None
        return self.so.unet_save(self.h, os.fsencode(path), m)

    def load(self, path):
        return self.so.unet_load(self.h, os.fsencode(path))


def _cfg(widths=(32, 64, 128, 256), context=None):
    c = lib.unet_cfg()
    c.in_ch, c.out_ch, c.levels, c.coarse_resnets = 4, 2, len(widths), 3
    for i, w in enumerate(widths):
        c.widths[i] = w
    for i, v in enumerate(context or []):
        c.context[i] = v
    return c


def test_round_trip_is_bit_exact(shim, tmp_path):
    src, dst = Net(shim, _cfg(), seed=1), Net(shim, _cfg(), seed=2)
    path = str(tmp_path / "net.ckpt")
    assert src.save(path, {"epochs": 96, "lr": 1e-3}) == 0
    assert dst.load(path) == 0
    assert np.array_equal(dst.params().view(np.uint32), src.params().view(np.uint32))
    assert np.array_equal(dst.bn().view(np.uint32), src.bn().view(np.uint32))
    # the Python reader of the layout sees the same file: configuration, arrays, meta
    cfg, p, b, meta = C.read(path)
    assert cfg == C.cfg_to_dict(src.cfg) and meta == {"epochs": 96, "lr": 1e-3}
    assert np.array_equal(p, src.params()) and np.array_equal(b, src.bn())


def test_python_written_file_loads_in_the_library(shim, tmp_path):
    cfg = _cfg(widths=(16, 32), context=[8, 16, 32])
    rng = np.random.default_rng(3)
    p, b = rng.standard_normal(1000).astype(np.float32), rng.standard_normal(64).astype(np.float32)
    path = tmp_path / "py.ckpt"
    path.write_bytes(C.encode(C.cfg_to_dict(cfg), p, b, {"note": "written by Python"}))
    net = Net(shim, cfg, seed=4)
    assert net.load(str(path)) == 0, shim.shim_error()
    assert np.array_equal(net.params(), p) and np.array_equal(net.bn(), b)


def test_cfg_survives_the_file(shim, tmp_path):
    cfg = _cfg(widths=(16, 32), context=[8, 16, 32])
    d = C.cfg_to_dict(cfg)
    back = C.cfg_to_dict(C.dict_to_cfg(d))
    assert back == d and back["widths"][:2] == [16, 32] and back["context"][:3] == [8, 16, 32]
    path = str(tmp_path / "net.ckpt")
    assert Net(shim, cfg).save(path) == 0
    assert C.read(path)[0] == d


def test_payload_is_16_byte_aligned_and_sized():
    blob = C.encode(C.cfg_to_dict(_cfg()), np.arange(10, dtype=np.float32), np.arange(3, dtype=np.float32))
    assert (len(blob) - 4 * 13) % 16 == 0
    cfg, p, bn, meta = C.decode(blob)
    assert np.array_equal(p, np.arange(10, dtype=np.float32)) and np.array_equal(bn, np.arange(3, dtype=np.float32))


def test_configuration_mismatch_is_refused(shim, tmp_path):
    path = str(tmp_path / "net.ckpt")
    assert Net(shim, _cfg(widths=(32, 64, 128, 256))).save(path) == 0
    other = Net(shim, _cfg(widths=(16, 32, 64, 128)), seed=5)
    before = other.params()
    assert other.load(path) == lib.HELM_EINVAL
    assert b"configuration" in shim.shim_error()
    assert np.array_equal(other.params(), before)
    assert Net(shim, _cfg(), n_params=999).load(path) == lib.HELM_EINVAL


def test_meta_must_be_one_json_object(shim, tmp_path):
    net = Net(shim, _cfg())
    assert net.so.unet_save(net.h, os.fsencode(str(tmp_path / "a.ckpt")), b"[1, 2]") == lib.HELM_EINVAL
    assert net.so.unet_save(net.h, os.fsencode(str(tmp_path / "b.ckpt")), b'{"a": 1} x') == lib.HELM_EINVAL


@pytest.mark.parametrize("damage", ["magic", "flip", "truncate", "version", "header"])
def test_damaged_files_are_refused(shim, tmp_path, damage):
    blob = bytearray(C.encode(C.cfg_to_dict(_cfg()), np.ones(100, np.float32), np.ones(8, np.float32)))
    if damage == "magic":
        blob[0] ^= 0xFF
    elif damage == "flip":
        blob[-5] ^= 0x01
    elif damage == "truncate":
        blob = blob[:-4]
    elif damage == "version":
        blob = bytearray(bytes(blob).replace(b'"version": 1', b'"version": 9'))
    else:
        blob[14] = 0xFF
    with pytest.raises(ValueError):
        C.decode(bytes(blob))
    path = tmp_path / "bad.ckpt"
    path.write_bytes(bytes(blob))
    net = Net(shim, _cfg(), n_params=100, n_bn=8)
    before = net.params()
    assert net.load(str(path)) == lib.HELM_EINVAL
    assert np.array_equal(net.params(), before)
