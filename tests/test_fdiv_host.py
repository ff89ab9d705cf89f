"""The multiply-shift division the convolution kernels use for item decoding and stage-ring
positions (csrc/fdiv.h, Granlund-Montgomery round-up multiplier), compiled with the host
compiler: equal to integer division for every divisor the kernels meet (tile counts, split
counts, stage counts; here all d < 4100 and powers of two up to 2^30) and every n they
divide (0 <= n < 2^31), including the edges n = k d - 1, k d and 2^31 - 1."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("fdiv") / "libfdiv.so")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-shared", "-fPIC",
                        "-I", os.path.join(ROOT, "paper_2203_11025_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "cpp", "fdiv_shim.cpp"), "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    so = ctypes.CDLL(out)
    so.fdiv_shim.argtypes = [ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                             ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)]
    return so


def divide(so, d, n):
    n = np.ascontiguousarray(n, dtype=np.int32)
    out = np.empty_like(n)
    m, s = ctypes.c_uint32(), ctypes.c_uint32()
    so.fdiv_shim(d, n.ctypes.data, n.size, out.ctypes.data, ctypes.byref(m), ctypes.byref(s))
    return out, m.value, s.value


def test_matches_integer_division(shim):
    rng = np.random.default_rng(0)
    divisors = list(range(1, 4100)) + [1 << k for k in range(13, 31)] + [3 * (1 << 20), 1000003, 2 ** 31 - 1]
    for d in divisors:
        k = np.arange(0, min((2 ** 31 - 1) // d, 64) + 1, dtype=np.int64)
        edges = np.concatenate([k * d, k * d - 1, [2 ** 31 - 1, 2 ** 31 - 2, 0, 1]])
        n = np.concatenate([edges[(edges >= 0) & (edges < 2 ** 31)], rng.integers(0, 2 ** 31, 512)])
        q, m, s = divide(shim, d, n)
        assert np.array_equal(q, n // d), d
        assert (1 << s) >= d and (s == 0 or (1 << (s - 1)) < d), (d, s)


def test_powers_of_two_reduce_to_a_shift(shim):
    # m = 1 and s = log2 d: n / 2^s = n >> s
    for s_ in range(0, 31):
        _, m, s = divide(shim, 1 << s_, np.array([0], np.int32))
        assert (m, s) == (1, s_)
