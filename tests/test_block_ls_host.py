"""The block-FGMRES host algebra (csrc/block_ls.h, plain C++) compiled on the CPU with the
host compiler and checked against numpy: the Cholesky factor of a Gram matrix with a
dependent column, and the incremental Householder least squares of a block Hessenberg
matrix against numpy's lstsq."""
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
    out = str(tmp_path_factory.mktemp("blockls") / "libblockls.so")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-shared", "-fPIC",
                        "-I", os.path.join(ROOT, "paper_2203_11025_gb300", "csrc"),
                        os.path.join(ROOT, "tests", "cpp", "block_ls_shim.cpp"), "-o", out],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    P = ctypes.POINTER(ctypes.c_double)
    lib.chol_upper_c.argtypes = [P, ctypes.c_int, P, P]
    lib.block_ls_run.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P, P]
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _chol(shim, G):
    p = G.shape[0]
    Gi = np.ascontiguousarray(G, dtype=np.complex128)
    R = np.zeros((p, p), np.complex128)
    Ri = np.zeros((p, p), np.complex128)
    shim.chol_upper_c(_ptr(Gi.view(np.float64)), p, _ptr(R.view(np.float64)), _ptr(Ri.view(np.float64)))
    return R, Ri


def _crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_cholesky_of_a_full_rank_gram_matrix(shim):
    W = _crandn(np.random.default_rng(1), (50, 6))
    G = W.conj().T @ W
    R, Ri = _chol(shim, G)
    assert np.allclose(np.tril(R, -1), 0) and np.all(np.diag(R).real > 0)
    assert np.allclose(R.conj().T @ R, G, rtol=1e-12, atol=1e-10)
    assert np.allclose(Ri @ R, np.eye(6), atol=1e-12)
    Q = W @ Ri
    assert np.allclose(Q.conj().T @ Q, np.eye(6), atol=1e-10)


def test_cholesky_marks_a_dependent_column(shim):
    W = _crandn(np.random.default_rng(2), (40, 5))
    W[:, 2] = W[:, 0] - 2j * W[:, 1]
    R, Ri = _chol(shim, W.conj().T @ W)
    assert np.allclose(R[2], 0) and np.allclose(Ri[:, 2], 0) and np.allclose(Ri[2], 0)
    Q = W @ Ri
    assert np.allclose(Q[:, 2], 0)
    keep = [0, 1, 3, 4]
    assert np.allclose(Q[:, keep].conj().T @ Q[:, keep], np.eye(4), atol=1e-10)
    assert np.allclose(Q @ R, W, atol=1e-10)          # W = (W Rinv) R


@pytest.mark.parametrize("p,m", [(1, 5), (3, 4), (4, 6)])
def test_block_least_squares_matches_lstsq(shim, p, m):
    rng = np.random.default_rng(10 * p + m)
    rows, cols = (m + 1) * p, m * p
    Hb = np.zeros((rows, cols), np.complex128)
    for j in range(m):                       # block upper Hessenberg, triangular subdiagonal blocks
        Hb[:(j + 1) * p, j * p:(j + 1) * p] = _crandn(rng, ((j + 1) * p, p))
        Hb[(j + 1) * p:(j + 2) * p, j * p:(j + 1) * p] = np.triu(_crandn(rng, (p, p)))
    S = np.triu(_crandn(rng, (p, p)))
    est = np.zeros((m, p))
    Y = np.zeros((cols, p), np.complex128)
    shim.block_ls_run(p, m, _ptr(np.ascontiguousarray(S).view(np.float64)),
                      _ptr(np.ascontiguousarray(Hb).view(np.float64)), _ptr(est), _ptr(Y.view(np.float64)))
    for j in range(m):
        n_r, n_c = (j + 2) * p, (j + 1) * p
        rhs = np.zeros((n_r, p), np.complex128)
        rhs[:p] = S
        Yj, *_ = np.linalg.lstsq(Hb[:n_r, :n_c], rhs, rcond=None)
        res = np.linalg.norm(rhs - Hb[:n_r, :n_c] @ Yj, axis=0)
        assert np.allclose(est[j], res, rtol=1e-9, atol=1e-12)
    assert np.allclose(Y, Yj, rtol=1e-9, atol=1e-10)
