"""Host-side orchestration without a GPU: the training schedule and batch composition
(Sec. 3.4, 4), and the benchmark's size rules."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2203_11025_gb300 import train as T  # noqa: E402


def test_lr_schedule_drops_at_the_papers_epochs():
    # Sec. 4: 10x drops at epoch 48, then after 24, 12, 6, ... further epochs
    lr0 = 1e-2
    drops = [e for e in range(1, 200) if T.lr_at(e, lr0) < T.lr_at(e - 1, lr0)]
    assert drops[:5] == [48, 72, 84, 90, 93]
    assert T.lr_at(0, lr0) == lr0 and abs(T.lr_at(48, lr0) - 1e-3) < 1e-15
    assert T.lr_at(10_000, 1e-4) == 1e-7


def test_batches_cover_every_pair_once_as_lead():
    rng = np.random.default_rng(0)
    seen = []
    for idx, coef in T.batches(rng, 64, 16, 2):
        assert idx.shape == (16, 2) and coef.shape == (16, 2) and idx.dtype == np.int32
        assert np.all((idx >= 0) & (idx < 64))
        seen.extend(idx[:, 0].tolist())
    assert sorted(seen) == list(range(64))


def test_batches_without_mixing_use_unit_coefficients():
    rng = np.random.default_rng(1)
    for idx, coef in T.batches(rng, 20, 8, 1):   # 2 full batches, the 4 left over are dropped
        assert idx.shape == (8, 1) and np.all(coef == 1.0)
    assert sum(1 for _ in T.batches(np.random.default_rng(1), 20, 8, 1)) == 2


def test_mixing_coefficients_are_complex_normal():
    rng = np.random.default_rng(2)
    c = np.concatenate([coef.ravel() for _, coef in T.batches(rng, 4096, 64, 2)])
    assert abs(np.mean(np.abs(c) ** 2) - 1.0) < 0.05          # E|c|^2 = 1
    assert abs(np.mean(c.real)) < 0.05 and abs(np.mean(c.imag)) < 0.05


def test_bench_batch_limit_and_default_rhs():
    # the network's tensor limit B*n*n*64 < 2^31 sets the training batch and the solve's
    # network chunk; the benchmark's default case is 2048^2 with 16 right-hand sides
    import bench
    for n, want in ((256, 16), (1024, 16), (2048, 4)):
        b = bench.max_batch(n, 16)
        assert b == want and b * n * n * 64 < 2 ** 31
    assert (bench.N_GRID, bench.NRHS) == (2048, 16)
