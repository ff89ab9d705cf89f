"""Named workloads: consistent with the paper's settings and with the benchmark's own
problem construction (same medium, same right-hand sides)."""
import math

import numpy as np
import pytest

from paper_2203_11025_gb300 import presets


def test_every_preset_is_well_formed():
    for p in presets.PRESETS.values():
        assert p.n % 4 == 0 and p.nrhs >= 1 and p.tol == 1e-7
        assert math.isclose(p.omega * p.h, 2 * math.pi / 10)          # 10 points per wavelength, kappa <= 1
        d = p.helmholtz_overrides()
        assert d["abc_width"] == 16 and d["levels"] == 3 and d["beta"] == 0.5
        assert (p.precond == "M_V") == (p.train_pairs == 0)
    with pytest.raises(ValueError):
        presets.get("nope")


def test_benchmark_preset_matches_the_benchmark_problem():
    import bench
    p = presets.get("retrain_2048")
    assert (p.n, p.nrhs) == (bench.N_GRID, bench.NRHS)
    assert (p.train_pairs, p.train_epochs, p.train_lr) == (bench.RETRAIN_PAIRS, bench.RETRAIN_EPOCHS,
                                                           bench.RETRAIN_LR)
    assert p.train_batch == bench.max_batch(p.n, 16)
    k2, b = bench.build_problem(0)
    assert np.array_equal(p.medium(0), k2) and np.array_equal(p.rhs(0), b)
    for name in ("retrain_1024", "unet_256"):
        r = presets.get(name)
        assert (r.n, r.nrhs) in bench.EXTRAS
        k2, b = bench.build_problem(0, r.n, r.nrhs)
        assert np.array_equal(r.medium(0), k2) and np.array_equal(r.rhs(0), b)
        assert (r.train_pairs, r.train_epochs, r.train_lr) == (bench.RETRAIN_PAIRS, bench.RETRAIN_EPOCHS,
                                                               bench.RETRAIN_LR)
    g = presets.get("general_256")
    assert g.train_pairs == bench.TRAIN_MEDIA * bench.TRAIN_PAIRS_PER_MEDIUM and g.train_epochs == bench.TRAIN_EPOCHS
    assert bench.TRAIN_PAIRS == g.train_pairs


def test_mixed_right_hand_sides():
    p = presets.get("encoder_solver_512")
    b = p.rhs(0)
    assert b.shape == (32, 512, 512)
    assert all(np.count_nonzero(b[k]) == 1 for k in range(16))
    assert all(np.count_nonzero(b[k]) == 512 * 512 for k in range(16, 32))
