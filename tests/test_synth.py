"""The seeded input generator shared by the CUDA path's tests and the oracle: SplitMix64
against the generator's published reference outputs, and the ranges, moments and
structure of the media, sources and draws it builds."""
import numpy as np

from paper_2203_11025_gb300 import synth


def test_splitmix64_reference_outputs():
    # reference outputs published with SplitMix64 (seed 0, and seed 1234567)
    assert [int(v) for v in synth.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in synth.splitmix64(1234567, 5)] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431, 16408922859458223821]


def test_counter_layout_is_splittable():
    a = synth.splitmix64(77, 10)
    assert np.array_equal(synth.splitmix64(77, 4, offset=6), a[6:])
    assert np.array_equal(synth.uniform01(77, 3, offset=2), synth.uniform01(77, 5)[2:])


def test_uniform_and_normal_moments():
    u = synth.uniform01(5, 200000)
    assert u.min() > 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    z = synth.normal(6, 200001)
    assert z.shape == (200001,) and abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 1e-2
    assert abs(np.mean(z ** 4) - 3.0) < 0.05                  # Gaussian kurtosis
    c = synth.complex_normal(7, (100, 1000))
    assert abs(np.mean(np.abs(c) ** 2) - 1.0) < 1e-2 and abs(np.mean(c.real * c.imag)) < 1e-2


def test_medium_range_and_smoothness():
    k2 = synth.grf_kappa2(96, 128, 1000)
    assert k2.dtype == np.float32 and k2.shape == (96, 128)
    assert np.isclose(k2.min(), 0.25 ** 2, rtol=1e-6) and np.isclose(k2.max(), 1.0, rtol=1e-6)
    k = np.sqrt(k2.astype(np.float64))
    assert np.abs(np.diff(k, axis=1)).max() < 0.1            # smooth on the 8-cell scale
    assert np.array_equal(k2, synth.grf_kappa2(96, 128, 1000)) and not np.array_equal(k2, synth.grf_kappa2(96, 128, 1001))


def test_sources_and_pair_draws():
    pos = synth.source_positions(64, 80, 50, 3, 16)
    assert len(pos) == 50 and all(16 <= iy < 48 and 16 <= ix < 64 for iy, ix in pos)
    g = synth.point_sources(64, 80, pos[:2], 1.0 / 64)
    assert g.shape == (2, 64, 80) and g[0][pos[0]] == 64.0 ** 2 and np.count_nonzero(g[1]) == 1
    assert np.isclose(synth.omega_for(256), 0.2 * np.pi * 256)
    x, ks = synth.pair_draws(11, 200, 4, 4, 10)
    assert x.shape == (200, 4, 4) and ks.min() >= 1 and ks.max() <= 10 and len(set(ks.tolist())) == 10
    assert np.array_equal(x[3], synth.complex_normal(11 + 1 + 3, (4, 4)))
