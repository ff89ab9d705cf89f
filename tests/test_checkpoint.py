"""Network checkpoint files (host side): round trip, configuration checks and the
detection of damaged files, with a stand-in network object (no GPU)."""
import numpy as np
import pytest

from paper_2203_11025_gb300 import checkpoint as C
from paper_2203_11025_gb300 import lib


class FakeNet:
    """Duck-typed stand-in for lib.UNet: configuration, flat weights, BN statistics."""

    def __init__(self, cfg, n_params=1000, n_bn=64, seed=0):
        rng = np.random.default_rng(seed)
        self.cfg = cfg
        self.n_params, self.n_bn = n_params, n_bn
        self.params = rng.standard_normal(n_params).astype(np.float32)
        self.bn = rng.standard_normal(n_bn).astype(np.float32)

    def get_params(self):
        return self.params.copy()

    def get_bn_stats(self):
        return self.bn.copy()

    def set_params(self, a):
        assert a.dtype == np.float32 and a.size == self.n_params
        self.params = a.copy()

    def set_bn_stats(self, a):
        assert a.dtype == np.float32 and a.size == self.n_bn
        self.bn = a.copy()


def _cfg(widths=(32, 64, 128, 256), context=None):
    c = lib.unet_cfg()
    c.in_ch, c.out_ch, c.levels, c.coarse_resnets = 4, 2, len(widths), 3
    for i, w in enumerate(widths):
        c.widths[i] = w
    for i, v in enumerate(context or []):
        c.context[i] = v
    return c


def test_round_trip_is_bit_exact(tmp_path):
    src = FakeNet(_cfg(), seed=1)
    path = str(tmp_path / "net.ckpt")
    C.save(src, path, meta={"epochs": 96, "lr": 1e-3})
    dst = FakeNet(_cfg(), seed=2)
    meta = C.load_into(dst, path)
    assert meta == {"epochs": 96, "lr": 1e-3}
    assert np.array_equal(dst.params.view(np.uint32), src.params.view(np.uint32))
    assert np.array_equal(dst.bn.view(np.uint32), src.bn.view(np.uint32))


def test_cfg_survives_the_file(tmp_path):
    cfg = _cfg(widths=(16, 32), context=[8, 16, 32])
    d = C.cfg_to_dict(cfg)
    back = C.cfg_to_dict(C.dict_to_cfg(d))
    assert back == d and back["widths"][:2] == [16, 32] and back["context"][:3] == [8, 16, 32]
    path = str(tmp_path / "net.ckpt")
    C.save(FakeNet(cfg), path)
    assert C.read(path)[0] == d


def test_payload_is_16_byte_aligned_and_sized():
    blob = C.encode(C.cfg_to_dict(_cfg()), np.arange(10, dtype=np.float32), np.arange(3, dtype=np.float32))
    assert (len(blob) - 4 * 13) % 16 == 0
    cfg, p, bn, meta = C.decode(blob)
    assert np.array_equal(p, np.arange(10, dtype=np.float32)) and np.array_equal(bn, np.arange(3, dtype=np.float32))


def test_configuration_mismatch_is_refused(tmp_path):
    path = str(tmp_path / "net.ckpt")
    C.save(FakeNet(_cfg(widths=(32, 64, 128, 256))), path)
    with pytest.raises(ValueError):
        C.load_into(FakeNet(_cfg(widths=(16, 32, 64, 128))), path)
    with pytest.raises(ValueError):
        C.load_into(FakeNet(_cfg(), n_params=999), path)


@pytest.mark.parametrize("damage", ["magic", "flip", "truncate", "version", "header"])
def test_damaged_files_are_refused(damage):
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
