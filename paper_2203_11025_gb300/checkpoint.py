"""Network checkpoints: save a trained U-Net (FP32 master weights and BatchNorm running
statistics, the state the preconditioners of Sec. 3 read) and load it back, so that a
network trained once can serve many solves.

File layout (little-endian):
    8 bytes   magic b"HLMUNET1"
    4 bytes   uint32 length L of the JSON header
    L bytes   JSON header: {"version", "cfg" (unet_cfg fields), "n_params", "n_bn",
              "crc32" (of the payload), "meta" (caller's dictionary)}
    padding   zeros up to a multiple of 16 bytes
    payload   float32[n_params] weights in the library's flat order (include/unet.h),
              then float32[n_bn] BatchNorm running means and variances

Adam moments are not part of the file: resuming training from a checkpoint restarts
the optimiser state.  Reading checks the magic, the version, the sizes and the CRC
and raises ValueError on any mismatch.

save / load_into / load go through the library's own reader and writer (unet_save,
unet_load in include/unet.h); encode / decode are the same layout in Python, for host-side
inspection and for checking the two against each other.
"""
from __future__ import annotations

import json
import struct
import zlib

import numpy as np

MAGIC = b"HLMUNET1"
VERSION = 1
_CFG_FIELDS = ("in_ch", "out_ch", "levels", "coarse_resnets", "widths", "context", "flags")


def cfg_to_dict(cfg) -> dict:
    """The unet_cfg fields as plain Python values (arrays as lists)."""
    out = {}
    for name in _CFG_FIELDS:
        v = getattr(cfg, name)
        out[name] = [int(e) for e in v] if not isinstance(v, int) else int(v)
    return out


def dict_to_cfg(d: dict):
    from . import lib
    cfg = lib.unet_cfg()
    for name in _CFG_FIELDS:
        v = d[name]
        if isinstance(v, list):
            arr = getattr(cfg, name)
            if len(v) != len(arr):
                raise ValueError(f"checkpoint cfg field {name} has {len(v)} entries, expected {len(arr)}")
            for i, e in enumerate(v):
                arr[i] = int(e)
        else:
            setattr(cfg, name, int(v))
    return cfg


def encode(cfg_dict: dict, params: np.ndarray, bn: np.ndarray, meta: dict | None = None) -> bytes:
    """The checkpoint bytes for a configuration, flat weights and BatchNorm statistics."""
    params = np.ascontiguousarray(params, dtype="<f4").ravel()
    bn = np.ascontiguousarray(bn, dtype="<f4").ravel()
    payload = params.tobytes() + bn.tobytes()
    header = json.dumps({"version": VERSION, "cfg": cfg_dict, "n_params": int(params.size), "n_bn": int(bn.size),
                         "crc32": zlib.crc32(payload), "meta": meta or {}}, sort_keys=True).encode()
    head = MAGIC + struct.pack("<I", len(header)) + header
    head += b"\0" * (-len(head) % 16)
    return head + payload


def decode(blob: bytes):
    """(cfg dict, weights, BatchNorm statistics, meta) from checkpoint bytes."""
    if len(blob) < 12 or blob[:8] != MAGIC:
        raise ValueError("not a U-Net checkpoint (bad magic)")
    (hlen,) = struct.unpack("<I", blob[8:12])
    if 12 + hlen > len(blob):
        raise ValueError("truncated checkpoint header")
    try:
        header = json.loads(blob[12:12 + hlen].decode())
    except (UnicodeDecodeError, json.JSONDecodeError) as exc:
        raise ValueError(f"unreadable checkpoint header: {exc}") from None
    if header.get("version") != VERSION:
        raise ValueError(f"checkpoint version {header.get('version')} (this reader: {VERSION})")
    start = 12 + hlen
    start += -start % 16
    n_params, n_bn = int(header["n_params"]), int(header["n_bn"])
    payload = blob[start:]
    if len(payload) != 4 * (n_params + n_bn):
        raise ValueError(f"checkpoint payload is {len(payload)} bytes, header says {4 * (n_params + n_bn)}")
    if zlib.crc32(payload) != header["crc32"]:
        raise ValueError("checkpoint payload CRC mismatch")
    data = np.frombuffer(payload, dtype="<f4")
    return header["cfg"], data[:n_params].astype(np.float32), data[n_params:].astype(np.float32), header["meta"]


def save(net, path: str, meta: dict | None = None) -> None:
    """Write net's weights and BatchNorm statistics (device state) with unet_save."""
    net.save(path, meta)


def read(path: str):
    with open(path, "rb") as f:
        return decode(f.read())


def load_into(net, path: str) -> dict:
    """Restore a checkpoint into an existing network of the same configuration (unet_load);
    returns meta."""
    from . import lib
    try:
        net.load(path)
    except lib.HelmError as exc:
        raise ValueError(str(exc)) from None
    return read(path)[3]


def load(path: str):
    """A new network (libhelm U-Net on the current GPU) restored from a checkpoint; returns (net, meta)."""
    from . import lib
    cfg, _, _, meta = read(path)
    net = lib.UNet(dict_to_cfg(cfg))
    try:
        net.load(path)
    except lib.HelmError as exc:
        net.close()
        raise ValueError(str(exc)) from None
    return net, meta
