"""Training of the U-Net preconditioners (Sec. 3.4, 3.5) through libhelm's C ABI.

Host-side orchestration only: choosing which pairs form a batch, the
augmentation coefficients, epochs and the learning-rate schedule.  Pair
generation (Eq. 3.8-3.9), batch assembly (unet_make_batch) and the training
step (unet_train_step: forward, MSE loss of Eq. 3.7 or the residual loss,
backward, Adam) run in the library's CUDA kernels.
"""
from __future__ import annotations

import numpy as np


def lr_at(epoch: int, lr0: float, t0: int = 48, floor: float = 1e-7) -> float:
    """Sec. 4 schedule: the learning rate drops 10x at epoch t0 and then after every
    t_i = t0 / 2^i further epochs (48, 72, 84, 90, ... for t0 = 48)."""
    lr, e, t = lr0, t0, t0
    while epoch >= e and t >= 1:
        lr /= 10.0
        t //= 2
        e += max(t, 1)
    return max(lr, floor)


def batches(rng, npairs: int, batch: int, nmix: int):
    """One epoch: every pair once as the lead term, mixed with nmix - 1 random partners
    using complex-normal coefficients (augmentation by linear combinations, Sec. 3.4)."""
    perm = rng.permutation(npairs)
    for s in range(0, npairs - batch + 1, batch):
        lead = perm[s:s + batch]
        idx = np.empty((batch, nmix), np.int32)
        idx[:, 0] = lead
        if nmix > 1:
            idx[:, 1:] = rng.integers(0, npairs, (batch, nmix - 1))
        coef = (rng.standard_normal((batch, nmix)) + 1j * rng.standard_normal((batch, nmix))) / np.sqrt(2)
        if nmix == 1:
            coef[:] = 1.0
        yield idx, coef


def train(hz, net, pairs=None, npairs: int = 256, epochs: int = 10, batch: int = 16, lr: float = 1e-3,
          seed: int = 0, nmix: int = 2, kmax: int = 10, schedule_t0: int | None = None, log=None,
          loss: str = "error"):
    """Train `net` on pairs of one medium (hz).  With an attached encoder the pair is
    trained jointly (encoder forward in training mode before each step).  loss="error"
    is Eq. 3.7 (supervised, the error of each pair); loss="residual" is the unsupervised
    residual norm of the Remark following Eq. 3.7 (only the residuals are used).
    Returns the per-epoch mean loss."""
    import torch
    if loss not in ("error", "residual"):
        raise ValueError(f"unknown loss {loss!r}")
    if pairs is None:
        pairs = hz.gen_pairs(npairs, seed, kmax)
    r, e = pairs
    rng = np.random.default_rng(seed + 1)
    history = []
    for ep in range(epochs):
        cur = lr if schedule_t0 is None else lr_at(ep, lr, schedule_t0)
        losses = []
        for idx, coef in batches(rng, r.shape[0], batch, nmix):
            x, t = hz.make_batch(r, e, idx, coef)
            # encoder forward (if attached), forward, loss, backward and Adam in one C-ABI call
            losses.append(net.train_step(hz, x, t if loss == "error" else None, lr=cur, loss=loss))
        m = float(torch.stack(losses).mean().item()) if losses else float("nan")
        history.append(m)
        if log:
            log(f"epoch {ep} lr {cur:.2e} loss {m:.4f}")
    return history


def train_media(media, net, epochs: int = 10, batch: int = 16, lr: float = 1e-3, seed: int = 0, nmix: int = 2,
                schedule_t0: int | None = None, log=None, loss: str = "error"):
    """Train `net` on pairs of many media (the general network of Sec. 3.4.1 / 4, trained on
    pairs generated on random media): media is a list of (hz, (r, e)), one Helmholtz handle
    per medium with its Eq. 3.8-3.9 pairs.  An epoch takes every medium's batches (pairs of
    one medium mixed with each other, as the augmentation reads) in a random interleaving,
    so consecutive steps see different media.  Returns the per-epoch mean loss."""
    import torch
    if loss not in ("error", "residual"):
        raise ValueError(f"unknown loss {loss!r}")
    rng = np.random.default_rng(seed + 1)
    history = []
    for ep in range(epochs):
        cur = lr if schedule_t0 is None else lr_at(ep, lr, schedule_t0)
        plan = []
        for mi, (_, (r, _)) in enumerate(media):
            plan += [(mi, idx, coef) for idx, coef in batches(rng, r.shape[0], batch, nmix)]
        order = rng.permutation(len(plan))
        losses = []
        for o in order:
            mi, idx, coef = plan[o]
            hz, (r, e) = media[mi]
            x, t = hz.make_batch(r, e, idx, coef)
            losses.append(net.train_step(hz, x, t if loss == "error" else None, lr=cur, loss=loss))
        m = float(torch.stack(losses).mean().item()) if losses else float("nan")
        history.append(m)
        if log:
            log(f"epoch {ep} lr {cur:.2e} loss {m:.4f}")
    return history


def relative_error(hz, net, pairs, count: int = 16) -> float:
    """Mean ||U-Net(r) - e|| / ||e|| over the first `count` pairs (the 'average relative
    error' of Sec. 4), with the network in inference mode."""
    import torch
    r, e = pairs
    n = min(count, r.shape[0])
    if net.encoder is not None:
        net.encode(hz, train=False)
    out = torch.empty_like(r[:n])
    # preconditioner-free application: U-Net alone (input scaling as in M_JU / M_VU)
    idx = np.arange(n, dtype=np.int32)[:, None]
    x, t = hz.make_batch(r, e, idx, np.ones((n, 1), complex))
    y = net.forward(x, train=False)
    num = torch.linalg.vector_norm((y - t).reshape(n, -1), dim=1)
    den = torch.linalg.vector_norm(t.reshape(n, -1), dim=1)
    del out
    return float((num / den).mean().item())
