"""FP64 CPU oracle: the U-Net preconditioner network, its backward pass, Adam.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy, float64,
activations NHWC (batch, y, x, channel), weights (ky, kx, cin, cout).

Architecture (Sec. 3.1; channel widths were only in a figure the text lacks,
so the widths are a reading: 4 levels, 32 -> 256 channels):
  down level l = 1..4 (Eq. 3.1): x_l = eLU(BN(R_l x_{l-1})), R_l a 5x5 stride-2
      convolution (pad 2) doubling the channels (input 4 -> 32);
      then one ResNet block (Eq. 3.2) on levels 1..3 and three on level 4:
      x <- eLU(BN(x + K2 eLU(BN(K1 x)))), K1, K2 3x3 convolutions (pad 1).
  up level l = 4..2 (Eq. 3.3): u <- cat(BN(P_l eLU(u)), x_{l-1}), P_l a 5x5
      stride-2 transposed convolution (pad 2, output padding 1) halving the
      channels; the last up layer maps eLU(u) to 2 output channels
      (Re e, Im e) with a bias and no BN.
  input channels: Re and Im of the scaled residual, kappa^2, gamma (Sec. 3.4).
Encoder-solver (Sec. 3.3, Eq. 3.5): the encoder is the same U-Net on
(kappa^2, gamma) with 4 output channels; its features f^(l) are the coarsest
ResNet output (level 4), the up-path BN(P eLU(u)) tensors (levels 3..1) and
its output (level 0).  The solver concatenates f^(l) to the input of every
down convolution R_l and of every up convolution P_l (before the eLU).

BatchNorm (Sec. 3.1): batch statistics in training, running statistics
(momentum 0.1, eps 1e-5) in inference.  eLU: x if x > 0 else exp(x) - 1.
Conv layers followed by BN carry no bias (BN's shift subsumes it).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BN_EPS = 1e-5
BN_MOMENTUM = 0.1


# ----------------------------------------------------------------------------
# primitive layers: forward and backward
# ----------------------------------------------------------------------------
def conv2d(x, W, stride, pad):
    """out[b,o,p,d] = sum_{ky,kx,c} x[b, s o + ky - pad, s p + kx - pad, c] W[ky,kx,c,d]."""
    B, H, Wd, C = x.shape
    k = W.shape[0]
    Ho = (H + 2 * pad - k) // stride + 1
    Wo = (Wd + 2 * pad - k) // stride + 1
    xp = np.zeros((B, H + 2 * pad, Wd + 2 * pad, C))
    xp[:, pad:pad + H, pad:pad + Wd] = x
    out = np.zeros((B, Ho, Wo, W.shape[3]))
    for ky in range(k):
        for kx in range(k):
            patch = xp[:, ky:ky + stride * (Ho - 1) + 1:stride, kx:kx + stride * (Wo - 1) + 1:stride]
            out += np.einsum("bhwc,cd->bhwd", patch, W[ky, kx], optimize=True)
    return out


def conv2d_backward(g, x, W, stride, pad):
    B, H, Wd, C = x.shape
    k = W.shape[0]
    Ho, Wo = g.shape[1:3]
    xp = np.zeros((B, H + 2 * pad, Wd + 2 * pad, C))
    xp[:, pad:pad + H, pad:pad + Wd] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for ky in range(k):
        for kx in range(k):
            sl = (slice(None), slice(ky, ky + stride * (Ho - 1) + 1, stride), slice(kx, kx + stride * (Wo - 1) + 1, stride))
            gW[ky, kx] = np.einsum("bhwc,bhwd->cd", xp[sl], g, optimize=True)
            gxp[sl] += np.einsum("bhwd,cd->bhwc", g, W[ky, kx], optimize=True)
    return gxp[:, pad:pad + H, pad:pad + Wd], gW


def conv2d_transposed(x, W, stride, pad, out_h, out_w):
    """Transposed convolution: out[b, s i + ky - pad, s j + kx - pad, d] += x[b,i,j,c] W[ky,kx,c,d],
    cropped to (out_h, out_w) (output padding fills the far edge)."""
    B, H, Wd, C = x.shape
    k = W.shape[0]
    full_h = max(stride * (H - 1) + k, out_h + pad)
    full_w = max(stride * (Wd - 1) + k, out_w + pad)
    outp = np.zeros((B, full_h, full_w, W.shape[3]))
    for ky in range(k):
        for kx in range(k):
            outp[:, ky:ky + stride * (H - 1) + 1:stride, kx:kx + stride * (Wd - 1) + 1:stride] += \
                np.einsum("bhwc,cd->bhwd", x, W[ky, kx], optimize=True)
    return outp[:, pad:pad + out_h, pad:pad + out_w]


def conv2d_transposed_backward(g, x, W, stride, pad):
    B, H, Wd, C = x.shape
    k = W.shape[0]
    out_h, out_w = g.shape[1:3]
    full_h = max(stride * (H - 1) + k, out_h + pad)
    full_w = max(stride * (Wd - 1) + k, out_w + pad)
    gp = np.zeros((B, full_h, full_w, g.shape[3]))
    gp[:, pad:pad + out_h, pad:pad + out_w] = g
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for ky in range(k):
        for kx in range(k):
            gs = gp[:, ky:ky + stride * (H - 1) + 1:stride, kx:kx + stride * (Wd - 1) + 1:stride]
            gx += np.einsum("bhwd,cd->bhwc", gs, W[ky, kx], optimize=True)
            gW[ky, kx] = np.einsum("bhwc,bhwd->cd", x, gs, optimize=True)
    return gx, gW


def elu(x):
    return np.where(x > 0, x, np.expm1(np.minimum(x, 0.0)))


def elu_backward(g, x):
    return g * np.where(x > 0, 1.0, np.exp(np.minimum(x, 0.0)))


def bn_train(x, gamma, beta):
    mu = x.mean(axis=(0, 1, 2))
    var = x.var(axis=(0, 1, 2))
    xhat = (x - mu) / np.sqrt(var + BN_EPS)
    return gamma * xhat + beta, (xhat, var, mu)


def bn_train_backward(g, cache, gamma):
    xhat, var, _ = cache
    n = g.shape[0] * g.shape[1] * g.shape[2]
    ggamma = np.sum(g * xhat, axis=(0, 1, 2))
    gbeta = np.sum(g, axis=(0, 1, 2))
    gx = gamma / np.sqrt(var + BN_EPS) * (g - gbeta / n - xhat * ggamma / n)
    return gx, ggamma, gbeta


def bn_eval(x, gamma, beta, rmean, rvar):
    return gamma * (x - rmean) / np.sqrt(rvar + BN_EPS) + beta


# ----------------------------------------------------------------------------
# network description
# ----------------------------------------------------------------------------
@dataclass
class UNetConfig:
    in_ch: int = 4                  # Re r, Im r, kappa^2, gamma
    out_ch: int = 2                 # Re e, Im e
    widths: tuple = (32, 64, 128, 256)
    coarse_resnets: int = 3
    context: tuple | None = None    # per-level feature channels (l = 0..4) for a solver net


def context_channels(cfg: UNetConfig):
    """Channels of the encoder features f^(0..4) for an encoder built from cfg."""
    w = cfg.widths
    return (cfg.out_ch,) + tuple(w[:-1]) + (w[-1],)


def layer_specs(cfg: UNetConfig):
    """Ordered list of (name, kind, ksize, cin, cout) for every convolution, plus BN names."""
    w = cfg.widths
    L = len(w)
    ctx = cfg.context or (0,) * (L + 1)
    convs, bns = [], []
    cin = cfg.in_ch
    for l in range(1, L + 1):
        convs.append((f"down{l}", "down", 5, cin + ctx[l - 1], w[l - 1]))
        bns.append((f"down{l}.bn", w[l - 1]))
        nres = cfg.coarse_resnets if l == L else 1
        for r in range(nres):
            convs.append((f"res{l}.{r}.k1", "same", 3, w[l - 1], w[l - 1]))
            bns.append((f"res{l}.{r}.bn1", w[l - 1]))
            convs.append((f"res{l}.{r}.k2", "same", 3, w[l - 1], w[l - 1]))
            bns.append((f"res{l}.{r}.bn2", w[l - 1]))
        cin = w[l - 1]
    ucin = w[L - 1]
    for l in range(L, 1, -1):
        cout = w[l - 2]
        convs.append((f"up{l}", "up", 5, ucin + ctx[l], cout))
        bns.append((f"up{l}.bn", cout))
        ucin = 2 * cout
    convs.append(("up1", "up", 5, ucin + ctx[1], cfg.out_ch))
    return convs, bns


def init_params(cfg: UNetConfig, seed: int):
    """He-normal weights (std sqrt(2 / fan_in)) from the seeded generator; BN gamma 1, beta 0."""
    from paper_2203_11025_gb300 import synth
    convs, bns = layer_specs(cfg)
    P = {}
    for i, (name, kind, k, cin, cout) in enumerate(convs):
        z = synth.normal(seed * 1000 + i, k * k * cin * cout).reshape(k, k, cin, cout)
        P[name] = z * np.sqrt(2.0 / (k * k * cin))
    P["up1.bias"] = np.zeros(cfg.out_ch)
    for name, c in bns:
        P[name + ".gamma"] = np.ones(c)
        P[name + ".beta"] = np.zeros(c)
    return P


def init_bn_stats(cfg: UNetConfig):
    _, bns = layer_specs(cfg)
    S = {}
    for name, c in bns:
        S[name + ".mean"] = np.zeros(c)
        S[name + ".var"] = np.ones(c)
    return S


# ----------------------------------------------------------------------------
# forward / backward, written block by block so each mirrors the equations
# ----------------------------------------------------------------------------
def _bn_fwd(x, name, P, S, train, new_stats):
    if not train:
        return bn_eval(x, P[name + ".gamma"], P[name + ".beta"], S[name + ".mean"], S[name + ".var"]), None
    y, cache = bn_train(x, P[name + ".gamma"], P[name + ".beta"])
    n = x.shape[0] * x.shape[1] * x.shape[2]
    mu, var = cache[2], cache[1]
    new_stats[name + ".mean"] = (1 - BN_MOMENTUM) * S[name + ".mean"] + BN_MOMENTUM * mu
    new_stats[name + ".var"] = (1 - BN_MOMENTUM) * S[name + ".var"] + BN_MOMENTUM * var * n / max(n - 1, 1)
    return y, cache


def _bn_bwd(g, name, cache, P, G):
    gx, gg, gb = bn_train_backward(g, cache, P[name + ".gamma"])
    G[name + ".gamma"] += gg
    G[name + ".beta"] += gb
    return gx


def _resnet_fwd(h, pre, P, S, train, st):
    """Eq. 3.2: eLU(BN(h + K2 eLU(BN(K1 h))))."""
    t1 = conv2d(h, P[pre + ".k1"], 1, 1)
    t1n, c1 = _bn_fwd(t1, pre + ".bn1", P, S, train, st)
    a1 = elu(t1n)
    t2 = conv2d(a1, P[pre + ".k2"], 1, 1)
    s = h + t2
    sn, c2 = _bn_fwd(s, pre + ".bn2", P, S, train, st)
    return elu(sn), (h, t1n, c1, a1, sn, c2)


def _resnet_bwd(g, pre, cache, P, G):
    h, t1n, c1, a1, sn, c2 = cache
    g = _bn_bwd(elu_backward(g, sn), pre + ".bn2", c2, P, G)
    g_h = g                                         # identity branch
    ga1, gW = conv2d_backward(g, a1, P[pre + ".k2"], 1, 1)
    G[pre + ".k2"] += gW
    gt1 = _bn_bwd(elu_backward(ga1, t1n), pre + ".bn1", c1, P, G)
    gh2, gW = conv2d_backward(gt1, h, P[pre + ".k1"], 1, 1)
    G[pre + ".k1"] += gW
    return g_h + gh2


def forward(cfg: UNetConfig, P, S, x, train=False, feats=None):
    """Run the network on x (B, n, n, in_ch).  feats: encoder features f^(0..4) for a
    solver network.  Returns (out, cache, new_bn_stats, my_features)."""
    L = len(cfg.widths)
    st = {}
    my_feats = [None] * (L + 1)
    cache = {"down": [], "up": [], "feats_given": feats is not None}

    def with_ctx(t, l):
        return t if feats is None else np.concatenate([t, feats[l]], axis=3)

    skips = []
    h = x
    for l in range(1, L + 1):
        inp = with_ctx(h, l - 1)
        z = conv2d(inp, P[f"down{l}"], 2, 2)                          # Eq. 3.1
        zn, cb = _bn_fwd(z, f"down{l}.bn", P, S, train, st)
        h = elu(zn)
        res = []
        for r in range(cfg.coarse_resnets if l == L else 1):
            h, c = _resnet_fwd(h, f"res{l}.{r}", P, S, train, st)
            res.append(c)
        cache["down"].append((inp, zn, cb, res, h.shape[3] if feats is None else inp.shape[3] - feats[l - 1].shape[3]))
        if l < L:
            skips.append(h)
    my_feats[L] = h
    u = h
    for l in range(L, 1, -1):                                          # Eq. 3.3
        inp = with_ctx(u, l)
        a = elu(inp)
        z = conv2d_transposed(a, P[f"up{l}"], 2, 2, 2 * u.shape[1], 2 * u.shape[2])
        zn, cb = _bn_fwd(z, f"up{l}.bn", P, S, train, st)
        my_feats[l - 1] = zn
        cache["up"].append((inp, a, cb, u.shape[3], zn.shape[3]))
        u = np.concatenate([zn, skips[l - 2]], axis=3)
    inp = with_ctx(u, 1)
    a = elu(inp)
    out = conv2d_transposed(a, P["up1"], 2, 2, 2 * u.shape[1], 2 * u.shape[2]) + P["up1.bias"]
    cache["final"] = (inp, a, u.shape[3])
    my_feats[0] = out
    return out, cache, st, my_feats


def backward(cfg: UNetConfig, P, cache, gout, g_own_feats=None):
    """Gradient of sum(gout * out) (+ sum over l of g_own_feats[l] * my_features[l] for an
    encoder) w.r.t. every parameter, the input and (solver) the context features.  Needs
    the cache of a train-mode forward.  Returns (G, g_x, g_context_feats)."""
    L = len(cfg.widths)
    G = {k: np.zeros_like(v) for k, v in P.items()}
    g_feats = [None] * (L + 1)
    G["up1.bias"] = gout.sum(axis=(0, 1, 2))
    inp, a, cu = cache["final"]
    ga, gW = conv2d_transposed_backward(gout, a, P["up1"], 2, 2)
    G["up1"] += gW
    g = elu_backward(ga, inp)
    if cache["feats_given"]:
        g_feats[1] = g[..., cu:]
    g_u = g[..., :cu]
    g_skip = {}
    for idx, l in enumerate(range(2, L + 1)):                          # reverse of the up loop
        inp, a, cb, cu, cz = cache["up"][L - l]
        g_z, g_skip[l - 1] = g_u[..., :cz], g_u[..., cz:]
        if g_own_feats is not None and g_own_feats[l - 1] is not None:
            g_z = g_z + g_own_feats[l - 1]
        g_z = _bn_bwd(g_z, f"up{l}.bn", cb, P, G)
        ga, gW = conv2d_transposed_backward(g_z, a, P[f"up{l}"], 2, 2)
        G[f"up{l}"] += gW
        g = elu_backward(ga, inp)
        if cache["feats_given"]:
            g_feats[l] = g[..., cu:]
        g_u = g[..., :cu]
    g_h = g_u
    if g_own_feats is not None and g_own_feats[L] is not None:
        g_h = g_h + g_own_feats[L]
    for l in range(L, 0, -1):
        inp, zn, cb, res, ch = cache["down"][l - 1]
        if l < L:
            g_h = g_h + g_skip[l]
        nres = cfg.coarse_resnets if l == L else 1
        for r in range(nres - 1, -1, -1):
            g_h = _resnet_bwd(g_h, f"res{l}.{r}", res[r], P, G)
        g_z = _bn_bwd(elu_backward(g_h, zn), f"down{l}.bn", cb, P, G)
        g_in, gW = conv2d_backward(g_z, inp, P[f"down{l}"], 2, 2)
        G[f"down{l}"] += gW
        if cache["feats_given"]:
            nctx = inp.shape[3] - (cfg.in_ch if l == 1 else cfg.widths[l - 2])
            gf = g_in[..., inp.shape[3] - nctx:]
            g_feats[l - 1] = gf if g_feats[l - 1] is None else g_feats[l - 1] + gf   # f^(1) also feeds up1
            g_in = g_in[..., :inp.shape[3] - nctx]
        g_h = g_in
    return G, g_h, g_feats


def backward_features(cfg: UNetConfig, P, cache, g_feats):
    """Parameter gradients of an encoder whose features f^(0..L) received g_feats."""
    return backward(cfg, P, cache, g_feats[0], g_own_feats=g_feats)[0]


# ----------------------------------------------------------------------------
# input scaling, loss, Adam
# ----------------------------------------------------------------------------
def make_input(r, kappa2, gamma, h):
    """Network input for residuals r (B, n, n) complex: channels (Re, Im) of h^2 r / s with
    s = RMS(h^2 r) per sample (Sec. 3.4 scales by h^2; the RMS normalisation is a reading),
    then kappa^2 and gamma.  Returns (x, s)."""
    rh = h * h * r
    s = np.sqrt(np.mean(np.abs(rh) ** 2, axis=(1, 2)))
    s = np.where(s > 0, s, 1.0)
    B, ny, nx = r.shape
    x = np.zeros((B, ny, nx, 4))
    x[..., 0] = rh.real / s[:, None, None]
    x[..., 1] = rh.imag / s[:, None, None]
    x[..., 2] = kappa2
    x[..., 3] = gamma
    return x, s


def mse_loss(out, target):
    """Eq. 3.7: mean over samples of ||out - target||^2 (sum over grid and the 2 channels)."""
    B = out.shape[0]
    d = out - target
    return float(np.sum(d * d) / B), 2.0 * d / B


def adam_step(P, G, M, V, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam (Kingma & Ba) with bias correction; updates P, M, V in place; t is 1-based."""
    for k in P:
        M[k] = b1 * M[k] + (1 - b1) * G[k]
        V[k] = b2 * V[k] + (1 - b2) * G[k] * G[k]
        mhat = M[k] / (1 - b1 ** t)
        vhat = V[k] / (1 - b2 ** t)
        P[k] = P[k] - lr * mhat / (np.sqrt(vhat) + eps)
