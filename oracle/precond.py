"""FP64 CPU oracle: U-Net preconditioners and the training-pair generator.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  M_JU (Alg. 2):  e1 = Jacobi(0, r); e2 = e1 + U-Net(r - A e1); e = Jacobi(e2, r)
                  (damped Jacobi on the Helmholtz operator A, w = 0.8: a reading,
                  the algorithm names A^h but not the damping).
  M_VU (Eq. 3.4): e = V-cycle(e0 = U-Net(r), r) on the shifted Laplacian.
  U-Net(r) = s * net([Re, Im](h^2 r / s), kappa^2, gamma), s = RMS(h^2 r): the
  network runs in inference mode (BatchNorm with running statistics).
  Pairs (Eq. 3.8-3.9): b = A x, x~ = k iterations of FGMRES(10) + M_V from 0,
  r = b - A x~, e = x - x~.
  Residual loss (Remark after Eq. 3.7): |h^2 A e_net - h^2 r|^2 per sample, scaled by 1/s.
  Training batch (Sec. 3.4): pairs of one medium mixed by complex coefficients
  (augmentation by linear combinations), then the network input of the mixed residual
  and the mixed error in the same units as the network output (e / s).
"""
from __future__ import annotations

import numpy as np

from oracle import helmholtz as H
from oracle import unet as U


def unet_apply(prob: H.Problem, cfg, P, S, r, feats=None):
    """U-Net(r) for residuals r (B, ny, nx) complex."""
    lv = prob.hierarchy[0]
    x, s = U.make_input(r, lv.kappa2, lv.gamma, lv.h)
    out, _, _, _ = U.forward(cfg, P, S, x, train=False, feats=feats)
    return s[:, None, None] * (out[..., 0] + 1j * out[..., 1])


def precond_ju(prob: H.Problem, cfg, P, S, r, feats=None):
    A = prob.A
    w = prob.jacobi_w
    e1 = H.jacobi(A, np.zeros_like(r), r, w)
    e2 = e1 + unet_apply(prob, cfg, P, S, H.residual(A, r, e1), feats)
    return H.jacobi(A, e2, r, w)


def precond_vu(prob: H.Problem, cfg, P, S, r, feats=None):
    e0 = unet_apply(prob, cfg, P, S, r, feats)
    return np.stack([H.vcycle(prob, r[k], e0[k]) for k in range(r.shape[0])])


def encoder_features(prob: H.Problem, enc_cfg, Pe, Se):
    lv = prob.hierarchy[0]
    med = np.stack([lv.kappa2, lv.gamma], axis=-1)[None]
    _, _, _, feats = U.forward(enc_cfg, Pe, Se, med, train=False)
    return feats


def gen_pairs(prob: H.Problem, x, ks, m=10):
    """Eq. 3.8-3.9 for given draws x (count, ny, nx) and iteration counts ks."""
    A = prob.A
    rs, es = [], []
    for j in range(x.shape[0]):
        b = H.apply_op(A, x[j])
        res = H.fgmres(A, H.precond_v(prob), b, m=m, tol=0.0, maxit=int(ks[j]))
        xt = res.x
        rs.append(b - H.apply_op(A, xt))
        es.append(x[j] - xt)
    return np.stack(rs), np.stack(es)


def make_batch(prob: H.Problem, r, e, idx, coef):
    """Training batch of Sec. 3.4 from pairs (r, e) (npairs, ny, nx) complex of one medium.
    Sample i mixes the pairs idx[i, q] with coefficients coef[i, q] (the augmentation by
    linear combinations; one term with coefficient 1 = the pair itself):
        r' = sum_q coef[i, q] r[idx[i, q]],   e' likewise,
    input x[i] = ([Re, Im](h^2 r' / s), kappa^2, gamma) with s = RMS(h^2 r') (the network
    input of the preconditioners), target t[i] = [Re, Im](e' / s), the error in the units
    the network output is scaled back from.  Returns (x (B, ny, nx, 4), t (B, ny, nx, 2))."""
    lv = prob.hierarchy[0]
    idx = np.asarray(idx)
    coef = np.asarray(coef, dtype=np.complex128)
    rm = np.stack([sum(coef[i, q] * r[idx[i, q]] for q in range(idx.shape[1])) for i in range(idx.shape[0])])
    em = np.stack([sum(coef[i, q] * e[idx[i, q]] for q in range(idx.shape[1])) for i in range(idx.shape[0])])
    x, s = U.make_input(rm, lv.kappa2, lv.gamma, lv.h)
    t = np.stack([em.real, em.imag], axis=-1) / s[:, None, None, None]
    return x, t


def residual_loss(prob: H.Problem, y, x):
    """Unsupervised residual loss (the Remark following Eq. 3.7): the norm of A e_net - r
    in place of the error norm.  y: network outputs (B, ny, nx, 2) in target units
    (e / s), x: network inputs (B, ny, nx, 4) whose channels 0, 1 are h^2 r / s, so that
        rho = h^2 A (y0 + i y1) - (x0 + i x1) = h^2 (A e_net - r) / s.
    Loss: sum over the grid of |rho|^2, mean over the batch (the convention of Eq. 3.7
    here).  Gradient with respect to (Re y, Im y): (2 / B) conj(h^2 A^T conj(rho)), since
    the gradient of |K y - x|^2 with respect to conj(y) is K^H (K y - x) and
    K^H = conj(K^T) (A^T = A but for reflection boundaries).  Returns (loss, gradient
    (B, ny, nx, 2))."""
    A = prob.A
    h2 = A.h ** 2
    yc = y[..., 0] + 1j * y[..., 1]
    xc = x[..., 0] + 1j * x[..., 1]
    rho = h2 * H.apply_op(A, yc) - xc
    B = y.shape[0]
    loss = float(np.sum(np.abs(rho) ** 2) / B)
    g = (2.0 / B) * np.conj(h2 * H.apply_op_T(A, np.conj(rho)))
    return loss, np.stack([g.real, g.imag], axis=-1)


def flatten_params(cfg, P):
    """Flat float parameter vector in the library's order (include/unet.h)."""
    convs, bns = U.layer_specs(cfg)
    parts = [P[name].ravel() for name, *_ in convs]
    parts.append(P["up1.bias"])
    for name, _ in bns:
        parts.append(P[name + ".gamma"])
        parts.append(P[name + ".beta"])
    return np.concatenate(parts)


def unflatten_params(cfg, flat):
    convs, bns = U.layer_specs(cfg)
    P, o = {}, 0
    for name, kind, k, cin, cout in convs:
        n = k * k * cin * cout
        P[name] = flat[o:o + n].reshape(k, k, cin, cout).astype(np.float64)
        o += n
    P["up1.bias"] = flat[o:o + cfg.out_ch].astype(np.float64)
    o += cfg.out_ch
    for name, c in bns:
        P[name + ".gamma"] = flat[o:o + c].astype(np.float64)
        P[name + ".beta"] = flat[o + c:o + 2 * c].astype(np.float64)
        o += 2 * c
    return P


def flatten_bn(cfg, S):
    _, bns = U.layer_specs(cfg)
    return np.concatenate([S[n + ".mean"] for n, _ in bns] + [S[n + ".var"] for n, _ in bns])


def unflatten_bn(cfg, flat):
    _, bns = U.layer_specs(cfg)
    S, o = {}, 0
    for n, c in bns:
        S[n + ".mean"] = flat[o:o + c].astype(np.float64)
        o += c
    for n, c in bns:
        S[n + ".var"] = flat[o:o + c].astype(np.float64)
        o += c
    return S
