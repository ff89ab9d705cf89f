"""Pins of the U-Net oracle: layer identities from the paper's multigrid analogy
(Eq. 2.9 kernels inside Eq. 3.1/3.3 convolutions), adjointness, finite-difference
gradients, BatchNorm/eLU/Adam closed forms."""
import numpy as np
import pytest

from conftest import load_golden_kernels
from oracle import helmholtz as H
from oracle import unet as U


def _rng(seed):
    return np.random.default_rng(seed)


def test_strided_conv_with_full_weighting_kernel_is_restriction():
    """A 5x5 stride-2 convolution (pad 2) whose centre 3x3 holds K_{I_h^H} equals R (Eq. 2.9)."""
    gold = load_golden_kernels()["restrict"]
    x = _rng(1).standard_normal((2, 12, 16, 1))
    W = np.zeros((5, 5, 1, 1))
    W[1:4, 1:4, 0, 0] = gold
    out = U.conv2d(x, W, 2, 2)[..., 0]
    assert np.allclose(out, H.restrict_fw(x[..., 0]), atol=1e-14)


def test_transposed_conv_with_bilinear_kernel_is_prolongation():
    gold = load_golden_kernels()["prolong"]
    e = _rng(2).standard_normal((2, 6, 8, 1))
    W = np.zeros((5, 5, 1, 1))
    W[1:4, 1:4, 0, 0] = gold
    out = U.conv2d_transposed(e, W, 2, 2, 12, 16)[..., 0]
    assert np.allclose(out, H.prolong_bilinear(e[..., 0], 12, 16), atol=1e-14)


@pytest.mark.parametrize("k,s,p", [(5, 2, 2), (3, 1, 1)])
def test_transposed_conv_is_adjoint_of_conv(k, s, p):
    rng = _rng(3)
    x = rng.standard_normal((2, 10, 12, 3))
    W = rng.standard_normal((k, k, 3, 5))
    y = U.conv2d(x, W, s, p)
    z = rng.standard_normal(y.shape)
    xt = U.conv2d_transposed(z, W.transpose(0, 1, 3, 2), s, p, 10, 12)
    assert np.isclose(np.sum(y * z), np.sum(x * xt), rtol=1e-12)


def test_conv_matches_direct_sum():
    rng = _rng(4)
    x = rng.standard_normal((1, 7, 9, 2))
    W = rng.standard_normal((5, 5, 2, 3))
    out = U.conv2d(x, W, 2, 2)
    o, q, d = 2, 3, 1
    acc = 0.0
    for ky in range(5):
        for kx in range(5):
            iy, ix = 2 * o + ky - 2, 2 * q + kx - 2
            if 0 <= iy < 7 and 0 <= ix < 9:
                acc += x[0, iy, ix] @ W[ky, kx, :, d]
    assert np.isclose(out[0, o, q, d], acc, rtol=1e-13)


def test_bn_eval_identity_and_train_statistics():
    x = _rng(5).standard_normal((3, 4, 5, 6)) * 2 + 1
    y = U.bn_eval(x, np.ones(6), np.zeros(6), np.zeros(6), np.ones(6))
    assert np.allclose(y, x / np.sqrt(1 + U.BN_EPS), rtol=1e-15)
    yt, _ = U.bn_train(x, np.full(6, 2.0), np.full(6, 0.5))
    assert np.allclose(yt.mean(axis=(0, 1, 2)), 0.5, atol=1e-12)
    assert np.allclose(yt.var(axis=(0, 1, 2)), 4.0 * x.var(axis=(0, 1, 2)) / (x.var(axis=(0, 1, 2)) + U.BN_EPS))


def test_elu_values():
    x = np.array([-50.0, -1.0, 0.0, 0.5])
    assert np.allclose(U.elu(x), [np.expm1(-50.0), np.expm1(-1.0), 0.0, 0.5], rtol=0, atol=0)
    g = U.elu_backward(np.ones(4), x)
    assert np.allclose(g, [np.exp(-50.0), np.exp(-1.0), 1.0, 1.0])


def test_adam_first_step_closed_form():
    P = {"w": np.array([1.0, -2.0, 3.0])}
    G = {"w": np.array([0.5, -4.0, 1e-3])}
    M = {"w": np.zeros(3)}
    V = {"w": np.zeros(3)}
    U.adam_step(P, G, M, V, 1, 1e-4)
    expect = np.array([1.0, -2.0, 3.0]) - 1e-4 * G["w"] / (np.abs(G["w"]) + 1e-8)
    assert np.allclose(P["w"], expect, rtol=1e-14)


def test_architecture_shapes_and_channels():
    cfg = U.UNetConfig()
    convs, bns = U.layer_specs(cfg)
    names = [c[0] for c in convs]
    assert names[:3] == ["down1", "res1.0.k1", "res1.0.k2"]
    assert sum(1 for n in names if n.startswith("res4")) == 6       # 3 ResNets at the coarsest level
    d = {c[0]: c for c in convs}
    assert d["down1"][3:] == (4, 32) and d["down4"][3:] == (128, 256)
    assert d["up4"][3:] == (256, 128) and d["up3"][3:] == (256, 64) and d["up2"][3:] == (128, 32)
    assert d["up1"][3:] == (64, 2)
    P = U.init_params(cfg, 0)
    S = U.init_bn_stats(cfg)
    x = _rng(6).standard_normal((1, 32, 32, 4))
    out, _, _, feats = U.forward(cfg, P, S, x)
    assert out.shape == (1, 32, 32, 2)
    assert [f.shape[1:] for f in feats] == [(32, 32, 2), (16, 16, 32), (8, 8, 64), (4, 4, 128), (2, 2, 256)]


def _tiny(context=None):
    return U.UNetConfig(in_ch=4, out_ch=2, widths=(4, 8), coarse_resnets=2, context=context)


def _fd_check(f, params, grads, keys, rng, n=4, eps=1e-5):
    worst = 0.0
    for k in keys:
        for _ in range(n):
            idx = tuple(rng.integers(0, s) for s in params[k].shape)
            old = params[k][idx]
            params[k][idx] = old + eps
            fp = f()
            params[k][idx] = old - eps
            fm = f()
            params[k][idx] = old
            fd = (fp - fm) / (2 * eps)
            worst = max(worst, abs(fd - grads[k][idx]) / max(abs(fd), 1e-3))
    return worst


def test_backward_matches_finite_differences():
    """Every parameter group and the input: analytic gradient of the train-mode MSE loss
    equals central finite differences (FP64, tiny net, 8x8 grid, batch 2)."""
    cfg = _tiny()
    rng = _rng(7)
    P = U.init_params(cfg, 3)
    for k in P:
        if k.endswith(".beta") or k.endswith(".gamma") or k.endswith("bias"):
            P[k] = P[k] + 0.1 * rng.standard_normal(P[k].shape)
    S = U.init_bn_stats(cfg)
    x = rng.standard_normal((2, 8, 8, 4))
    tgt = rng.standard_normal((2, 8, 8, 2))
    out, cache, _, _ = U.forward(cfg, P, S, x, train=True)
    loss, gout = U.mse_loss(out, tgt)
    G, gx, _ = U.backward(cfg, P, cache, gout)

    def f():
        return U.mse_loss(U.forward(cfg, P, S, x, train=True)[0], tgt)[0]

    assert _fd_check(f, P, G, list(P.keys()), rng, n=2) < 1e-6
    # input gradient
    worst = 0.0
    for _ in range(6):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        old = x[idx]
        x[idx] = old + 1e-5
        fp = f()
        x[idx] = old - 1e-5
        fm = f()
        x[idx] = old
        fd = (fp - fm) / 2e-5
        worst = max(worst, abs(fd - gx[idx]) / max(abs(fd), 1e-3))
    assert worst < 1e-6


def test_encoder_solver_backward_matches_finite_differences():
    """Solver with encoder context (Eq. 3.5): gradients w.r.t. solver parameters and the
    context features (through which the encoder is trained) match finite differences."""
    enc_cfg = U.UNetConfig(in_ch=2, out_ch=4, widths=(4, 8), coarse_resnets=1)
    ctx = U.context_channels(enc_cfg)
    cfg = _tiny(context=ctx)
    rng = _rng(8)
    Pe = U.init_params(enc_cfg, 4)
    Pe.update({k: v + 0.1 * rng.standard_normal(v.shape) for k, v in Pe.items() if k.endswith("beta")})
    P = U.init_params(cfg, 5)
    Se, S = U.init_bn_stats(enc_cfg), U.init_bn_stats(cfg)
    med = rng.standard_normal((2, 8, 8, 2))
    x = rng.standard_normal((2, 8, 8, 4))
    tgt = rng.standard_normal((2, 8, 8, 2))

    def total():
        _, _, _, fe = U.forward(enc_cfg, Pe, Se, med, train=True)
        out = U.forward(cfg, P, S, x, train=True, feats=fe)[0]
        return U.mse_loss(out, tgt)[0]

    _, ce, _, fe = U.forward(enc_cfg, Pe, Se, med, train=True)
    out, cache, _, _ = U.forward(cfg, P, S, x, train=True, feats=fe)
    _, gout = U.mse_loss(out, tgt)
    G, _, gfe = U.backward(cfg, P, cache, gout)
    assert _fd_check(total, P, G, ["down1", "down2", "up2", "up1", "res2.0.k1"], rng, n=3) < 1e-6
    Ge = U.backward_features(enc_cfg, Pe, ce, gfe)
    assert _fd_check(total, Pe, Ge, ["down1", "res2.0.k2", "up2", "up1", "up2.bn.gamma"], rng, n=3) < 1e-6


def _small_problem(n=8, seed=3, bc="dirichlet"):
    rng = np.random.default_rng(seed)
    k2 = rng.uniform(0.25, 1.0, (n, n))
    return H.Problem(k2, omega=0.2 * np.pi * n, h=1.0 / n, abc_width=2, levels=1, bc=bc), rng


@pytest.mark.parametrize("bc", ["dirichlet", "reflect", "replicate"])
def test_residual_loss_gradient_matches_finite_differences(bc):
    # the residual-loss gradient (Remark after Eq. 3.7) against central differences of the
    # loss, for every boundary mode (reflection makes A unsymmetric: the gradient needs A^T)
    from oracle import precond as PR
    prob, rng = _small_problem(bc=bc)
    y = rng.standard_normal((2, 8, 8, 2))
    x = rng.standard_normal((2, 8, 8, 4))
    loss, g = PR.residual_loss(prob, y, x)
    for _ in range(4):
        d = rng.standard_normal(y.shape)
        eps = 1e-6
        fd = (PR.residual_loss(prob, y + eps * d, x)[0] - PR.residual_loss(prob, y - eps * d, x)[0]) / (2 * eps)
        assert abs(fd - np.sum(g * d)) <= 1e-7 * max(1.0, abs(fd))
    # and against the closed form sum |K y - x|^2 / B with the dense operator
    K = H.assemble_dense(prob.A) * prob.h ** 2
    yc = (y[..., 0] + 1j * y[..., 1]).reshape(2, -1)
    xc = (x[..., 0] + 1j * x[..., 1]).reshape(2, -1)
    ref = sum(np.linalg.norm(K @ yc[b] - xc[b]) ** 2 for b in range(2)) / 2
    assert abs(loss - ref) <= 1e-10 * ref


def test_residual_loss_vanishes_at_the_error():
    # y = e / s with A e = r: rho = 0 (the unsupervised loss is minimal at the exact error)
    from oracle import precond as PR
    prob, rng = _small_problem(seed=4)
    x = rng.standard_normal((1, 8, 8, 4))
    K = H.assemble_dense(prob.A) * prob.h ** 2
    e = np.linalg.solve(K, (x[0, ..., 0] + 1j * x[0, ..., 1]).ravel()).reshape(8, 8)
    y = np.stack([e.real, e.imag], axis=-1)[None]
    loss, g = PR.residual_loss(prob, y, x)
    assert loss <= 1e-20 * np.sum(x[..., :2] ** 2) and np.abs(g).max() <= 1e-9


# ---------------------------------------------------------------- preconditioners and pairs
def _precond_problem(n=16, seed=11):
    k2 = _rng(seed).uniform(0.25, 1.0, (n, n))
    return H.Problem(k2, omega=0.2 * np.pi * n, h=1.0 / n, abc_width=3, levels=2)


def _net(seed, silent=False):
    cfg = _tiny()
    P = U.init_params(cfg, seed)
    S = U.init_bn_stats(cfg)
    if silent:
        P["up1"][:] = 0.0
        P["up1.bias"][:] = 0.0
    return cfg, P, S


def _crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_silent_network_reduces_the_preconditioners_to_their_multigrid_parts():
    """A network whose output layer is zero returns 0: M_VU (Eq. 3.4) is then the SL
    V-cycle from zero (M_V), and M_JU (Alg. 2) two damped Jacobi sweeps on A."""
    from oracle import precond as PR
    prob = _precond_problem()
    cfg, P, S = _net(1, silent=True)
    r = _crandn(_rng(12), (2, 16, 16))
    assert np.array_equal(PR.unet_apply(prob, cfg, P, S, r), np.zeros_like(r))
    vu = PR.precond_vu(prob, cfg, P, S, r)
    ju = PR.precond_ju(prob, cfg, P, S, r)
    w = prob.jacobi_w
    for k in range(2):
        assert np.allclose(vu[k], H.vcycle(prob, r[k]), rtol=1e-14, atol=0)
        e1 = H.jacobi(prob.A, np.zeros_like(r[k]), r[k], w)
        assert np.allclose(ju[k], H.jacobi(prob.A, e1, r[k], w), rtol=1e-14, atol=0)


def test_network_preconditioner_is_positively_homogeneous():
    """The input is h^2 r / s with s = RMS(h^2 r) and the output is scaled back by s, so
    U-Net(c r) = c U-Net(r) for c > 0, whatever the weights; M_VU and M_JU inherit it
    (their multigrid parts are linear)."""
    from oracle import precond as PR
    prob = _precond_problem()
    cfg, P, S = _net(2)
    r = _crandn(_rng(13), (2, 16, 16))
    for c in (1e-6, 3.7, 1e5):
        assert np.allclose(PR.unet_apply(prob, cfg, P, S, c * r), c * PR.unet_apply(prob, cfg, P, S, r), rtol=1e-9)
        assert np.allclose(PR.precond_vu(prob, cfg, P, S, c * r), c * PR.precond_vu(prob, cfg, P, S, r), rtol=1e-9)
        assert np.allclose(PR.precond_ju(prob, cfg, P, S, c * r), c * PR.precond_ju(prob, cfg, P, S, r), rtol=1e-9)
    # and not in the phase: the network sees Re and Im as separate channels
    assert not np.allclose(PR.unet_apply(prob, cfg, P, S, 1j * r), 1j * PR.unet_apply(prob, cfg, P, S, r))


def test_network_input_channels():
    """Channels 0-1 of the input have unit mean square per sample; 2-3 carry the medium;
    a zero residual gives a zero input (s = 1)."""
    lv = _precond_problem().A
    r = _crandn(_rng(14), (3, 16, 16)) * np.array([1e-3, 1.0, 1e4])[:, None, None]
    r[1] = 0.0
    x, s = U.make_input(r, lv.kappa2, lv.gamma, lv.h)
    ms = np.mean(x[..., 0] ** 2 + x[..., 1] ** 2, axis=(1, 2))
    assert np.allclose(ms[[0, 2]], 1.0, rtol=1e-12) and ms[1] == 0.0 and s[1] == 1.0
    assert np.allclose(s[0], lv.h ** 2 * np.sqrt(np.mean(np.abs(r[0]) ** 2)), rtol=1e-12)
    assert np.array_equal(x[0, ..., 2], lv.kappa2) and np.array_equal(x[2, ..., 3], lv.gamma)


def test_generated_pairs_satisfy_the_error_equation():
    """Eq. 3.8-3.9: A e = r for every pair; k = 0 leaves x~ = 0 (r = A x, e = x); the
    FGMRES residual, and so ||r||, does not grow with k."""
    from oracle import precond as PR
    prob = _precond_problem()
    x = np.repeat(_crandn(_rng(15), (1, 16, 16)), 6, axis=0)
    ks = np.array([0, 1, 3, 9, 10, 14])
    r, e = PR.gen_pairs(prob, x, ks)
    for j in range(len(ks)):
        assert np.allclose(H.apply_op(prob.A, e[j]), r[j], rtol=1e-10, atol=1e-10 * np.abs(r[j]).max())
    assert np.array_equal(e[0], x[0]) and np.allclose(r[0], H.apply_op(prob.A, x[0]))
    norms = [np.linalg.norm(r[j]) for j in range(len(ks))]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(norms, norms[1:]))
    assert norms[-1] < 0.5 * norms[0]


def test_training_batch_keeps_the_error_equation_in_network_units():
    """Sec. 3.4's batch: mixing pairs of one medium by the same complex coefficients keeps
    A e' = r' (linearity), and the target is the error in the units of the network output,
    so h^2 A (t0 + i t1) = x0 + i x1 exactly: the residual loss of the target is zero.  A
    coefficient applied to r but not to e (or conjugated for one of them), or a target
    without the 1/s or with an extra h^2, breaks it."""
    from oracle import precond as PR
    prob = _precond_problem()
    A = prob.A
    rng = _rng(21)
    e = _crandn(rng, (5, 16, 16))
    r = np.stack([H.apply_op(A, e[j]) for j in range(5)])
    idx = np.array([[0, 3], [4, 4], [2, 1]])
    coef = _crandn(rng, (3, 2)) / np.sqrt(2)
    x, t = PR.make_batch(prob, r, e, idx, coef)
    assert x.shape == (3, 16, 16, 4) and t.shape == (3, 16, 16, 2)
    h2 = A.h ** 2
    for i in range(3):
        tc = t[i, ..., 0] + 1j * t[i, ..., 1]
        xc = x[i, ..., 0] + 1j * x[i, ..., 1]
        assert np.abs(h2 * H.apply_op(A, tc) - xc).max() <= 1e-11 * np.abs(xc).max()
    loss, _ = PR.residual_loss(prob, t, x)
    assert loss <= 1e-20 * np.sum(x[..., :2] ** 2)
    # channels 0-1 of the mixed input have unit mean square; 2-3 carry the medium
    ms = np.mean(x[..., 0] ** 2 + x[..., 1] ** 2, axis=(1, 2))
    assert np.allclose(ms, 1.0, rtol=1e-12)
    assert np.array_equal(x[1, ..., 2], A.kappa2) and np.array_equal(x[2, ..., 3], A.gamma)


def test_training_batch_selects_and_mixes_the_named_pairs():
    """One term with coefficient 1 is the pair itself (the network input of the
    preconditioners and e / s); a zero coefficient drops its pair; the mixture with
    coefficients (a, b) is a r_i + b r_j, scaled by its own RMS."""
    from oracle import precond as PR
    prob = _precond_problem()
    lv = prob.A
    rng = _rng(22)
    r, e = _crandn(rng, (4, 16, 16)), _crandn(rng, (4, 16, 16))
    x, t = PR.make_batch(prob, r, e, np.array([[2]]), np.ones((1, 1)))
    xr, s = U.make_input(r[2:3], lv.kappa2, lv.gamma, lv.h)
    assert np.array_equal(x, xr)
    assert np.allclose(t[0, ..., 0] + 1j * t[0, ..., 1], e[2] / s[0], rtol=1e-15, atol=0)
    x2, t2 = PR.make_batch(prob, r, e, np.array([[2, 0]]), np.array([[1.0, 0.0]]))
    assert np.allclose(x2, x, rtol=1e-14, atol=0) and np.allclose(t2, t, rtol=1e-14, atol=0)
    a, b = 0.3 - 1.1j, -0.7 + 0.2j
    x3, t3 = PR.make_batch(prob, r, e, np.array([[1, 3]]), np.array([[a, b]]))
    mix = a * r[1] + b * r[3]
    s3 = lv.h ** 2 * np.sqrt(np.mean(np.abs(mix) ** 2))
    assert np.allclose(x3[0, ..., 0] + 1j * x3[0, ..., 1], lv.h ** 2 * mix / s3, rtol=1e-13, atol=0)
    assert np.allclose(t3[0, ..., 0] + 1j * t3[0, ..., 1], (a * e[1] + b * e[3]) / s3, rtol=1e-13, atol=0)


def test_solver_with_silent_context_is_the_standalone_network():
    """Eq. 3.5: the solver network sees cat(own channels, f^(l)) at every level.  With the
    weights on the context channels zero, it equals the standalone network built from its
    other weights, whatever the encoder features are."""
    ctx = (3, 5, 6)
    solver = U.UNetConfig(in_ch=4, out_ch=2, widths=(4, 8), coarse_resnets=2, context=ctx)
    plain = _tiny()
    Pp = U.init_params(plain, 4)
    S = U.init_bn_stats(plain)
    rng = _rng(31)
    for k in S:
        S[k] = 0.1 * rng.standard_normal(S[k].shape) if k.endswith(".mean") else rng.uniform(0.5, 2.0, S[k].shape)
    Ps = dict(Pp)
    convs_s, _ = U.layer_specs(solver)
    convs_p = {c[0]: c for c in U.layer_specs(plain)[0]}
    for name, kind, k, cin, cout in convs_s:
        cin_plain = convs_p[name][3]
        W = np.zeros((k, k, cin, cout))
        W[:, :, :cin_plain, :] = Pp[name]
        Ps[name] = W
    x = rng.standard_normal((2, 8, 8, 4))
    feats = [rng.standard_normal((2, 8 >> l, 8 >> l, c)) for l, c in enumerate(ctx)]
    out_s, _, _, _ = U.forward(solver, Ps, S, x, train=False, feats=feats)
    out_p, _, _, _ = U.forward(plain, Pp, S, x, train=False)
    assert np.allclose(out_s, out_p, rtol=1e-13, atol=1e-13)
    Ps["down1"][:, :, 4:, :] = 1.0              # and the context does enter once its weights do
    assert not np.allclose(U.forward(solver, Ps, S, x, train=False, feats=feats)[0], out_p)


def test_flat_parameter_layout_round_trips():
    """The flat layouts the library's state functions use (weights layer by layer, the
    output bias, BN gamma/beta; BN means then variances) invert exactly, with the sizes
    the layer list implies."""
    from oracle import precond as PR
    for cfg in (_tiny(), _tiny(context=(3, 5, 6)), U.UNetConfig()):
        P = U.init_params(cfg, 9)
        flat = PR.flatten_params(cfg, P)
        convs, bns = U.layer_specs(cfg)
        assert flat.size == sum(k * k * ci * co for _, _, k, ci, co in convs) + cfg.out_ch + 2 * sum(c for _, c in bns)
        back = PR.unflatten_params(cfg, flat)
        assert back.keys() == P.keys() and all(np.array_equal(back[k], P[k]) for k in P)
        S = {k: _rng(10).standard_normal(v.shape) for k, v in U.init_bn_stats(cfg).items()}
        Sb = PR.unflatten_bn(cfg, PR.flatten_bn(cfg, S))
        assert all(np.array_equal(Sb[k], S[k]) for k in S)
        assert np.array_equal(PR.flatten_bn(cfg, S)[:bns[0][1]], S[bns[0][0] + ".mean"])
