"""GPU parity of the U-Net path against the FP64 oracle: forward (inference and
training BatchNorm), backward (every parameter group and the input), the
encoder-solver pair, Adam, the preconditioners M_JU / M_VU, and the
training-pair generator.

Tolerance: the network runs in BF16 (weights and activations, 8-bit mantissa,
unit roundoff 2^-9) with FP32 accumulation; over ~20 layers the normwise
relative error of the output stays near 5e-3 (measured on the full-width default
network: 5.3e-3 at 64^2, 5.8e-3 at 128^2), so forward checks use 2e-2 normwise
(the BF16 tolerance the design states) and gradient checks 5e-2 per parameter
group."""
import numpy as np
import pytest

from gpu_util import crandn, medium
from oracle import helmholtz as H
from oracle import precond as PR
from oracle import unet as U
from paper_2203_11025_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2203_11025_gb300 import build
    from paper_2203_11025_gb300 import lib as L
    build.build()
    return L


def nrel(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def make_cfgs(lib, widths=(8, 16), resnets=2, in_ch=4, out_ch=2, context=None, simt=False):
    """simt: False (tensor cores fed by TMA), True (CUDA cores) or "cpasync" (tensor cores fed by cp.async)."""
    c = lib.unet_cfg()
    c.in_ch, c.out_ch, c.levels, c.coarse_resnets = in_ch, out_ch, len(widths), resnets
    c.flags = {False: 0, True: lib.UNET_FLAG_SIMT, "cpasync": lib.UNET_FLAG_NO_TMA}[simt]
    for i, w in enumerate(widths):
        c.widths[i] = w
    if context:
        for i, v in enumerate(context):
            c.context[i] = v
    oc = U.UNetConfig(in_ch=in_ch, out_ch=out_ch, widths=tuple(widths), coarse_resnets=resnets,
                      context=tuple(context) if context else None)
    return c, oc


def randomise(lib, net, oc, seed):
    """Non-trivial BN parameters and running statistics, identical on both sides."""
    rng = np.random.default_rng(seed)
    P = U.init_params(oc, seed)
    for k in P:
        if k.endswith(".gamma"):
            P[k] = 1.0 + 0.2 * rng.standard_normal(P[k].shape)
        elif k.endswith(".beta") or k.endswith("bias"):
            P[k] = 0.1 * rng.standard_normal(P[k].shape)
    P = PR.unflatten_params(oc, PR.flatten_params(oc, P).astype(np.float32))   # the same float32 values
    S = U.init_bn_stats(oc)
    for k in S:
        S[k] = (0.05 * rng.standard_normal(S[k].shape)) if k.endswith(".mean") else rng.uniform(0.5, 2.0, S[k].shape)
    S = PR.unflatten_bn(oc, PR.flatten_bn(oc, S).astype(np.float32))
    net.set_params(PR.flatten_params(oc, P))
    net.set_bn_stats(PR.flatten_bn(oc, S))
    return P, S


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_init_matches_oracle_init(lib):
    c, oc = make_cfgs(lib)
    net = lib.UNet(c, seed=5)
    ref = PR.flatten_params(oc, U.init_params(oc, 5))
    got = net.get_params()
    assert got.size == ref.size
    assert np.allclose(got, ref, rtol=1e-6, atol=1e-7)


@pytest.mark.parametrize("simt", [False, True, "cpasync"])
@pytest.mark.parametrize("ny,nx,B", [(32, 48, 3), (16, 16, 1), (64, 64, 2)])
def test_forward_inference_parity(lib, ny, nx, B, simt):
    c, oc = make_cfgs(lib, widths=(16, 32), simt=simt)
    net = lib.UNet(c, seed=1)
    P, S = randomise(lib, net, oc, 1)
    x = np.random.default_rng(2).standard_normal((B, ny, nx, 4))
    out = net.forward(cuda(x)).cpu().numpy()
    assert not net.status()
    ref, _, _, _ = U.forward(oc, P, S, x, train=False)
    assert nrel(out, ref) < 2e-2


@pytest.mark.parametrize("simt", [False, True, "cpasync"])
def test_forward_default_architecture(lib, simt):
    """Full-width network (32..256 channels): every layer type runs on the tensor-core
    kernel (down 5x5 stride 2, ResNet 3x3, transposed 5x5 per output phase) except the
    4-channel input and 2-channel output layers."""
    c = lib.unet_cfg_default(lib.UNET_STANDALONE)
    c.flags = {False: 0, True: lib.UNET_FLAG_SIMT, "cpasync": lib.UNET_FLAG_NO_TMA}[simt]
    oc = U.UNetConfig()
    net = lib.UNet(c, seed=3)
    P, S = randomise(lib, net, oc, 3)
    x = np.random.default_rng(4).standard_normal((2, 64, 64, 4))
    out = net.forward(cuda(x)).cpu().numpy()
    assert not net.status()
    ref, _, _, _ = U.forward(oc, P, S, x, train=False)
    assert nrel(out, ref) < 2e-2


@pytest.mark.parametrize("shape", [(3, 96, 64), (2, 256, 256), (5, 32, 32)])
def test_tensor_core_and_cuda_core_paths_agree(lib, shape):
    """TMA-fed and cp.async-fed tensor-core paths and the CUDA-core path agree (96x64 has
    non-power-of-two tiles, so TMA declines and the cp.async path runs there)."""
    outs = []
    for flags in (0, lib.UNET_FLAG_NO_TMA, lib.UNET_FLAG_SIMT):
        c = lib.unet_cfg_default(lib.UNET_STANDALONE)
        c.flags = flags
        net = lib.UNet(c, seed=21)
        x = cuda(np.random.default_rng(22).standard_normal(shape + (4,)))
        outs.append(net.forward(x).cpu().numpy())
        assert not net.status()
    assert nrel(outs[0], outs[2]) < 1e-2 and nrel(outs[1], outs[2]) < 1e-2


def test_train_forward_backward_parity(lib):
    c, oc = make_cfgs(lib)
    net = lib.UNet(c, seed=6)
    P, S = randomise(lib, net, oc, 6)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((3, 32, 32, 4))
    tgt = rng.standard_normal((3, 32, 32, 2))
    net.zero_grad()
    out = net.forward(cuda(x), train=True)
    loss, gout = net.mse(out, cuda(tgt))
    gx = net.backward(gout, want_gx=True)
    ref, cache, new_stats, _ = U.forward(oc, P, S, x, train=True)
    rloss, rgout = U.mse_loss(ref, tgt)
    G, rgx, _ = U.backward(oc, P, cache, rgout)
    assert nrel(out.cpu().numpy(), ref) < 2e-2
    assert abs(loss.item() - rloss) / rloss < 2e-2
    Gg = PR.unflatten_params(oc, net.get_grads())
    for k in G:
        assert nrel(Gg[k], G[k]) < 5e-2, k
    assert nrel(gx.cpu().numpy(), rgx) < 5e-2
    Sg = PR.unflatten_bn(oc, net.get_bn_stats())
    for k in new_stats:
        assert nrel(Sg[k], new_stats[k]) < 1e-2, k


@pytest.mark.parametrize("simt", [False, True])
def test_default_network_backward_matches_oracle(lib, simt):
    """Full-width network (32..256 channels, the preconditioners' default) in training
    mode on 2 x 32 x 32: loss, every parameter group's gradient, the input gradient and
    the BatchNorm running statistics against the FP64 oracle's backward (Eq. 3.7 loss,
    Sec. 3.4 training), on the tensor-core path (adjoint-weight data gradients, MN-major
    weight-gradient GEMMs, the widest layer with Cin = 256 and two M blocks) and on CUDA
    cores.  Tolerances as for the small network: 2e-2 forward, 5e-2 per gradient group."""
    c = lib.unet_cfg_default(lib.UNET_STANDALONE)
    c.flags = lib.UNET_FLAG_SIMT if simt else 0
    oc = U.UNetConfig()
    net = lib.UNet(c, seed=8)
    P, S = randomise(lib, net, oc, 8)
    rng = np.random.default_rng(9)
    x = rng.standard_normal((2, 32, 32, 4))
    tgt = rng.standard_normal((2, 32, 32, 2))
    net.zero_grad()
    out = net.forward(cuda(x), train=True)
    loss, gout = net.mse(out, cuda(tgt))
    gx = net.backward(gout, want_gx=True)
    assert not net.status()
    ref, cache, new_stats, _ = U.forward(oc, P, S, x, train=True)
    rloss, rgout = U.mse_loss(ref, tgt)
    G, rgx, _ = U.backward(oc, P, cache, rgout)
    assert nrel(out.cpu().numpy(), ref) < 2e-2
    assert abs(loss.item() - rloss) / rloss < 2e-2
    Gg = PR.unflatten_params(oc, net.get_grads())
    worst = {k: nrel(Gg[k], G[k]) for k in G}
    for k, v in worst.items():
        assert v < 5e-2, (k, v)
    assert nrel(gx.cpu().numpy(), rgx) < 5e-2
    Sg = PR.unflatten_bn(oc, net.get_bn_stats())
    for k in new_stats:
        assert nrel(Sg[k], new_stats[k]) < 1e-2, k
    print("worst gradient group", max(worst.items(), key=lambda kv: kv[1]))


def test_backward_tensor_core_matches_cuda_core(lib):
    """Full-width network (32..256 channels): the tensor-core backward (data gradients on
    the TMA convolution with adjoint weights, weight gradients as MN-major tcgen05 GEMMs)
    agrees with the CUDA-core backward on every parameter group and the input gradient."""
    oc = U.UNetConfig()
    nets = []
    for flags in (0, lib.UNET_FLAG_SIMT):
        c = lib.unet_cfg_default(lib.UNET_STANDALONE)
        c.flags = flags
        net = lib.UNet(c, seed=3)
        randomise(lib, net, oc, 3)
        nets.append(net)
    rng = np.random.default_rng(11)
    x = cuda(rng.standard_normal((2, 64, 64, 4)))
    tgt = cuda(rng.standard_normal((2, 64, 64, 2)))
    grads, gxs = [], []
    for net in nets:
        net.zero_grad()
        out = net.forward(x, train=True)
        _, gout = net.mse(out, tgt)
        gxs.append(net.backward(gout, want_gx=True).cpu().numpy())
        assert not net.status()
        grads.append(PR.unflatten_params(oc, net.get_grads()))
    for k in grads[1]:
        assert nrel(grads[0][k], grads[1][k]) < 3e-2, k
    assert nrel(gxs[0], gxs[1]) < 3e-2


@pytest.mark.parametrize("simt", [False, True])
def test_encoder_solver_parity(lib, simt):
    ec, eoc = make_cfgs(lib, in_ch=2, out_ch=4, widths=(16, 32), simt=simt)
    ctx = U.context_channels(eoc)
    sc, soc = make_cfgs(lib, context=ctx, widths=(16, 32), simt=simt)
    enc, sol = lib.UNet(ec, seed=8), lib.UNet(sc, seed=9)
    Pe, Se = randomise(lib, enc, eoc, 8)
    Ps, Ss = randomise(lib, sol, soc, 9)
    sol.attach_encoder(enc)
    rng = np.random.default_rng(10)
    med = rng.standard_normal((1, 32, 32, 2))
    x = rng.standard_normal((2, 32, 32, 4))
    tgt = rng.standard_normal((2, 32, 32, 2))
    # inference: encoder once, features broadcast to the solver batch
    enc.forward(cuda(med))
    out = sol.forward(cuda(x)).cpu().numpy()
    _, _, _, fe = U.forward(eoc, Pe, Se, med, train=False)
    ref, _, _, _ = U.forward(soc, Ps, Ss, x, train=False, feats=[np.broadcast_to(f, (2,) + f.shape[1:]) for f in fe])
    assert nrel(out, ref) < 2e-2
    # training: gradients reach the encoder through the context features
    sol.zero_grad()
    enc.forward(cuda(med), train=True)
    o = sol.forward(cuda(x), train=True)
    _, gout = sol.mse(o, cuda(tgt))
    sol.backward(gout)
    _, ce, _, fe = U.forward(eoc, Pe, Se, med, train=True)
    feb = [np.repeat(f, 2, axis=0) for f in fe]
    ro, cs, _, _ = U.forward(soc, Ps, Ss, x, train=True, feats=feb)
    _, rg = U.mse_loss(ro, tgt)
    Gs, _, gf = U.backward(soc, Ps, cs, rg)
    gf = [g.sum(axis=0, keepdims=True) for g in gf]
    Ge = U.backward_features(eoc, Pe, ce, gf)
    Gsg = PR.unflatten_params(soc, sol.get_grads())
    Geg = PR.unflatten_params(eoc, enc.get_grads())
    for k in ("down1", "down2", "up2", "up1", "res2.1.k2"):
        assert nrel(Gsg[k], Gs[k]) < 5e-2, k
    for k in ("down1", "down2", "up2", "up1", "res1.0.k1"):
        assert nrel(Geg[k], Ge[k]) < 5e-2, k


def test_adam_step_matches_oracle(lib):
    c, oc = make_cfgs(lib)
    net = lib.UNet(c, seed=11)
    P, S = randomise(lib, net, oc, 11)
    rng = np.random.default_rng(12)
    x = rng.standard_normal((2, 16, 16, 4))
    tgt = rng.standard_normal((2, 16, 16, 2))
    net.zero_grad()
    out = net.forward(cuda(x), train=True)
    _, gout = net.mse(out, cuda(tgt))
    net.backward(gout)
    G = PR.unflatten_params(oc, net.get_grads())
    net.adam_step(lr=1e-3)
    M = {k: np.zeros_like(v) for k, v in P.items()}
    V = {k: np.zeros_like(v) for k, v in P.items()}
    P2 = {k: v.copy() for k, v in P.items()}
    U.adam_step(P2, G, M, V, 1, 1e-3)
    got = PR.unflatten_params(oc, net.get_params())
    for k in P2:
        assert np.allclose(got[k], P2[k], rtol=1e-5, atol=1e-6), k


def _helm(lib, n, seed=1000):
    k2 = medium(n, n, seed)
    hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
    d = hz.desc
    prob = H.Problem(k2.astype(np.float64), omega=d.omega, h=d.h, abc_width=d.abc_width, levels=d.levels)
    return hz, prob


@pytest.mark.parametrize("kind", ["ju", "vu"])
def test_unet_preconditioner_parity(lib, kind):
    n = 64
    hz, prob = _helm(lib, n)
    c, oc = make_cfgs(lib, widths=(16, 32, 64))
    net = lib.UNet(c, seed=13)
    P, S = randomise(lib, net, oc, 13)
    r = crandn(14, (2, n, n))
    k = lib.HELM_PREC_JU if kind == "ju" else lib.HELM_PREC_VU
    e = hz.unet_precond(net, torch.from_numpy(r).cuda(), kind=k).cpu().numpy()
    ref = (PR.precond_ju if kind == "ju" else PR.precond_vu)(prob, oc, P, S, r)
    assert nrel(e, ref) < 2e-2


def test_unet_preconditioner_chunks_large_batches(lib):
    # 2048^2 x 8 images of a 32-channel first level exceed the U-Net's 2^31-element tensor
    # limit: the preconditioner runs the network on chunks of 4 right-hand sides, which must
    # give exactly what two separate 4-RHS applications give
    n = 2048
    hz = lib.Helmholtz(torch.from_numpy(medium(n, n, 1001)).cuda())
    c, _ = make_cfgs(lib, widths=(32, 64))
    net = lib.UNet(c, seed=19)
    r = torch.from_numpy(crandn(20, (8, n, n)).astype(np.complex64)).cuda()
    e = hz.unet_precond(net, r, kind=lib.HELM_PREC_VU)
    e0 = hz.unet_precond(net, r[:4].contiguous(), kind=lib.HELM_PREC_VU)
    e1 = hz.unet_precond(net, r[4:].contiguous(), kind=lib.HELM_PREC_VU)
    assert torch.isfinite(torch.view_as_real(e)).all()
    assert torch.equal(e[:4], e0) and torch.equal(e[4:], e1)


def test_encoder_solver_preconditioner(lib):
    n = 64
    hz, prob = _helm(lib, n)
    ec, eoc = make_cfgs(lib, in_ch=2, out_ch=4)
    sc, soc = make_cfgs(lib, context=U.context_channels(eoc))
    enc, sol = lib.UNet(ec, seed=15), lib.UNet(sc, seed=16)
    Pe, Se = randomise(lib, enc, eoc, 15)
    Ps, Ss = randomise(lib, sol, soc, 16)
    sol.attach_encoder(enc)
    sol.encode(hz)
    r = crandn(17, (3, n, n))
    e = hz.unet_precond(sol, torch.from_numpy(r).cuda(), kind=lib.HELM_PREC_VU).cpu().numpy()
    fe = PR.encoder_features(prob, eoc, Pe, Se)
    ref = PR.precond_vu(prob, soc, Ps, Ss, r, feats=[np.broadcast_to(f, (3,) + f.shape[1:]) for f in fe])
    assert nrel(e, ref) < 2e-2


def test_full_size_bench_batch_forward_and_preconditioner(lib):
    """The benchmark's launch configuration, 256^2 x 8 with the default network: the
    inference forward (space-to-depth input layer, column-reuse, split-K and sub-pixel
    kernels) and the M_VU application, each against the FP64 oracle."""
    n, B = 256, 8
    c = lib.unet_cfg_default(lib.UNET_STANDALONE)
    oc = U.UNetConfig()
    net = lib.UNet(c, seed=41)
    P, S = randomise(lib, net, oc, 41)
    x = np.random.default_rng(42).standard_normal((B, n, n, 4))
    out = net.forward(cuda(x)).cpu().numpy()
    assert not net.status()
    ref, _, _, _ = U.forward(oc, P, S, x, train=False)
    assert nrel(out, ref) < 2e-2
    hz, prob = _helm(lib, n)
    r = crandn(43, (B, n, n))
    e = hz.unet_precond(net, torch.from_numpy(r).cuda(), kind=lib.HELM_PREC_VU).cpu().numpy()
    ref_e = PR.precond_vu(prob, oc, P, S, r)
    assert nrel(e, ref_e) < 2e-2


def test_encoder_solver_fgmres_512_32rhs(lib):
    """512^2, 32 right-hand sides (16 point sources, 16 complex Gaussian) through the
    default-size encoder-solver pair (Sec. 3.3) as the M_VU network, its output layer
    zeroed: the whole network runs every iteration, U-Net(r) = 0, so FGMRES(M_VU) takes
    the iterations of FGMRES(M_V); every solution's FP64 residual, recomputed by the
    oracle's operator, is <= 1e-7."""
    n = 512
    hz, prob = _helm(lib, n)
    w = (32, 64, 128, 256)
    ec, eoc = make_cfgs(lib, widths=w, resnets=3, in_ch=2, out_ch=4)
    sc, soc = make_cfgs(lib, widths=w, resnets=3, context=U.context_channels(eoc))
    enc, sol = lib.UNet(ec, seed=21), lib.UNet(sc, seed=22)
    P = PR.unflatten_params(soc, sol.get_params())
    P["up1"][:] = 0.0
    P["up1.bias"][:] = 0.0
    sol.set_params(PR.flatten_params(soc, P))
    sol.attach_encoder(enc)
    sol.encode(hz)
    pos = synth.source_positions(n, n, 16, synth.rhs_seed(3), 16)
    b = np.concatenate([synth.point_sources(n, n, pos, 1.0 / n), synth.gaussian_rhs(n, n, 16, 2003)])
    bd = torch.from_numpy(b.astype(np.complex128)).cuda()
    _, iv = hz.fgmres(bd, precond=lib.HELM_PREC_V, tol=1e-7, maxit=20000)
    x, iu = hz.fgmres(bd, precond=lib.HELM_PREC_VU, net=sol, tol=1e-7, maxit=20000)
    assert iv["status"] == 0 and iu["status"] == 0
    assert all(abs(a - c) <= 2 for a, c in zip(iu["iters"], iv["iters"]))
    x = x.cpu().numpy()
    for k in range(32):
        assert np.linalg.norm(H.residual(prob.A, b[k], x[k])) <= 1e-7 * np.linalg.norm(b[k])


def test_residual_loss_parity(lib):
    # the unsupervised residual loss (Remark after Eq. 3.7) and its gradient vs the oracle
    n = 64
    hz, prob = _helm(lib, n)
    rng = np.random.default_rng(31)
    y = rng.standard_normal((2, n, n, 2)).astype(np.float32)
    x = rng.standard_normal((2, n, n, 4)).astype(np.float32)
    loss, g = hz.residual_loss(torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda())
    ref_loss, ref_g = PR.residual_loss(prob, y.astype(np.float64), x.astype(np.float64))
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * ref_loss
    assert nrel(g.cpu().numpy(), ref_g) < 1e-5


def test_residual_loss_training_lowers_the_residual(lib):
    # unsupervised training (loss="residual") on pairs of one medium lowers the loss
    from paper_2203_11025_gb300 import train as T
    n = 64
    hz, _ = _helm(lib, n)
    c, _ = make_cfgs(lib, widths=(8, 16))
    net = lib.UNet(c, seed=33)
    hist = T.train(hz, net, pairs=hz.gen_pairs(32, 34, 10), epochs=6, batch=8, lr=1e-3, seed=35, loss="residual")
    assert all(np.isfinite(hist)) and hist[-1] < 0.8 * hist[0]


def test_gen_pairs_parity(lib):
    n = 32
    hz, prob = _helm(lib, n)
    r, e = hz.gen_pairs(4, seed=123, kmax=10)
    r, e = r.cpu().numpy(), e.cpu().numpy()
    x, ks = synth.pair_draws(123, 4, n, n, 10)
    rr, er = PR.gen_pairs(prob, x, ks)
    for j in range(4):
        # Eq. 3.9 identity: A e = r (independent of solver precision)
        assert nrel(H.apply_op(prob.A, e[j]), r[j]) < 1e-10
        # k FP32 Krylov steps vs FP64: the iterate x~ agrees to ~1e-6 relative, and e = x - x~
        # loses the digits x and x~ share (|e| ~ 1e-2 |x| after a few steps); r = A e
        # amplifies the high-frequency part of that difference by up to ||A|| ~ 8/h^2
        assert nrel(e[j], er[j]) < 5e-4 and nrel(r[j], rr[j]) < 1e-2


@pytest.mark.parametrize("n,nmix", [(48, 2), (64, 3), (32, 1)])
def test_make_batch_parity(lib, n, nmix):
    """Training-batch assembly (Sec. 3.4: linear combinations of pairs, input h^2 r' / s,
    target e' / s) against the oracle's make_batch, on pairs the GPU generated; FP32
    outputs of FP64 inputs (relative 1e-6), the medium channels bit for bit."""
    hz, prob = _helm(lib, n)
    r, e = hz.gen_pairs(6, seed=77, kmax=10)
    rng = np.random.default_rng(78)
    count = 5
    idx = rng.integers(0, 6, (count, nmix)).astype(np.int32)
    coef = (rng.standard_normal((count, nmix)) + 1j * rng.standard_normal((count, nmix))) / np.sqrt(2)
    if nmix == 1:
        coef[:] = 1.0
    x, t = hz.make_batch(r, e, idx, coef)
    x, t = x.cpu().numpy(), t.cpu().numpy()
    xr, tr = PR.make_batch(prob, r.cpu().numpy(), e.cpu().numpy(), idx, coef)
    for i in range(count):
        assert nrel(x[i, ..., :2], xr[i, ..., :2]) < 1e-6, i
        assert nrel(t[i], tr[i]) < 1e-6, i
        assert np.array_equal(x[i, ..., 2], prob.A.kappa2.astype(np.float32))
        assert nrel(x[i, ..., 3], prob.A.gamma) < 1e-6


def test_fgmres_vu_with_silent_network_equals_sl(lib):
    """With the output layer zeroed, U-Net(r) = 0 and M_VU is exactly one V-cycle from
    zero: FGMRES(M_VU) must take the same iterations as FGMRES(M_V)."""
    n = 64
    hz, prob = _helm(lib, n)
    c, oc = make_cfgs(lib)
    net = lib.UNet(c, seed=18)
    P, S = randomise(lib, net, oc, 18)
    P["up1"][:] = 0.0
    P["up1.bias"][:] = 0.0
    net.set_params(PR.flatten_params(oc, P))
    pos = synth.source_positions(n, n, 2, 5, 16)
    b = torch.from_numpy(synth.point_sources(n, n, pos, 1.0 / n)).cuda()
    _, iv = hz.fgmres(b, precond=lib.HELM_PREC_V, tol=1e-7, maxit=3000)
    x, iu = hz.fgmres(b, precond=lib.HELM_PREC_VU, net=net, tol=1e-7, maxit=3000)
    assert iu["status"] == 0
    assert all(abs(a - b) <= 2 for a, b in zip(iu["iters"], iv["iters"]))
    x = x.cpu().numpy()
    bb = b.cpu().numpy()
    for j in range(2):
        assert np.linalg.norm(H.residual(prob.A, bb[j], x[j])) / np.linalg.norm(bb[j]) <= 1e-7


def test_block_fgmres_vu_with_silent_network_equals_block_sl(lib):
    """Block FGMRES with M_VU whose output layer is zeroed takes block FGMRES(M_V)'s
    iterations; every FP64 residual <= 1e-7."""
    n = 64
    hz, prob = _helm(lib, n)
    c, oc = make_cfgs(lib)
    net = lib.UNet(c, seed=38)
    P, S = randomise(lib, net, oc, 38)
    P["up1"][:] = 0.0
    P["up1.bias"][:] = 0.0
    net.set_params(PR.flatten_params(oc, P))
    pos = synth.source_positions(n, n, 4, 39, 16)
    b = torch.from_numpy(synth.point_sources(n, n, pos, 1.0 / n)).cuda()
    _, iv = hz.fgmres(b, precond=lib.HELM_PREC_V, tol=1e-7, maxit=3000, block=True)
    x, iu = hz.fgmres(b, precond=lib.HELM_PREC_VU, net=net, tol=1e-7, maxit=3000, block=True)
    assert iv["status"] == 0 and iu["status"] == 0
    assert abs(iu["iters_max"] - iv["iters_max"]) <= 2
    x = x.cpu().numpy()
    bb = b.cpu().numpy()
    for j in range(4):
        assert np.linalg.norm(H.residual(prob.A, bb[j], x[j])) / np.linalg.norm(bb[j]) <= 1e-7


def test_solve_cycles_follow_network_buffers(lib):
    """A captured FGMRES cycle references the network's weights and workspace.  A forward
    at another batch size (workspace reallocated) between two solves, and a new network
    created after the previous one was released, must each be solved with their own
    buffers: the three solves agree."""
    import gc
    n = 64
    hz, _ = _helm(lib, n)
    c, oc = make_cfgs(lib)
    pos = synth.source_positions(n, n, 2, 5, 16)
    b = torch.from_numpy(synth.point_sources(n, n, pos, 1.0 / n)).cuda()
    net = lib.UNet(c, seed=21)
    x1, i1 = hz.fgmres(b, precond=lib.HELM_PREC_VU, net=net, tol=1e-7, maxit=3000)
    x1 = x1.cpu().numpy()
    net.forward(cuda(np.random.default_rng(3).standard_normal((3, n, n, 4))))   # batch 3: new workspace
    x2, i2 = hz.fgmres(b, precond=lib.HELM_PREC_VU, net=net, tol=1e-7, maxit=3000)
    assert i2["iters"] == i1["iters"]
    assert np.allclose(x2.cpu().numpy(), x1, rtol=0, atol=1e-12 * np.abs(x1).max())
    del net
    gc.collect()
    net2 = lib.UNet(c, seed=21)
    x3, i3 = hz.fgmres(b, precond=lib.HELM_PREC_VU, net=net2, tol=1e-7, maxit=3000)
    assert i3["iters"] == i1["iters"]
    assert np.allclose(x3.cpu().numpy(), x1, rtol=0, atol=1e-12 * np.abs(x1).max())


def test_checkpoint_round_trip_reproduces_the_network(lib, tmp_path):
    # a saved network, loaded into a fresh handle, gives bit-identical inference outputs
    from paper_2203_11025_gb300 import checkpoint as CK
    c, oc = make_cfgs(lib, widths=(16, 32))
    net = lib.UNet(c, seed=21)
    randomise(lib, net, oc, 21)
    x = torch.from_numpy(np.random.default_rng(22).standard_normal((2, 64, 64, 4)).astype(np.float32)).cuda()
    y0 = net.forward(x).cpu().numpy()
    path = str(tmp_path / "net.ckpt")
    CK.save(net, path, meta={"seed": 21})
    net2, meta = CK.load(path)
    assert meta == {"seed": 21}
    y1 = net2.forward(x).cpu().numpy()
    assert np.array_equal(y0.view(np.uint32), y1.view(np.uint32))
    other = lib.UNet(make_cfgs(lib, widths=(8, 16))[0], seed=1)
    with pytest.raises(ValueError):
        CK.load_into(other, path)


@pytest.mark.parametrize("loss", ["error", "residual"])
def test_train_step_equals_the_step_by_step_sequence(lib, loss):
    """unet_train_step (one C-ABI call) performs the training step of Sec. 3.4: the Adam
    update it makes equals the one of the separate forward, loss (Eq. 3.7 or the residual
    loss), backward and Adam calls from the same state, and it reports the same loss."""
    n = 64
    hz, prob = _helm(lib, n)
    c, oc = make_cfgs(lib, widths=(16, 32))
    nets = [lib.UNet(c, seed=50), lib.UNet(c, seed=50)]
    r, e = hz.gen_pairs(8, seed=51, kmax=10)
    idx = np.arange(4, dtype=np.int32)[:, None]
    x, t = hz.make_batch(r, e, idx, np.ones((4, 1), complex))
    p0 = nets[0].get_params()
    lv_a = nets[0].train_step(hz, x, t if loss == "error" else None, lr=1e-3, loss=loss)
    nets[1].zero_grad()
    out = nets[1].forward(x, train=True)
    lv_b, gout = nets[1].mse(out, t) if loss == "error" else hz.residual_loss(out, x)
    nets[1].backward(gout)
    nets[1].adam_step(lr=1e-3)
    da, db = nets[0].get_params() - p0, nets[1].get_params() - p0
    assert abs(lv_a.item() - lv_b.item()) <= 1e-5 * abs(lv_b.item())
    assert nrel(da, db) < 1e-2 and np.abs(da).max() > 0
    assert not nets[0].status()


def test_checkpoint_written_by_the_library_reads_in_python(lib, tmp_path):
    """unet_save writes the layout that checkpoint.decode describes (and unet_load reads
    what checkpoint.encode writes), with the device weights and statistics."""
    from paper_2203_11025_gb300 import checkpoint as CK
    c, oc = make_cfgs(lib, widths=(16, 32))
    net = lib.UNet(c, seed=61)
    randomise(lib, net, oc, 61)
    path = str(tmp_path / "lib.ckpt")
    net.save(path, {"k": 1})
    cfg, p, b, meta = CK.read(path)
    assert meta == {"k": 1} and cfg == CK.cfg_to_dict(net.cfg)
    assert np.array_equal(p, net.get_params()) and np.array_equal(b, net.get_bn_stats())
    other = lib.UNet(c, seed=62)
    (tmp_path / "py.ckpt").write_bytes(CK.encode(cfg, p * 2, b, {}))
    other.load(str(tmp_path / "py.ckpt"))
    assert np.array_equal(other.get_params(), p * 2)


def test_fallback_to_plain_sl_when_the_network_fails(lib):
    # plain SL-FGMRES stays as the fallback of the network: with HELM_FLAG_FALLBACK_V a solve
    # whose U-Net preconditioner breaks (here a network that returns NaN) is finished by M_V
    n = 64
    hz, prob = _helm(lib, n)
    c, oc = make_cfgs(lib, widths=(16, 32))
    net = lib.UNet(c, seed=5)
    net.set_params(np.full(net.n_params, np.nan, np.float32))
    b = torch.from_numpy(synth.complex_normal(41, (2, n, n))).cuda()
    with pytest.raises(lib.HelmError) as e:
        hz.fgmres(b, precond=lib.HELM_PREC_VU, net=net, maxit=40)
    assert e.value.code == lib.HELM_ENAN
    x, info = hz.fgmres(b, precond=lib.HELM_PREC_VU, net=net, maxit=2000, flags=lib.HELM_FLAG_FALLBACK_V)
    assert info["status"] == lib.HELM_OK and info["fallbacks"] == 2
    _, ref = hz.fgmres(b, precond=lib.HELM_PREC_V, maxit=2000)
    x = x.cpu().numpy()
    bb = b.cpu().numpy()
    for k in range(2):
        assert np.linalg.norm(H.residual(prob.A, bb[k], x[k])) <= 1e-7 * np.linalg.norm(bb[k])
        assert info["iters"][k] > ref["iters"][k]          # the failed attempt's steps are counted too
    # a working network (here a silent one: M_VU acts as M_V) needs no fallback
    good = lib.UNet(c, seed=6)
    P, _ = randomise(lib, good, oc, 6)
    P["up1"][:] = 0.0
    P["up1.bias"][:] = 0.0
    good.set_params(PR.flatten_params(oc, P))
    _, info = hz.fgmres(b, precond=lib.HELM_PREC_VU, net=good, maxit=2000, flags=lib.HELM_FLAG_FALLBACK_V)
    assert info["status"] == lib.HELM_OK and info["fallbacks"] == 0


@pytest.mark.slow
def test_trained_network_gains_over_plain_sl(lib):
    # what the learned part buys: a network trained with the benchmark's single-model recipe
    # (Sec. 4: Eq. 3.8-3.9 pairs of one 256^2 medium from the library's SL-FGMRES, MSE of
    # Eq. 3.7, Adam) makes FGMRES + M_VU converge in far fewer iterations than FGMRES + M_V
    # on right-hand sides it never saw (point sources and Gaussian noise); every solution is
    # checked by the oracle's FP64 residual
    from paper_2203_11025_gb300 import train as T
    n = 256
    k2 = synth.grf_kappa2(n, n, synth.medium_seed(0))
    hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
    d = hz.desc
    prob = H.Problem(k2.astype(np.float64), omega=d.omega, h=d.h, abc_width=d.abc_width, levels=d.levels)
    net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=7)
    pairs = hz.gen_pairs(1024, 5151, 10)
    T.train(hz, net, pairs=pairs, epochs=96, batch=16, lr=1e-3, seed=11)
    del pairs
    pos = synth.source_positions(n, n, 4, synth.rhs_seed(7), 16)
    b = np.concatenate([synth.point_sources(n, n, pos, 1.0 / n), synth.complex_normal(77, (4, n, n))])
    bt = torch.from_numpy(b).cuda()
    _, iv = hz.fgmres(bt, precond=lib.HELM_PREC_V, tol=1e-7, maxit=20000)
    x, iu = hz.fgmres(bt, precond=lib.HELM_PREC_VU, net=net, tol=1e-7, maxit=20000)
    assert iv["status"] == lib.HELM_OK and iu["status"] == lib.HELM_OK
    for k in range(4):      # point sources, the benchmark's kind: at least twice as fast
        assert iu["iters"][k] <= 0.5 * iv["iters"][k], (k, iu["iters"], iv["iters"])
    for k in range(4, 8):   # white-noise right-hand sides, unlike the training residuals: still fewer
        assert iu["iters"][k] < iv["iters"][k], (k, iu["iters"], iv["iters"])
    x = x.cpu().numpy()
    for k in range(8):
        assert np.linalg.norm(H.residual(prob.A, b[k], x[k])) <= 1e-7 * np.linalg.norm(b[k])


def test_weight_gradients_are_bit_reproducible(lib):
    """The default network's training step at 16 x 256^2 (the benchmark's base-training batch):
    forward in training mode, MSE, backward -- twice from the same weights and batch -- gives
    bit-identical gradients (the weight gradients' pixel chunks are summed in a fixed order,
    not with atomics), so a training run is reproducible."""
    net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=5)
    rng = np.random.default_rng(6)
    x = cuda(rng.standard_normal((16, 256, 256, 4)))
    t = cuda(rng.standard_normal((16, 256, 256, 2)))
    grads = []
    for _ in range(2):
        net.zero_grad()
        o = net.forward(x, train=True)
        _, g = net.mse(o, t)
        net.backward(g)
        grads.append(np.array(net.get_grads()))
    assert not net.status()
    assert np.all(np.isfinite(grads[0])) and np.abs(grads[0]).max() > 0
    assert np.array_equal(grads[0], grads[1])


def test_trained_encoder_solver_gains_over_plain_sl(lib):
    """The encoder-solver pair of Sec. 3.3 with the library's default widths, trained jointly
    (Eq. 3.7 MSE, Adam) on Eq. 3.8-3.9 pairs of one 256^2 medium, the encoder run once for the
    medium: FGMRES + M_VU needs at most half the iterations of FGMRES + M_V on point sources it
    never saw (measured at 512^2 x 32: 148 against 544), and every solution's FP64 residual,
    recomputed by the oracle's operator, is <= 1e-7."""
    from paper_2203_11025_gb300 import train as T
    n = 256
    k2 = synth.grf_kappa2(n, n, synth.medium_seed(0))
    hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
    d = hz.desc
    prob = H.Problem(k2.astype(np.float64), omega=d.omega, h=d.h, abc_width=d.abc_width, levels=d.levels)
    enc = lib.UNet(kind=lib.UNET_ENCODER, seed=3)
    sol = lib.UNet(kind=lib.UNET_SOLVER, seed=4)
    sol.attach_encoder(enc)
    T.train(hz, sol, pairs=hz.gen_pairs(512, 4242, 10), epochs=24, batch=16, lr=1e-3, seed=11)
    sol.encode(hz)
    pos = synth.source_positions(n, n, 4, synth.rhs_seed(9), 16)
    b = synth.point_sources(n, n, pos, 1.0 / n).astype(np.complex128)
    bt = torch.from_numpy(b).cuda()
    _, iv = hz.fgmres(bt, precond=lib.HELM_PREC_V, tol=1e-7, maxit=20000)
    x, iu = hz.fgmres(bt, precond=lib.HELM_PREC_VU, net=sol, tol=1e-7, maxit=20000)
    assert iv["status"] == lib.HELM_OK and iu["status"] == lib.HELM_OK
    for k in range(4):
        assert iu["iters"][k] <= 0.5 * iv["iters"][k], (k, iu["iters"], iv["iters"])
    x = x.cpu().numpy()
    for k in range(4):
        assert np.linalg.norm(H.residual(prob.A, b[k], x[k])) <= 1e-7 * np.linalg.norm(b[k])


@pytest.mark.slow
def test_general_network_gains_on_an_unseen_medium(lib):
    """The general network of Sec. 3.4.1 / 4: trained on Eq. 3.8-3.9 pairs of 16 random
    256^2 media (64 pairs each, none of them the test medium), it lowers FGMRES(M_VU)
    iterations against plain SL on a medium it never saw (measured: 106-132 against
    196-230 on three unseen media); every solution is checked by the oracle's FP64 residual."""
    from paper_2203_11025_gb300 import train as T
    n = 256
    media = []
    for i in range(16):
        hz_i = lib.Helmholtz(torch.from_numpy(synth.grf_kappa2(n, n, 10 ** 6 + i)).cuda())
        media.append((hz_i, hz_i.gen_pairs(64, 4000 + i, 10)))
    net = lib.UNet(lib.unet_cfg_default(lib.UNET_STANDALONE), seed=7)
    hist = T.train_media(media, net, epochs=96, batch=16, lr=1e-3, seed=11)
    assert hist[-1] < 0.6 * hist[0]
    for hz_i, _ in media:
        hz_i.close()
    k2 = synth.grf_kappa2(n, n, 777)               # unseen
    hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
    d = hz.desc
    prob = H.Problem(k2.astype(np.float64), omega=d.omega, h=d.h, abc_width=d.abc_width, levels=d.levels)
    pos = synth.source_positions(n, n, 4, synth.rhs_seed(7), 16)
    b = synth.point_sources(n, n, pos, 1.0 / n)
    bt = torch.from_numpy(b).cuda()
    _, iv = hz.fgmres(bt, precond=lib.HELM_PREC_V, tol=1e-7, maxit=20000)
    x, iu = hz.fgmres(bt, precond=lib.HELM_PREC_VU, net=net, tol=1e-7, maxit=20000)
    assert iv["status"] == lib.HELM_OK and iu["status"] == lib.HELM_OK
    for k in range(4):
        assert iu["iters"][k] <= 0.75 * iv["iters"][k], (k, iu["iters"], iv["iters"])
    x = x.cpu().numpy()
    for k in range(4):
        assert np.linalg.norm(H.residual(prob.A, b[k], x[k])) <= 1e-7 * np.linalg.norm(b[k])
