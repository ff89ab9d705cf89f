"""GPU parity: libhelm's stencil, transfer, coarse-solve, V-cycle and FGMRES
kernels against the FP64 oracle, element by element, on seeded inputs.

Tolerances: FP64 kernels 1e-12 relative (max-norm), FP32 stencils 1e-5; a
composed V-cycle in FP32 1e-4 (about twenty stencil sweeps plus the nonlinear
coarse GMRES, each adding ~1e-6); solutions at FP64 true residual <= 1e-7."""
import numpy as np
import pytest

from gpu_util import crandn, medium, relerr
from oracle import helmholtz as H
from paper_2203_11025_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    from paper_2203_11025_gb300 import build
    from paper_2203_11025_gb300 import lib as L
    build.build()
    return L


def make(lib, ny, nx, seed=1000, levels=3, abc=16, omega=None, sigma=8.0, **kw):
    k2 = medium(ny, nx, seed, sigma)
    h = 1.0 / nx
    om = synth.omega_for(nx) if omega is None else omega
    hz = lib.Helmholtz(torch.from_numpy(k2).cuda(), levels=levels, abc_width=abc, omega=om, h=h, **kw)
    d = hz.desc
    prob = H.Problem(k2.astype(np.float64), omega=om, h=h, abc_width=abc, gamma_max=d.abc_gamma_max,
                     beta=d.beta, levels=levels, nu1=d.nu1, nu2=d.nu2, jacobi_w=d.jacobi_w,
                     coarse_its=d.coarse_its)
    return hz, prob


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


SHAPES = [(48, 80), (64, 64), (40, 24)]   # several 32x8 tiles with ragged tails, non-square


@pytest.mark.parametrize("ny,nx", SHAPES)
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 1e-5)])
def test_apply_residual_parity(lib, ny, nx, dtype, tol):
    hz, prob = make(lib, ny, nx, abc=6)
    x = crandn(1, (3, ny, nx))
    b = crandn(2, (3, ny, nx))
    for op, lv in ((lib.HELM_OP_A, prob.A), (lib.HELM_OP_M, prob.M)):
        y = hz.apply(dev(x, dtype), op=op).cpu().numpy()
        assert relerr(y, H.apply_op(lv, x)) < tol
        r = hz.residual(dev(b, dtype), dev(x, dtype), op=op).cpu().numpy()
        assert relerr(r, H.residual(lv, b, x)) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 1e-5)])
def test_coarse_levels_parity(lib, dtype, tol):
    hz, prob = make(lib, 48, 80, abc=6)
    for level in range(1, 3):
        k2 = hz.level_kappa2(level).cpu().numpy()
        assert np.abs(k2 - prob.hierarchy[level].kappa2).max() < 1e-14
        lvM = prob.hierarchy[level]
        ny, nx = lvM.ny, lvM.nx
        x = crandn(3 + level, (2, ny, nx))
        y = hz.apply(dev(x, dtype), op=lib.HELM_OP_M, level=level).cpu().numpy()
        assert relerr(y, H.apply_op(lvM, x)) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-12), (torch.complex64, 1e-5)])
def test_jacobi_parity(lib, dtype, tol):
    hz, prob = make(lib, 48, 80, abc=6)
    f = crandn(5, (2, 48, 80))
    x = crandn(6, (2, 48, 80))
    out = hz.jacobi(dev(f, dtype), dev(x, dtype), op=lib.HELM_OP_M).cpu().numpy()
    assert relerr(out, H.jacobi(prob.M, x, f, 0.8)) < tol
    out0 = hz.jacobi(dev(f, dtype), None, op=lib.HELM_OP_A).cpu().numpy()
    assert relerr(out0, H.jacobi(prob.A, np.zeros_like(f), f, 0.8)) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-13), (torch.complex64, 1e-6)])
def test_transfer_parity(lib, dtype, tol):
    hz, prob = make(lib, 48, 80, abc=6)
    r = crandn(7, (3, 48, 80))
    rc = hz.restrict(dev(r, dtype)).cpu().numpy()
    assert relerr(rc, H.restrict_fw(r)) < tol
    e = crandn(8, (3, 24, 40))
    xf = crandn(9, (3, 48, 80))
    out = hz.prolong_add(dev(e, dtype), dev(xf, dtype)).cpu().numpy()
    assert relerr(out, xf + H.prolong_bilinear(e, 48, 80)) < tol


COARSE_PATHS = [0, 1, 2]   # cluster (default), multi-kernel, one CTA per right-hand side


@pytest.mark.parametrize("path", COARSE_PATHS)
@pytest.mark.parametrize("shape", [(128, 96), (256, 256), (64, 256)])
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-11), (torch.complex64, 2e-5)])
def test_coarse_gmres_parity(lib, dtype, tol, path, shape):
    hz, prob = make(lib, shape[0], shape[1], abc=16, flags=path)
    lc = prob.hierarchy[-1]
    f = crandn(10, (4, lc.ny, lc.nx))
    f[2] = 0.0  # a zero right-hand side returns zero
    x = hz.coarse_solve(dev(f, dtype)).cpu().numpy()
    for k in range(4):
        ref = H.gmres_jacobi(lc, f[k], prob.coarse_its)
        if k == 2:
            assert np.all(x[k] == 0)
        else:
            assert relerr(x[k], ref) < tol


@pytest.mark.parametrize("seg", [4, 8, 16, 32, -1])
@pytest.mark.parametrize("ny,nx", [(96, 160), (128, 128), (40, 248)])
def test_vcycle_parity_every_tile_form(lib, ny, nx, seg):
    """Each form of the fused cycle kernels (column strips with segments of 4-32 rows, the
    shared-memory tile) gives the oracle's V-cycle in FP32 (ragged strips: 160, 248 are no
    multiples of the 60-column strip, 96 / 40 rows no multiples of the segment)."""
    hz, prob = make(lib, ny, nx, abc=16)
    nrhs = 3
    for lev in range(prob.levels - 1):
        for kern in (0, 1):
            hz.set_tile_choice(kern, lev, nrhs, seg)
            assert hz.tile_choice(kern, lev, nrhs) == seg
    f = crandn(12, (nrhs, ny, nx))
    z = hz.vcycle(dev(f, torch.complex64)).cpu().numpy()
    for k in range(nrhs):
        assert relerr(z[k], H.vcycle(prob, f[k])) < 1e-4


def test_tuner_picks_a_tile_form_per_level(lib):
    hz, prob = make(lib, 128, 128, abc=16)
    b = crandn(13, (4, 128, 128))
    x, info = hz.fgmres(dev(b, torch.complex128), tol=1e-7, maxit=2000)
    for lev in range(prob.levels - 1):
        for kern in (0, 1):
            assert hz.tile_choice(kern, lev, 4) in (4, 8, 16, 32, -1)
    xs = x.cpu().numpy()
    for k in range(4):
        assert np.linalg.norm(H.residual(prob.A, b[k], xs[k])) / np.linalg.norm(b[k]) <= 1e-7


@pytest.mark.parametrize("ny,nx,path", [(64, 64, 0), (96, 160, 0), (96, 160, 1), (96, 160, 2), (256, 256, 0)])
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-11), (torch.complex64, 1e-4)])
def test_vcycle_parity_zero_guess(lib, ny, nx, path, dtype, tol):
    hz, prob = make(lib, ny, nx, abc=16, flags=path)
    f = crandn(11, (3, ny, nx))
    z = hz.vcycle(dev(f, dtype)).cpu().numpy()
    for k in range(3):
        assert relerr(z[k], H.vcycle(prob, f[k])) < tol


@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-11), (torch.complex64, 1e-4)])
def test_vcycle_parity_initial_guess(lib, dtype, tol):
    hz, prob = make(lib, 64, 96, abc=16)
    f = crandn(12, (2, 64, 96))
    x0 = crandn(13, (2, 64, 96)) * 1e-3
    x = dev(x0, dtype)
    hz.vcycle(dev(f, dtype), x)
    x = x.cpu().numpy()
    for k in range(2):
        assert relerr(x[k], H.vcycle(prob, f[k], x0[k])) < tol


@pytest.mark.parametrize("nu", [(0, 1), (2, 2), (1, 0)])
def test_vcycle_parity_other_smoothing_counts(lib, nu):
    hz, prob = make(lib, 64, 64, abc=16, nu1=nu[0], nu2=nu[1])
    f = crandn(14, (2, 64, 64))
    z = hz.vcycle(dev(f, torch.complex128)).cpu().numpy()
    for k in range(2):
        assert relerr(z[k], H.vcycle(prob, f[k])) < 1e-11


def _oracle_relres(prob, b, x):
    return np.linalg.norm(H.residual(prob.A, b, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("flags", [0, 8])   # FP32 Krylov vectors / FP64 checking mode
def test_fgmres_vcycle_matches_oracle(lib, flags):
    n = 64
    hz, prob = make(lib, n, n, abc=16)
    pos = synth.source_positions(n, n, 2, 77, 16)
    b = synth.point_sources(n, n, pos, 1.0 / n) + 0.1 * crandn(15, (2, n, n))
    x, info = hz.fgmres(dev(b, torch.complex128), tol=1e-7, maxit=2000, flags=flags)
    x = x.cpu().numpy()
    for k in range(2):
        ref = H.fgmres(prob.A, H.precond_v(prob), b[k], tol=1e-7, maxit=2000)
        rr = _oracle_relres(prob, b[k], x[k])
        assert rr <= 1e-7 and abs(rr - info["relres"][k]) <= 1e-9
        if flags & 8:
            assert info["iters"][k] == ref.iters
            assert relerr(x[k], ref.x) < 1e-8
        else:
            assert abs(info["iters"][k] - ref.iters) <= max(2, ref.iters // 20)
            assert relerr(x[k], ref.x) < 1e-4


def test_fgmres_graph_and_direct_launch_agree(lib):
    n = 64
    hz, prob = make(lib, n, n, abc=16)
    b = crandn(16, (2, n, n))
    xa, ia = hz.fgmres(dev(b, torch.complex128), flags=0)
    xb, ib = hz.fgmres(dev(b, torch.complex128), flags=lib.HELM_FLAG_NO_GRAPH)
    assert ia["iters"] == ib["iters"]
    assert torch.equal(xa, xb)


def test_fgmres_edge_cases(lib):
    n = 32
    hz, prob = make(lib, n, n, abc=8)
    b = crandn(17, (3, n, n))
    b[1] = 0.0                                  # zero rhs: x = 0 without iterating
    x, info = hz.fgmres(dev(b, torch.complex128), maxit=500)
    assert info["iters"][1] == 0 and torch.count_nonzero(x[1]) == 0
    assert info["relres"][0] <= 1e-7 and info["relres"][2] <= 1e-7
    x, info = hz.fgmres(dev(b, torch.complex128), maxit=3)      # iteration cap
    assert info["status"] == lib.HELM_MAXIT and info["iters_max"] == 3
    bn = b.copy()
    bn[0, 5, 5] = np.nan                       # non-finite input reported, not hidden
    with pytest.raises(lib.HelmError) as e:
        hz.fgmres(dev(bn, torch.complex128), maxit=50)
    assert e.value.code == lib.HELM_ENAN


def test_fgmres_host_io_matches_device(lib):
    n = 64
    hz, prob = make(lib, n, n, abc=16)
    b = crandn(18, (2, n, n))
    xd, idv = hz.fgmres(dev(b, torch.complex128))
    bh = torch.from_numpy(b).pin_memory()
    xh = torch.zeros_like(bh).pin_memory()
    _, ih = hz.fgmres(bh, xh, flags=lib.HELM_FLAG_HOST_IO | lib.HELM_FLAG_X0_ZERO)
    assert ih["iters"] == idv["iters"]
    assert torch.equal(xh, xd.cpu())


@pytest.mark.parametrize("n", [576, 1024])
def test_coarse_gmres_large_grid_parity(lib, n):
    """Coarsest grids whose Krylov basis does not fit in a cluster's shared memory (144²
    and 256²) take the cluster kernel with the basis in global memory (1024 threads per
    CTA); parity with the oracle's GMRES(10) holds there too."""
    hz, prob = make(lib, n, n, abc=16)
    lc = prob.hierarchy[-1]
    f = crandn(19, (2, lc.ny, lc.nx))
    x = hz.coarse_solve(dev(f, torch.complex64)).cpu().numpy()
    for k in range(2):
        assert relerr(x[k], H.gmres_jacobi(lc, f[k], prob.coarse_its)) < 2e-5


def test_fgmres_full_size_bench_config(lib):
    """256^2, 8 point sources (the benchmark workload): every solution's true FP64
    residual, recomputed by the oracle, is <= 1e-7, and sampled entries of A x
    computed one by one by the oracle's stencil match b."""
    n = 256
    hz, prob = make(lib, n, n, abc=16)
    pos = synth.source_positions(n, n, 8, synth.rhs_seed(0), 16)
    b = synth.point_sources(n, n, pos, 1.0 / n)
    x, info = hz.fgmres(dev(b, torch.complex128), tol=1e-7, maxit=5000)
    x = x.cpu().numpy()
    assert info["status"] == 0
    for k in range(8):
        assert _oracle_relres(prob, b[k], x[k]) <= 1e-7


# ---------------------------------------------------------------- block FGMRES
def _block_rhs(n, count, seed):
    pos = synth.source_positions(n, n, count - 1, seed, 4)
    return np.concatenate([synth.point_sources(n, n, pos, 1.0 / n), crandn(seed + 1, (1, n, n))])


def test_block_fgmres_fp64_matches_oracle(lib):
    """Block FGMRES(10) + M_V with FP64 Krylov vectors: the oracle's block iterations (its
    QR by Householder, ours by Cholesky QR twice) and FP64 residuals <= tol."""
    n = 32
    hz, prob = make(lib, n, n, abc=4)
    b = _block_rhs(n, 3, 51)
    x, info = hz.fgmres(dev(b, torch.complex128), tol=1e-9, maxit=500, flags=8, block=True)
    ref = H.block_fgmres(prob.A, H.precond_v(prob), b, m=10, tol=1e-9, maxit=500)
    assert info["status"] == 0 and ref.converged
    assert abs(info["iters_max"] - ref.iters) <= 1
    x = x.cpu().numpy()
    for k in range(3):
        assert _oracle_relres(prob, b[k], x[k]) <= 1e-9


@pytest.mark.parametrize("p", [1, 8])
def test_block_fgmres_fp32(lib, p):
    """FP32 block FGMRES(10) + M_V on 64^2: converged FP64 residuals <= 1e-7 (oracle
    recomputed), block iterations within 15 % of the oracle's; one column matches FGMRES."""
    n = 64
    hz, prob = make(lib, n, n, abc=16)
    b = _block_rhs(n, p, 52)
    x, info = hz.fgmres(dev(b, torch.complex128), tol=1e-7, maxit=2000, block=True)
    ref = H.block_fgmres(prob.A, H.precond_v(prob), b, m=10, tol=1e-7, maxit=2000)
    assert info["status"] == 0
    assert abs(info["iters_max"] - ref.iters) <= max(1, 0.15 * ref.iters)
    x = x.cpu().numpy()
    for k in range(p):
        assert _oracle_relres(prob, b[k], x[k]) <= 1e-7
    if p == 1:
        _, i1 = hz.fgmres(dev(b, torch.complex128), tol=1e-7, maxit=2000)
        assert abs(i1["iters_max"] - info["iters_max"]) <= 1


def test_block_and_subspace_size_sweep(lib):
    """The influence of the block size and of the subspace size (Sec. 4, the paper's sweep
    over both): block FGMRES(m) with M_V for block sizes 1, 2, 4 and restart lengths 5, 10,
    20 on the same point sources; every run reaches the FP64 true residual 1e-7 (the oracle
    recomputes it for the widest block), and a longer restart never needs more iterations
    than restart 5 at the same block size by more than 10 %.  profcase sweep prints the
    full table (profiles/block_subspace_sweep_256x256x16.md)."""
    n = 128
    hz, prob = make(lib, n, n, abc=16)
    pos = synth.source_positions(n, n, 4, synth.rhs_seed(3), 16)
    b = synth.point_sources(n, n, pos, 1.0 / n)
    bt = torch.from_numpy(b).cuda()
    its = {}
    for m in (5, 10, 20):
        for bs in (1, 2, 4):
            x, info = hz.fgmres(bt[:bs].contiguous(), tol=1e-7, maxit=5000, restart=m, block=True)
            assert info["status"] == lib.HELM_OK and info["relres_max"] <= 1e-7, (m, bs, info)
            its[(m, bs)] = info["iters_max"]
            if bs == 4:
                xs = x.cpu().numpy()
                for k in range(4):
                    assert np.linalg.norm(H.residual(prob.A, b[k], xs[k])) <= 1e-7 * np.linalg.norm(b[k])
    for bs in (1, 2, 4):
        for m in (10, 20):
            assert its[(m, bs)] <= 1.1 * its[(5, bs)], its
