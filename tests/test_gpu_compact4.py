"""GPU parity for the compact fourth-order 9-point scheme (the higher-order operators the
convolution form of Sec. 2.4 admits): operator, residual and Jacobi on every level, the
scheme's right-hand side, the coarsest-grid GMRES paths, V-cycles and FGMRES against the
FP64 oracle with the same scheme; and, independently of the oracle, fourth-order
convergence of the GPU solution to a smooth continuum solution.

Tolerances as for the 5-point parity tests: FP64 kernels 1e-12 (max-norm), FP32
stencils 1e-5, composed V-cycles 1e-4 in FP32."""
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


def make(lib, ny, nx, seed=1000, levels=3, abc=16, **kw):
    k2 = medium(ny, nx, seed)
    h, om = 1.0 / nx, synth.omega_for(nx)
    hz = lib.Helmholtz(torch.from_numpy(k2).cuda(), levels=levels, abc_width=abc, omega=om, h=h,
                       stencil=lib.HELM_STENCIL_COMPACT4, **kw)
    d = hz.desc
    prob = H.Problem(k2.astype(np.float64), omega=om, h=h, abc_width=abc, gamma_max=d.abc_gamma_max,
                     beta=d.beta, levels=levels, nu1=d.nu1, nu2=d.nu2, jacobi_w=d.jacobi_w,
                     coarse_its=d.coarse_its, order=4)
    return hz, prob


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


DTYPES = [(torch.complex128, 1e-12), (torch.complex64, 1e-5)]


@pytest.mark.parametrize("ny,nx", [(48, 80), (40, 24)])
@pytest.mark.parametrize("dtype,tol", DTYPES)
def test_apply_residual_jacobi_rhs_parity(lib, ny, nx, dtype, tol):
    hz, prob = make(lib, ny, nx, abc=6)
    x = crandn(1, (3, ny, nx))
    b = crandn(2, (3, ny, nx))
    for op, lv in ((lib.HELM_OP_A, prob.A), (lib.HELM_OP_M, prob.M)):
        assert relerr(hz.apply(dev(x, dtype), op=op).cpu().numpy(), H.apply_op(lv, x)) < tol
        r = hz.residual(dev(b, dtype), dev(x, dtype), op=op).cpu().numpy()
        assert relerr(r, H.residual(lv, b, x)) < tol
        out = hz.jacobi(dev(b, dtype), dev(x, dtype), op=op).cpu().numpy()
        assert relerr(out, H.jacobi(lv, x, b, 0.8)) < tol
    assert relerr(hz.apply(dev(b, dtype), op=lib.HELM_OP_RHS).cpu().numpy(), H.rhs_weight(prob.A, b)) < tol
    for level in (1, 2):
        lv = prob.hierarchy[level]
        xc = crandn(3 + level, (2, lv.ny, lv.nx))
        y = hz.apply(dev(xc, dtype), op=lib.HELM_OP_M, level=level).cpu().numpy()
        assert relerr(y, H.apply_op(lv, xc)) < tol


def test_setup_and_entry_points_reject_unsupported_combinations(lib):
    k2 = torch.from_numpy(medium(32, 32)).cuda()
    with pytest.raises(Exception):      # the compact scheme is built for Dirichlet boundaries only
        lib.Helmholtz(k2, stencil=lib.HELM_STENCIL_COMPACT4, bc=lib.HELM_BC_REFLECT)
    with pytest.raises(Exception):
        lib.Helmholtz(k2, stencil=2)
    hz = lib.Helmholtz(k2, stencil=lib.HELM_STENCIL_COMPACT4)
    y = torch.zeros(1, 32, 32, 2, device="cuda")
    x = torch.zeros(1, 32, 32, 4, device="cuda")
    with pytest.raises(Exception):      # the residual loss is built for the 5-point stencil
        hz.residual_loss(y, x)
    v = dev(crandn(3, (1, 32, 32)), torch.complex64)
    with pytest.raises(Exception):      # helm_residual takes A or M only
        hz.residual(v, v.clone(), op=lib.HELM_OP_RHS)
    with pytest.raises(Exception):      # outputs must not alias inputs
        hz.apply(v, out=v)
    with pytest.raises(Exception):
        hz.residual(v, v.clone(), out=v)


@pytest.mark.parametrize("path", [0, 1, 2])   # cluster (declines: one-CTA kernel), multi-kernel, one CTA
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-11), (torch.complex64, 2e-5)])
def test_coarse_gmres_parity(lib, path, dtype, tol):
    hz, prob = make(lib, 128, 96, flags=path)
    lc = prob.hierarchy[-1]
    f = crandn(10, (3, lc.ny, lc.nx))
    x = hz.coarse_solve(dev(f, dtype)).cpu().numpy()
    for k in range(3):
        assert relerr(x[k], H.gmres_jacobi(lc, f[k], prob.coarse_its)) < tol


@pytest.mark.parametrize("ny,nx,path", [(96, 160, 0), (96, 160, 1), (64, 64, 2)])
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-11), (torch.complex64, 1e-4)])
def test_vcycle_parity(lib, ny, nx, path, dtype, tol):
    hz, prob = make(lib, ny, nx, flags=path)
    f = crandn(11, (2, ny, nx))
    z = hz.vcycle(dev(f, dtype)).cpu().numpy()
    x0 = crandn(12, (2, ny, nx)) * 1e-3
    x = dev(x0, dtype)
    hz.vcycle(dev(f, dtype), x)
    x = x.cpu().numpy()
    for k in range(2):
        assert relerr(z[k], H.vcycle(prob, f[k])) < tol
        assert relerr(x[k], H.vcycle(prob, f[k], x0[k])) < tol


def test_fgmres_fp64_matches_oracle_and_dense_solve(lib):
    n = 32
    hz, prob = make(lib, n, n, abc=8)
    b = np.concatenate([synth.point_sources(n, n, [(10, 20)], 1.0 / n), crandn(16, (1, n, n))])
    x, info = hz.fgmres(dev(b, torch.complex128), tol=1e-10, maxit=2000, flags=lib.HELM_FLAG_FP64)
    x = x.cpu().numpy()
    K = H.assemble_dense(prob.A)
    for k in range(2):
        ref = H.fgmres(prob.A, H.precond_v(prob), b[k], tol=1e-10, maxit=2000)
        assert info["iters"][k] == ref.iters
        exact = H.lu_solve(K, b[k].ravel()).reshape(n, n)
        assert np.linalg.norm(x[k] - exact) <= 1e-8 * np.linalg.norm(exact)


def test_fgmres_fp32_reaches_tolerance(lib):
    n = 128
    hz, prob = make(lib, n, n)
    b = crandn(17, (4, n, n))
    x, info = hz.fgmres(dev(b, torch.complex128), tol=1e-7, maxit=3000)
    x = x.cpu().numpy()
    assert info["status"] == lib.HELM_OK
    for k in range(4):
        assert np.linalg.norm(H.residual(prob.A, b[k], x[k])) <= 1e-7 * np.linalg.norm(b[k])


def test_fourth_order_convergence_on_the_gpu(lib):
    """u = sin(pi x) sin(2 pi y) in k^2 = 1 + 0.5 sin(pi x) cos(pi y), no layer, nodes at
    (i+1)h with h = 1/(n+1): the GPU solution of K u = (1/12) M5 f (right-hand side from
    helm_apply with HELM_OP_RHS) approaches u by (33/17)^4 = 14.2 from n = 16 to 32."""
    errs = []
    for n in (16, 32):
        h = 1.0 / (n + 1)
        x = (np.arange(n) + 1) * h
        X, Y = x[None, :], x[:, None]
        U = np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
        k2 = (1.0 + 0.5 * np.sin(np.pi * X) * np.cos(np.pi * Y)).astype(np.float32)
        omega = 6.0
        hz = lib.Helmholtz(torch.from_numpy(k2).cuda(), levels=3, abc_width=0, omega=omega, h=h,
                           stencil=lib.HELM_STENCIL_COMPACT4)
        f = ((5 * np.pi ** 2 - omega ** 2 * k2.astype(np.float64)) * U)[None] + 0j
        b = hz.apply(dev(f, torch.complex128), op=lib.HELM_OP_RHS)
        xs, info = hz.fgmres(b, tol=1e-11, maxit=3000, flags=lib.HELM_FLAG_FP64)
        assert info["status"] == lib.HELM_OK
        errs.append(np.abs(xs.cpu().numpy()[0] - U).max())
    ratio = errs[0] / errs[1]
    assert 0.9 * (33 / 17) ** 4 < ratio < 1.1 * (33 / 17) ** 4
