"""GPU parity for Neumann boundaries (Sec. 2.4: the stencil's convolution padded by
reflection or replication instead of zeros): every kernel that applies the 5-point
stencil — operator and residual, Jacobi, the fused restriction and prolongation
sweeps, the three coarsest-grid GMRES paths, the FGMRES Arnoldi and FP64 true-residual
kernels and the residual loss — against the FP64 oracle with the same boundary mode.

Tolerances as for the Dirichlet parity tests: FP64 kernels 1e-12 (max-norm), FP32
stencils 1e-5, composed V-cycles 1e-4 in FP32."""
import numpy as np
import pytest

from gpu_util import crandn, medium, relerr
from oracle import helmholtz as H
from paper_2203_11025_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BCS = ["reflect", "replicate"]


@pytest.fixture(scope="module")
def lib():
    from paper_2203_11025_gb300 import build
    from paper_2203_11025_gb300 import lib as L
    build.build()
    return L


def make(lib, ny, nx, bc, seed=1000, levels=3, abc=16, **kw):
    code = {"dirichlet": lib.HELM_BC_DIRICHLET, "reflect": lib.HELM_BC_REFLECT,
            "replicate": lib.HELM_BC_REPLICATE}[bc]
    k2 = medium(ny, nx, seed)
    h, om = 1.0 / nx, synth.omega_for(nx)
    hz = lib.Helmholtz(torch.from_numpy(k2).cuda(), levels=levels, abc_width=abc, omega=om, h=h, bc=code, **kw)
    d = hz.desc
    prob = H.Problem(k2.astype(np.float64), omega=om, h=h, abc_width=abc, gamma_max=d.abc_gamma_max,
                     beta=d.beta, levels=levels, nu1=d.nu1, nu2=d.nu2, jacobi_w=d.jacobi_w,
                     coarse_its=d.coarse_its, bc=bc)
    return hz, prob


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


DTYPES = [(torch.complex128, 1e-12), (torch.complex64, 1e-5)]


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("ny,nx", [(48, 80), (40, 24)])
@pytest.mark.parametrize("dtype,tol", DTYPES)
def test_apply_residual_jacobi_parity(lib, bc, ny, nx, dtype, tol):
    hz, prob = make(lib, ny, nx, bc, abc=6)
    x = crandn(1, (3, ny, nx))
    b = crandn(2, (3, ny, nx))
    for op, lv in ((lib.HELM_OP_A, prob.A), (lib.HELM_OP_M, prob.M)):
        assert relerr(hz.apply(dev(x, dtype), op=op).cpu().numpy(), H.apply_op(lv, x)) < tol
        r = hz.residual(dev(b, dtype), dev(x, dtype), op=op).cpu().numpy()
        assert relerr(r, H.residual(lv, b, x)) < tol
        out = hz.jacobi(dev(b, dtype), dev(x, dtype), op=op).cpu().numpy()
        assert relerr(out, H.jacobi(lv, x, b, 0.8)) < tol
    for level in (1, 2):
        lv = prob.hierarchy[level]
        xc = crandn(3 + level, (2, lv.ny, lv.nx))
        y = hz.apply(dev(xc, dtype), op=lib.HELM_OP_M, level=level).cpu().numpy()
        assert relerr(y, H.apply_op(lv, xc)) < tol


def test_setup_rejects_bad_boundary_modes(lib):
    k2 = torch.from_numpy(medium(16, 16)).cuda()
    with pytest.raises(Exception):
        lib.Helmholtz(k2, levels=3, bc=3)
    with pytest.raises(Exception):   # reflection needs a coarsest level of at least 2 x 2
        lib.Helmholtz(k2, levels=5, abc_width=0, bc=lib.HELM_BC_REFLECT)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("path", [0, 1, 2])   # cluster (default), multi-kernel, one CTA per right-hand side
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-11), (torch.complex64, 2e-5)])
def test_coarse_gmres_parity(lib, bc, path, dtype, tol):
    hz, prob = make(lib, 128, 96, bc, flags=path)
    lc = prob.hierarchy[-1]
    f = crandn(10, (3, lc.ny, lc.nx))
    x = hz.coarse_solve(dev(f, dtype)).cpu().numpy()
    for k in range(3):
        assert relerr(x[k], H.gmres_jacobi(lc, f[k], prob.coarse_its)) < tol


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("ny,nx,path", [(96, 160, 0), (96, 160, 1), (64, 64, 2)])
@pytest.mark.parametrize("dtype,tol", [(torch.complex128, 1e-11), (torch.complex64, 1e-4)])
def test_vcycle_parity(lib, bc, ny, nx, path, dtype, tol):
    hz, prob = make(lib, ny, nx, bc, flags=path)
    f = crandn(11, (2, ny, nx))
    z = hz.vcycle(dev(f, dtype)).cpu().numpy()
    x0 = crandn(12, (2, ny, nx)) * 1e-3
    x = dev(x0, dtype)
    hz.vcycle(dev(f, dtype), x)
    x = x.cpu().numpy()
    for k in range(2):
        assert relerr(z[k], H.vcycle(prob, f[k])) < tol
        assert relerr(x[k], H.vcycle(prob, f[k], x0[k])) < tol


@pytest.mark.parametrize("bc", BCS)
def test_fgmres_fp64_matches_oracle_and_dense_solve(lib, bc):
    n = 32
    hz, prob = make(lib, n, n, bc, abc=8)
    b = synth.point_sources(n, n, [(10, 20)], 1.0 / n) + 0.1 * crandn(15, (1, n, n))
    b = np.concatenate([b, crandn(16, (1, n, n))])
    x, info = hz.fgmres(dev(b, torch.complex128), tol=1e-10, maxit=2000, flags=lib.HELM_FLAG_FP64)
    x = x.cpu().numpy()
    K = H.assemble_dense(prob.A)
    for k in range(2):
        ref = H.fgmres(prob.A, H.precond_v(prob), b[k], tol=1e-10, maxit=2000)
        assert info["iters"][k] == ref.iters
        exact = H.lu_solve(K, b[k].ravel()).reshape(n, n)
        assert np.linalg.norm(x[k] - exact) <= 1e-8 * np.linalg.norm(exact)


@pytest.mark.parametrize("bc", ["dirichlet"] + BCS)
def test_residual_loss_parity(lib, bc):
    from oracle import precond as PR
    n = 64
    hz, prob = make(lib, n, n, bc, levels=1)
    rng = np.random.default_rng(31)
    y = rng.standard_normal((2, n, n, 2)).astype(np.float32)
    x = rng.standard_normal((2, n, n, 4)).astype(np.float32)
    loss, g = hz.residual_loss(torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda())
    ref_loss, ref_g = PR.residual_loss(prob, y.astype(np.float64), x.astype(np.float64))
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * ref_loss
    g = g.cpu().numpy()
    assert np.linalg.norm(g - ref_g) <= 1e-5 * np.linalg.norm(ref_g)
