"""Guard zones: each output a library call writes is a view in the middle of a larger
buffer whose margins hold a sentinel; after the call the margins must be unchanged (no
write out of bounds).  Ragged grids (tiles of 32 x 8 with tails; a 9 x 17 coarsest level),
every boundary mode and both stencils, FP32 and FP64 vectors.  (Reads out of bounds are
not visible this way; the parity tests compare every written value.)"""
import math

import pytest

from gpu_util import crandn, medium

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

G = 4096                        # margin elements on each side
SENTINEL = complex(1234.5, -678.25)


@pytest.fixture(scope="module")
def lib():
    from paper_2203_11025_gb300 import build
    from paper_2203_11025_gb300 import lib as L
    build.build()
    return L


def guarded(shape, dtype, fill=None):
    """(buffer, view): a contiguous view of `shape` inside sentinel margins."""
    n = math.prod(shape)
    val = SENTINEL if dtype.is_complex else SENTINEL.real
    buf = torch.full((G + n + G,), val, dtype=dtype, device="cuda")
    view = buf[G:G + n].view(shape)
    if fill is not None:
        view.copy_(fill)
    return buf, view


def intact(buf, shape):
    n = math.prod(shape)
    val = SENTINEL if buf.dtype.is_complex else SENTINEL.real
    ref = torch.full((G,), val, dtype=buf.dtype, device="cuda")
    torch.cuda.synchronize()
    return torch.equal(buf[:G], ref) and torch.equal(buf[G + n:], ref)


CASES = [("dirichlet", 0), ("reflect", 0), ("replicate", 0), ("dirichlet", 1)]   # (boundary, stencil)
GRIDS = [(40, 24, 3), (18, 34, 2)]


def make(lib, ny, nx, levels, bc, stencil):
    code = {"dirichlet": lib.HELM_BC_DIRICHLET, "reflect": lib.HELM_BC_REFLECT,
            "replicate": lib.HELM_BC_REPLICATE}[bc]
    k2 = torch.from_numpy(medium(ny, nx, 1000 + ny)).cuda()
    return lib.Helmholtz(k2, levels=levels, abc_width=4, omega=20.0, h=1.0 / nx, bc=code, stencil=stencil)


@pytest.mark.parametrize("bc,stencil", CASES)
@pytest.mark.parametrize("ny,nx,levels", GRIDS)
@pytest.mark.parametrize("dtype", [torch.complex64, torch.complex128])
def test_stencil_transfer_and_coarse_outputs_stay_in_bounds(lib, bc, stencil, ny, nx, levels, dtype):
    hz = make(lib, ny, nx, levels, bc, stencil)
    x = torch.from_numpy(crandn(1, (3, ny, nx))).to(dtype).cuda()
    b = torch.from_numpy(crandn(2, (3, ny, nx))).to(dtype).cuda()
    shape = (3, ny, nx)
    for op in (lib.HELM_OP_A, lib.HELM_OP_M, lib.HELM_OP_RHS):
        buf, out = guarded(shape, dtype)
        hz.apply(x, op=op, out=out)
        assert intact(buf, shape) and torch.isfinite(torch.view_as_real(out)).all()
    buf, out = guarded(shape, dtype)
    hz.residual(b, x, out=out)
    assert intact(buf, shape)
    for x_in in (x, None):
        buf, out = guarded(shape, dtype)
        hz.jacobi(b, x_in, out=out)
        assert intact(buf, shape)
    cy, cx = hz.level_shape(1)
    buf, out = guarded((3, cy, cx), dtype)
    hz.restrict(b, out=out)
    assert intact(buf, (3, cy, cx))
    ec = torch.from_numpy(crandn(3, (3, cy, cx))).to(dtype).cuda()
    buf, fine = guarded(shape, dtype, fill=x)
    hz.prolong_add(ec, fine)
    assert intact(buf, shape)
    ly, lx = hz.level_shape(levels - 1)
    f = torch.from_numpy(crandn(4, (3, ly, lx))).to(dtype).cuda()
    buf, out = guarded((3, ly, lx), dtype)
    hz.coarse_solve(f, out=out)
    assert intact(buf, (3, ly, lx))
    buf, xv = guarded(shape, dtype, fill=torch.zeros(shape, dtype=dtype, device="cuda"))
    hz.vcycle(b, xv)
    assert intact(buf, shape)


@pytest.mark.parametrize("bc,stencil", CASES)
@pytest.mark.parametrize("flags", [0, 8])          # FP32 Krylov vectors / FP64 checking mode
def test_fgmres_solution_stays_in_bounds(lib, bc, stencil, flags):
    ny, nx, levels = 40, 24, 3
    hz = make(lib, ny, nx, levels, bc, stencil)
    b = torch.from_numpy(crandn(5, (3, ny, nx))).cuda()
    buf, xv = guarded((3, ny, nx), torch.complex128, fill=torch.zeros(3, ny, nx, dtype=torch.complex128,
                                                                       device="cuda"))
    _, info = hz.fgmres(b, xv, tol=1e-7, maxit=2000, flags=flags)
    assert info["status"] in (lib.HELM_OK, lib.HELM_MAXIT) and intact(buf, (3, ny, nx))


@pytest.mark.parametrize("kind", ["ju", "vu"])
def test_network_preconditioner_output_stays_in_bounds(lib, kind):
    ny, nx = 32, 48
    hz = make(lib, ny, nx, 3, "dirichlet", 0)
    c = lib.unet_cfg()
    c.in_ch, c.out_ch, c.levels, c.coarse_resnets = 4, 2, 2, 1
    c.widths[0], c.widths[1] = 16, 32
    net = lib.UNet(c, seed=3)
    pc = lib.HELM_PREC_JU if kind == "ju" else lib.HELM_PREC_VU
    for dtype in (torch.complex64, torch.complex128):
        r = torch.from_numpy(crandn(6, (3, ny, nx))).to(dtype).cuda()
        buf, out = guarded((3, ny, nx), dtype)
        hz.unet_precond(net, r, kind=pc, out=out)
        assert intact(buf, (3, ny, nx)) and torch.isfinite(torch.view_as_real(out)).all()
