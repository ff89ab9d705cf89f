"""The allocation-free coarsest-grid solve (helm_coarse_solve_static) gives the same
result as the handle-based entry point (helm_coarse_solve) and as the FP64 oracle's
GMRES(10) with diagonal right preconditioning (Sec. 2.4, 4), on two calls in a row.

It exists for callers that cannot call cudaMalloc (graph capture in progress,
real-time loops that must avoid cudaMalloc's implicit synchronisation, fixed
memory budgets): its Krylov basis lives in a static device array, so the test
also checks that a second call, which finds the previous call's data in that
array, is unaffected.  Collected last so that a stop at the first failure has
already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_static_coarse_solve_matches_handle_entry_point():
    from paper_2203_11025_gb300 import build
    from paper_2203_11025_gb300 import lib
    from paper_2203_11025_gb300 import synth
    build.build()
    n = 128
    k2 = synth.grf_kappa2(n, n, 1000)
    hz = lib.Helmholtz(torch.from_numpy(k2).cuda())
    d = hz.desc
    lc = d.levels - 1
    ny, nx = hz.level_shape(lc)
    k2c = hz.level_kappa2(lc).to(torch.float32).contiguous()
    hc = d.h * (1 << lc)
    width = d.abc_width >> lc
    from oracle import helmholtz as H
    prob = H.Problem(k2.astype(np.float64), omega=d.omega, h=d.h, abc_width=d.abc_width,
                     gamma_max=d.abc_gamma_max, beta=d.beta, levels=d.levels, coarse_its=d.coarse_its)
    lc_oracle = prob.hierarchy[-1]
    for call, seed in enumerate((31, 32)):
        f = torch.from_numpy(synth.complex_normal(seed, (5, ny, nx))).to(torch.complex64).cuda()
        ref = hz.coarse_solve(f)
        x = torch.full_like(f, float("nan"))
        lib.helm_coarse_solve_static(nx, ny, hc, d.omega, d.beta, width, d.abc_gamma_max, k2c, f, x, 5,
                                     d.coarse_its)
        torch.cuda.synchronize()
        a, b = x.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a)), f"call {call}"
        assert np.abs(a - b).max() / np.abs(b).max() < 2e-5, f"call {call}"
        fh = f.cpu().numpy().astype(np.complex128)
        for k in range(5):
            ref_k = H.gmres_jacobi(lc_oracle, fh[k], d.coarse_its)
            assert np.abs(a[k] - ref_k).max() / np.abs(ref_k).max() < 2e-5, f"call {call}, rhs {k}"
    # sizes beyond the static array are refused with a clear error, before any launch
    big = torch.zeros(64, ny, nx, dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.HelmError) as e:
        lib.helm_coarse_solve_static(nx, ny, hc, d.omega, d.beta, width, d.abc_gamma_max, k2c, big,
                                     torch.empty_like(big), 64, 32)
    assert "static scratch" in str(e.value)
    # f and x must not share bytes: x one right-hand side past f is refused
    buf = torch.zeros(6, ny, nx, dtype=torch.complex64, device="cuda")
    with pytest.raises(lib.HelmError) as e:
        lib.helm_coarse_solve_static(nx, ny, hc, d.omega, d.beta, width, d.abc_gamma_max, k2c, buf[:5],
                                     buf[1:], 5, d.coarse_its)
    assert "overlap" in str(e.value)
