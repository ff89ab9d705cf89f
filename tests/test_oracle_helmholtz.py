"""Pins of the FP64 oracle (operator, transfers, V-cycle, GMRES, FGMRES) against
what the paper and the mathematics fix, independently of the oracle itself."""
import numpy as np
import pytest

from conftest import load_golden_kernels
from oracle import helmholtz as H
from paper_2203_11025_gb300 import synth


def _level(ny, nx, seed=0, omega=20.0, beta=0.3, width=3):
    rng = np.random.default_rng(seed)
    k2 = rng.uniform(0.1, 1.0, (ny, nx))
    g = H.abc_gamma(ny, nx, width, 1.0)
    return H.Level(ny, nx, 1.0 / nx, omega, k2, g, beta)


def _crandn(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- operator
def test_stencil_matches_printed_kernel():
    """Eq. 2.2: h^2 (A u) at an interior node of a delta reproduces the printed
    off-centre stencil; the centre is 4 - w^2 k^2 h^2 (1 - g i)."""
    gold = load_golden_kernels()["stencil_offdiag"]
    lv = _level(9, 11, beta=0.0)
    u = np.zeros((9, 11), complex)
    u[4, 5] = 1.0
    y = H.apply_op(lv, u) * lv.h ** 2
    off = y[3:6, 4:7].copy()
    centre = off[1, 1]
    off[1, 1] = 0
    assert np.allclose(off, gold, atol=1e-14)
    k2, g = lv.kappa2[4, 5], lv.gamma[4, 5]
    assert np.isclose(centre, 4 - lv.omega ** 2 * k2 * lv.h ** 2 * (1 - g * 1j), rtol=1e-14)
    # a node inside the absorbing layer (g > 0): the attenuation enters as (1 - g i)
    u = np.zeros((9, 11), complex)
    u[1, 5] = 1.0
    k2, g = lv.kappa2[1, 5], lv.gamma[1, 5]
    assert g > 0
    c = (H.apply_op(lv, u) * lv.h ** 2)[1, 5]
    assert np.isclose(c, 4 - lv.omega ** 2 * k2 * lv.h ** 2 * (1 - g * 1j), rtol=1e-14)


def test_apply_matches_nodewise_assembly():
    """Array-shift formulation == explicit node-by-node assembly (non-square grid)."""
    lv = _level(7, 10, seed=1)
    u = _crandn(np.random.default_rng(2), (7, 10))
    K = H.assemble_dense(lv)
    assert np.allclose(H.apply_op(lv, u).ravel(), K @ u.ravel(), rtol=1e-14, atol=1e-12)


@pytest.mark.parametrize("ny,nx", [(12, 12), (10, 14)])
def test_discrete_laplacian_eigenpairs(ny, nx):
    """Constant medium, no attenuation: sin modes are eigenvectors with the closed-form
    eigenvalue (4/h^2)[sin^2(j pi/(2(nx+1))) + sin^2(k pi/(2(ny+1)))] - w^2 k^2."""
    h, omega, k2 = 1.0 / nx, 17.0, 0.7
    lv = H.Level(ny, nx, h, omega, np.full((ny, nx), k2), np.zeros((ny, nx)), 0.0)
    p = np.arange(ny)[:, None]
    q = np.arange(nx)[None, :]
    for j, k in [(1, 1), (2, 5), (ny, nx), (3, 1)]:
        v = np.sin(j * np.pi * (p + 1) / (ny + 1)) * np.sin(k * np.pi * (q + 1) / (nx + 1)) + 0j
        lam = (4 / h ** 2) * (np.sin(j * np.pi / (2 * (ny + 1))) ** 2
                              + np.sin(k * np.pi / (2 * (nx + 1))) ** 2) - omega ** 2 * k2
        assert np.allclose(H.apply_op(lv, v), lam * v, rtol=1e-12, atol=1e-9 * abs(lam))


def test_complex_symmetric_and_absorbing():
    """A^T = A (complex symmetric), and Im(x^H A x) = w^2 sum k^2 (g+beta) |x|^2 >= 0."""
    lv = _level(6, 8, seed=3, beta=0.5)
    K = H.assemble_dense(lv)
    assert np.allclose(K, K.T, atol=0)
    rng = np.random.default_rng(4)
    for _ in range(5):
        x = _crandn(rng, (6, 8))
        q = np.vdot(x, H.apply_op(lv, x))
        expect = lv.omega ** 2 * np.sum(lv.kappa2 * (lv.gamma + lv.beta) * np.abs(x) ** 2)
        assert q.imag >= 0 and np.isclose(q.imag, expect, rtol=1e-12)


def test_abc_profile():
    """Quadratic layer: 1 on the outermost unknowns, (1 - d/W)^2 inside, 0 in the interior."""
    g = H.abc_gamma(40, 40, 16, 1.0)
    assert g[0, 20] == 1.0 and g[20, 0] == 1.0 and g[39, 20] == 1.0
    assert np.isclose(g[20, 3], (1 - 3 / 16) ** 2)
    assert g[20, 16] == 0.0 and g[20, 20] == 0.0
    assert np.isclose(g[5, 7], (1 - 5 / 16) ** 2)   # nearest edge decides


# ---------------------------------------------------------------- transfers
def test_transfer_kernels_match_paper():
    """Eq. 2.9: P of a coarse delta is the printed bilinear kernel centred on the fine
    node 2I; R^T of a coarse delta is the printed full-weighting kernel."""
    gold = load_golden_kernels()
    n = 12
    e = np.zeros((6, 6))
    e[2, 3] = 1.0
    Pe = H.prolong_bilinear(e, n, n)
    assert np.allclose(Pe[3:6, 5:8], gold["prolong"], atol=0)
    assert np.isclose(Pe.sum(), gold["prolong"].sum())
    # R^T e: column of R for a coarse delta, via R applied to fine deltas
    Rt = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            d = np.zeros((n, n))
            d[i, j] = 1.0
            Rt[i, j] = H.restrict_fw(d)[2, 3]
    assert np.allclose(Rt[3:6, 5:8], gold["restrict"], atol=0)
    assert np.isclose(Rt.sum(), 1.0)


def test_restriction_is_quarter_prolongation_transpose():
    ny, nx = 8, 10
    N, Nc = ny * nx, (ny // 2) * (nx // 2)
    P = np.zeros((N, Nc))
    R = np.zeros((Nc, N))
    for k in range(Nc):
        e = np.zeros(Nc)
        e[k] = 1
        P[:, k] = H.prolong_bilinear(e.reshape(ny // 2, nx // 2), ny, nx).ravel()
    for k in range(N):
        e = np.zeros(N)
        e[k] = 1
        R[:, k] = H.restrict_fw(e.reshape(ny, nx)).ravel()
    assert np.array_equal(R, P.T / 4)


def test_transfers_reproduce_constants_and_bilinears():
    n = 16
    c = np.full((n, n), 3.5)
    Rc = H.restrict_fw(c)
    assert np.allclose(Rc[1:, 1:], 3.5)            # interior coarse nodes (not touching node -1)
    I = np.arange(n // 2)[:, None]
    J = np.arange(n // 2)[None, :]
    lin = 1.0 + 0.3 * (2 * I) - 0.7 * (2 * J) + 0.05 * (2 * I) * (2 * J)
    Pl = H.prolong_bilinear(lin, n, n)
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    exact = 1.0 + 0.3 * i - 0.7 * j + 0.05 * i * j
    assert np.allclose(Pl[:n - 1, :n - 1], exact[:n - 1, :n - 1], atol=1e-13)


def test_coarse_operator_consistent_with_galerkin():
    """Rediscretisation on H = 2h agrees with R A_h P on smooth interior functions to
    O(H^2): the error drops ~4x per refinement (pins the coarse spacing and medium)."""
    errs = []
    for n in (32, 64, 128):
        yy, xx = np.meshgrid(np.arange(n) / n, np.arange(n) / n, indexing="ij")
        k2 = 0.5 + 0.3 * np.sin(2 * np.pi * xx) * np.cos(np.pi * yy)
        prob = H.Problem(k2, omega=30.0, h=1.0 / n, abc_width=0, beta=0.5, levels=2)
        f0, f1 = prob.hierarchy
        Y, X = np.meshgrid(np.arange(n // 2) * 2 / n, np.arange(n // 2) * 2 / n, indexing="ij")
        phi = np.sin(3 * X + 1) * np.cos(2 * Y) + 0j
        gal = H.restrict_fw(H.apply_op(f0, H.prolong_bilinear(phi, n, n)))
        red = H.apply_op(f1, phi)
        s = slice(2, n // 2 - 2)
        errs.append(np.abs(gal - red)[s, s].max() / np.abs(red[s, s]).max())
    assert errs[0] < 0.02
    assert 3.2 < errs[0] / errs[1] < 4.8 and 3.2 < errs[1] / errs[2] < 4.8


def test_coarse_medium_is_weighted_average():
    k2 = np.random.default_rng(5).uniform(0.0625, 1.0, (16, 16))
    c = H.coarsen_kappa2(k2)
    assert c.min() >= k2.min() - 1e-15 and c.max() <= k2.max() + 1e-15
    assert np.isclose(c[3, 4], np.sum(load_golden_kernels()["restrict"] * k2[5:8, 7:10]))
    # corner (0,0): weights 4,2,2,1 over the in-domain 2x2 block, renormalised by 9
    assert np.isclose(c[0, 0], (4 * k2[0, 0] + 2 * k2[0, 1] + 2 * k2[1, 0] + k2[1, 1]) / 9)


# ---------------------------------------------------------------- smoothing / V-cycle
def test_jacobi_on_eigenmodes_closed_form():
    """Damped Jacobi on a Dirichlet sin mode of the constant-coefficient operator multiplies
    the error by 1 - w lambda / D exactly; the Poisson high-frequency factor is <= 0.6."""
    n, h = 14, 1.0 / 14
    lv = H.Level(n, n, h, 0.0, np.ones((n, n)), np.zeros((n, n)), 0.0)
    p = np.arange(n)[:, None]
    worst = 0.0
    for j in range(1, n + 1):
        for k in range(1, n + 1):
            v = np.sin(j * np.pi * (p + 1) / (n + 1)) * np.sin(k * np.pi * (p.T + 1) / (n + 1)) + 0j
            lam = (4 / h ** 2) * (np.sin(j * np.pi / (2 * (n + 1))) ** 2 + np.sin(k * np.pi / (2 * (n + 1))) ** 2)
            e1 = H.jacobi(lv, v, np.zeros_like(v), 0.8)   # error propagation with f = 0
            fac = 1 - 0.8 * lam / (4 / h ** 2)
            assert np.allclose(e1, fac * v, atol=1e-12)
            if max(j, k) > (n + 1) / 2:
                worst = max(worst, abs(fac))
    assert worst <= 0.6 + 1e-12


def test_two_grid_equals_error_propagation_matrix():
    """Alg. 1 with two levels and an exact coarse solve is the linear map whose error
    propagation is S (I - P M_H^-1 R M) S, S = I - w D^-1 M (16x16 SL problem)."""
    n = 16
    k2 = synth.grf_kappa2(n, n, 7, sigma=2.0).astype(np.float64)
    prob = H.Problem(k2, omega=synth.omega_for(n), h=1.0 / n, abc_width=4, levels=2)
    M = H.assemble_dense(prob.hierarchy[0])
    MH = H.assemble_dense(prob.hierarchy[1])
    N, Nc = n * n, (n // 2) ** 2
    P = np.zeros((N, Nc))
    for k in range(Nc):
        e = np.zeros(Nc)
        e[k] = 1
        P[:, k] = H.prolong_bilinear(e.reshape(n // 2, n // 2), n, n).ravel()
    R = P.T / 4
    S = np.eye(N) - 0.8 * M / np.diag(M)[:, None]
    E = S @ (np.eye(N) - P @ np.linalg.solve(MH, R @ M)) @ S
    B = np.zeros((N, N), complex)
    for k in range(N):
        e = np.zeros(N, complex)
        e[k] = 1
        B[:, k] = H.vcycle(prob, e.reshape(n, n), coarse="direct").ravel()
    assert np.abs((np.eye(N) - B @ M) - E).max() < 1e-12


def _prolongation_matrix(n_f, n_c):
    """Dense P of Eq. 2.9 (column k = P applied to the k-th coarse unit vector)."""
    P = np.zeros((n_f * n_f, n_c * n_c))
    for k in range(n_c * n_c):
        e = np.zeros(n_c * n_c)
        e[k] = 1
        P[:, k] = H.prolong_bilinear(e.reshape(n_c, n_c), n_f, n_f).ravel()
    return P


def _vcycle_inverse_dense(prob, level=0):
    """The V-cycle of Alg. 1 with an exact coarsest solve as a dense matrix B_l (the cycle
    from a zero guess maps f to B_l f), built level by level from assembled matrices:
    B_L = M_L^-1 on the coarsest level, and on level l
        E_l = S_l (I - P_l B_{l+1} R_l M_l) S_l,   B_l = (I - E_l) M_l^-1,
    S_l = I - w D_l^-1 M_l one damped Jacobi sweep, R_l = P_l^T / 4 (V(1,1))."""
    lv = prob.hierarchy[level]
    M = H.assemble_dense(lv)
    if level == len(prob.hierarchy) - 1:
        return np.linalg.inv(M)
    N = M.shape[0]
    P = _prolongation_matrix(lv.nx, prob.hierarchy[level + 1].nx)
    S = np.eye(N) - prob.jacobi_w * M / np.diag(M)[:, None]
    E = S @ (np.eye(N) - P @ _vcycle_inverse_dense(prob, level + 1) @ (P.T / 4) @ M) @ S
    return (np.eye(N) - E) @ np.linalg.inv(M)


def _sl_problem(n, levels=3):
    k2 = synth.grf_kappa2(n, n, 7, sigma=2.0).astype(np.float64)
    return H.Problem(k2, omega=synth.omega_for(n), h=1.0 / n, abc_width=4, levels=levels)


def test_three_level_vcycle_equals_error_propagation_matrix():
    """Alg. 1 with three levels (16, 8, 4) and an exact coarsest solve: the oracle's
    recursion, applied to every unit vector, is the dense map B built from the level
    matrices, so its error propagation I - B M equals S (I - P B_1 R M) S with B_1 the
    two-grid cycle of level 1 (the recursion the solver uses, one level deeper than the
    two-grid pin)."""
    n = 16
    prob = _sl_problem(n)
    B = _vcycle_inverse_dense(prob)
    N = n * n
    Bo = np.zeros((N, N), complex)
    for k in range(N):
        e = np.zeros(N, complex)
        e[k] = 1
        Bo[:, k] = H.vcycle(prob, e.reshape(n, n), coarse="direct").ravel()
    M = H.assemble_dense(prob.hierarchy[0])
    assert np.abs(Bo - B).max() <= 1e-12 * np.abs(B).max()
    E = np.eye(N) - B @ M
    assert np.abs((np.eye(N) - Bo @ M) - E).max() < 1e-11


@pytest.mark.parametrize("n,rho_lo,rho_hi", [(16, 0.58, 0.63), (32, 0.57, 0.61)])
def test_three_level_sl_factor_is_the_epm_spectral_radius(n, rho_lo, rho_hi):
    """The asymptotic convergence factor of the 3-level SL V-cycle (shift 0.5, the
    benchmark's medium generator, a 4-cell layer) is the spectral radius of its exact
    error-propagation matrix: repeated oracle cycles on e_{k+1} = e_k - V(M e_k) settle at
    rho(E) (power iteration).  Measured here: 0.606 at 16^2 and 0.590 at 32^2, the same at
    both sizes, as a multigrid factor should be."""
    prob = _sl_problem(n)
    M = H.assemble_dense(prob.hierarchy[0])
    B = _vcycle_inverse_dense(prob)
    rho = np.abs(np.linalg.eigvals(np.eye(n * n) - B @ M)).max()
    assert rho_lo < rho < rho_hi
    e = np.random.default_rng(3).standard_normal((n, n)) + 0j
    norms = []
    for _ in range(70):
        e = e - H.vcycle(prob, H.apply_op(prob.M, e), coarse="direct")
        norms.append(np.linalg.norm(e))
    measured = (norms[-1] / norms[-31]) ** (1 / 30)
    assert abs(measured - rho) < 0.01 * rho


def test_poisson_vcycle_under_the_grid_alignment():
    """Unshifted Poisson (w = 0, no layer) under the stride-2 / pad-1 alignment of Eq. 2.9
    on an even grid: coarse node I sits on fine node 2I, so the coarse grid's low-side
    boundary lies one fine cell beyond the fine grid's.  The interior LFA factor (mu^2 =
    0.36 for V(1,1) with w = 0.8) is then not reached: the exact two-grid factor is 0.470
    at 16^2 and 0.559 at 32^2, and the 3-level factor 0.842 at 16^2 and 1.18 at 32^2 (the
    3-level Poisson cycle diverges).  The shifted Laplacian of the solver is not affected
    in this way (the 3-level SL factor above is 0.59-0.61)."""
    for n, levels, lo, hi in ((16, 2, 0.46, 0.48), (32, 2, 0.55, 0.57), (16, 3, 0.83, 0.85), (32, 3, 1.15, 1.21)):
        prob = H.Problem(np.ones((n, n)), omega=0.0, h=1.0 / n, abc_width=0, beta=0.0, levels=levels)
        M = H.assemble_dense(prob.hierarchy[0])
        rho = np.abs(np.linalg.eigvals(np.eye(n * n) - _vcycle_inverse_dense(prob) @ M)).max()
        assert lo < rho < hi, (n, levels, rho)


def test_two_grid_poisson_contracts():
    """Two-grid Poisson cycle with exact coarse solve contracts (rho < 0.5 at n = 16).
    (With the stride-2 / pad-1 grid alignment the low-side boundaries of fine and
    coarse grids differ by h, so deeper Poisson hierarchies do not reach the LFA value.)"""
    n = 16
    prob = H.Problem(np.ones((n, n)), omega=0.0, h=1.0 / n, abc_width=0, beta=0.0, levels=2)
    A = H.assemble_dense(prob.hierarchy[0])
    N = n * n
    B = np.zeros((N, N), complex)
    for k in range(N):
        e = np.zeros(N, complex)
        e[k] = 1
        B[:, k] = H.vcycle(prob, e.reshape(n, n), coarse="direct").ravel()
    rho = np.abs(np.linalg.eigvals(np.eye(N) - B @ A)).max()
    assert 0.3 < rho < 0.5


# ---------------------------------------------------------------- GMRES / Givens
def test_givens_least_squares_matches_lstsq():
    rng = np.random.default_rng(8)
    m = 7
    Hh = np.triu(_crandn(rng, (m + 1, m)), -1)
    Hh[np.arange(1, m + 1), np.arange(m)] = np.abs(Hh[np.arange(1, m + 1), np.arange(m)])
    ls = H.ArnoldiLS(m, 2.5)
    for j in range(m):
        est = ls.add_column(Hh[:j + 2, j])
        rhs = np.zeros(j + 2, complex)
        rhs[0] = 2.5
        y_ref, *_ = np.linalg.lstsq(Hh[:j + 2, :j + 1], rhs, rcond=None)
        assert np.isclose(est, np.linalg.norm(rhs - Hh[:j + 2, :j + 1] @ y_ref), rtol=1e-10)
    assert np.allclose(ls.solve(), y_ref, rtol=1e-10)


def test_gmres_minimises_over_explicit_krylov_space():
    """GMRES(m) from 0 returns D^-1 y, y = argmin_{y in K_m(K D^-1, f)} ||f - K D^-1 y||,
    checked against a least-squares solve over an explicitly built Krylov basis."""
    n, m = 8, 6
    lv = _level(n, n, seed=9, omega=9.0, beta=0.5, width=2)
    f = _crandn(np.random.default_rng(10), (n, n))
    x = H.gmres_jacobi(lv, f, m)
    K = H.assemble_dense(lv)
    dinv = 1.0 / np.diag(K)
    B = K * dinv[None, :]
    cols = [f.ravel() / np.linalg.norm(f)]
    for _ in range(m - 1):
        w = B @ cols[-1]
        cols.append(w / np.linalg.norm(w))
    Q, _ = np.linalg.qr(np.stack(cols, 1))
    c, *_ = np.linalg.lstsq(B @ Q, f.ravel(), rcond=None)
    x_ref = dinv * (Q @ c)
    assert np.linalg.norm(x.ravel() - x_ref) / np.linalg.norm(x_ref) < 1e-8


def test_gmres_exact_in_n_steps():
    lv = _level(3, 4, seed=11, omega=5.0)
    f = _crandn(np.random.default_rng(12), (3, 4))
    x = H.gmres_jacobi(lv, f, 12)
    assert np.linalg.norm(H.apply_op(lv, x) - f) / np.linalg.norm(f) < 1e-10


def test_lu_solve_matches_numpy():
    rng = np.random.default_rng(13)
    K = _crandn(rng, (30, 30))
    f = _crandn(rng, 30)
    assert np.allclose(H.lu_solve(K, f), np.linalg.solve(K, f), rtol=1e-11)


# ---------------------------------------------------------------- FGMRES
def _small_problem(n=16, seed=14):
    k2 = synth.grf_kappa2(n, n, seed, sigma=2.0).astype(np.float64)
    return H.Problem(k2, omega=synth.omega_for(n), h=1.0 / n, abc_width=4, levels=3)


def test_fgmres_vcycle_matches_dense_direct_16():
    """FGMRES(10) + M_V on a 16x16 heterogeneous problem reproduces the dense LU solve."""
    prob = _small_problem()
    b = synth.point_sources(16, 16, [(8, 8)], prob.h)[0] + _crandn(np.random.default_rng(15), (16, 16))
    res = H.fgmres(prob.A, H.precond_v(prob), b, tol=1e-13, maxit=400)
    x_ref = H.lu_solve(H.assemble_dense(prob.A), b.ravel()).reshape(16, 16)
    assert res.converged
    assert np.linalg.norm(res.x - x_ref) / np.linalg.norm(x_ref) < 1e-10


def test_fgmres_exact_preconditioner_one_step():
    prob = _small_problem(8, 16)
    Ainv = np.linalg.inv(H.assemble_dense(prob.A))
    b = _crandn(np.random.default_rng(17), (8, 8))
    res = H.fgmres(prob.A, lambda r: (Ainv @ r.ravel()).reshape(r.shape), b, tol=1e-12)
    assert res.converged and res.iters == 1


def test_fgmres_estimates_monotone_and_match_true_residual():
    """Within a cycle the Givens estimate never grows; at each restart it equals the
    true residual recomputed from x (to FP64 rounding)."""
    prob = _small_problem()
    b = _crandn(np.random.default_rng(18), (16, 16))
    res = H.fgmres(prob.A, H.precond_v(prob), b, m=5, tol=1e-10, maxit=200)
    ests = [e for _, e in res.history]
    for c in range(0, len(ests), 5):
        cyc = ests[c:c + 5]
        assert all(cyc[i + 1] <= cyc[i] * (1 + 1e-12) for i in range(len(cyc) - 1))
    for c, true in enumerate(res.true_history[1:]):
        assert np.isclose(ests[5 * c + 4] if 5 * c + 4 < len(ests) else ests[-1], true, rtol=1e-6)


def test_fgmres_identity_preconditioner_is_gmres():
    """With M = I and one cycle, FGMRES gives the GMRES minimiser over K_m(A, b)."""
    prob = _small_problem(8, 19)
    b = _crandn(np.random.default_rng(20), (8, 8))
    m = 6
    res = H.fgmres(prob.A, lambda r: r, b, m=m, tol=0.0, maxit=m)
    K = H.assemble_dense(prob.A)
    cols = [b.ravel() / np.linalg.norm(b)]
    for _ in range(m - 1):
        w = K @ cols[-1]
        cols.append(w / np.linalg.norm(w))
    Q, _ = np.linalg.qr(np.stack(cols, 1))
    c, *_ = np.linalg.lstsq(K @ Q, b.ravel(), rcond=None)
    assert np.linalg.norm(res.x.ravel() - Q @ c) / np.linalg.norm(Q @ c) < 1e-8


def test_manufactured_continuum_second_order():
    """u = sin(pi x) sin(pi y) in a constant medium with no layer, nodes at (i+1)h,
    h = 1/(n+1): the discrete solution error is O(h^2) (ratio ~4 on refinement)."""
    errs = []
    for n in (16, 32):
        h = 1.0 / (n + 1)
        x = (np.arange(n) + 1) * h
        U = np.sin(np.pi * x)[:, None] * np.sin(np.pi * x)[None, :]
        omega, k2 = 6.0, 1.0
        prob = H.Problem(np.full((n, n), k2), omega=omega, h=h, abc_width=0, levels=3)
        f = (2 * np.pi ** 2 - omega ** 2 * k2) * U + 0j
        res = H.fgmres(prob.A, H.precond_v(prob), f, tol=1e-12, maxit=300)
        errs.append(np.abs(res.x - U).max())
    assert 3.5 < errs[0] / errs[1] < 4.5


def test_manufactured_discrete_solution():
    prob = _small_problem(32, 21)
    u_star = _crandn(np.random.default_rng(22), (32, 32))
    f = H.apply_op(prob.A, u_star)
    res = H.fgmres(prob.A, H.precond_v(prob), f, tol=1e-11, maxit=1000)
    assert res.converged
    assert np.linalg.norm(res.x - u_star) / np.linalg.norm(u_star) < 1e-7


@pytest.mark.slow
def test_sl_iterations_in_paper_regime():
    """Paper setting (Sec. 4): 128^2, omega = 20 pi, kappa^2 in [0.25, 1], M_V with
    shift 0.5, 3 levels, V(1,1), w_J = 0.8, coarse GMRES(10): the paper reports
    rho_V ~ 0.9 and > 130 iterations for a 10^6 reduction (block FGMRES, 10 RHS).
    Our independent-RHS FGMRES must land in the same regime: T within +-40% of 137,
    i.e. rho = 10^(-6/T) between 0.84 and 0.95."""
    n = 128
    kappa = np.sqrt(synth.grf_kappa2(n, n, 31, kappa_min=0.5).astype(np.float64))
    prob = H.Problem(kappa ** 2, omega=20 * np.pi, h=1.0 / n, abc_width=10, levels=3)
    b = synth.gaussian_rhs(n, n, 1, 32)[0]
    res = H.fgmres(prob.A, H.precond_v(prob), b, tol=1e-6, maxit=400)
    rho = H.convergence_factor(1.0, res.relres, res.iters)
    assert res.converged
    assert 80 <= res.iters <= 200, res.iters
    assert 0.84 <= rho <= 0.95, rho


# ---------------------------------------------------------------- block FGMRES
def test_block_fgmres_one_column_is_fgmres():
    """With one right-hand side the block method is FGMRES: same iterations and solution."""
    prob = _small_problem()
    b = _crandn(np.random.default_rng(40), (16, 16))
    r1 = H.fgmres(prob.A, H.precond_v(prob), b, m=10, tol=1e-9)
    rb = H.block_fgmres(prob.A, H.precond_v(prob), b[None], m=10, tol=1e-9)
    assert rb.converged and rb.iters == r1.iters
    assert np.linalg.norm(rb.X[0] - r1.x) / np.linalg.norm(r1.x) < 1e-7


def test_block_fgmres_exact_on_full_block_krylov_space():
    """p = 2 columns and m p >= n unknowns: one cycle spans the whole space."""
    lv = _level(4, 4, seed=41, omega=6.0, beta=0.0)
    B = _crandn(np.random.default_rng(42), (2, 4, 4))
    res = H.block_fgmres(lv, lambda v: v, B, m=8, tol=1e-11)
    assert res.converged and res.iters <= 8
    for k in range(2):
        assert np.linalg.norm(H.apply_op(lv, res.X[k]) - B[k]) / np.linalg.norm(B[k]) < 1e-10


def test_block_gmres_minimises_over_explicit_block_krylov_space():
    """Identity preconditioner, first cycle: after j block steps each column's residual
    estimate equals min ||r_c - K y|| over y in span{R, K R, ..., K^(j-1) R} (all p
    columns of R), from a least-squares solve over an explicitly built block basis."""
    n, p, j = 8, 3, 3
    lv = _level(n, n, seed=43, omega=9.0, beta=0.0, width=2)
    B = _crandn(np.random.default_rng(44), (p, n, n))
    res = H.block_fgmres(lv, lambda v: v, B, m=j, tol=1e-30, maxit=j)
    K = H.assemble_dense(lv)
    R = B.reshape(p, -1).T
    blocks, Q = [R], None
    for _ in range(j - 1):
        blocks.append(K @ blocks[-1])
    Q, _ = np.linalg.qr(np.concatenate(blocks, axis=1))
    for c in range(p):
        y, *_ = np.linalg.lstsq(K @ Q, R[:, c], rcond=None)
        ref = np.linalg.norm(R[:, c] - K @ Q @ y) / np.linalg.norm(R[:, c])
        assert abs(res.estimates[j - 1][c] - ref) <= 1e-9 * max(ref, 1e-3)


# ---------------------------------------------------------------- Neumann boundaries
# Sec. 2.4: the stencil's convolution with reflection or replication padding in place
# of zero padding gives Neumann boundaries.  The closed forms below are the discrete
# cosine eigenbases of the two second-difference operators (DCT-I for reflection about
# the boundary node, DCT-II for replication across a half-cell boundary).
def _neumann_modes(n, bc):
    p = np.arange(n)
    if bc == "reflect":
        th = np.arange(n) * np.pi / (n - 1)
        return [(j, np.cos(th[j] * p), 4 * np.sin(th[j] / 2) ** 2) for j in range(n)]
    th = np.arange(n) * np.pi / n
    return [(j, np.cos(th[j] * (p + 0.5)), 4 * np.sin(th[j] / 2) ** 2) for j in range(n)]


@pytest.mark.parametrize("bc", ["reflect", "replicate"])
@pytest.mark.parametrize("ny,nx", [(8, 8), (6, 11)])
def test_neumann_laplacian_eigenpairs(bc, ny, nx):
    """Constant medium, no attenuation: tensor products of the cosine modes are
    eigenvectors with eigenvalue (mu_j + mu_k)/h^2 - w^2 k^2 (the constant mode, j = k = 0,
    gives L 1 = 0)."""
    h, omega, k2 = 1.0 / nx, 9.0, 0.6
    lv = H.Level(ny, nx, h, omega, np.full((ny, nx), k2), np.zeros((ny, nx)), 0.0, bc)
    my, mx = _neumann_modes(ny, bc), _neumann_modes(nx, bc)
    for (j, vy, ly) in my:
        for (k, vx, lx) in mx[:: max(1, nx // 4)]:
            v = np.outer(vy, vx) + 0j
            lam = (ly + lx) / h ** 2 - omega ** 2 * k2
            assert np.allclose(H.apply_op(lv, v), lam * v, rtol=1e-12, atol=1e-9 * (abs(lam) + 1 / h ** 2))


@pytest.mark.parametrize("bc", ["reflect", "replicate"])
def test_neumann_constant_is_in_laplacian_kernel(bc):
    lv = H.Level(7, 9, 0.1, 0.0, np.ones((7, 9)), np.zeros((7, 9)), 0.0, bc)
    assert np.abs(H.apply_op(lv, np.ones((7, 9), complex))).max() < 1e-10


@pytest.mark.parametrize("bc", ["reflect", "replicate"])
def test_neumann_apply_diagonal_and_assembly_agree(bc):
    """Padded-array formulation == node-by-node ghost mapping; the Jacobi diagonal is
    the assembled matrix's diagonal (replication folds one neighbour per boundary side
    onto the node itself)."""
    lv = _level(7, 10, seed=3)
    lv = H.Level(lv.ny, lv.nx, lv.h, lv.omega, lv.kappa2, lv.gamma, lv.beta, bc)
    K = H.assemble_dense(lv)
    u = _crandn(np.random.default_rng(4), (2, 7, 10))
    for t in range(2):
        assert np.allclose(H.apply_op(lv, u)[t].ravel(), K @ u[t].ravel(), rtol=1e-14, atol=1e-12)
    assert np.allclose(np.diag(K).reshape(7, 10), H.diagonal(lv) * np.ones((7, 10)), rtol=1e-14)
    if bc == "replicate":
        # corner: two sides fold back -> 2/h^2 off the centre weight
        assert np.isclose((4 / lv.h ** 2 - K[0, 0].real) * lv.h ** 2,
                          2 + lv.omega ** 2 * lv.kappa2[0, 0] * lv.h ** 2, rtol=1e-12)


def test_neumann_reflect_symmetric_under_trapezoid_weights():
    """Reflection doubles the inward coupling of boundary rows; the operator is complex
    symmetric after scaling rows by the trapezoidal weights (1/2 per boundary side),
    replication's operator is complex symmetric as it stands."""
    lv = _level(6, 9, seed=5)
    refl = H.Level(lv.ny, lv.nx, lv.h, lv.omega, lv.kappa2, lv.gamma, lv.beta, "reflect")
    rep = H.Level(lv.ny, lv.nx, lv.h, lv.omega, lv.kappa2, lv.gamma, lv.beta, "replicate")
    wy = np.ones(6); wy[[0, -1]] = 0.5
    wx = np.ones(9); wx[[0, -1]] = 0.5
    W = np.diag(np.outer(wy, wx).ravel())
    Kr = W @ H.assemble_dense(refl)
    assert np.allclose(Kr, Kr.T, atol=1e-10)
    assert not np.allclose(H.assemble_dense(refl), H.assemble_dense(refl).T)
    Kp = H.assemble_dense(rep)
    assert np.allclose(Kp, Kp.T, atol=1e-10)


@pytest.mark.parametrize("bc", ["reflect", "replicate"])
def test_neumann_fgmres_vcycle_matches_dense_direct(bc):
    """The whole hierarchy carries the boundary mode; FGMRES(10) + M_V reaches the
    dense LU solution of the Neumann problem."""
    k2 = synth.grf_kappa2(16, 16, 14, sigma=2.0).astype(np.float64)
    prob = H.Problem(k2, omega=synth.omega_for(16), h=1.0 / 16, abc_width=4, levels=3, bc=bc)
    assert all(lv.bc == bc for lv in prob.hierarchy)
    b = _crandn(np.random.default_rng(16), (16, 16))
    res = H.fgmres(prob.A, H.precond_v(prob), b, tol=1e-12, maxit=400)
    x_ref = H.lu_solve(H.assemble_dense(prob.A), b.ravel()).reshape(16, 16)
    assert res.converged
    assert np.linalg.norm(res.x - x_ref) / np.linalg.norm(x_ref) < 1e-9
    dir_prob = H.Problem(k2, omega=synth.omega_for(16), h=1.0 / 16, abc_width=4, levels=3)
    assert not np.allclose(H.assemble_dense(dir_prob.A), H.assemble_dense(prob.A))


@pytest.mark.parametrize("bc", ["dirichlet", "reflect", "replicate"])
def test_transpose_action_matches_assembled_transpose(bc):
    """K^T u by scatter-and-fold equals the transposed node-wise assembly."""
    lv = _level(6, 9, seed=7)
    lv = H.Level(lv.ny, lv.nx, lv.h, lv.omega, lv.kappa2, lv.gamma, lv.beta, bc)
    K = H.assemble_dense(lv)
    u = _crandn(np.random.default_rng(8), (2, 6, 9))
    for t in range(2):
        assert np.allclose(H.apply_op_T(lv, u)[t].ravel(), K.T @ u[t].ravel(), rtol=1e-14, atol=1e-11)


# ---------------------------------------------------------------- compact fourth-order scheme
def _compact_level(ny, nx, seed=0, bc="dirichlet", beta=0.3):
    lv = _level(ny, nx, seed=seed, beta=beta)
    return H.Level(lv.ny, lv.nx, lv.h, lv.omega, lv.kappa2, lv.gamma, lv.beta, bc, 4)


@pytest.mark.parametrize("ny,nx", [(10, 10), (8, 13)])
def test_compact4_eigenpairs(ny, nx):
    """Constant medium, no attenuation: sin modes are eigenvectors of the compact scheme with
    eigenvalue [20 - 8 cos a - 8 cos b - 4 cos a cos b] / (6 h^2) - w^2 k^2 (8 + 2 cos a + 2 cos b) / 12,
    a = j pi / (ny + 1), b = k pi / (nx + 1)."""
    h, omega, k2 = 1.0 / nx, 11.0, 0.8
    lv = H.Level(ny, nx, h, omega, np.full((ny, nx), k2), np.zeros((ny, nx)), 0.0, "dirichlet", 4)
    p = np.arange(ny)[:, None]
    q = np.arange(nx)[None, :]
    for j, k in [(1, 1), (2, 5), (ny, nx), (3, 1)]:
        a, b = j * np.pi / (ny + 1), k * np.pi / (nx + 1)
        v = np.sin(a * (p + 1)) * np.sin(b * (q + 1)) + 0j
        lam = ((20 - 8 * np.cos(a) - 8 * np.cos(b) - 4 * np.cos(a) * np.cos(b)) / (6 * h ** 2)
               - omega ** 2 * k2 * (8 + 2 * np.cos(a) + 2 * np.cos(b)) / 12)
        assert np.allclose(H.apply_op(lv, v), lam * v, rtol=1e-12, atol=1e-9 * (abs(lam) + 1 / h ** 2))


@pytest.mark.parametrize("order", [2, 4])
def test_manufactured_continuum_order(order):
    """u = sin(pi x) sin(2 pi y) in a smooth heterogeneous medium k^2 = 1 + 0.5 sin(pi x) cos(pi y),
    no layer, nodes at (i+1)h, h = 1/(n+1); the right-hand side weighted as the scheme
    asks: from n = 16 to 32 the error falls by (33/17)^order (3.8 for the 5-point
    stencil, 14.2 for the compact fourth-order scheme), to within 10 %."""
    expect = (33.0 / 17.0) ** order
    lo, hi = 0.9 * expect, 1.1 * expect
    errs = []
    for n in (16, 32):
        h = 1.0 / (n + 1)
        x = (np.arange(n) + 1) * h
        X, Y = x[None, :], x[:, None]
        U = np.sin(np.pi * X) * np.sin(2 * np.pi * Y)
        k2 = 1.0 + 0.5 * np.sin(np.pi * X) * np.cos(np.pi * Y)
        omega = 6.0
        prob = H.Problem(k2, omega=omega, h=h, abc_width=0, levels=3, order=order)
        f = (5 * np.pi ** 2 - omega ** 2 * k2) * U + 0j
        b = H.rhs_weight(prob.A, f)
        x_h = H.lu_solve(H.assemble_dense(prob.A), b.ravel()).reshape(n, n)
        errs.append(np.abs(x_h - U).max())
    assert lo < errs[0] / errs[1] < hi


@pytest.mark.parametrize("bc", ["dirichlet", "reflect", "replicate"])
def test_compact4_apply_diagonal_and_assembly_agree(bc):
    lv = _compact_level(7, 10, seed=9, bc=bc)
    K = H.assemble_dense(lv)
    u = _crandn(np.random.default_rng(10), (2, 7, 10))
    for t in range(2):
        assert np.allclose(H.apply_op(lv, u)[t].ravel(), K @ u[t].ravel(), rtol=1e-14, atol=1e-11)
    assert np.allclose(np.diag(K).reshape(7, 10), H.diagonal(lv), rtol=1e-14)


def test_compact4_fgmres_vcycle_matches_dense_direct():
    """The whole hierarchy rediscretises with the compact scheme; FGMRES(10) + M_V reaches
    the dense LU solution."""
    k2 = synth.grf_kappa2(16, 16, 14, sigma=2.0).astype(np.float64)
    prob = H.Problem(k2, omega=synth.omega_for(16), h=1.0 / 16, abc_width=4, levels=3, order=4)
    assert all(lv.order == 4 for lv in prob.hierarchy)
    b = _crandn(np.random.default_rng(17), (16, 16))
    res = H.fgmres(prob.A, H.precond_v(prob), b, tol=1e-12, maxit=400)
    x_ref = H.lu_solve(H.assemble_dense(prob.A), b.ravel()).reshape(16, 16)
    assert res.converged
    assert np.linalg.norm(res.x - x_ref) / np.linalg.norm(x_ref) < 1e-9
