"""The oracle's pins catch plausible mistakes: each case plants one mistake in the oracle
(in memory, on the CPU, through monkeypatch) and checks that a pin written against the
paper or the mathematics fails, after checking that the same pin passes unmutated."""
import numpy as np
import pytest

import test_oracle_helmholtz as TH
import test_oracle_unet as TU
from oracle import helmholtz as H
from oracle import unet as U


def _fails(fn, *args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


def _wrong_mass_sign(mp):
    mp.setattr(H, "_center", lambda lv: 4.0 / lv.h ** 2 - lv.omega ** 2 * lv.kappa2 * (1.0 + (lv.gamma + lv.beta) * 1j))


def _reflect_as_symmetric(mp):
    # numpy's "symmetric" padding (ghost u_-1 = u_0) taken for reflection (ghost u_-1 = u_1)
    orig = H.apply_op

    def mutant(lv, u):
        if lv.bc == "reflect":
            lv = H.Level(lv.ny, lv.nx, lv.h, lv.omega, lv.kappa2, lv.gamma, lv.beta, "replicate", lv.order)
        return orig(lv, u)
    mp.setattr(H, "apply_op", mutant)


def _pointwise_mass_in_compact(mp):
    mp.setattr(H, "MASS5", np.array([[0.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 0.0]]))


def _restriction_scaled_by_eighth(mp):
    mp.setattr(H, "K_RESTRICT", np.array([[1, 2, 1], [2, 4, 2], [1, 2, 1]], dtype=np.float64) / 8.0)


def _gradient_without_transpose(mp):
    mp.setattr(H, "apply_op_T", H.apply_op)


def _jacobi_damping_squared(mp):
    mp.setattr(H, "jacobi", lambda lv, u, f, w: u + w * w * (f - H.apply_op(lv, u)) / H.diagonal(lv))


def _replicate_diagonal_uncorrected(mp):
    orig = H.diagonal
    mp.setattr(H, "diagonal", lambda lv: H._center(lv) if (lv.bc == "replicate" and lv.order == 2) else orig(lv))


def _lap9_corner_weight(mp):
    mp.setattr(H, "LAP9", np.array([[-2.0, -4.0, -2.0], [-4.0, 24.0, -4.0], [-2.0, -4.0, -2.0]]) / 6.0)


def _givens_without_phase(mp):
    # (dropping conj(b) instead would be an equivalent mistake: the Arnoldi subdiagonal is real)
    def mutant(a, b):
        if b == 0:
            return 1.0, 0.0j, a
        if a == 0:
            return 0.0, 1.0 + 0.0j, b
        t = np.hypot(abs(a), abs(b))
        return abs(a) / t, np.conj(b) / t, (a / abs(a)) * t          # the phase of a dropped from s
    mp.setattr(H, "givens", mutant)


def _coarse_correction_subtracted(mp):
    orig = H.prolong_bilinear
    mp.setattr(H, "prolong_bilinear", lambda e, ny, nx: -orig(e, ny, nx))


def _unweighted_coarse_medium(mp):
    mp.setattr(H, "coarsen_kappa2", lambda k2: k2[::2, ::2].copy())     # injection, not full weighting


def _inner_product_without_conjugate(mp):
    mp.setattr(H, "_dot", lambda u, v: complex(np.sum(u.ravel() * v.ravel())))


def _elu_without_minus_one(mp):
    mp.setattr(U, "elu", lambda x: np.where(x > 0, x, np.exp(np.minimum(x, 0.0))))


def _bn_backward_without_mean_term(mp):
    def mutant(g, cache, gamma):
        xhat, var, _ = cache
        n = g.shape[0] * g.shape[1] * g.shape[2]
        ggamma = np.sum(g * xhat, axis=(0, 1, 2))
        gbeta = np.sum(g, axis=(0, 1, 2))
        return gamma / np.sqrt(var + U.BN_EPS) * (g - xhat * ggamma / n), ggamma, gbeta   # - gbeta / n dropped
    mp.setattr(U, "bn_train_backward", mutant)


def _adam_without_bias_correction(mp):
    def mutant(P, G, M, V, t, lr, b1=0.9, b2=0.999, eps=1e-8):
        for k in P:
            M[k] = b1 * M[k] + (1 - b1) * G[k]
            V[k] = b2 * V[k] + (1 - b2) * G[k] * G[k]
            P[k] = P[k] - lr * M[k] / (np.sqrt(V[k]) + eps)
    mp.setattr(U, "adam_step", mutant)


def _input_without_h2(mp):
    orig = U.make_input
    mp.setattr(U, "make_input", lambda r, kappa2, gamma, h: orig(r, kappa2, gamma, 1.0))


CASES = [
    ("attenuation sign", _wrong_mass_sign, TH.test_stencil_matches_printed_kernel, ()),
    ("attenuation sign (energy identity)", _wrong_mass_sign, TH.test_complex_symmetric_and_absorbing, ()),
    ("reflection taken as symmetric padding", _reflect_as_symmetric, TH.test_neumann_laplacian_eigenpairs,
     ("reflect", 8, 8)),
    ("compact scheme with a pointwise mass term", _pointwise_mass_in_compact, TH.test_manufactured_continuum_order,
     (4,)),
    ("compact scheme with a pointwise mass term (eigenpairs)", _pointwise_mass_in_compact, TH.test_compact4_eigenpairs,
     (10, 10)),
    ("compact Laplacian corner weight", _lap9_corner_weight, TH.test_compact4_eigenpairs, (8, 13)),
    ("restriction scaled by 1/8", _restriction_scaled_by_eighth, TH.test_transfer_kernels_match_paper, ()),
    ("residual-loss gradient without the transpose", _gradient_without_transpose,
     TU.test_residual_loss_gradient_matches_finite_differences, ("reflect",)),
    ("Jacobi damping applied twice", _jacobi_damping_squared, TH.test_jacobi_on_eigenmodes_closed_form, ()),
    ("replication's diagonal left uncorrected", _replicate_diagonal_uncorrected,
     TH.test_neumann_apply_diagonal_and_assembly_agree, ("replicate",)),
    ("Givens rotation without the phase", _givens_without_phase, TH.test_givens_least_squares_matches_lstsq, ()),
    ("coarse-grid correction subtracted", _coarse_correction_subtracted, TH.test_two_grid_poisson_contracts, ()),
    ("coarse medium by injection", _unweighted_coarse_medium, TH.test_coarse_medium_is_weighted_average, ()),
    ("Arnoldi inner product without the conjugate", _inner_product_without_conjugate,
     TH.test_gmres_minimises_over_explicit_krylov_space, ()),
    ("Arnoldi inner product without the conjugate (FGMRES)", _inner_product_without_conjugate,
     TH.test_fgmres_estimates_monotone_and_match_true_residual, ()),
    ("eLU without the -1", _elu_without_minus_one, TU.test_elu_values, ()),
    ("BatchNorm backward without the mean term", _bn_backward_without_mean_term,
     TU.test_backward_matches_finite_differences, ()),
    ("Adam without bias correction", _adam_without_bias_correction, TU.test_adam_first_step_closed_form, ()),
    ("network input without the h^2 scaling", _input_without_h2, TU.test_network_input_channels, ()),
]


@pytest.mark.parametrize("name,mutate,pin,args", CASES, ids=[c[0] for c in CASES])
def test_pin_catches_planted_mistake(monkeypatch, name, mutate, pin, args):
    pin(*args)                      # passes on the oracle as written
    with monkeypatch.context() as mp:
        mutate(mp)
        assert _fails(pin, *args), f"pin {pin.__name__} did not catch: {name}"
