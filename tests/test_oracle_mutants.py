"""Planted mistakes in the oracle must be caught by its pins.

Each case patches one oracle routine with a plausible error (a dropped
factor, a wrong sign, a swapped operand) on the CPU and checks that at least
one pin in ``test_oracle_pins`` then fails.  This shows that the pins constrain
every part of the oracle rather than agreeing with it by construction.
"""
import numpy as np
import pytest

import oracle.lsplit as L
from tests import test_oracle_pins as pins

PINS = [
    pins.test_dft_matrix_against_numpy_fft_and_unitarity,
    pins.test_grid_potential_closed_form_cos,
    pins.test_constant_potential_is_global_phase,
    pins.test_commensurate_fiber_sum_matches_supercell,
    pins.test_single_layer_reduces_to_bloch_split_step,
    pins.test_observables_against_dense_quadratic_forms,
    pins.test_gaussian_packet_reduces_to_paper_initial_state,
    pins.test_2d_order_against_dense_exponential,
    pins.test_2d_free_particle_and_mass,
    pins.test_stochastic_sampled_factor_matches_dense,
    lambda: pins.test_free_particle_exact_phase("strang"),
    lambda: pins.test_convergence_order_against_dense_exponential("strang", 2),
    lambda: pins.test_convergence_order_against_dense_exponential("lie", 1),
    lambda: pins.test_convergence_order_against_dense_exponential("yoshida4", 4),
    pins.test_yoshida_weights_conditions,
    pins.test_toeplitz_potential_matches_quadrature,
    pins.test_cn_mass_conservation,
    pins.test_cn_free_particle_cayley_phases,
    pins.test_cn_second_order_against_dense_galerkin_exponential,
    pins.test_semi_implicit_step_matches_dense_formula,
    pins.test_semi_implicit_free_particle_closed_form,
    pins.test_random_batch_is_unbiased,
    pins.test_density_single_plane_wave,
    pins.test_density_periodic_for_commensurate_layers,
    pins.test_adjoint_matches_central_differences,
    pins.test_one_step_equals_dense_factor_product,
    lambda: pins.test_stochastic_steps_match_dense_sampled_factors("strang_stoch"),
    lambda: pins.test_stochastic_steps_match_dense_sampled_factors("lie_stoch"),
    pins.test_gaussian_packet_position_and_momentum,
    pins.test_example3_free_particle_exact_phase,
    pins.test_example3_y_independent_reduces_to_1d_planes,
    pins.test_example3_one_step_and_order_against_dense,
]

_orig_dft = L.dft_matrix
_orig_kin = L.kinetic_energy_diag
_orig_axis = L._axis_dft
_orig_grid = L.grid_potential
_orig_factors = L.scheme_factors
_orig_P = L.apply_P
_orig_yw = L.yoshida_weights
_orig_toep = L.toeplitz_potential
_orig_C = L.apply_C
_orig_SI = L.apply_semi_implicit
_orig_dens = L.density_on_line
_orig_wv = L.wavevectors
_orig_exp = L.expanded_factors
_orig_gp = L.gaussian_packet
_orig_lg = L.layer_grid
_orig_ls = L.layer_slices


def _stoch_scale_inverted(prob, scheme, tau, nsteps, seed=0, step0=0, frac_den=8):
    # sampled factors with duration s p / S instead of s S / p
    out = []
    for f in _orig_exp(prob, scheme, tau, nsteps, seed, step0, frac_den):
        if f[0] == "P" and f[3] is not None:
            S = prob.M2 if f[1] == 1 else prob.M1
            r = len(f[3]) / S
            f = ("P", f[1], f[2] * r * r, f[3])
        out.append(f)
    return out


def _strang_wrong(scheme, tau):
    f = _orig_factors(scheme, tau)
    if scheme.startswith("strang") and not scheme.startswith("strang_kp"):
        f = [(x[0], x[1], x[2] / 2) if x[0] == "P" and x[1] == 2 else x for x in f]
    return f


def _lie_wrong_order(scheme, tau):
    f = _orig_factors(scheme, tau)
    if scheme.startswith("lie"):
        f = [f[1], f[0], f[2]]
    return f


MUTANTS = {
    "kinetic_missing_half": ("kinetic_energy_diag", lambda p: 2.0 * _orig_kin(p)),
    "kinetic_wrong_sign": ("kinetic_energy_diag", lambda p: -_orig_kin(p)),
    "dft_conjugated": ("dft_matrix", lambda q: _orig_dft(q).conj()),
    "dft_index_off_by_one": ("dft_matrix", lambda q: np.roll(_orig_dft(q), 1, axis=0)),
    "forward_missing_1_over_q": ("_axis_dft",
                                 lambda x, q, inverse: _orig_axis(x, q, inverse) * (1.0 if inverse else float(np.prod(q)))),
    "potential_sign": ("grid_potential", lambda h, c, q: -_orig_grid(h, c, q)),
    "potential_h_negated": ("grid_potential", lambda h, c, q: _orig_grid(-np.asarray(h), c, q)),
    "layers_swapped": ("apply_P", lambda p, phi, layer, s, slices=None, _v=None:
                       _orig_P(p, phi, 3 - layer, s, slices, None)),
    "strang_wrong_duration": ("scheme_factors", _strang_wrong),
    "lie_wrong_order": ("scheme_factors", _lie_wrong_order),
    "yoshida_weights_swapped": ("yoshida_weights", lambda: _orig_yw()[::-1]),
    "yoshida_middle_forward": ("yoshida_weights", lambda: (_orig_yw()[0], -_orig_yw()[1])),
    "toeplitz_transposed": ("toeplitz_potential", lambda h, c, q: _orig_toep(h, c, q).T),
    "toeplitz_wrapped": ("toeplitz_potential", lambda h, c, q: _orig_toep(np.asarray(h) - q, c, q)
                         + _orig_toep(h, c, q) + _orig_toep(np.asarray(h) + q, c, q)),
    "cn_half_duration": ("apply_C", lambda p, phi, layer, s, _kin=None: _orig_C(p, phi, layer, s / 2, _kin)),
    "density_conjugate_phase": ("density_on_line", lambda p, phi, x: np.conj(_orig_dens(p, np.conj(phi), x))),
    "density_wrong_wavevector": ("wavevectors", lambda p: _orig_wv(p) * 1.0001),
    "semi_implicit_no_kinetic_solve": ("apply_semi_implicit", lambda p, phi, tau, rows=None, cols=None, _kin=None:
                                       _orig_SI(p, phi, tau, rows, cols, _kin) * (1 + 1j * tau * L.kinetic_energy_diag(p))),
    "random_batch_ignores_sample": ("apply_semi_implicit", lambda p, phi, tau, rows=None, cols=None, _kin=None:
                                    _orig_SI(p, phi, tau, None, None, _kin)),
    "stoch_scale_inverted": ("expanded_factors", _stoch_scale_inverted),
    "stoch_scale_dropped": ("expanded_factors", lambda prob, scheme, tau, nsteps, seed=0, step0=0, frac_den=8: [
        ("P", f[1], f[2] * len(f[3]) / (prob.M2 if f[1] == 1 else prob.M1), f[3])
        if f[0] == "P" and f[3] is not None else f
        for f in _orig_exp(prob, scheme, tau, nsteps, seed, step0, frac_den)]),
    "packet_x0_sign": ("gaussian_packet", lambda prob, x0, w, k0: _orig_gp(prob, -np.asarray(x0, dtype=float), w, k0)),
    "packet_k0_sign": ("gaussian_packet", lambda prob, x0, w, k0: _orig_gp(prob, x0, w, -np.asarray(k0, dtype=float))),
    "shared_grid_extents_swapped": ("layer_grid", lambda prob, layer: (
        lambda h, c, q: (h, c, q[::-1] if getattr(prob, "shared", 0) else q))(*_orig_lg(prob, layer))),
    "shared_layer2_p_fastest": ("layer_slices", lambda prob, phi, layer: (
        phi.reshape(prob.q2[1], prob.q2[0], prob.q1[0]).transpose(2, 1, 0).reshape(prob.q1[0], -1)
        if getattr(prob, "shared", 0) and layer == 2 else _orig_ls(prob, phi, layer))),
    "cn_layer2_half": ("apply_C", lambda p, phi, layer, s, _kin=None:
                       _orig_C(p, phi, layer, s / 2 if layer == 2 else s, _kin)),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    attr, fn = MUTANTS[name]
    monkeypatch.setattr(L, attr, fn)
    caught = 0
    for pin in PINS:
        try:
            pin()
        except (AssertionError, ValueError, IndexError):
            caught += 1
    assert caught > 0, f"no pin caught mutant {name}"
