"""The oracle's pins are strong enough to catch plausible mistakes: each test plants one
mistake in a copy of an oracle function (on the CPU; the oracle module itself is put
back afterwards) and checks that the pin written for that function then fails.  The
planted versions live only here."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as ML
from oracle import ns_oracle as O
from tests import test_oracle_adjoint as TA
from tests import test_oracle_bc as TB
from tests import test_oracle_lambda as TL
from tests import test_oracle_mlp as TM
from tests import test_oracle_primal as TP
from tests import test_oracle_rk3 as TR
from tests import test_oracle_roe as TRoe
from tests import test_oracle_sigma as TS


def _fails(pin, *args):
    try:
        pin(*args)
    except AssertionError:
        return True
    return False


# ---- the closure label: nu* = max(0, v^T M v) / |grad v|^2 -------------------------
def _label(variant):
    def f(w, lam, P, eps=1e-30):
        vh = O.symmetric_adjoint(w, lam, P)
        M = O.growth_matrix_field(w, P)
        if w.shape[1] == 1 and variant != "u3_in_2d_block":
            idx = [0, 1, 2, 4]
            M = M[..., idx, :][..., :, idx]
            vh = vh[idx]
        vc = np.moveaxis(vh, 0, -1)
        growth = np.einsum("...i,...ij,...j->...", vc, M, vc)
        grad2 = np.zeros(w.shape[1:])
        for d in range(3):
            ax = d + 1 if variant == "axis_mixup" else 3 - d
            den = P.dx[d] if variant == "difference_over_h" else 2.0 * P.dx[d]
            gd = (np.roll(vh, -1, axis=ax) - np.roll(vh, 1, axis=ax)) / den
            grad2 += np.sum(gd * gd, axis=0)
        if variant == "no_clamp":
            g = growth
        elif variant == "growth_sign":
            g = np.maximum(-growth, 0.0)
        else:
            g = np.maximum(growth, 0.0)
        return g / (grad2 + eps)
    return f


@pytest.mark.parametrize("variant", ["u3_in_2d_block", "axis_mixup", "difference_over_h", "no_clamp",
                                     "growth_sign"])
def test_label_pin_catches(monkeypatch, variant):
    monkeypatch.setattr(ML, "label_rate", _label("none"))
    assert not _fails(TM.test_label_closed_form_on_a_sinusoidal_shear, 1)
    assert not _fails(TM.test_label_closed_form_on_a_sinusoidal_shear, 3)
    monkeypatch.setattr(ML, "label_rate", _label(variant))
    assert (_fails(TM.test_label_closed_form_on_a_sinusoidal_shear, 1) or
            _fails(TM.test_label_closed_form_on_a_sinusoidal_shear, 3))


# ---- the energy-growth fit --------------------------------------------------------
def _efolds(variant):
    def f(E):
        E = np.asarray(E, dtype=np.float64)
        N = E.shape[0] - 1
        M = N // 2
        if M < 1:
            raise ValueError("the window needs N >= 2")
        win = E[N - M:] if variant == "first_half_of_sweep" else E[: M + 1]
        if not np.all(np.isfinite(win)) or np.any(win <= 0.0):
            return math.inf
        m = np.arange(M + 1, dtype=np.float64) + (N - M if variant == "first_half_of_sweep" else 0)
        if variant == "no_normalisation":
            y = np.log(win)
        elif variant == "normalised_by_N_minus_m":
            y = np.log(win / (N - m) ** 2) if np.all(N - m > 0) else np.log(win)
        else:
            y = np.log(win / (N - m + 1.0) ** 2)
        mc = m - m.mean()
        slope = float(np.sum(mc * (y - y.mean())) / np.sum(mc * mc))
        scale = N if variant == "scaled_by_N" else M
        return scale * slope if variant == "sign" else -scale * slope
    return f


@pytest.mark.parametrize("variant", ["first_half_of_sweep", "no_normalisation", "normalised_by_N_minus_m",
                                     "scaled_by_N", "sign"])
def test_efolds_pins_catch(monkeypatch, variant):
    monkeypatch.setattr(O, "energy_efolds", _efolds("none"))
    for N in (2, 3, 10, 41):
        assert not _fails(TL.test_efolds_of_an_exact_exponential, N)
    assert not _fails(TL.test_efolds_window_scale_and_degenerate_cases)
    monkeypatch.setattr(O, "energy_efolds", _efolds(variant))
    caught = any(_fails(TL.test_efolds_of_an_exact_exponential, N) for N in (2, 3, 10, 41))
    caught = caught or _fails(TL.test_efolds_window_scale_and_degenerate_cases)
    assert caught


# ---- the plateau rule -------------------------------------------------------------
def _select(variant):
    def f(efolds, change, efold_tol, rel_tol):
        for i in range(len(change)):
            if efolds[i] <= efold_tol and change[i] <= rel_tol:
                return i + 1 if variant == "takes_the_larger_of_the_pair" else i
        return -1
    return f


def _change(variant):
    def f(g_a, g_b):
        g_a = np.asarray(g_a, dtype=np.float64)
        g_b = np.asarray(g_b, dtype=np.float64)
        d = math.sqrt(float(np.sum((g_b - g_a) ** 2)))
        nb = math.sqrt(float(np.sum((g_a if variant == "relative_to_smaller_lambda" else g_b) ** 2)))
        if nb == 0.0:
            return 0.0 if d == 0.0 else math.inf
        return d / nb
    return f


def test_plateau_pin_catches_choosing_the_larger_factor(monkeypatch):
    monkeypatch.setattr(O, "select_lambda", _select("none"))
    assert not _fails(TL.test_plateau_rule_picks_the_row_where_the_paper_matches_fd)
    monkeypatch.setattr(O, "select_lambda", _select("takes_the_larger_of_the_pair"))
    assert _fails(TL.test_plateau_rule_picks_the_row_where_the_paper_matches_fd)


def test_change_pin_catches_the_wrong_reference_norm(monkeypatch):
    monkeypatch.setattr(O, "sensitivity_change", _change("none"))
    assert not _fails(TL.test_sensitivity_change_and_selection_edge_cases)
    monkeypatch.setattr(O, "sensitivity_change", _change("relative_to_smaller_lambda"))
    assert _fails(TL.test_sensitivity_change_and_selection_edge_cases)


# ---- the primal's viscous flux, heat flux and objective ----------------------------

def _stress(variant):
    def f(g, d, P):
        div = g[0, 0] + g[1, 1] + g[2, 2]
        sig = np.empty((3,) + g.shape[2:])
        for j in range(3):
            sig[j] = P.mu * (g[j, d] + (0.0 if variant == "no_transpose_term" else g[d, j]))
            if j == d and variant != "no_dilatation_term":
                sig[j] -= (2.0 / 3.0) * P.mu * div
        return sig
    return f


@pytest.mark.parametrize("variant", ["no_dilatation_term", "no_transpose_term"])
def test_stress_pins_catch(monkeypatch, variant):
    pins = [TP.test_viscous_flux_of_linear_shear_and_heat,
            TP.test_viscous_flux_of_linear_compression_stokes_hypothesis]
    monkeypatch.setattr(O, "stress_row", _stress("none"))
    assert not any(_fails(p) for p in pins)
    monkeypatch.setattr(O, "stress_row", _stress(variant))
    assert any(_fails(p) for p in pins)


def test_heat_flux_pin_catches_alpha_without_gamma(monkeypatch):
    monkeypatch.setattr(O.Params, "alpha", property(lambda self: self.mu / self.Pr))
    assert _fails(TP.test_heat_flux_through_the_temperature)


def _objective(variant):
    def f(w, P):
        wf = O.plane_state(w, P)
        pt = O.stagnation_pressure(wf[0], wf[1:4], wf[4], P)
        if variant == "unweighted":
            return float(np.mean(P.pt_in - pt)) / P.pt_in
        if variant == "sign":
            return float(np.sum(wf[0] * (pt - P.pt_in)) / np.sum(wf[0])) / P.pt_in
        if variant == "not_normalised":
            return float(np.sum(wf[0] * (P.pt_in - pt)) / np.sum(wf[0]))
        return float(np.sum(wf[0] * (P.pt_in - pt)) / np.sum(wf[0])) / P.pt_in
    return f


@pytest.mark.parametrize("variant", ["unweighted", "sign", "not_normalised"])
def test_objective_pin_catches(monkeypatch, variant):
    monkeypatch.setattr(O, "objective", _objective("none"))
    assert not _fails(TP.test_objective_closed_form_on_a_two_state_plane)
    monkeypatch.setattr(O, "objective", _objective(variant))
    assert _fails(TP.test_objective_closed_form_on_a_two_state_plane)


def test_stagnation_pin_catches_the_wrong_exponent(monkeypatch):
    def pt(rho, m, rhoE, P):
        u2 = (m[0] ** 2 + m[1] ** 2 + m[2] ** 2) / rho ** 2
        p = (P.gamma - 1.0) * (rhoE - 0.5 * rho * u2)
        M2 = u2 / (P.gamma * p / rho)
        return p * (1.0 + 0.5 * (P.gamma - 1.0) * M2) ** (1.0 / (P.gamma - 1.0))
    monkeypatch.setattr(O, "stagnation_pressure", pt)
    assert _fails(TP.test_stagnation_pressure_closed_forms)
    assert _fails(TP.test_objective_closed_form_on_a_two_state_plane)


# ---- the hand-derived transpose and the RK4 adjoint step ---------------------------
def test_transpose_pins_catch_a_dropped_viscous_part_and_an_untransposed_jacobian(monkeypatch):
    import dataclasses
    true_T = O.residual_transpose
    pin = TA.test_transpose_dot_product_identity
    assert not _fails(pin, (7, 5, 3))
    monkeypatch.setattr(O, "residual_transpose", lambda w, a, P: true_T(w, a, dataclasses.replace(P, mu=0.0)))
    assert _fails(pin, (7, 5, 3))
    monkeypatch.setattr(O, "residual_transpose", lambda w, a, P: O.residual_tangent(w, a, P))
    assert _fails(pin, (7, 5, 3))


def _rk4_adjoint(variant):
    def f(w, lam, P, s=None, nu=None):
        dt = P.dt
        _, (W1, W2, W3, W4) = O.rk4_step(w, P, s)

        def JT(W, ab):
            g = O.residual_transpose(W, ab, P)
            if nu is not None:
                g = g + O.viscosity_apply(ab, nu, P)
            return g

        a4 = dt / 6.0 * lam
        g4 = JT(W3 if variant == "stage_state_off_by_one" else W4, a4)
        a3 = (dt / 6.0 if variant == "weight_b3" else dt / 3.0) * lam + dt * g4
        g3 = JT(W3, a3)
        a2 = dt / 3.0 * lam + (dt if variant == "coefficient_a32" else 0.5 * dt) * g3
        g2 = JT(W2, a2)
        a1 = dt / 6.0 * lam + 0.5 * dt * g2
        g1 = JT(W1, a1)
        seeds = a1 + a2 + a3 + (0.0 if variant == "seed_sum_without_a4" else a4)
        return lam + g1 + g2 + g3 + g4, seeds
    return f


@pytest.mark.parametrize("variant", ["stage_state_off_by_one", "weight_b3", "coefficient_a32",
                                     "seed_sum_without_a4"])
def test_rk4_adjoint_pins_catch(monkeypatch, variant):
    pins = [TA.test_rk4_step_adjoint_dot_product, TA.test_trajectory_dot_product_with_source]
    monkeypatch.setattr(O, "rk4_adjoint_step", _rk4_adjoint("none"))
    assert not any(_fails(p) for p in pins)
    monkeypatch.setattr(O, "rk4_adjoint_step", _rk4_adjoint(variant))
    assert any(_fails(p) for p in pins)


# ---- the growth matrix and sigma_1 ------------------------------------------------
def test_growth_matrix_pin_catches_rows_and_columns_exchanged(monkeypatch):
    true_M = O.growth_matrix_closed
    pin = TS.test_closed_form_growth_matrix_equals_definition
    assert not _fails(pin)
    monkeypatch.setattr(O, "growth_matrix_closed", lambda *a: np.swapaxes(true_M(*a), -1, -2))
    assert _fails(pin)


def _sigma1(variant):
    def f(w, P):
        M = O.growth_matrix_field(w, P)
        if w.shape[1] == 1:
            idx = [0, 1, 2, 3] if variant == "u3_instead_of_p_in_2d" else [0, 1, 2, 4]
            M = M[..., idx, :][..., :, idx]
        if variant == "symmetric_part":
            M = 0.5 * (M + np.swapaxes(M, -1, -2))
        return np.linalg.svd(M, compute_uv=False)[..., 0]
    return f


@pytest.mark.parametrize("variant", ["symmetric_part", "u3_instead_of_p_in_2d"])
def test_sigma1_pin_catches(monkeypatch, variant):
    pin = TS.test_sigma1_field_uniform_zero_and_svd_vs_eig
    monkeypatch.setattr(O, "sigma1_field", _sigma1("none"))
    assert not _fails(pin)
    monkeypatch.setattr(O, "sigma1_field", _sigma1(variant))
    assert _fails(pin)


# ---- the adjoint energy -----------------------------------------------------------
@pytest.mark.parametrize("variant", ["no_cell_volume", "norm_not_squared"])
def test_energy_pin_catches(monkeypatch, variant):
    def E(w, lam, P):
        vh = O.symmetric_adjoint(w, lam, P)
        s = float(np.sum(vh * vh))
        if variant == "norm_not_squared":
            s = math.sqrt(s)
        return s if variant == "no_cell_volume" else s * P.dx[0] * P.dx[1] * P.dx[2]
    monkeypatch.setattr(O, "adjoint_energy", E)
    assert (_fails(TS.test_adjoint_energy_is_the_integral_of_vhat_squared, (12, 5, 3)) or
            _fails(TS.test_adjoint_energy_is_the_integral_of_vhat_squared, (7, 4, 1)))


# ---- characteristic inflow and outflow ----------------------------------------------

def test_boundary_pins_catch_the_sides_exchanged(monkeypatch):
    true_state = O.characteristic_state
    pin = TB.test_boundary_states_carry_the_right_invariants
    assert not _fails(pin)
    monkeypatch.setattr(O, "characteristic_state",
                        lambda wc, P, side: true_state(wc, P, "in" if side == "out" else "out"))
    assert _fails(pin)


def test_boundary_transpose_pin_catches_a_missing_ghost_pullback(monkeypatch):
    import dataclasses

    def transpose(w, a, P):
        ap = np.pad(a, [(0, 0)] * 3 + [(1, 1)])
        return O.residual_transpose(O.pad_x(w, P), ap, dataclasses.replace(P, bc="periodic"))[..., 1:-1]

    assert not _fails(TB.test_tangent_and_transpose_equal_fd_jacobian, "central")
    monkeypatch.setattr(O, "_bounded_transpose", transpose)
    assert _fails(TB.test_tangent_and_transpose_equal_fd_jacobian, "central")


# ---- the paper's own scheme: SSP-RK3 adjoint and the Roe entropy fix ----------------
def _ssprk3_adjoint(variant):
    def f(w, lam, P, s=None, nu=None):
        dt = P.dt
        _, (W1, W2, W3) = O.ssprk3_step(w, P, s)

        def JT(W, ab):
            g = O.residual_transpose(W, ab, P)
            if nu is not None:
                g = g + O.viscosity_apply(ab, nu, P)
            return g

        wbar = lam / 3.0
        r3 = 2.0 / 3.0 * dt * lam
        W3bar = 2.0 / 3.0 * lam + JT(W3, r3)
        wbar = wbar + (0.25 if variant == "convex_weights_swapped" else 0.75) * W3bar
        r2 = (0.75 if variant == "convex_weights_swapped" else 0.25) * dt * W3bar
        W2bar = 0.25 * W3bar + JT(W2, r2)
        wbar = wbar + W2bar
        r1 = dt * W2bar
        wbar = wbar + JT(W2 if variant == "first_stage_at_W2" else W1, r1)
        return wbar, r1 + r2 + (0.0 if variant == "seed_without_r3" else r3)
    return f


@pytest.mark.parametrize("variant", ["convex_weights_swapped", "first_stage_at_W2", "seed_without_r3"])
def test_ssprk3_adjoint_pins_catch(monkeypatch, variant):
    pins = [(TR.test_adjoint_step_dot_product, (False,)), (TR.test_trajectory_dot_product_with_source, ())]
    monkeypatch.setattr(O, "ssprk3_adjoint_step", _ssprk3_adjoint("none"))
    assert not any(_fails(p, *a) for p, a in pins)
    monkeypatch.setattr(O, "ssprk3_adjoint_step", _ssprk3_adjoint(variant))
    assert any(_fails(p, *a) for p, a in pins)


def test_entropy_fix_pin_catches_a_kink(monkeypatch):
    def fix(lam, delta, signed):
        if signed:
            return lam
        re = np.real(lam)
        mag = np.where(re >= 0, lam, -lam)
        # a value-continuous but kinked blend: delta at |lam| = 0 rising linearly to |lam|
        return np.where(np.abs(re) < np.real(delta), 0.5 * (delta + mag), mag)
    assert not _fails(TRoe.test_entropy_fix_is_c1_at_delta)
    monkeypatch.setattr(O, "_abs_fix", fix)
    assert _fails(TRoe.test_entropy_fix_is_c1_at_delta)


def _wall(variant):
    def f(wc, P, side):
        ew = P.wall_e[0] if side == "bottom" else P.wall_e[1]
        rho = wc[0]
        u = wc[1:4] / rho
        e = wc[4] / rho - 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
        eg = ew if variant == "ghost_at_wall_energy" else 2.0 * ew - e
        out = np.empty(wc.shape, dtype=wc.dtype)
        out[0] = rho
        out[1:4] = wc[1:4] if variant == "slip_velocity" else -wc[1:4]
        out[4] = rho * (eg + 0.5 * (u[0] ** 2 + u[1] ** 2 + u[2] ** 2))
        return out
    return f


@pytest.mark.parametrize("variant", ["slip_velocity", "ghost_at_wall_energy"])
def test_wall_pins_catch(monkeypatch, variant):
    pins = [TB.test_wall_heat_flux_and_pressure_closed_forms, TB.test_wall_drag_on_a_uniform_stream]
    monkeypatch.setattr(O, "wall_state", _wall("none"))
    assert not any(_fails(p) for p in pins)
    monkeypatch.setattr(O, "wall_state", _wall(variant))
    assert any(_fails(p) for p in pins)
