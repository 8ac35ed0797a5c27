"""Planted mistakes in the oracle (on the CPU, via monkeypatch) must be caught by the
pins: a dropped term, a wrong sign, a swapped operand.  Each test plants one mistake
and asserts that the corresponding pin then fails."""
import math

import numpy as np
import pytest

import lpgen
from oracle import pdlp_oracle as O
from tests import test_oracle_pins as P


def test_dual_step_sign_error_is_caught(monkeypatch):
    def bad(y, Ax, Ax_new, lc, uc, sigma):
        yhat = y + sigma * (2.0 * Ax_new - Ax)  # wrong sign
        return yhat - O.proj_box(yhat, -sigma * uc, -sigma * lc)
    monkeypatch.setattr(O, "dual_step", bad)
    with pytest.raises(AssertionError):
        P.test_dual_step_equals_prox_argmin()


def test_dual_step_dropped_extrapolation_is_caught(monkeypatch):
    def bad(y, Ax, Ax_new, lc, uc, sigma):
        yhat = y - sigma * Ax_new  # A x' instead of A(2x' - x)
        return yhat - O.proj_box(yhat, -sigma * uc, -sigma * lc)
    monkeypatch.setattr(O, "dual_step", bad)
    with pytest.raises(AssertionError):
        P.test_fixed_step_iterates_equal_chambolle_pock()


def test_normalized_gap_dropped_dual_term_is_caught(monkeypatch):
    orig = O.normalized_gap

    def bad(lp, x, y, Ax, ATy, x_ref, y_ref, omega):
        # forget the row terms: evaluate with every row free (y part fixed at 0 move)
        lp2 = O.ScaledLP(**{**lp.__dict__, "lc": np.full_like(lp.lc, -np.inf),
                            "uc": np.full_like(lp.uc, np.inf)})
        return orig(lp2, x, np.zeros_like(y), Ax, ATy, x_ref, y_ref, omega)
    monkeypatch.setattr(O, "normalized_gap", bad)
    with pytest.raises(AssertionError):
        P.test_normalized_gap_vs_sorted_breakpoints(0)


def test_primal_weight_inverted_ratio_is_caught(monkeypatch):
    def bad(x_new, y_new, x_old, y_old, omega, theta=0.5, eps_zero=1e-10):
        dx = O.norm2(x_new - x_old)
        dy = O.norm2(y_new - y_old)
        return math.exp(theta * math.log(dx / dy) + (1 - theta) * math.log(omega))
    monkeypatch.setattr(O, "primal_weight_update", bad)
    with pytest.raises(AssertionError):
        P.test_primal_weight_closed_form()


def test_pc_row_col_swap_is_caught(monkeypatch):
    orig = O._row_pnorm

    def bad(M, p):
        return orig(M, 2.0 if p == 1.0 else p)  # l2 instead of l1
    monkeypatch.setattr(O, "_row_pnorm", bad)
    with pytest.raises(AssertionError):
        P.test_pock_chambolle_alpha1_row_col_l1()


def test_dual_objective_swapped_bounds_is_caught(monkeypatch):
    orig = O.p_fn

    def bad(y, lo, hi):
        return orig(y, hi, lo)  # lower and upper bound swapped in p(y; l, u)
    monkeypatch.setattr(O, "p_fn", bad)
    with pytest.raises(AssertionError):
        P.test_weak_duality_any_dual_point()


# --- feasibility polishing (Sec. 5, Algorithm 4) -----------------------------------
from tests import test_oracle_polishing as PP  # noqa: E402


def test_primal_phase_keeping_the_objective_is_caught(monkeypatch):
    monkeypatch.setattr(O, "primal_feasibility_lp", lambda lp: lp)
    with pytest.raises(AssertionError):
        PP.test_phases_never_move_away_from_their_saddle_points(3)


def test_dual_phase_zeroing_infinite_bounds_is_caught(monkeypatch):
    import dataclasses

    def bad(lp):
        z = np.zeros_like
        return dataclasses.replace(lp, lc=z(lp.lc), uc=z(lp.uc), lv=z(lp.lv), uv=z(lp.uv))
    monkeypatch.setattr(O, "dual_feasibility_lp", bad)
    with pytest.raises(AssertionError):
        PP.test_feasibility_problems_of_sec5()


def test_dual_phase_keeping_the_bounds_is_caught(monkeypatch):
    monkeypatch.setattr(O, "dual_feasibility_lp", lambda lp: lp)
    with pytest.raises(AssertionError):
        PP.test_phases_never_move_away_from_their_saddle_points(3)


def test_wrong_pause_schedule_is_caught(monkeypatch):
    def bad():
        k = 100
        while True:
            yield k
            k += 100
    monkeypatch.setattr(O, "polish_pauses", bad)
    with pytest.raises(AssertionError):
        PP.test_pause_schedule_and_phase_budgets()


# --- infeasibility detection (Sec. 3, App. C) --------------------------------------
from tests import test_oracle_infeasibility as PI  # noqa: E402


def test_wrong_dual_cone_is_caught(monkeypatch):
    # Y taken as R^+ for rows with only an upper bound (sign flipped)
    def bad(y, lc, uc):
        lf, uf = np.isfinite(lc), np.isfinite(uc)
        out = y.copy()
        out = np.where(lf & ~uf, np.maximum(y, 0.0), out)
        out = np.where(~lf & uf, np.maximum(y, 0.0), out)
        return np.where(~lf & ~uf, 0.0, out)
    monkeypatch.setattr(O, "proj_Y", bad)
    with pytest.raises(AssertionError):
        PI.test_two_variable_closed_forms()


def test_dropped_reduced_cost_term_is_caught(monkeypatch):
    # objective of the certificate without the lv'r+ - uv'r- term
    def bad(inst, A_orig, y):
        yb = O.proj_Y(y, inst.lc, inst.uc)
        q = A_orig.T @ yb
        r = O.proj_R(-q, inst.lv, inst.uv)
        return yb, -O.p_fn(-yb, inst.lc, inst.uc), float(np.max(np.abs(q + r)))
    monkeypatch.setattr(O, "primal_infeasibility_measures", bad)
    with pytest.raises(AssertionError):
        PI.test_bound_driven_infeasibility_closed_form()


def test_wrong_slack_cone_is_caught(monkeypatch):
    # S-bar with the one-sided cases swapped
    def bad(s, lc, uc):
        lf, uf = np.isfinite(lc), np.isfinite(uc)
        out = s.copy()
        out = np.where(lf & uf, 0.0, out)
        out = np.where(~lf & uf, np.minimum(s, 0.0), out)
        return np.where(lf & ~uf, np.maximum(s, 0.0), out)
    monkeypatch.setattr(O, "proj_Sbar", bad)
    with pytest.raises(AssertionError):
        PI.test_two_variable_closed_forms()


# --- adjoint of unrolled PDHG -------------------------------------------------------
import inspect  # noqa: E402
import textwrap  # noqa: E402

from tests import test_oracle_adjoint as PA  # noqa: E402


def _mutated_vjp(old, new):
    src = textwrap.dedent(inspect.getsource(O.unrolled_pdhg_vjp))
    assert old in src
    ns = dict(vars(O))
    exec(src.replace(old, new), ns)  # noqa: S102  (a planted mistake, CPU only)
    return ns["unrolled_pdhg_vjp"]


@pytest.mark.parametrize("old,new", [
    ("bxn = bx - 2.0 * sigma * q", "bxn = bx - sigma * q"),            # extrapolation factor
    ("by_k += tau * (A @ bu)", "by_k += 0.0 * (A @ bu)"),             # dropped A'y path
    ('g["uc"] += np.where(below, sigma * by, 0.0)', 'g["uc"] += np.where(above, sigma * by, 0.0)'),
    ("inside = ~(lo | hi)", "inside = ~lo"),                          # upper clamp ignored
])
def test_adjoint_mistakes_are_caught(monkeypatch, old, new):
    monkeypatch.setattr(O, "unrolled_pdhg_vjp", _mutated_vjp(old, new))
    with pytest.raises(AssertionError):
        PA.test_vjp_matches_central_differences(5)


# --- restart bookkeeping --------------------------------------------------------------
def _mutated_run(old, new):
    src = textwrap.dedent(inspect.getsource(O.PdlpRun.run))
    assert src.count(old) == 1
    ns = dict(vars(O))
    exec(src.replace(old, new), ns)  # noqa: S102  (a planted mistake, CPU only)
    return ns["run"]


@pytest.mark.parametrize("old,new", [
    ("self.t = 0\n", "self.t = self.t\n"),                            # t kept across a restart
    ("(t >= prm.beta_art * k)", "(t > prm.beta_art * k)"),            # strict criterion (iii)
    ("self.k += 1", "self.k += 1 + (self.t == 1)"),                   # k counts an extra step
])
def test_restart_bookkeeping_mistakes_are_caught(monkeypatch, old, new):
    monkeypatch.setattr(O.PdlpRun, "run", _mutated_run(old, new))
    with pytest.raises(AssertionError):
        P.test_artificial_restarts_follow_the_closed_form_schedule(0.5, 2, 1)


@pytest.mark.parametrize("old,new", [
    ("if prm.restarts and is_check and self.mu_ref is not None:",
     "if prm.restarts and self.mu_ref is not None:"),                # (i) between checks
    ("if kind == RESTART_NONE and is_art:", "if is_art:"),            # (iii) overrides (i)
])
def test_restart_criterion_order_mistakes_are_caught(monkeypatch, old, new):
    monkeypatch.setattr(O.PdlpRun, "run", _mutated_run(old, new))
    with pytest.raises(AssertionError):
        P.test_sufficient_decay_restarts_only_at_checks()


def _mutated_run_multi(pairs):
    src = textwrap.dedent(inspect.getsource(O.PdlpRun.run))
    for old, new in pairs:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    ns = dict(vars(O))
    exec(src, ns)  # noqa: S102  (a planted mistake, CPU only)
    return ns["run"]


@pytest.mark.parametrize("pairs,pin", [
    # (ii) taken with a non-strict rise of the candidate gap
    ([("mu_c > self.mu_c_prev", "mu_c >= self.mu_c_prev")],
     P.test_necessary_decay_needs_a_strict_increase),
    # the previous candidate gap kept across a restart
    ([("self.mu_c_prev = math.inf\n", "pass\n")],
     P.test_restart_criteria_i_and_ii_at_the_paper_thresholds),
    # (ii) evaluated at (iii) iterations between the checks, (i) still only at checks
    ([("if prm.restarts and is_check and self.mu_ref is not None:",
       "if prm.restarts and self.mu_ref is not None:"),
      ("if mu_c <= prm.beta_suff * self.mu_ref:", "if is_check and mu_c <= prm.beta_suff * self.mu_ref:")],
     P.test_restart_criteria_i_and_ii_at_the_paper_thresholds),
    # beta_suff and beta_nec swapped
    ([("prm.beta_suff * self.mu_ref", "@SWAP@"), ("prm.beta_nec * self.mu_ref", "prm.beta_suff * self.mu_ref"),
      ("@SWAP@", "prm.beta_nec * self.mu_ref")],
     P.test_restart_criteria_i_and_ii_at_the_paper_thresholds),
    # (ii) without the decay bound
    ([("elif mu_c <= prm.beta_nec * self.mu_ref and mu_c > self.mu_c_prev:",
       "elif mu_c > self.mu_c_prev:")],
     P.test_necessary_decay_needs_the_decay_bound),
    # the candidate chosen the other way round on a tie or in general
    ([("if mu_cur < mu_avg:", "if mu_cur <= mu_avg and False:")],
     P.test_restart_criteria_i_and_ii_at_the_paper_thresholds),
])
def test_restart_criteria_ii_mistakes_are_caught(monkeypatch, pairs, pin):
    monkeypatch.setattr(O.PdlpRun, "run", _mutated_run_multi(pairs))
    with pytest.raises(AssertionError):
        pin()


# --- Eq. (10)'s scaled residuals ------------------------------------------------------
def _q_max_finite(lc, uc):  # planted: the zero-exclusion of Eq. (10a) dropped
    lf, uf = np.isfinite(lc), np.isfinite(uc)
    return np.where(lf | uf, np.maximum(np.where(lf, np.abs(lc), 0.0), np.where(uf, np.abs(uc), 0.0)), 1.0)


_row_scale_q = O.row_scale_q


def _q_one_when_both(lc, uc):  # planted: two-sided rows given scale 1
    lf = np.isfinite(lc) & (lc != 0)
    uf = np.isfinite(uc) & (uc != 0)
    return np.where(lf & uf, 1.0, _row_scale_q(lc, uc))


@pytest.mark.parametrize("bad", [_q_max_finite, _q_one_when_both])
def test_row_scale_mistakes_are_caught(monkeypatch, bad):
    monkeypatch.setattr(O, "row_scale_q", bad)
    with np.errstate(all="ignore"), pytest.raises(AssertionError):
        P.test_rescaled_criteria_q_and_w_by_hand()


def test_scaled_residual_multiplied_is_caught(monkeypatch):
    orig = O.kkt_stats

    def bad(inst, A, x, y, reduced_costs=0):
        st = orig(inst, A, x, y, reduced_costs)
        st["primal_res_rel_inf"] = st["primal_res_inf"]  # the scale not applied
        return st
    monkeypatch.setattr(O, "kkt_stats", bad)
    with pytest.raises(AssertionError):
        P.test_rescaled_criteria_equal_absolute_residuals_of_the_rescaled_instance()
