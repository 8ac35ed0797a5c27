"""Plain FP64 CPU oracle of PDLP (restarted PDHG for LP).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` use it.  It shares no code with the CUDA path.

It restates the method of "PDLP: A Practical First-Order Method for Large-Scale
Linear Programming" step by step, in the paper's order and notation, with numpy
vector operations and scipy's CSR matrix-vector product as the only library
primitives.  Everything is float64, evaluated in plain index order.

Problem (Sec. 2, Eq. (1)):   min c'x  s.t.  lc <= Ax <= uc,  lv <= x <= uv.
Saddle form (Eq. (2)):       L(x,y) = c'x - y'Ax - p(y; -uc, -lc)  over X x Y.

Readings taken where the paper is silent or ambiguous (each is repeated where it is
used):
  R1  z^{0,0}: x = proj_X(0), y = 0.
  R2  ||A||_inf in eta_hat^{0,0} = 1/||A||_inf is the largest absolute entry of the
      preconditioned matrix (1 if the matrix has no nonzero).
  R3  k in Algorithm 2 counts accepted iterations only, and the step-size factors use
      (k+2) with that 0-based k: with (k+1) the very first step would give
      (1 - 1^-0.3) = 0 and eta_hat would stay 0 forever.
  R4  Restart/termination are evaluated when the total count k is a multiple of 64;
      condition (iii) is tested after every accepted iteration.
  R5  (i)/(ii) need mu(z^{n,0}, z^{n-1,0}); they are off until the first restart.
  R6  mu_c of the "previous" candidate in (ii) is the candidate mu from the previous
      evaluation in the same outer loop (+inf if none).
  R7  mu(z^{n,0}, z^{n-1,0}) is evaluated once, right after the restart, with the
      updated primal weight.
  R8  A tie mu(current) == mu(average) picks the average ("otherwise").
  R9  Termination is tested on the restart candidate at each 64-check (and on z^{0,0}
      before the first step); the returned point is that candidate.
  R10 Relative KKT error on the unscaled LP (see ``kkt_stats``).
  R11 0 * inf = 0 in the dual objective (the sign sets make the multiplier 0).
  R12 Relative gap 0/0 = 0.
  R13 A zero row/column gets scaling factor 1.
  R14 Ruiz row and column factors are both computed from the same current matrix.
  R16 The retry loop of Algorithm 2 is capped (``max_step_retries``).
  R17 The dual step is evaluated as  y' = yhat - proj_[-sigma uc, -sigma lc](yhat)
      with yhat = y - sigma (2 A x' - A x): the same map as Eq. (3b) (Appendix B's
      Moreau form with sigma pulled into the interval), written so that the case
      analysis of Sec. 2 holds exactly in floating point (y' in Y bit for bit).
  R18 A x of the running average is obtained from the running sum of A x^{n,i}
      (linearity), A'y likewise.
  R19 The interaction term of Eq. (5) / Algorithm 2 is taken in magnitude,
      2|(y'-y)'A(x'-x)|.  Eq. (5) is Chambolle-Pock's condition written for their
      operator K = -A (App. B); under the dual step (3b), which moves y along
      -A(2x'-x), the signed term (y'-y)'A(x'-x) is negative on typical steps, and the
      literal formula then never limits eta (eta grows without bound and the
      iteration diverges).  With the magnitude, eta_bar >= 1/||A||_2 still holds.
  R20 The dual feasibility problem of Sec. 5 is solved as the LP with every finite
      bound set to 0: its dual objective vanishes on the dual feasible set, which is
      unchanged because Y and R depend only on which bounds are finite.
  R21 Feasibility polishing (Algorithm 4): the pause test uses the relative gap of
      Eq. (8) of the average iterate since the last restart, after the k-th
      iteration's own checks and restart (right after a restart that average is the
      restart point); each polishing phase is a fresh PDLP run (own iteration count
      for the step-size factors, checks and restarts; z^{n,0} = its start) with
      normal PDLP's current primal weight and step estimate; "primal (dual)
      constraint violation below the termination tolerance" is the primal (dual) half
      of the termination criteria in force, tested on the restart candidate at the
      checks and at the phase's last iteration; the primal phase's output is its
      returned candidate, the dual phase's likewise even when it hits its budget.
  R22 Infeasibility detection (Sec. 3, App. C) runs at every check of normal PDLP,
      after the termination test, on three candidate directions in this order: the
      difference of the last two iterates, the current iterate, the average since the
      last restart (positive scalings of the paper's "normalized" sequences; the tests
      are scale invariant).  Each candidate's y is projected onto Y and paired with
      r = proj_R(-A'y), its x onto the recession cone of the box and paired with
      s = proj_Sbar(-Ax); the tests run on the unscaled LP.  The returned point is
      (current x, certificate y) for primal infeasibility and (certificate x, current
      y) for dual infeasibility.
  R23 The differentiated map is K steps of Eq. (3) on the LP as given (no
      preconditioning, restarts or adaptive steps: the step sizes are inputs), from
      R1's start, with the dual step of R17/R18; at a clamp boundary (u = lv, yh =
      -sigma uc, ...) the derivative of the inside branch is taken as 0 for the
      iterate (measure-zero set).
  R25 The paper's experiments stop at absolute l_inf residuals of 1e-8 on instances
      rescaled first (Sec. 6: right-hand sides and costs of magnitude 1); on the LP as
      given that is Eq. (10) (row tolerance 1e-8 q_i, column tolerance 1e-8 w_j).
      ``termination_mode`` 2 applies it to instances that were not rescaled; mode 1 is
      the absolute criterion as written.

Pins (tests/): closed forms, brute force, HiGHS, finite differences and hand-solved LPs
for every function.  The restart decisions of ``PdlpRun`` are pinned by closed-form
schedules: (iii) alone; an always-true (i); and (i) and (ii) at the paper's thresholds
on fixed-step PDHG for a 1 x 1 equality-constrained LP with a free variable, where the
iteration is a 2 x 2 linear map and the normalized gap is the omega-dual norm of the
gradient, plus a nilpotent instance on which (ii) must wait for a strict rise.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

# status codes (same meaning as the C-ABI's)
OPTIMAL = 0
ITERATION_LIMIT = 1
TIME_LIMIT = 2
PRIMAL_INFEASIBLE = 3
DUAL_INFEASIBLE = 4
NUMERICAL_ERROR = 5

RESTART_NONE, RESTART_SUFFICIENT, RESTART_NECESSARY, RESTART_ARTIFICIAL = 0, 1, 2, 3


@dataclasses.dataclass
class Params:
    """Algorithm constants; defaults are the paper's (Sec. 3 and Sec. 7)."""

    eps_rel_kkt: float = 1e-8
    termination_mode: int = 0  # 0: relative KKT (R10); 1: Eq. (9) + Eq. (8); 2: Eq. (10) + Eq. (8)
    eps_abs_feas: float = 1e-8
    eps_rel_gap: float = 1e-2
    max_iters: int = 1_000_000
    ruiz_iters: int = 10
    pc_alpha: float = 1.0
    check_period: int = 64
    beta_suff: float = 0.1
    beta_nec: float = 0.9
    beta_art: float = 0.5
    theta: float = 0.5
    eps_zero: float = 1e-10
    max_step_retries: int = 60
    # oracle-only switches used by pin tests (no counterpart in the CUDA path)
    fixed_step: float | None = None  # constant eta, no adaptive step (Chambolle-Pock)
    fixed_omega: float | None = None
    restarts: bool = True
    feasibility_polishing: bool = False  # Algorithm 4 (Sec. 5)
    detect_infeasibility: bool = True  # Sec. 3 "Infeasibility detection", App. C
    eps_infeas: float = 1e-9
    reduced_costs: int = 0  # 0: proj_R(c - A'y) (Sec. 2); 1: App. A's bound proximity


# ----------------------------------------------------------------------------
# small helpers, each a definition from Sec. 2
# ----------------------------------------------------------------------------

def proj_box(v, lo, hi):
    """Orthogonal projection onto the box [lo, hi] (Sec. 2, "Notation")."""
    return np.minimum(np.maximum(v, lo), hi)


def pos(v):
    """v^+ = max(0, v) (Sec. 2, "Notation")."""
    return np.maximum(v, 0.0)


def neg(v):
    """v^- = -min(0, v) (Sec. 2, "Notation")."""
    return -np.minimum(v, 0.0)


def p_fn(y, lo, hi):
    """p(y; l, u) = u'y^+ - l'y^- (Sec. 2), with 0*inf = 0 (R11)."""
    yp, yn = pos(y), neg(y)
    with np.errstate(invalid="ignore"):
        t1 = np.where(yp > 0, hi * yp, 0.0)
        t2 = np.where(yn > 0, lo * yn, 0.0)
    return float(np.sum(t1) - np.sum(t2))


def combine(lc, uc):
    """Combine(lc, uc)_i = max{0, |lc_i|*, |uc_i|*} with |v|* = |v| if finite else 0
    (Sec. 3, "Initialization of the primal weights")."""
    lf = np.where(np.isfinite(lc), np.abs(lc), 0.0)
    uf = np.where(np.isfinite(uc), np.abs(uc), 0.0)
    return np.maximum(0.0, np.maximum(lf, uf))


def norm2(v):
    return math.sqrt(float(np.dot(v, v)))


def proj_R(g, lv, uv):
    """Projection onto the reduced-cost sign set R (Sec. 2, Eq. (1)): {0} for a free
    variable, R^- for only an upper bound, R^+ for only a lower bound, R otherwise."""
    lf, uf = np.isfinite(lv), np.isfinite(uv)
    r = g.copy()
    r = np.where(lf & ~uf, np.maximum(g, 0.0), r)
    r = np.where(~lf & uf, np.minimum(g, 0.0), r)
    r = np.where(~lf & ~uf, 0.0, r)
    return r


def proj_Y(y, lc, uc):
    """Projection onto the dual sign set Y (Sec. 2): R^+ for a row with only a finite
    lower bound, R^- with only a finite upper bound, {0} for a free row, R otherwise."""
    lf, uf = np.isfinite(lc), np.isfinite(uc)
    out = y.copy()
    out = np.where(lf & ~uf, np.maximum(y, 0.0), out)
    out = np.where(~lf & uf, np.minimum(y, 0.0), out)
    out = np.where(~lf & ~uf, 0.0, out)
    return out


def proj_Xbar(x, lv, uv):
    """Projection onto the recession cone of the variable box (App. C): {0} for a
    variable with two finite bounds, R^+ with only a finite lower bound, R^- with only a
    finite upper bound, R for a free variable."""
    lf, uf = np.isfinite(lv), np.isfinite(uv)
    out = x.copy()
    out = np.where(lf & uf, 0.0, out)
    out = np.where(lf & ~uf, np.maximum(x, 0.0), out)
    out = np.where(~lf & uf, np.minimum(x, 0.0), out)
    return out


def proj_Sbar(s, lc, uc):
    """Projection onto the slack cone S-bar of App. C: {0} for a row with two finite
    bounds, R^+ with only a finite upper bound, R^- with only a finite lower bound, R
    for a free row."""
    lf, uf = np.isfinite(lc), np.isfinite(uc)
    out = s.copy()
    out = np.where(lf & uf, 0.0, out)
    out = np.where(~lf & uf, np.maximum(s, 0.0), out)
    out = np.where(lf & ~uf, np.minimum(s, 0.0), out)
    return out


# ----------------------------------------------------------------------------
# diagonal preconditioning (Sec. 3, "Diagonal Preconditioning")
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class ScaledLP:
    """The preconditioned instance: A~ = D1 A D2, c~ = D2 c, (lc~, uc~) = D1 (lc, uc),
    (lv~, uv~) = D2^-1 (lv, uv); x = D2 x~ and y = D1 y~ map back."""

    A: sp.csr_matrix
    AT: sp.csr_matrix
    c: np.ndarray
    lc: np.ndarray
    uc: np.ndarray
    lv: np.ndarray
    uv: np.ndarray
    d1: np.ndarray
    d2: np.ndarray
    orig: object  # the unscaled instance (lpgen.LPInstance-like)
    A_orig: sp.csr_matrix


def _row_max_abs(M):
    """||M_j,.||_inf for every row (0 for an empty row)."""
    M = M.tocsr()
    out = np.zeros(M.shape[0])
    nz = np.diff(M.indptr) > 0
    if M.nnz:
        out[nz] = np.maximum.reduceat(np.abs(M.data), M.indptr[:-1][nz])
    return out


def _row_pnorm(M, p):
    """||M_j,.||_p for every row (0 for an empty row)."""
    M = M.tocsr()
    out = np.zeros(M.shape[0])
    nz = np.diff(M.indptr) > 0
    if M.nnz:
        a = np.abs(M.data)
        if p == 1.0:
            out[nz] = np.add.reduceat(a, M.indptr[:-1][nz])
        else:
            out[nz] = np.add.reduceat(a ** p, M.indptr[:-1][nz]) ** (1.0 / p)
    return out


def _apply_factors(M, fr, fs):
    """A~_ij <- (A~_ij * fr_i) * fs_j, the same rounding order for every entry."""
    M = M.tocsr(copy=True)
    rows = np.repeat(np.arange(M.shape[0]), np.diff(M.indptr))
    M.data = (M.data * fr[rows]) * fs[M.indices]
    return M


def precondition(inst, ruiz_iters=10, pc_alpha=1.0) -> ScaledLP:
    """``ruiz_iters`` Ruiz passes, then one Pock-Chambolle pass with ``pc_alpha``.

    Ruiz (Sec. 3): (D1)_jj = 1/sqrt(||A_j,.||_inf), (D2)_ii = 1/sqrt(||A_.,i||_inf),
    both from the current matrix (R14), applied repeatedly.  Pock-Chambolle:
    (D1)_jj = 1/sqrt(||A_j,.||_{2-alpha}), (D2)_ii = 1/sqrt(||A_.,i||_alpha).
    A zero row/column keeps factor 1 (R13)."""
    A = sp.csr_matrix((inst.val.astype(np.float64), inst.col_idx, inst.row_ptr),
                      shape=(inst.m, inst.n))
    m, n = A.shape
    d1 = np.ones(m)
    d2 = np.ones(n)
    At = A.copy()
    for _ in range(ruiz_iters):
        r = _row_max_abs(At)
        s = _row_max_abs(At.T.tocsr())
        with np.errstate(divide="ignore"):
            fr = np.where(r > 0, 1.0 / np.sqrt(r), 1.0)
            fs = np.where(s > 0, 1.0 / np.sqrt(s), 1.0)
        At = _apply_factors(At, fr, fs)
        d1 = d1 * fr
        d2 = d2 * fs
    if pc_alpha is not None and pc_alpha > 0:
        r = _row_pnorm(At, 2.0 - pc_alpha)
        s = _row_pnorm(At.T.tocsr(), pc_alpha)
        with np.errstate(divide="ignore"):
            fr = np.where(r > 0, 1.0 / np.sqrt(r), 1.0)
            fs = np.where(s > 0, 1.0 / np.sqrt(s), 1.0)
        At = _apply_factors(At, fr, fs)
        d1 = d1 * fr
        d2 = d2 * fs
    return ScaledLP(
        A=At,
        AT=At.T.tocsr(),
        c=d2 * inst.c,
        lc=d1 * inst.lc,
        uc=d1 * inst.uc,
        lv=inst.lv / d2,
        uv=inst.uv / d2,
        d1=d1,
        d2=d2,
        orig=inst,
        A_orig=A,
    )


def initial_primal_weight(c, lc, uc):
    """InitializePrimalWeight (Sec. 3): ||c||_2 / ||Combine(lc,uc)||_2 if both are
    positive, else 1."""
    nc = norm2(c)
    nb = norm2(combine(lc, uc))
    if nc > 0.0 and nb > 0.0:
        return nc / nb
    return 1.0


def primal_weight_update(x_new, y_new, x_old, y_old, omega, theta=0.5, eps_zero=1e-10):
    """Algorithm 3: log-space smoothing of Delta_y / Delta_x when both distances lie in
    (eps_zero, 1/eps_zero); otherwise the weight is kept."""
    dx = norm2(x_new - x_old)
    dy = norm2(y_new - y_old)
    if eps_zero < dx < 1.0 / eps_zero and eps_zero < dy < 1.0 / eps_zero:
        return math.exp(theta * math.log(dy / dx) + (1.0 - theta) * math.log(omega))
    return omega


# ----------------------------------------------------------------------------
# the PDHG step (Eq. (3), Algorithm 2)
# ----------------------------------------------------------------------------

def primal_step(x, ATy, c, lv, uv, tau):
    """Eq. (3a): x' = proj_X(x - tau (c - A'y))."""
    return proj_box(x - tau * (c - ATy), lv, uv)


def dual_step(y, Ax, Ax_new, lc, uc, sigma):
    """Eq. (3b): y' = y - sigma A(2x'-x) - sigma proj_[-uc,-lc](y/sigma - A(2x'-x)),
    evaluated as yhat - proj_[-sigma uc, -sigma lc](yhat) with
    yhat = y - sigma (2 A x' - A x) (R17, R18)."""
    yhat = y - sigma * (2.0 * Ax_new - Ax)
    return yhat - proj_box(yhat, -sigma * uc, -sigma * lc)


def step_factors(k):
    """The reduction and growth factors of Algorithm 2 at accepted count k (R3)."""
    kk = float(k + 2)
    return 1.0 - kk ** (-0.3), 1.0 + kk ** (-0.6)


def adaptive_step(lp: ScaledLP, x, y, Ax, ATy, omega, eta_hat, k, max_retries):
    """Algorithm 2 (AdaptiveStepOfPDHG).  Returns (x', y', Ax', eta, eta', attempts,
    ok); ``ok`` is False when the retry cap (R16) is hit or the step is not finite."""
    eta = eta_hat
    red, grow = step_factors(k)
    for attempt in range(1, max_retries + 1):
        xn = primal_step(x, ATy, lp.c, lp.lv, lp.uv, eta / omega)
        Axn = lp.A @ xn
        yn = dual_step(y, Ax, Axn, lp.lc, lp.uc, eta * omega)
        dx = xn - x
        dy = yn - y
        num = omega * float(np.dot(dx, dx)) + float(np.dot(dy, dy)) / omega
        den = 2.0 * abs(float(np.dot(dy, Axn - Ax)))  # R19
        eta_bar = num / den if den > 0.0 else math.inf
        eta_new = min(red * eta_bar, grow * eta)
        if not (math.isfinite(eta_new) and math.isfinite(num)):
            return xn, yn, Axn, eta, eta_new, attempt, False
        if eta <= eta_bar:
            return xn, yn, Axn, eta, eta_new, attempt, True
        eta = eta_new
    return xn, yn, Axn, eta, eta, max_retries, False


# ----------------------------------------------------------------------------
# normalized duality gap (Sec. 3, "Adaptive restarts")
# ----------------------------------------------------------------------------

def normalized_gap(lp: ScaledLP, x, y, Ax, ATy, x_ref, y_ref, omega):
    """mu_n(z, z_ref) = rho_r(z) with r = ||z - z_ref||_omega, where
    rho_r(z) = (1/r) max { L(x, yh) - L(xh, y) : zh in X x Y, ||zh - z||_omega <= r }.

    L(x,yh) - L(xh,y) = -g'(xh - x) + sum_i [h_i(yh_i) - h_i(y_i)] with g = c - A'y and
    h_i(s) = (lc_i - (Ax)_i) s for s > 0, (uc_i - (Ax)_i) s for s < 0 (the objective of
    the max, written relative to its value 0 at zh = z).  For a multiplier on the
    ball, parametrised by s = 1/lambda >= 0, the maximiser is coordinate-wise
        xh = proj_[lv,uv](x - (s/omega) g),
        yh = y + s omega a   if lc finite and that is > 0      (a = lc - Ax),
             y + s omega b   elif uc finite and that is < 0    (b = uc - Ax),
             0               otherwise,
    and ||zh(s) - z||_omega is nondecreasing in s.  The radius is met by bisection
    on s to relative width 1e-14; if every coordinate saturates at a finite
    distance within the ball, the saturated point is the maximiser."""
    dxr = x - x_ref
    dyr = y - y_ref
    r = math.sqrt(omega * float(np.dot(dxr, dxr)) + float(np.dot(dyr, dyr)) / omega)
    if r == 0.0:
        return 0.0
    g = lp.c - ATy
    lcf = np.isfinite(lp.lc)
    ucf = np.isfinite(lp.uc)
    with np.errstate(invalid="ignore"):
        a = np.where(lcf, lp.lc - Ax, -np.inf)
        b = np.where(ucf, lp.uc - Ax, np.inf)

    def hfun(v):
        with np.errstate(invalid="ignore"):
            return np.where(v > 0, a * v, np.where(v < 0, b * v, 0.0))

    hy = hfun(y)

    def trial(s):
        xh = proj_box(x - (s / omega) * g, lp.lv, lp.uv)
        with np.errstate(invalid="ignore", over="ignore"):
            sp_ = y + (s * omega) * np.where(lcf, a, 0.0)
            sm_ = y + (s * omega) * np.where(ucf, b, 0.0)
        yh = np.where(lcf & (sp_ > 0), sp_, np.where(ucf & (sm_ < 0), sm_, 0.0))
        return xh, yh

    def dist(s):
        xh, yh = trial(s)
        ex, ey = xh - x, yh - y
        return math.sqrt(omega * float(np.dot(ex, ex)) + float(np.dot(ey, ey)) / omega)

    def objective(s):
        xh, yh = trial(s)
        return float(-np.dot(g, xh - x) + np.sum(hfun(yh) - hy))

    # Does every coordinate stop moving at a finite s?
    x_unb = ((g > 0) & ~np.isfinite(lp.lv)) | ((g < 0) & ~np.isfinite(lp.uv))
    y_unb = (lcf & (a > 0)) | (ucf & (b < 0))
    if not (x_unb.any() or y_unb.any()):
        bps = [0.0]
        with np.errstate(divide="ignore", invalid="ignore"):
            gx = np.abs(g)
            room = np.where(g > 0, x - lp.lv, np.where(g < 0, lp.uv - x, 0.0))
            bx = np.where(gx > 0, omega * room / gx, 0.0)
            by1 = np.where(lcf & (a < 0), -y / (omega * a), 0.0)
            by2 = np.where(ucf & (b > 0), -y / (omega * b), 0.0)
        for arr in (bx, by1, by2):
            arr = arr[np.isfinite(arr)]
            if arr.size:
                bps.append(float(arr.max()))
        s_sat = max(bps)
        if dist(s_sat) <= r:
            return objective(s_sat) / r
    # bracket [s_lo, s_hi] with dist(s_lo) < r <= dist(s_hi), s_hi = 2 s_lo
    s_hi = 1.0
    if dist(s_hi) < r:
        for _ in range(4000):
            s_hi *= 2.0
            if dist(s_hi) >= r:
                break
        s_lo = 0.5 * s_hi
    else:
        s_lo = 1.0
        for _ in range(4000):
            s_lo *= 0.5
            if dist(s_lo) < r or s_lo == 0.0:
                break
        s_hi = 2.0 * s_lo
    for _ in range(200):
        if s_hi - s_lo <= 1e-14 * s_hi:
            break
        mid = 0.5 * (s_lo + s_hi)
        if dist(mid) < r:
            s_lo = mid
        else:
            s_hi = mid
    return objective(s_hi) / r


# ----------------------------------------------------------------------------
# optimality measures on the unscaled LP (R10)
# ----------------------------------------------------------------------------

def reduced_costs_bound_proximity(g, x, lv, uv):
    """App. A's alternative reduced costs: r_i = g_i when g_i > 0 and x_i - lv_i <= |x_i|,
    or g_i < 0 and uv_i - x_i <= |x_i|; 0 otherwise (g = c - A'y)."""
    with np.errstate(invalid="ignore"):
        near_lo = (x - lv) <= np.abs(x)
        near_hi = (uv - x) <= np.abs(x)
    return np.where((g > 0) & near_lo, g, np.where((g < 0) & near_hi, g, 0.0))


def kkt_stats(inst, A_orig, x, y, reduced_costs=0):
    """Residuals, objectives and gaps of (x, y) for the unscaled LP, with the reduced
    costs r = proj_R(c - A'y) (Sec. 2, "natural choice"), or App. A's bound-proximity
    choice when ``reduced_costs`` = 1.

    primal residual  Ax - proj_[lc,uc](Ax)        relative: /(1 + ||Combine(lc,uc)||_2)
    dual residual    (c - A'y) - r                relative: /(1 + ||c||_2)
    pobj = c'x, dobj = lc'y^+ - uc'y^- + lv'r^+ - uv'r^- (Eq. (1) and App. D's expansion)
    gap              |pobj - dobj| / (1 + |pobj| + |dobj|)
    rel_kkt = max of the three; paper_gap = |pobj - dobj| / (|pobj| + |dobj|) (Eq. (8)).
    primal_res_rel_inf, dual_res_rel_inf: the l_inf residuals with each row divided by
    q_i and each column by w_j of Sec. 7's Eq. (10) -- the absolute 1e-8 criterion of
    Eq. (9) on the paper's rescaled instances, read on the LP as given (see
    ``row_scale_q``, ``col_scale_w``)."""
    Ax = A_orig @ x
    ATy = A_orig.T @ y
    pres = Ax - proj_box(Ax, inst.lc, inst.uc)
    g = inst.c - ATy
    if reduced_costs == 1:
        r = reduced_costs_bound_proximity(g, x, inst.lv, inst.uv)
    else:
        r = proj_R(g, inst.lv, inst.uv)
    dres = g - r
    pobj = float(np.dot(inst.c, x))
    dobj = -p_fn(-y, inst.lc, inst.uc) - p_fn(-r, inst.lv, inst.uv)
    p2 = norm2(pres)
    d2 = norm2(dres)
    eps_p = p2 / (1.0 + norm2(combine(inst.lc, inst.uc)))
    eps_d = d2 / (1.0 + norm2(inst.c))
    eps_g = abs(pobj - dobj) / (1.0 + abs(pobj) + abs(dobj))
    den = abs(pobj) + abs(dobj)
    paper_gap = abs(pobj - dobj) / den if den > 0 else 0.0
    return dict(
        primal_res_l2=p2,
        dual_res_l2=d2,
        primal_res_inf=float(np.max(np.abs(pres))) if pres.size else 0.0,
        dual_res_inf=float(np.max(np.abs(dres))) if dres.size else 0.0,
        pobj=pobj,
        dobj=dobj,
        rel_primal=eps_p,
        rel_dual=eps_d,
        rel_gap=eps_g,
        rel_kkt=max(eps_p, eps_d, eps_g),
        paper_gap=paper_gap,
        primal_res_rel_inf=float(np.max(np.abs(pres) / row_scale_q(inst.lc, inst.uc))) if pres.size else 0.0,
        dual_res_rel_inf=float(np.max(np.abs(dres) / col_scale_w(inst.c))) if dres.size else 0.0,
    )


def row_scale_q(lc, uc):
    """q_i of Sec. 7's Eq. (10a): the scale of row i's tolerance once the paper's
    instance rescaling (right-hand sides in {-inf, -1, 0, 1, inf}, Sec. 6) is undone --
    |lc_i| when only lc_i is finite and nonzero, |uc_i| when only uc_i is, the larger of
    the two when both are, and 1 when neither is."""
    lf = np.isfinite(lc) & (lc != 0)
    uf = np.isfinite(uc) & (uc != 0)
    with np.errstate(invalid="ignore"):
        alc, auc = np.abs(np.where(lf, lc, 0.0)), np.abs(np.where(uf, uc, 0.0))
    return np.where(lf & ~uf, alc, np.where(~lf & uf, auc, np.where(lf & uf, np.maximum(alc, auc), 1.0)))


def col_scale_w(c):
    """w_j of Sec. 7's Eq. (10b): |c_j| when c_j != 0, else 1."""
    return np.where(c != 0, np.abs(c), 1.0)


# ----------------------------------------------------------------------------
# infeasibility certificates (Sec. 3 "Infeasibility detection", App. C)
# ----------------------------------------------------------------------------

def primal_infeasibility_measures(inst, A_orig, y):
    """For a direction y (unscaled LP): y-bar = proj_Y(y), the reduced costs that make
    ||A'y-bar + r||_inf smallest over R, r = proj_R(-A'y-bar), and the two numbers of
    App. C's test: the dual objective lc'y+ - uc'y- + lv'r+ - uv'r- of (y-bar, r) and
    ||A'y-bar + r||_inf.  Returns (y_bar, objective, residual)."""
    yb = proj_Y(y, inst.lc, inst.uc)
    q = A_orig.T @ yb
    r = proj_R(-q, inst.lv, inst.uv)
    obj = -p_fn(-yb, inst.lc, inst.uc) - p_fn(-r, inst.lv, inst.uv)
    res = float(np.max(np.abs(q + r))) if q.size else 0.0
    return yb, obj, res


def dual_infeasibility_measures(inst, A_orig, x):
    """For a direction x (unscaled LP): x-bar = proj_Xbar(x), s = proj_Sbar(-A x-bar)
    (the slack that makes ||A x-bar + s||_inf smallest), and App. C's numbers c'x-bar and
    ||A x-bar + s||_inf.  Returns (x_bar, c'x_bar, residual)."""
    xb = proj_Xbar(x, inst.lv, inst.uv)
    p = A_orig @ xb
    sl = proj_Sbar(-p, inst.lc, inst.uc)
    res = float(np.max(np.abs(p + sl))) if p.size else 0.0
    return xb, float(np.dot(inst.c, xb)), res


def infeasibility_certificate(inst, A_orig, candidates, eps):
    """App. C's tests on the candidate directions (unscaled (x, y) pairs, in order):
    primal infeasibility -- objective > 0 and residual <= eps * objective -- on each
    candidate's y, then dual infeasibility -- c'x-bar < 0 and residual <= eps |c'x-bar| --
    on each candidate's x.  Returns (PRIMAL_INFEASIBLE, y_bar), (DUAL_INFEASIBLE, x_bar)
    or None."""
    for _, y in candidates:
        yb, obj, res = primal_infeasibility_measures(inst, A_orig, y)
        if obj > 0.0 and res <= eps * obj:
            return PRIMAL_INFEASIBLE, yb
    for x, _ in candidates:
        xb, cx, res = dual_infeasibility_measures(inst, A_orig, x)
        if cx < 0.0 and res <= eps * abs(cx):
            return DUAL_INFEASIBLE, xb
    return None


def converged(st, prm: Params):
    """Termination test: 0 relative KKT (R10); 1 the l_inf criteria of Eq. (9) with the
    relative gap of Eq. (8); 2 the same with Eq. (10)'s scaled residuals (Eq. (9) on the
    paper's rescaled instance)."""
    if prm.termination_mode == 0:
        return st["rel_kkt"] <= prm.eps_rel_kkt
    return primal_feasible(st, prm) and dual_feasible(st, prm) and st["paper_gap"] <= prm.eps_rel_gap


# ----------------------------------------------------------------------------
# PDLP (Algorithm 1)
# ----------------------------------------------------------------------------

@dataclasses.dataclass
class Result:
    status: int
    x: np.ndarray
    y: np.ndarray
    stats: dict
    trace: list


class PdlpRun:
    """One run of Algorithm 1 (Algorithm 2 steps, the restart scheme of Sec. 3,
    Algorithm 3's primal weight) on the scaled LP ``lp``, from the start (x, y) with
    primal weight ``omega`` and step estimate ``eta_hat``.

    ``goal(x, y)`` is the termination test of a candidate (scaled point, R9);
    ``max_iters`` caps the accepted iterations.  ``run(pause_at)`` advances until the
    goal is met, the cap is reached or a step fails -- returning (status, x, y) -- or,
    if ``pause_at`` is given, until ``pause_at`` iterations are complete (with that
    iteration's checks and restart done), returning None; the state stays in the
    object, so a paused run continues where it stopped."""

    def __init__(self, lp, prm: Params, x, y, omega, eta_hat, goal, max_iters, trace_iters=0,
                 infeas=None):
        m, n = lp.A.shape
        self.lp, self.prm, self.goal, self.max_iters = lp, prm, goal, max_iters
        self.infeas = infeas  # infeas(candidates) -> (status, x, y) or None (scaled)
        self.m, self.n = m, n
        self.x, self.y = np.array(x, dtype=float), np.array(y, dtype=float)
        self.Ax, self.ATy = lp.A @ self.x, lp.AT @ self.y
        self.x_prev, self.y_prev = self.x.copy(), self.y.copy()  # z before the last step
        self.omega, self.eta_hat = omega, eta_hat
        self.k = self.t = 0
        self.x0, self.y0 = self.x.copy(), self.y.copy()  # z^{n,0}
        self.mu_ref = None  # mu(z^{n,0}, z^{n-1,0})  (R5, R7)
        self.mu_c_prev = math.inf  # R6
        self._zero_sums()
        self.stats = dict(iterations=0, attempts=0, rejected_steps=0, restarts=[0, 0, 0],
                          kkt_passes=0.0)
        self.trace = []
        self.trace_iters = trace_iters
        self.started = False

    def _zero_sums(self):
        self.Sx, self.Sy = np.zeros(self.n), np.zeros(self.m)
        self.SAx, self.SATy = np.zeros(self.m), np.zeros(self.n)
        self.W = 0.0

    def average(self):
        """Running weighted average since the last restart (Algorithm 1); right after
        a restart (no step since) it is the restart point itself."""
        if self.W == 0.0:
            return self.x.copy(), self.y.copy()
        return self.Sx / self.W, self.Sy / self.W

    def run(self, pause_at=None):
        prm, lp = self.prm, self.lp
        if not self.started:
            self.started = True
            # termination check before the first step (Sec. 3, "Periodic checks")
            if self.goal(self.x, self.y):
                return OPTIMAL, self.x, self.y
        while True:
            if pause_at is not None and self.k >= pause_at:
                return None
            x, y, Ax, ATy, omega = self.x, self.y, self.Ax, self.ATy, self.omega
            if prm.fixed_step is not None:
                tau, sig = prm.fixed_step / omega, prm.fixed_step * omega
                xn = primal_step(x, ATy, lp.c, lp.lv, lp.uv, tau)
                Axn = lp.A @ xn
                yn = dual_step(y, Ax, Axn, lp.lc, lp.uc, sig)
                eta, eta_new, attempts, ok = prm.fixed_step, prm.fixed_step, 1, True
            else:
                xn, yn, Axn, eta, eta_new, attempts, ok = adaptive_step(
                    lp, x, y, Ax, ATy, omega, self.eta_hat, self.k, prm.max_step_retries)
            self.stats["attempts"] += attempts
            self.stats["rejected_steps"] += attempts - 1
            self.stats["kkt_passes"] += 0.5 * attempts + 0.5
            if not ok:
                return NUMERICAL_ERROR, x, y
            ATyn = lp.AT @ yn
            # running weighted average since the last restart (Algorithm 1)
            self.Sx += eta * xn
            self.Sy += eta * yn
            self.SAx += eta * Axn
            self.SATy += eta * ATyn
            self.W += eta
            self.x_prev, self.y_prev = x, y
            self.x, self.y, self.Ax, self.ATy = xn, yn, Axn, ATyn
            self.eta_hat = eta_new
            self.t += 1
            self.k += 1
            k, t = self.k, self.t
            self.stats["iterations"] = k
            rec = None
            if len(self.trace) < self.trace_iters:
                rec = dict(k=k, x=xn.copy(), y=yn.copy(), eta=eta, omega=omega,
                           eta_hat=eta_new, attempts=attempts, restart=RESTART_NONE,
                           mu_cur=math.nan, mu_avg=math.nan)
                self.trace.append(rec)

            is_check = (k % prm.check_period) == 0  # R4
            is_art = prm.restarts and (t >= prm.beta_art * k)
            is_limit = k >= self.max_iters
            if not (is_check or is_art or is_limit):
                continue
            # GetRestartCandidate (Sec. 3): current iterate vs the average (R8, R18)
            W = self.W
            xa, ya, Axa, ATya = self.Sx / W, self.Sy / W, self.SAx / W, self.SATy / W
            x0, y0 = self.x0, self.y0
            mu_cur = normalized_gap(lp, xn, yn, Axn, ATyn, x0, y0, omega)
            mu_avg = normalized_gap(lp, xa, ya, Axa, ATya, x0, y0, omega)
            if mu_cur < mu_avg:
                cand, mu_c = (xn, yn, Axn, ATyn), mu_cur
            else:
                cand, mu_c = (xa, ya, Axa, ATya), mu_avg
            if rec is not None:
                rec["mu_cur"], rec["mu_avg"] = mu_cur, mu_avg
            if is_check or is_limit:  # R9
                if self.goal(cand[0], cand[1]):
                    return OPTIMAL, cand[0], cand[1]
                if self.infeas is not None:  # R22
                    out = self.infeas([(xn - self.x_prev, yn - self.y_prev), (xn, yn), (xa, ya)])
                    if out is not None:
                        return out
                if is_limit:
                    return ITERATION_LIMIT, cand[0], cand[1]
            kind = RESTART_NONE
            if prm.restarts and is_check and self.mu_ref is not None:
                if mu_c <= prm.beta_suff * self.mu_ref:
                    kind = RESTART_SUFFICIENT
                elif mu_c <= prm.beta_nec * self.mu_ref and mu_c > self.mu_c_prev:
                    kind = RESTART_NECESSARY
            if kind == RESTART_NONE and is_art:
                kind = RESTART_ARTIFICIAL
            if is_check:
                self.mu_c_prev = mu_c
            if kind == RESTART_NONE:
                continue
            # restart the outer loop: z^{n+1,0} <- candidate, eta_hat carried
            self.stats["restarts"][kind - 1] += 1
            if rec is not None:
                rec["restart"] = kind
            self.x, self.y, self.Ax, self.ATy = (v.copy() for v in cand)
            if prm.fixed_omega is None:
                self.omega = primal_weight_update(self.x, self.y, x0, y0, omega, prm.theta,
                                                  prm.eps_zero)
            self.mu_ref = normalized_gap(lp, self.x, self.y, self.Ax, self.ATy, x0, y0,
                                         self.omega)  # R7
            self.x0, self.y0 = self.x.copy(), self.y.copy()
            self.t = 0
            self.mu_c_prev = math.inf
            self._zero_sums()


def solve(inst, prm: Params | None = None, trace_iters: int = 0, lp: ScaledLP | None = None,
          x_init=None, y_init=None) -> Result:
    """Algorithm 1 after preconditioning (with feasibility polishing, Algorithm 4,
    when ``prm.feasibility_polishing``).  ``trace_iters`` > 0 records, for each of the
    first accepted iterations, the scaled iterate and the step/weight scalars.
    ``x_init``/``y_init`` (scaled space) override R1's starting point."""
    prm = prm or Params()
    if lp is None:
        lp = precondition(inst, prm.ruiz_iters, prm.pc_alpha)
    m, n = inst.m, inst.n
    maxabs = float(np.max(np.abs(lp.A.data))) if lp.A.nnz else 0.0
    eta_hat = 1.0 / maxabs if maxabs > 0 else 1.0  # R2
    if prm.fixed_step is not None:
        eta_hat = prm.fixed_step
    omega = initial_primal_weight(lp.c, lp.lc, lp.uc)
    if prm.fixed_omega is not None:
        omega = prm.fixed_omega
    # R1
    x = proj_box(np.zeros(n), lp.lv, lp.uv) if x_init is None else np.array(x_init, dtype=float)
    y = np.zeros(m) if y_init is None else np.array(y_init, dtype=float)

    def measures(xs, ys):
        return kkt_stats(inst, lp.A_orig, lp.d2 * xs, lp.d1 * ys, prm.reduced_costs)

    def infeas(cands):
        """Certificate directions are tested on the unscaled LP; a certificate is
        returned in the scaled space like every other result (R22)."""
        out = infeasibility_certificate(
            inst, lp.A_orig, [(lp.d2 * cx, lp.d1 * cy) for cx, cy in cands], prm.eps_infeas)
        if out is None:
            return None
        status, v = out
        xs, ys = cands[1]
        if status == PRIMAL_INFEASIBLE:
            return status, xs, v / lp.d1
        return status, v / lp.d2, ys

    run = PdlpRun(lp, prm, x, y, omega, eta_hat, lambda xs, ys: converged(measures(xs, ys), prm),
                  prm.max_iters, trace_iters, infeas if prm.detect_infeasibility else None)
    polish = None
    if prm.feasibility_polishing:
        status, xs, ys, polish = _solve_polished(lp, prm, run, measures)
    else:
        status, xs, ys = run.run()
    stats = dict(run.stats)
    stats.update(measures(xs, ys))
    stats.update(iterations=run.k, omega=run.omega, eta_hat=run.eta_hat)
    if polish is not None:
        stats["polish"] = polish
        stats["polish_primal_iters"] = sum(p["primal_iters"] for p in polish)
        stats["polish_dual_iters"] = sum(p["dual_iters"] for p in polish)
    return Result(status, lp.d2 * xs, lp.d1 * ys, stats, run.trace)


# ----------------------------------------------------------------------------
# feasibility polishing (Sec. 5, Algorithm 4)
# ----------------------------------------------------------------------------

def primal_feasibility_lp(lp: ScaledLP) -> ScaledLP:
    """The primal feasibility problem of Sec. 5: the LP with objective 0."""
    return dataclasses.replace(lp, c=np.zeros_like(lp.c))


def dual_feasibility_lp(lp: ScaledLP) -> ScaledLP:
    """The LP whose dual is the dual feasibility problem of Sec. 5: every finite bound
    set to 0 (infinite ones kept), so that p(.) vanishes on the dual feasible set while
    the sets Y and R, which depend only on which bounds are finite, are unchanged (R20)."""
    z = lambda v: np.where(np.isfinite(v), 0.0, v)  # noqa: E731
    return dataclasses.replace(lp, lc=z(lp.lc), uc=z(lp.uc), lv=z(lp.lv), uv=z(lp.uv))


def primal_feasible(st, prm: Params):
    """The primal half of the termination criteria."""
    if prm.termination_mode == 0:
        return st["rel_primal"] <= prm.eps_rel_kkt
    if prm.termination_mode == 2:
        return st["primal_res_rel_inf"] <= prm.eps_abs_feas
    return st["primal_res_inf"] <= prm.eps_abs_feas


def dual_feasible(st, prm: Params):
    """The dual half of the termination criteria."""
    if prm.termination_mode == 0:
        return st["rel_dual"] <= prm.eps_rel_kkt
    if prm.termination_mode == 2:
        return st["dual_res_rel_inf"] <= prm.eps_abs_feas
    return st["dual_res_inf"] <= prm.eps_abs_feas


def polish_pauses():
    """Iteration counts after which normal PDLP may pause: 100, 200, 400, ... (Alg. 4)."""
    k = 100
    while True:
        yield k
        k *= 2


def _solve_polished(lp, prm: Params, run: PdlpRun, measures):
    """Algorithm 4.  Normal PDLP (``run``) pauses after k = 100, 200, 400, ... iterations
    when the relative gap of Eq. (8) of its average iterate (x^k, y^k) is below
    eps_rel_gap.  Then PDLP on the primal feasibility problem runs from (x^k, 0), and
    PDLP on the dual feasibility problem from (0, y^k), each with normal PDLP's current
    primal weight and step estimate, for at most k/8 iterations and with its own
    iteration count (R21).  If the primal phase does not reach primal feasibility,
    normal PDLP resumes; otherwise the pair (x~ from the primal phase, y~ from the
    dual phase) is returned if it meets the termination criteria, else normal PDLP
    resumes.  Returns (status, x, y, log) with one log entry per pause."""
    m, n = run.m, run.n
    lp_p, lp_d = primal_feasibility_lp(lp), dual_feasibility_lp(lp)
    log = []
    for k_pause in polish_pauses():
        out = run.run(pause_at=k_pause)
        if out is not None:
            return (*out, log)
        xk, yk = run.average()
        gap = measures(xk, yk)["paper_gap"]
        entry = dict(k=k_pause, paper_gap=gap, primal_iters=0, primal_ok=False, dual_iters=0,
                     dual_ok=False, accepted=False)
        log.append(entry)
        if not gap < prm.eps_rel_gap:
            continue
        budget = k_pause // 8
        pr = PdlpRun(lp_p, prm, xk, np.zeros(m), run.omega, run.eta_hat,
                     lambda xs, ys: primal_feasible(measures(xs, ys), prm), budget)
        st_p, x_t, _ = pr.run()
        entry.update(primal_iters=pr.k, primal_ok=st_p == OPTIMAL)
        if st_p != OPTIMAL:
            continue
        dr = PdlpRun(lp_d, prm, np.zeros(n), yk, run.omega, run.eta_hat,
                     lambda xs, ys: dual_feasible(measures(xs, ys), prm), budget)
        st_d, _, y_t = dr.run()
        entry.update(dual_iters=dr.k, dual_ok=st_d == OPTIMAL)
        if converged(measures(x_t, y_t), prm):
            entry["accepted"] = True
            return OPTIMAL, x_t, y_t, log


# ----------------------------------------------------------------------------
# differentiation of unrolled PDHG (the adjoint of K steps of Eq. (3))
# ----------------------------------------------------------------------------

def unrolled_pdhg(inst, K, eta, omega):
    """K steps of PDHG, Eq. (3), on the LP as given (no preconditioning, restarts or
    adaptive steps): constant tau = eta/omega, sigma = eta*omega, start (proj_X(0), 0)
    (R1), dual step in the form of R17 with A x' - A x by linearity (R18).  Returns the
    list of iterates (x_k, y_k, Ax_k, A'y_k), k = 0..K (R23)."""
    A = inst.scipy_csr()
    AT = A.T.tocsr()
    tau, sigma = eta / omega, eta * omega
    x = proj_box(np.zeros(inst.n), inst.lv, inst.uv)
    y = np.zeros(inst.m)
    Ax, ATy = A @ x, AT @ y
    traj = [(x, y, Ax, ATy)]
    for _ in range(K):
        xn = primal_step(x, ATy, inst.c, inst.lv, inst.uv, tau)
        Axn = A @ xn
        yn = dual_step(y, Ax, Axn, inst.lc, inst.uc, sigma)
        x, y, Ax, ATy = xn, yn, Axn, AT @ yn
        traj.append((x, y, Ax, ATy))
    return traj


def unrolled_pdhg_vjp(inst, K, eta, omega, gx, gy):
    """Reverse-mode derivative of (x_K, y_K) = unrolled_pdhg(...)[K] contracted with
    (gx, gy): the gradients of L = gx'x_K + gy'y_K with respect to c, lc, uc, lv, uv
    (infinite bounds get 0).  Each step is differentiated piece by piece:
      x' = clamp(u, lv, uv), u = x - tau (c - A'y): d/du = 1 strictly inside, d/dlv = 1
        where u < lv, d/duv = 1 where u > uv;
      y' = yh - clamp(yh, -sigma uc, -sigma lc), yh = y - sigma (2 A x' - A x):
        d/dyh = 1 where yh < -sigma uc (then d/duc = sigma) or yh > -sigma lc (then
        d/dlc = sigma), 0 in between;
    and the start x_0 = clamp(0, lv, uv) likewise.  Returns (x_K, y_K, grads dict)."""
    A = inst.scipy_csr()
    AT = A.T.tocsr()
    tau, sigma = eta / omega, eta * omega
    traj = unrolled_pdhg(inst, K, eta, omega)
    g = {k: np.zeros(v) for k, v in (("c", inst.n), ("lc", inst.m), ("uc", inst.m),
                                     ("lv", inst.n), ("uv", inst.n))}
    bx, by = np.array(gx, dtype=float), np.array(gy, dtype=float)
    for k in range(K - 1, -1, -1):
        x, y, Ax, ATy = traj[k]
        xn, _, Axn, _ = traj[k + 1]
        # dual step
        yh = y - sigma * (2.0 * Axn - Ax)
        below, above = yh < -sigma * inst.uc, yh > -sigma * inst.lc
        byh = np.where(below | above, by, 0.0)
        g["uc"] += np.where(below, sigma * by, 0.0)
        g["lc"] += np.where(above, sigma * by, 0.0)
        q = AT @ byh                      # yh = y - sigma A (2x' - x)
        bxn = bx - 2.0 * sigma * q        # total adjoint of x'
        by_k = byh.copy()
        bx_k = sigma * q
        # primal step
        u = x - tau * (inst.c - ATy)
        lo, hi = u < inst.lv, u > inst.uv
        inside = ~(lo | hi)
        bu = np.where(inside, bxn, 0.0)
        g["lv"] += np.where(lo, bxn, 0.0)
        g["uv"] += np.where(hi, bxn, 0.0)
        g["c"] += -tau * bu
        bx_k += bu
        by_k += tau * (A @ bu)            # u depends on y through A'y
        bx, by = bx_k, by_k
    lo0, hi0 = 0.0 < inst.lv, 0.0 > inst.uv    # x_0 = clamp(0, lv, uv); y_0 = 0
    g["lv"] += np.where(lo0, bx, 0.0)
    g["uv"] += np.where(hi0, bx, 0.0)
    for key in ("lc", "uc", "lv", "uv"):
        g[key] = np.where(np.isfinite(getattr(inst, key)), g[key], 0.0)
    xK, yK = traj[K][0], traj[K][1]
    return xK, yK, g
