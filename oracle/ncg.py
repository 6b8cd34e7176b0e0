"""Algorithm 4: projected, preconditioned nonlinear conjugate gradient method
for micromagnetics, with the beta*ZA restart rule (Sec. 2.2), the descent
safeguard, a line search that avoids too long steps, and the stopping rules
t1-t3 (Sec. 3.1).

Steps per field (the order of Algorithm 4):
  init: x_0 = N(m_0); g_0 = Pi(grad F(x_0)); solve P_0 y_0 = g_0; d_0 = -y_0
  loop: alpha_j from the line search on F(N(x_j + alpha d_j));
        x_{j+1} = N(x_j + alpha_j d_j); g_{j+1} = Pi(grad F(x_{j+1}));
        solve P_{j+1} y_{j+1} = g_{j+1};
        d_{j+1} = -y_{j+1} + beta*ZA d_j;
        stop when t1, t2 and t3 all hold.

beta*ZA = (g+ - g).y+ / (g+ - g).d  if y+.g+ > y+.g, else 0.  The paper's
other preconditioned rules (Sec. 2.1, Algorithm 3) are selectable:
beta*FR = g+.y+ / g.y and beta*PRP = (g+ - g).y+ / g.y.

Readings where the paper is silent or garbled (shared exactly with the CUDA
path):
  * Descent safeguard ("replace y by g if g.d > 0", indices garbled): if the
    new direction has g.d >= 0, y is replaced by g, beta is recomputed with
    it, and if g.d is still >= 0 the direction becomes d = -g.  The initial
    direction gets the same treatment.
  * Line search (defined only by reference to Fischbacher et al. 2017, "which
    avoids too long steps"): phi(a) = F(N(x + a d)), phi'(a) from Eq. (opt2).
    Step cap a_max = theta_max / max_i |d_i|.  Trial a_t = min(a_prev, a_max)
    (a_prev = 1 at the start of each field).  One evaluation at a_t, then the
    minimiser a_s of the cubic Hermite interpolant of (phi(0), phi'(0),
    phi(a_t), phi'(a_t)), clamped to [0.1 a_t, min(4 a_t, a_max)] (when the
    cubic has no minimiser: 4 a_t if phi'(a_t) < 0 else a_t/2, then clamped),
    and one evaluation at a_s.  The lower of the two (a_s on ties) is taken
    if it satisfies phi(a) <= phi(0) + c1 a phi'(0); otherwise a halves from
    min(a_t, a_s)/2 until that holds (at most max_backtrack evaluations).  If
    nothing qualifies the minimiser stops with status "stalled" and x
    unchanged.  This gives exactly two evaluations per iteration in the
    common case, matching evals = 2 nli + n_fields in Tables 1 and 2.
  * Stopping rules t1-t3 use internal units (fem.Units) and the max norm
    over all 3N components.
  * Potential tolerance (the paper does not state one): poisson_tol for
    every solve, or with poisson_sched a schedule tied to t1 (see
    scheduled_tolerance): looser solves while the previous energy decrease
    is more than 100 times the t1 threshold.
  * beta*FR / beta*PRP need g_j.y_j of the previous direction; after the
    safeguard replaced y by g, that is g_j.g_j.
  * Counters: evals (function evaluations), nli (iterations), li (products
    with H in the inner solves), mi (products with K_phi in the loop of the
    Poisson solves; 0 with the direct solver), ls_extra (evaluations spent
    backtracking); the branches taken: li2 (inner solves ended by negative
    curvature), li2_first (of them on the first step: y = g), restarts (y
    replaced by g in the safeguard), steepest (d = -g).

Pins (tests/test_oracle_ncg.py): the Stoner-Wohlfarth switching field of a
small particle (exchange-coupled uniform rotation, demag off), the exact
beta*ZA branches on hand-made vectors, the iteration identities
evals = 2 nli + 1 and li = j_max (nli + 1) when every inner solve runs to
j_max, monotone energy decrease, and |m_i| = 1 at every accepted iterate.
"""
from dataclasses import dataclass, field

import numpy as np

from .energy import evaluate, normalize, ftilde_derivative
from .precond import precond_solve


@dataclass
class Params:
    tau_F: float = 1e-10
    jmax: int = 4
    max_iter: int = 10000
    theta_max: float = 0.1
    c1: float = 1e-4
    max_backtrack: int = 10
    keep_last_term: bool = False
    poisson: str = "direct"        # "direct" or "cg"
    poisson_tol: float = 1e-10
    beta_rule: str = "ZA"          # "ZA", "FR" or "PRP" (Sec. 2.1, Eqs. FRstar, PRPstar)
    poisson_sched: bool = False    # potential tolerance tied to t1 (CG potential solve only)
    poisson_tol_max: float = 1e-6


@dataclass
class Result:
    m: np.ndarray
    F: float
    terms: dict
    g: np.ndarray
    phi: np.ndarray
    status: str
    stats: dict = field(default_factory=dict)


def beta_za(g_new, g_old, y_new, d_old):
    """beta*ZA (Hestenes-Stiefel with restart)."""
    if float(np.sum(y_new * g_new)) > float(np.sum(y_new * g_old)):
        dg = g_new - g_old
        den = float(np.sum(dg * d_old))
        if den == 0.0:
            return 0.0
        return float(np.sum(dg * y_new)) / den
    return 0.0


def beta_fr(g_new, y_new, gy_old):
    """beta*FR = g_{j+1}.y_{j+1} / g_j.y_j (Eq. FRstar); 0 if g_j.y_j = 0."""
    return 0.0 if gy_old == 0.0 else float(np.sum(g_new * y_new)) / gy_old


def beta_prp(g_new, g_old, y_new, gy_old):
    """beta*PRP = (g_{j+1} - g_j).y_{j+1} / g_j.y_j (Eq. PRPstar)."""
    return 0.0 if gy_old == 0.0 else float(np.sum((g_new - g_old) * y_new)) / gy_old


def _beta(rule, g_new, g_old, y_new, d_old, gy_old):
    if rule == "FR":
        return beta_fr(g_new, y_new, gy_old)
    if rule == "PRP":
        return beta_prp(g_new, g_old, y_new, gy_old)
    return beta_za(g_new, g_old, y_new, d_old)


def direction(g_new, g_old, y_new, d_old, counts=None, rule="ZA", gy_old=0.0):
    """d = -y + beta d_old (beta*ZA, or beta*FR / beta*PRP with gy_old =
    g_j.y_j of the previous direction) with the descent safeguard: if
    g.d >= 0, y is replaced by g and beta recomputed; if still g.d >= 0,
    d = -g.  Returns (d, g_{j+1}.y) with y the vector the direction was built
    from (g itself after the safeguard), which the next beta*FR / beta*PRP
    needs.  With a dict `counts`, the safeguard's branches are tallied:
    counts["restarts"] when y is replaced by g, counts["steepest"] when d
    falls back to -g (bookkeeping only)."""
    beta = _beta(rule, g_new, g_old, y_new, d_old, gy_old)
    d = -y_new + beta * d_old
    gy = float(np.sum(g_new * y_new))
    if float(np.sum(g_new * d)) >= 0.0:
        if counts is not None:
            counts["restarts"] = counts.get("restarts", 0) + 1
        beta = _beta(rule, g_new, g_old, g_new, d_old, gy_old)
        d = -g_new + beta * d_old
        gy = float(np.sum(g_new * g_new))
        if float(np.sum(g_new * d)) >= 0.0:
            if counts is not None:
                counts["steepest"] = counts.get("steepest", 0) + 1
            d = -g_new.copy()
    return d, gy


def scheduled_tolerance(p, dF_prev, F0):
    """Potential tolerance of one iteration with the schedule tied to t1
    (a reading: the paper leaves the potential tolerance open): while the
    previous energy decrease dF_prev exceeds 100 times the t1 threshold
    tau_F (1 + |F|), the solve may stop at poisson_tol sqrt(dF / threshold)
    / 10 (at most poisson_tol_max) -- the energy error of the variational
    form is quadratic in the potential error, so it stays far below the
    decrease the line search resolves; otherwise poisson_tol."""
    if not p.poisson_sched or dF_prev is None or not dF_prev > 0.0:
        return p.poisson_tol
    q = dF_prev / (p.tau_F * (1.0 + abs(F0)))
    if q <= 100.0:
        return p.poisson_tol
    return min(p.poisson_tol_max, max(p.poisson_tol, p.poisson_tol * np.sqrt(q) / 10.0))


def cubic_step(f0, g0, a, f1, g1):
    """Minimiser of the cubic Hermite interpolant through (0, f0, g0) and
    (a, f1, g1), or None if it has none."""
    d1 = g0 + g1 - 3.0 * (f1 - f0) / a
    disc = d1 * d1 - g0 * g1
    if disc <= 0.0:                  # no stationary point, or only an inflection
        return None
    d2 = np.sqrt(disc)
    den = g1 - g0 + 2.0 * d2
    if den == 0.0:
        return None
    return a - a * (g1 + d2 - d1) / den


def minimize(P, m0, h, params=None, phi0=None):
    """Minimise F at reduced field h starting from m0 (Nm, 3)."""
    p = params or Params()
    st = {"evals": 0, "nli": 0, "li": 0, "mi": 0, "ls_extra": 0,
          "li2": 0, "li2_first": 0, "restarts": 0, "steepest": 0}

    tol = [p.poisson_tol]

    def ev(m, phi_warm):
        e = evaluate(P, m, h, p.poisson, phi0=phi_warm, tol=tol[0])
        st["evals"] += 1
        st["mi"] += e["poisson_steps"]
        return e

    def pre(m, e):
        y, steps = precond_solve(P, m, e["grad"], e["g"], p.jmax, p.keep_last_term, counts=st)
        st["li"] += steps
        return y

    x = normalize(np.asarray(m0, dtype=np.float64))
    e = ev(x, phi0)
    phi = e["phi"]
    y = pre(x, e)
    d = -y
    gy = float(np.sum(e["g"] * y))
    if float(np.sum(e["g"] * d)) >= 0.0:
        st["steepest"] += 1
        d = -e["g"].copy()
        gy = float(np.sum(e["g"] * e["g"]))
    dF_prev = None
    a_prev = 1.0
    status = "max_iter"
    if not np.isfinite(e["F"]):
        status = "nonfinite"
    elif np.max(np.abs(e["g"])) == 0.0:
        status = "converged"
    while status == "max_iter" and st["nli"] < p.max_iter:
        F0 = e["F"]
        tol[0] = scheduled_tolerance(p, dF_prev, F0)
        dphi0 = float(np.sum(e["g"] * d))
        a_max = p.theta_max / np.max(np.linalg.norm(d, axis=1))
        a_t = min(a_prev, a_max)
        u_t = x + a_t * d
        x_t = normalize(u_t)
        e_t = ev(x_t, phi)
        phi = e_t["phi"]
        dphi_t = ftilde_derivative(e_t["g"], u_t, d)
        a_s = cubic_step(F0, dphi0, a_t, e_t["F"], dphi_t)
        if a_s is None or not np.isfinite(a_s):
            a_s = 4.0 * a_t if dphi_t < 0.0 else 0.5 * a_t
        a_s = min(max(a_s, 0.1 * a_t), min(4.0 * a_t, a_max))
        x_s = normalize(x + a_s * d)
        e_s = ev(x_s, phi)
        phi = e_s["phi"]
        if e_s["F"] <= e_t["F"]:
            a_b, x_b, e_b = a_s, x_s, e_s
        else:
            a_b, x_b, e_b = a_t, x_t, e_t
        if not (e_b["F"] <= F0 + p.c1 * a_b * dphi0):
            found = False
            a = 0.5 * min(a_t, a_s)
            for _ in range(p.max_backtrack):
                x_k = normalize(x + a * d)
                e_k = ev(x_k, phi)
                st["ls_extra"] += 1
                phi = e_k["phi"]
                if e_k["F"] <= F0 + p.c1 * a * dphi0:
                    a_b, x_b, e_b = a, x_k, e_k
                    found = True
                    break
                a *= 0.5
            if not found:
                status = "stalled"
                break
        st["nli"] += 1
        dF_prev = F0 - e_b["F"]
        if not np.isfinite(e_b["F"]):
            status = "nonfinite"
            break
        t1 = F0 - e_b["F"] < p.tau_F * (1.0 + abs(e_b["F"]))
        t2 = np.max(np.abs(x - x_b)) < np.sqrt(p.tau_F) * (1.0 + np.max(np.abs(x_b)))
        t3 = np.max(np.abs(e_b["g"])) < p.tau_F ** (1.0 / 3.0) * (1.0 + abs(e_b["F"]))
        y_new = pre(x_b, e_b)
        d, gy = direction(e_b["g"], e["g"], y_new, d, counts=st, rule=p.beta_rule, gy_old=gy)
        x, e, a_prev = x_b, e_b, a_b
        if t1 and t2 and t3:
            status = "converged"
    return Result(m=x, F=e["F"], terms=e["terms"], g=e["g"], phi=phi,
                  status=status, stats=st)
