"""The sparse approximate Hessian preconditioner and its truncated solve.

Eq. (precond): only the short-range (exchange + anisotropy) part of the
Hessian of the Lagrangian (Eq. hessact) is kept:

  (H(m) v)_i = (C v)_i - (m_i . (C v)_i) m_i - (m_i . grad F_i) v_i
               [ - (v_i . grad F_i) m_i ]

with C = C_A + C_K (magnetostatics dropped, Sec. 3.4).  The bracketed last
term is dropped by default: the paper reports that H without it performed
best.  P y = g is solved by Algorithm 1 with y_0 = 0 and the Jacobi matrix
built from the exchange interactions, P_ij = delta_ij C_A,ij, stopped by
  li1: at most j_max steps,
  li2: d^T H d <= 0 (negative curvature),
  li3: |g_{j+1}| < min(0.5, sqrt(|b|)) |g_0|, b = the right-hand side g.
j_max = 0 means no preconditioning (y = g).  A negative-curvature exit on
the very first step leaves y = 0, which is replaced by y = g.  Nodes whose
C_A diagonal is zero (no exchange) use 1 in the Jacobi matrix.

Pins (tests/test_oracle_precond.py): with all four terms and no
magnetostatics H v equals the directional derivative of Pi_{m perp} grad F
(central differences); the default operator differs from it by exactly
(v_i . grad F_i) m_i; H maps tangent vectors to tangent vectors; the solve
matches a dense solve of the projected system when j_max is large.
"""
import numpy as np

from .linear_cg import alg1


def apply_C_local(P, v):
    """(C_A + C_K) v for v (Nm, 3)."""
    return 2.0 * (P.KA @ v) + np.einsum("iab,ib->ia", P.CK, v)


def apply_H(P, m, grad, v, keep_last=False):
    """Eq. (precond) applied to v (Nm, 3)."""
    Cv = apply_C_local(P, v)
    lam = np.sum(m * grad, axis=1)
    Hv = Cv - np.sum(m * Cv, axis=1, keepdims=True) * m - lam[:, None] * v
    if keep_last:
        Hv -= np.sum(v * grad, axis=1, keepdims=True) * m
    return Hv


def jacobi_diag(P):
    d = P.diag_CA.copy()
    d[d == 0.0] = 1.0
    return d


def precond_solve(P, m, grad, g, jmax, keep_last=False, counts=None):
    """Solve H(m) y = g approximately.  Returns (y, steps).  With a dict
    `counts`, the exits by negative curvature (li2) are tallied in
    counts["li2"] and, of them, those on the first step in
    counts["li2_first"] (bookkeeping only)."""
    if jmax <= 0:
        return g.copy(), 0
    nm = m.shape[0]
    dinv = 1.0 / jacobi_diag(P)

    def H(vflat):
        return apply_H(P, m, grad, vflat.reshape(nm, 3), keep_last).reshape(-1)

    def Pinv(gflat):
        return (gflat.reshape(nm, 3) * dinv[:, None]).reshape(-1)

    rhs = g.reshape(-1)
    ng = np.linalg.norm(rhs)
    eps = min(0.5, np.sqrt(ng)) * ng
    # Algorithm 1 solves C x = -b_alg1 with C = H, b_alg1 = -g, x0 = 0
    y, steps, reason = alg1(H, -rhs, np.zeros_like(rhs), Pinv, eps, jmax,
                            neg_curvature=True)
    if counts is not None and reason == "neg_curvature":
        counts["li2"] = counts.get("li2", 0) + 1
        if steps == 1:
            counts["li2_first"] = counts.get("li2_first", 0) + 1
    if reason == "neg_curvature" and steps == 1:
        y = rhs.copy()
    return y.reshape(nm, 3), steps
