"""Algorithm 1: preconditioned linear conjugate gradient for C x = -b.

Written in the paper's notation (Sec. 2.1): residual g = C x + b, the
preconditioned residual y solves P y = g, the direction starts at d = -y;
each step takes alpha = g.y / d.C d, moves x by alpha d, updates
g by alpha C d, exits once |g| < eps, then forms beta = g+.y+ / g.y and
d = -y + beta d.

Two optional exits serve the truncated preconditioner solve (Sec. 3.1):
``max_iter`` (li1: at most j_max steps) and ``neg_curvature`` (li2: stop
when d^T C d <= 0 before using the step).  The step counter returned is the
number of products C d formed inside the loop.

Pins (tests/test_oracle_cg.py): agreement with a dense direct solve on
random SPD systems, exact termination within n steps, the monotone decrease
of the C-norm error, and the li2 exit on an indefinite matrix.
"""
import numpy as np


def alg1(apply_C, b, x0, apply_Pinv, eps, max_iter, neg_curvature=False):
    """Returns (x, steps, reason) with reason in {"tol", "max_iter",
    "neg_curvature"}; reason "neg_curvature" at steps == 1 means no step
    was taken (x = x0)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    g = apply_C(x) + b
    if np.linalg.norm(g) < eps:
        return x, 0, "tol"
    y = apply_Pinv(g)
    d = -y
    gy = float(g @ y)
    steps = 0
    while steps < max_iter:
        Cd = apply_C(d)
        steps += 1
        dCd = float(d @ Cd)
        if neg_curvature and dCd <= 0.0:
            return x, steps, "neg_curvature"
        alpha = gy / dCd
        x = x + alpha * d
        g = g + alpha * Cd
        if np.linalg.norm(g) < eps:
            return x, steps, "tol"
        y = apply_Pinv(g)
        gy_new = float(g @ y)
        beta = gy_new / gy
        gy = gy_new
        d = -y + beta * d
    return x, steps, "max_iter"
