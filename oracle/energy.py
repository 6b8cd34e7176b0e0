"""Energy, gradient and projections of Sec. 2.2.

Eq. (energy) in the assembled form of ``fem``:

  F(m) = 1/2 m^T C_A m + 1/2 m^T C_K m + E_demag(m) - sum_i w_i h . m_i
  grad F = C_A m + C_K m + D^T phi - w h,      K_phi phi = D m

E_demag = 1/2 phi^T D m at the exact potential.  The value is evaluated in
the equivalent variational form phi^T b - 1/2 phi^T K_phi phi (b = D m),
whose error is quadratic in the error of an approximate potential; at the
exact potential the two agree.

Eq. (proj):   (Pi_{m perp} v)_i = v_i - (v_i . m_i) m_i
Eq. (nablaLF): the projected gradient g = Pi_{m perp} grad F, with the KKT
               multiplier lambda_i = m_i . grad F_i
Eq. (opt2):   grad Ftilde(u)_i = (grad F(N u)_i - (u_i.grad F(N u)_i)/|u_i|^2 u_i)/|u_i|
              = g(N u)_i / |u_i|,  N u = u_i/|u_i| per node.

Pins (tests/test_oracle_energy.py): central differences of F equal grad F to
round-off (F is quadratic); the derivative of F(N(x + a d)) equals the opt2
expression; the demagnetising energy of a uniformly magnetised cube tends to
mu0 Ms^2 V/6 (factor 1/3, Richardson in box size); adjointness of D and D^T;
E_demag >= 0; the direct and iterative potentials give the same energy.
"""
import numpy as np
import scipy.sparse.linalg as spla

from .linear_cg import alg1


def normalize(v):
    """(N v)_i = v_i / |v_i|."""
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def project(m, v):
    """Eq. (proj)."""
    return v - np.sum(v * m, axis=1, keepdims=True) * m


def poisson_rhs(P, m):
    return P.D @ m.reshape(-1)


def solve_potential(P, m, method="direct", phi0=None, tol=1e-10, max_iter=100000):
    """Solve K_phi phi = D m.  "direct": sparse LU (the definition, exact to
    round-off).  "cg": Algorithm 1 with the Jacobi preconditioner
    diag(K_phi), started from phi0 (or zero), stopped at
    |K phi - b| < tol |b|.  Returns (phi, steps)."""
    b = poisson_rhs(P, m)
    if method == "direct":
        lu = P.cache.get("lu")
        if lu is None:
            lu = spla.splu(P.Kphi.tocsc())
            P.cache["lu"] = lu
        return lu.solve(b), 0
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return np.zeros_like(b), 0
    dinv = 1.0 / P.Kphi.diagonal()
    x0 = np.zeros_like(b) if phi0 is None else phi0
    # Algorithm 1 solves C x = -b_alg1: here C = K_phi and b_alg1 = -b
    phi, steps, _ = alg1(lambda v: P.Kphi @ v, -b, x0, lambda g: dinv * g,
                         tol * nb, max_iter)
    return phi, steps


def energy_terms(P, m, phi, h):
    """Energy contributions (internal units) for unit vectors m (Nm, 3),
    potential phi and uniform reduced field h (3,)."""
    KAm = P.KA @ m
    ex = float(np.sum(m * KAm))                       # 1/2 m^T (2 K_A x I3) m
    an = 0.5 * float(np.einsum("ia,iab,ib->", m, P.CK, m))
    b = poisson_rhs(P, m)
    r = b - P.Kphi @ phi
    dm = float(phi @ b) - 0.5 * float(phi @ (b - r))  # phi.b - 1/2 phi.K phi
    ze = -float(np.sum(P.w[:, None] * (m @ np.asarray(h))[:, None]))
    return {"exchange": ex, "anisotropy": an, "demag": dm, "zeeman": ze,
            "total": ex + an + dm + ze}


def gradient(P, m, phi, h):
    """grad F = C_A m + C_K m + D^T phi - w h, shape (Nm, 3)."""
    g = 2.0 * (P.KA @ m)
    g += np.einsum("iab,ib->ia", P.CK, m)
    g += (P.D.T @ phi).reshape(-1, 3)
    g -= P.w[:, None] * np.asarray(h)[None, :]
    return g


def evaluate(P, m, h, poisson="direct", phi0=None, tol=1e-10):
    """One function evaluation at unit vectors m: potential, energy, gradient
    and projected gradient.  Returns a dict."""
    phi, steps = solve_potential(P, m, poisson, phi0=phi0, tol=tol)
    terms = energy_terms(P, m, phi, h)
    grad = gradient(P, m, phi, h)
    return {"F": terms["total"], "terms": terms, "grad": grad,
            "g": project(m, grad), "phi": phi, "poisson_steps": steps}


def ftilde_derivative(g_at, u, d):
    """d/da F(N(x + a d)) at u = x + a d, given the projected gradient at N u
    (Eq. opt2): sum_i g_i . d_i / |u_i|."""
    return float(np.sum(np.sum(g_at * d, axis=1) / np.linalg.norm(u, axis=1)))
