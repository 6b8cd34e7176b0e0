"""The demagnetisation curve (Sec. 3.1): the field changes in small steps and
at each field a minimum is computed by Algorithm 4, starting from the
minimum of the previous field.

Per field step k the record holds the reduced magnetisation
M_k = sum_i w_i m_i / sum_i w_i (w = lumped Ms weights), the energy and the
counters of ``ncg.minimize``.  The coercive field is the applied field at
which M.u changes sign, u the unit vector of the sweep direction
(fields[-1] - fields[0]), by linear interpolation between the two bracketing
steps; it is reported as |mu0 H . u| in tesla.

Pins (tests/test_oracle_ncg.py): the Stoner-Wohlfarth switching field of a
small exchange-coupled particle, and the zero-crossing interpolation on
hand-made records.
"""
import numpy as np

from .energy import normalize
from .ncg import minimize, Params


def sweep_axis(fields):
    f = np.asarray(fields, dtype=np.float64)
    u = f[-1] - f[0]
    n = np.linalg.norm(u)
    if n == 0.0:
        n = np.linalg.norm(f[-1])
        u = f[-1]
    return u / n


def coercive_field(fields, M, u=None):
    """Interpolated |mu0 H . u| at the first sign change of M . u (or None)."""
    f = np.asarray(fields, dtype=np.float64)
    u = sweep_axis(f) if u is None else u
    mu = np.asarray(M) @ u
    hu = f @ u
    for k in range(1, len(mu)):
        if mu[k - 1] == 0.0:
            return abs(hu[k - 1])
        if mu[k - 1] * mu[k] < 0.0:
            t = mu[k - 1] / (mu[k - 1] - mu[k])
            return abs(hu[k - 1] + t * (hu[k] - hu[k - 1]))
    return None


def demag_curve(P, fields_T, m0_nodes, params=None, n_steps=None):
    """Run the field loop.  fields_T: (F, 3) mu0*H in tesla; m0_nodes: (N, 3)
    initial magnetisation per mesh node (magnetic nodes used)."""
    p = params or Params()
    m = normalize(np.asarray(m0_nodes, dtype=np.float64)[P.mag_nodes])
    phi = None
    wsum = P.w.sum()
    records = []
    fields_T = np.asarray(fields_T, dtype=np.float64)
    if n_steps is not None:
        fields_T = fields_T[:n_steps]
    for b in fields_T:
        h = P.units.field_int(b)
        r = minimize(P, m, h, p, phi0=phi)
        m, phi = r.m, r.phi
        Mvec = (P.w[:, None] * m).sum(axis=0) / wsum
        records.append({"field_T": b.copy(), "M": Mvec, "F": r.F,
                        "F_J": r.F * P.units.energy_J, "status": r.status, **r.stats})
    M = np.array([rec["M"] for rec in records])
    return {"records": records, "M": M, "m": m, "phi": phi,
            "Hc_T": coercive_field(fields_T, M)}
