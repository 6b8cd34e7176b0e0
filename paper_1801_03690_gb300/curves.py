"""Helpers for demagnetisation curves (Sec. 3.1): the sweep axis and the
coercive field as the interpolated zero crossing of M along it."""
import numpy as np


def sweep_axis(fields):
    f = np.asarray(fields, dtype=np.float64)
    u = f[-1] - f[0]
    if not np.any(u):
        u = f[-1]
    return u / np.linalg.norm(u)


def coercive_field(fields, M):
    """|mu0 H . u| (tesla) at the first sign change of M . u, linearly
    interpolated between the bracketing field steps; None if M never
    changes sign."""
    f = np.asarray(fields, dtype=np.float64)
    u = sweep_axis(f)
    mu = np.asarray(M, dtype=np.float64) @ u
    hu = f @ u
    for k in range(1, len(mu)):
        if mu[k - 1] == 0.0:
            return float(abs(hu[k - 1]))
        if mu[k - 1] * mu[k] < 0.0:
            t = mu[k - 1] / (mu[k - 1] - mu[k])
            return float(abs(hu[k - 1] + t * (hu[k] - hu[k - 1])))
    return None
