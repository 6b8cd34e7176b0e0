"""muMAG standard problem 3 (Sec. 3.3): the single-domain limit of a soft
cube with uniaxial anisotropy K = 0.1 Km (Km = mu0 Ms^2 / 2) along z.  The
twisted flower state (relaxed from saturation) and the vortex state
(relaxed from two domains with a sharp wall) are minimised at zero field
with tau_F = 1e-12; their energies cross at the critical edge, which the
paper finds at 8.52 l_ex (Hertel and Kronmueller: 8.56 l_ex).  The mesh is
h ~ 0.35 l_ex (24 voxels per edge) in a graded air box of 8 times the edge
(measured: 8.51 l_ex; a box of 4 edges lowers the flower state's
stray-field energy enough to move the crossover to 8.64 l_ex); the
crossover is required within 1.5% of 8.52 l_ex.  On the smallest edge both
states are checked against the oracle on the same mesh at 12 voxels per
edge (the parity check needs the same mesh on both sides, not the fine one;
the oracle's vortex relaxation takes about 2 minutes there, 6 at 16).""" 
import numpy as np
import pytest

import synth
from oracle import fem, energy, ncg

pytestmark = pytest.mark.gpu

EDGES = (8.3, 8.5, 8.7, 8.9)
TAU = dict(tau_F=1e-12, jmax=12, poisson_tol=1e-12, max_iter=100000)


def _relax(L, start, n_mag, box=8.0):
    from paper_1801_03690_gb300 import Magnet, Params
    wl = synth.sp3_cube(L, n_mag=n_mag, start=start, box_factor=box)
    mag = Magnet(device=0)
    mag.upload_workload(wl)
    mag.set_magnetization(wl.m0)
    st = mag.minimize(Params(**TAU))
    m = mag.get_magnetization()
    mag.close()
    km, Lm = wl.meta["Km"], wl.meta["L"]
    return wl, st, m, st["F"] / (km * Lm ** 3)


def test_flower_vortex_crossover_near_8_52_lex():
    de = []
    for L in EDGES:
        _, sf, _, ef = _relax(L, "flower", 24)
        _, sv, _, ev = _relax(L, "vortex", 24)
        assert sf["status"] == "ok" and sv["status"] == "ok"
        assert sf["M"][2] > 0.9                                   # flower: nearly saturated along z
        assert np.linalg.norm(sv["M"]) < 0.5                      # vortex: flux closure
        de.append(ef - ev)
    de = np.array(de)
    changes = np.nonzero(de[:-1] * de[1:] < 0)[0]
    assert len(changes) == 1, de                                  # the flower is lower below, the vortex above
    i = changes[0]
    cross = EDGES[i] + de[i] / (de[i] - de[i + 1]) * (EDGES[i + 1] - EDGES[i])
    print(f"flower/vortex crossover at {cross:.3f} l_ex (paper 8.52)")
    assert abs(cross - 8.52) <= 0.015 * 8.52


def test_states_match_oracle_on_the_smallest_edge():
    """Flower (deterministic from saturation): energy 1e-8 relative, max
    nodal |dm| 1e-5, the same iteration count.  Vortex (from a symmetric
    two-domain start, so the side the wall curls to is decided by rounding
    and mirror images on the Kuhn lattice differ slightly): the same
    energy within 1e-4 relative and the same closure |M| within 0.02."""
    L = EDGES[0]
    for start in ("flower", "vortex"):
        wl, st, m, e = _relax(L, start, 12)
        P = fem.assemble_workload(wl)
        r = ncg.minimize(P, energy.normalize(wl.m0[P.mag_nodes]), np.zeros(3),
                         ncg.Params(tau_F=1e-12, jmax=12, max_iter=100000))
        assert r.status == "converged"
        F_or = r.F * P.units.energy_J
        M_or = (P.w[:, None] * r.m).sum(0) / P.w.sum()
        if start == "flower":
            assert st["F"] == pytest.approx(F_or, rel=1e-8)
            assert np.abs(m[P.mag_nodes] - r.m).max() < 1e-5
            assert st["nli"] == r.stats["nli"]
        else:
            assert st["F"] == pytest.approx(F_or, rel=1e-4)
            assert abs(np.linalg.norm(st["M"]) - np.linalg.norm(M_or)) < 0.02
