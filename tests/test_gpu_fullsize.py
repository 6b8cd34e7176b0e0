"""Parity at full size for the 80 nm hard-magnet cube (48^3 voxels,
857,375 potential unknowns; its full demagnetisation curve is part of the
bench line): sampled rows of the potential stiffness against the oracle
assembled on the sampled nodes' neighbourhoods, closed-form energies of
uniform states, the converged first field step against the properties of
a minimum, and one field step of both GPU forms against the oracle's own
minimisation at this size."""
import numpy as np
import pytest

import synth
from oracle import fem

pytestmark = pytest.mark.gpu

MU0 = 4e-7 * np.pi


@pytest.fixture(scope="module")
def full():
    from paper_1801_03690_gb300 import Magnet
    wl = synth.hard_cube()
    mag = Magnet(device=0)
    mag.upload_workload(wl)
    return wl, mag


def test_sizes(full):
    wl, mag = full
    s = mag.sizes()
    assert s["n_mag"] == 49 ** 3
    assert s["n_phi"] == 95 ** 3


def test_sampled_stiffness_rows_match_local_oracle_assembly(full):
    wl, mag = full
    mesh = wl.mesh
    rng = np.random.default_rng(0)
    v = rng.normal(size=mesh.n_nodes)
    nx = mesh.shape[0]
    ijk = lambda n: (n % nx, (n // nx) % nx, n // (nx * nx))
    boundary = np.zeros(mesh.n_nodes, bool)
    idx = np.arange(mesh.n_nodes)
    i, j, k = ijk(idx)
    boundary[(i == 0) | (j == 0) | (k == 0) | (i == nx - 1) | (j == nx - 1) | (k == nx - 1)] = True
    out = mag.potential_matvec(v)
    assert np.all(out[boundary] == 0.0)
    samples = rng.choice(np.nonzero(~boundary)[0], size=64, replace=False)
    # tets touching the samples; assemble the oracle on that sub-mesh
    touch = np.isin(mesh.tets, samples).any(axis=1)
    sub_tets = mesh.tets[touch]
    nodes = np.unique(sub_tets)
    loc = -np.ones(mesh.n_nodes, dtype=np.int64)
    loc[nodes] = np.arange(nodes.size)
    P = fem.assemble(mesh.xyz[nodes], loc[sub_tets], mesh.region[touch], wl.materials)
    vv = np.where(boundary[nodes], 0.0, v[nodes])          # outer-surface values do not enter
    ref = P.Kfull[loc[samples]] @ vv
    np.testing.assert_allclose(out[samples], ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_uniform_state_energies(full):
    from paper_1801_03690_gb300 import Params
    wl, mag = full
    u = np.array([0.3, -0.4, np.sqrt(1 - 0.25)])
    b = np.array([0.0, 0.2, -1.0])
    mag.set_field(b)
    F, terms = mag.energy(np.tile(u, (wl.mesh.n_nodes, 1)), Params(precision=1, poisson_tol=1e-10))
    Ms, K = wl.materials[1, 0], wl.materials[1, 2]
    ax = wl.materials[1, 3:6] / np.linalg.norm(wl.materials[1, 3:6])
    V = (80e-9) ** 3
    ex, an, dm, ze = terms
    assert abs(ex) < 1e-9 * abs(an)                      # uniform m: no exchange energy
    assert an == pytest.approx(-K * V * (u @ ax) ** 2, rel=1e-10)
    assert ze == pytest.approx(-Ms * V * (b @ u), rel=1e-10)
    assert 0.0 < dm < 0.5 * MU0 * Ms ** 2 * V            # 0 < N < 1
    assert F == pytest.approx(ex + an + dm + ze, rel=1e-12)


def test_first_field_step_reaches_a_minimum(full):
    from paper_1801_03690_gb300 import Params
    wl, mag = full
    mag.set_magnetization(wl.m0)
    mag.set_field(wl.fields[1])
    F0, _ = mag.energy(wl.m0, Params(precision=1))
    st = mag.minimize(Params(precision=1))
    assert st["status"] == "ok"
    assert st["F"] < F0
    m = mag.get_magnetization()
    mag_nodes = np.linalg.norm(m, axis=1) > 0
    np.testing.assert_allclose(np.linalg.norm(m[mag_nodes], axis=1), 1.0, atol=1e-13)
    g = mag.gradient(None, projected=True, params=Params(precision=1))
    # t3 at the returned state (internal units)
    assert np.abs(g).max() < 1e-10 ** (1 / 3) * (1 + abs(st["F_internal"]))
    assert st["evals"] == 2 * st["nli"] + 1 + st["ls_extra"]


def test_multigrid_form_first_field_step_matches_jacobi_form(full):
    """The bench's headline form (precision form, multigrid-preconditioned
    potential solve) at full size, in the launch configuration bench.py
    times: same minimum as the Jacobi-preconditioned precision form (energy
    1e-8 relative, max nodal |dm| 1e-5), |m| = 1, t3 at the returned state,
    and far fewer potential steps."""
    from paper_1801_03690_gb300 import Params
    wl, mag = full
    assert len(mag.amg_levels()) >= 3
    out = []
    for prm in (Params(precision=1), Params(precision=1, amg=1, inner_tol=1e-3)):
        mag.set_magnetization(wl.m0)
        mag.set_field(wl.fields[1])
        st = mag.minimize(prm)
        assert st["status"] == "ok"
        out.append((st, mag.get_magnetization()))
    (sj, mj), (sm, mm_) = out
    assert sm["F"] == pytest.approx(sj["F"], rel=1e-8)
    assert np.abs(mm_ - mj).max() < 1e-5
    mag_nodes = np.linalg.norm(mm_, axis=1) > 0
    np.testing.assert_allclose(np.linalg.norm(mm_[mag_nodes], axis=1), 1.0, atol=1e-13)
    g = mag.gradient(None, projected=True, params=Params(precision=1, amg=1, inner_tol=1e-3))
    assert np.abs(g).max() < 1e-10 ** (1 / 3) * (1 + abs(sm["F_internal"]))
    assert sm["mi"] / sm["evals"] < 0.25 * sj["mi"] / sj["evals"]


@pytest.mark.parametrize("form", ["plain_fp64", "multigrid_precision"])
def test_field_step_matches_oracle_minimization(full, form):
    """One field step of the curve (field index 1, from m0) at full size:
    the GPU plain FP64 form and the multigrid precision form against the
    oracle's Algorithm 4 with its own Jacobi-CG potential solve on the same
    mesh: energy 1e-8 relative, max nodal |dm| 1e-5; the FP64 form along the
    same path (same iteration, evaluation and inner-step counts)."""
    from paper_1801_03690_gb300 import Params
    from oracle import energy, ncg
    wl, mag = full
    P = _oracle_full(wl)
    b = wl.fields[1]
    prm = (Params(jmax=4, poisson_tol=1e-10) if form == "plain_fp64"
           else Params(jmax=4, poisson_tol=1e-10, precision=1, amg=1, inner_tol=1e-3))
    mag.set_magnetization(wl.m0)
    mag.set_field(b)
    st = mag.minimize(prm)
    m = mag.get_magnetization()[P.mag_nodes]
    r = _oracle_step(P, wl)
    assert st["status"] == "ok" and r.status == "converged"
    assert st["F"] == pytest.approx(r.F * P.units.energy_J, rel=1e-8)
    assert np.abs(m - r.m).max() < 1e-5
    if form == "plain_fp64":
        for k in ("nli", "evals", "li", "ls_extra"):
            assert st[k] == r.stats[k], (k, st[k], r.stats[k])


_ORACLE = {}


def _oracle_full(wl):
    if "P" not in _ORACLE:
        _ORACLE["P"] = fem.assemble_workload(wl)
    return _ORACLE["P"]


def _oracle_step(P, wl):
    from oracle import energy, ncg
    if "r" not in _ORACLE:
        _ORACLE["r"] = ncg.minimize(P, energy.normalize(wl.m0[P.mag_nodes]), P.units.field_int(wl.fields[1]),
                                    ncg.Params(jmax=4, poisson="cg", poisson_tol=1e-10))
    return _ORACLE["r"]
