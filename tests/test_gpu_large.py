"""Parity at the benchmark's full size: the large polycrystalline magnet
(149^3 voxels, 125 grains with a grain-boundary phase, graded air box;
3,375,000 magnetic nodes, 8,741,816 potential unknowns) in the launch
configuration bench.py times.

The oracle cannot assemble this mesh in seconds, so the operators are
checked on sampled rows: the oracle assembles the tetrahedra around 48
sampled nodes, and the input vectors vanish on the outer surface of that
sub-mesh, so that every sampled row of D v, D^T phi, (C_A + C_K) v and
K_phi v is exact there (1e-12 relative).  Closed forms pin the energies of
uniform states; the headline form's first field step is checked against
the plain FP64 form on the same mesh (energy 1e-8, max nodal |dm| 1e-5) and
against the properties of a minimum."""
import numpy as np
import pytest

import synth
from oracle import fem, precond

pytestmark = pytest.mark.gpu

MU0 = 4e-7 * np.pi


@pytest.fixture(scope="module")
def big():
    from paper_1801_03690_gb300 import Magnet
    wl = synth.large_polycrystal()
    mag = Magnet(device=0)
    mag.upload_workload(wl)
    yield wl, mag
    mag.close()


@pytest.fixture(scope="module")
def sampled(big):
    """48 sampled magnetic nodes (interior of the mesh, some on grain
    boundaries), the oracle on the sub-mesh of their tetrahedra, and the
    sub-mesh's outer-surface nodes (where the inputs are set to zero)."""
    wl, mag = big
    mesh = wl.mesh
    rng = np.random.default_rng(0)
    magn = np.unique(mesh.tets[wl.materials[mesh.region, 0] > 0])
    # nodes touching more than one region: interfaces of grains / boundary phase / air
    lo = np.full(mesh.n_nodes, 1 << 30)
    hi = np.full(mesh.n_nodes, -1)
    for c in range(4):
        np.minimum.at(lo, mesh.tets[:, c], mesh.region)
        np.maximum.at(hi, mesh.tets[:, c], mesh.region)
    inter = magn[lo[magn] != hi[magn]]
    samples = np.concatenate([rng.choice(magn, 24, replace=False), rng.choice(inter, 24, replace=False)])
    touch = np.isin(mesh.tets, samples).any(axis=1)
    sub = mesh.tets[touch]
    nodes = np.unique(sub)
    loc = -np.ones(mesh.n_nodes, dtype=np.int64)
    loc[nodes] = np.arange(nodes.size)
    P = fem.assemble(mesh.xyz[nodes], loc[sub], mesh.region[touch], wl.materials)
    zero = np.zeros(mesh.n_nodes, bool)
    zero[nodes[P.dirichlet_nodes]] = True
    return samples, nodes, loc, P, zero


def _close(out, ref):
    scale = np.abs(ref).max()
    assert scale > 0
    assert np.abs(out - ref).max() <= 1e-12 * scale, np.abs(out - ref).max() / scale


def test_sizes(big):
    wl, mag = big
    s = mag.sizes()
    assert s["n_mag"] == 150 ** 3
    assert s["n_phi"] == 8741816
    assert len(mag.amg_levels()) >= 3


def test_sampled_operator_rows(big, sampled):
    wl, mag = big
    samples, nodes, loc, P, zero = sampled
    rng = np.random.default_rng(1)
    N = wl.mesh.n_nodes
    v3 = rng.normal(size=(N, 3))
    v3[zero] = 0.0
    v1 = rng.normal(size=N)
    v1[zero] = 0.0
    vs3 = v3[nodes]
    vs1 = v1[nodes]
    rows = loc[samples]
    # D v at the sampled potential rows
    ref = np.zeros(nodes.size)
    ref[P.free_nodes] = P.D @ vs3[P.mag_nodes].reshape(-1)
    _close(mag.divergence(v3)[samples], ref[rows])
    # D^T phi at the sampled magnetic rows
    ref3 = np.zeros((nodes.size, 3))
    ref3[P.mag_nodes] = (P.D.T @ vs1[P.free_nodes]).reshape(-1, 3)
    _close(mag.divergence_t(v1)[samples], ref3[rows])
    # (C_A + C_K) v
    ref3 = np.zeros((nodes.size, 3))
    ref3[P.mag_nodes] = precond.apply_C_local(P, vs3[P.mag_nodes])
    _close(mag.local_apply(v3)[samples], ref3[rows])
    # K_phi v (the stored operator is the assembled one without its rounding residues)
    ref = P.Kfull @ vs1
    _close(mag.potential_matvec(v1)[samples], ref[rows])


def test_uniform_state_energies(big):
    from paper_1801_03690_gb300 import Params
    wl, mag = big
    mesh = wl.mesh
    u = np.array([0.3, -0.4, np.sqrt(1 - 0.25)])
    b = np.array([0.0, 0.2, -1.0])
    mag.set_field(b)
    F, terms = mag.energy(np.tile(u, (mesh.n_nodes, 1)), Params(precision=1, amg=1, inner_tol=1e-3,
                                                                 poisson_tol=1e-10))
    x = mesh.xyz[mesh.tets]
    V = np.abs(np.einsum("ti,ti->t", np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]), x[:, 3] - x[:, 0])) / 6
    mat = wl.materials[mesh.region]
    k = mat[:, 3:6] / np.linalg.norm(mat[:, 3:6], axis=1, keepdims=True)
    an_ref = -np.sum(mat[:, 2] * V * (k @ u) ** 2)
    ze_ref = -np.sum(mat[:, 0] * V) * (b @ u)
    ex, an, dm, ze = terms
    assert abs(ex) < 1e-9 * abs(an)                      # uniform m: no exchange energy
    assert an == pytest.approx(an_ref, rel=1e-10)
    assert ze == pytest.approx(ze_ref, rel=1e-10)
    Vm = np.sum(V[mat[:, 0] > 0])
    assert 0.0 < dm < 0.5 * MU0 * wl.materials[:, 0].max() ** 2 * Vm
    assert F == pytest.approx(ex + an + dm + ze, rel=1e-12)


def test_headline_form_first_field_step_matches_plain_fp64(big):
    """The bench's headline form (multigrid precision form with the
    potential tolerance tied to t1) and plain FP64 on field index 1 from m0:
    the same minimum, |m| = 1, t3 at the returned state, iteration counts
    within two, and the identity evals = 2 nli + 1 + ls_extra."""
    from paper_1801_03690_gb300 import Params
    wl, mag = big
    out = []
    for prm in (Params(precision=1, amg=1, inner_tol=1e-3, poisson_sched=1), Params(precision=0)):
        mag.set_magnetization(wl.m0)
        mag.set_field(wl.fields[1])
        st = mag.minimize(prm)
        assert st["status"] == "ok"
        assert st["evals"] == 2 * st["nli"] + 1 + st["ls_extra"]
        out.append((st, mag.get_magnetization()))
    (sh, mh), (s64, m64) = out
    assert sh["F"] == pytest.approx(s64["F"], rel=1e-8)
    assert np.abs(mh - m64).max() < 1e-5
    assert abs(sh["nli"] - s64["nli"]) <= 2
    mag_nodes = np.linalg.norm(mh, axis=1) > 0
    np.testing.assert_allclose(np.linalg.norm(mh[mag_nodes], axis=1), 1.0, atol=1e-13)
    g = mag.gradient(None, projected=True, params=Params(precision=0))
    assert np.abs(g).max() < 1e-10 ** (1 / 3) * (1 + abs(s64["F_internal"]))
