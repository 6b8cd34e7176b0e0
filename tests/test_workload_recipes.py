"""The seeded workloads behind the bench line and the parity cases have the
sizes and structure the documentation states (no GPU): a change to a
generator that would silently change the benchmarked problem fails here.
Potential unknowns are the lattice nodes off the grounded outer surface,
(n - 2)^3 for an n^3-node box lattice."""
import numpy as np

import synth


def _box_nodes_per_axis(mesh):
    n = int(round(mesh.n_nodes ** (1.0 / 3.0)))
    assert n ** 3 == mesh.n_nodes
    return n


def _magnet(wl):
    magnetic = wl.materials[wl.mesh.region, 0] > 0
    return magnetic, np.unique(wl.mesh.tets[magnetic])


def test_large_polycrystal_recipe():
    wl = synth.large_polycrystal()
    n = _box_nodes_per_axis(wl.mesh)
    assert (wl.mesh.n_nodes, wl.mesh.n_tets, n) == (8_998_912, 53_218_458, 208)
    assert (n - 2) ** 3 == 8_741_816                                  # potential unknowns
    magnetic, nodes = _magnet(wl)
    assert nodes.size == 150 ** 3 and magnetic.sum() == 6 * 149 ** 3
    ms = wl.materials[wl.mesh.region[magnetic], 0]
    gb = ms < ms.max()
    assert np.isclose(ms[gb], 0.4 * ms.max()).all()                   # grain boundary at 40% Ms
    assert 0.08 < gb.mean() < 0.11
    bulk_regions = np.unique(wl.mesh.region[magnetic][~gb])
    assert bulk_regions.size == 125                                   # one region per grain
    ax = wl.materials[bulk_regions, 3:6]
    ax = ax / np.linalg.norm(ax, axis=1, keepdims=True)
    assert (ax[:, 2] >= np.cos(np.radians(15.0)) - 1e-12).all()       # 15 degree cone about +z
    assert np.allclose(wl.m0, [0.0, 0.0, 1.0])
    assert len(wl.fields) == 60 and np.allclose(wl.fields[-1], [0.0, 0.0, -8.0])


def test_hard_and_soft_cube_recipes():
    hc = synth.hard_cube()
    n = _box_nodes_per_axis(hc.mesh)
    assert (hc.mesh.n_nodes, hc.mesh.n_tets, (n - 2) ** 3) == (912_673, 5_308_416, 857_375)
    _, nodes = _magnet(hc)
    assert nodes.size == 117_649 and len(hc.fields) == 40
    sc = synth.soft_cube()
    n = _box_nodes_per_axis(sc.mesh)
    assert (sc.mesh.n_nodes, (n - 2) ** 3) == (35_937, 29_791)
    _, nodes = _magnet(sc)
    assert nodes.size == 4_913 and len(sc.fields) == 21
    assert np.allclose(np.linalg.norm(sc.m0, axis=1), 1.0)
