"""Pins of the oracle's P1 assembly (Sec. 2.2, Eq. energy) against closed
forms, invariants and brute force."""
import numpy as np
import pytest

import synth
from oracle import fem, energy

MU0 = fem.MU0


def _tet_brute(xyz4):
    """Barycentric gradients by central differences of the barycentric
    coordinates (each from a 4x4 linear solve), volume by the triple product."""
    A = np.vstack([xyz4.T, np.ones(4)])
    c = xyz4.mean(axis=0)

    def lam(p):
        return np.linalg.solve(A, np.append(p, 1.0))

    grads = np.zeros((4, 3))
    for ax in range(3):
        e = np.zeros(3)
        e[ax] = 1e-3
        grads[:, ax] = (lam(c + e) - lam(c - e)) / 2e-3
    a, b, cc, d = xyz4
    vol = abs(np.dot(a - d, np.cross(b - d, cc - d))) / 6.0
    return vol, grads


def test_tet_geometry_matches_brute_force():
    rng = np.random.default_rng(0)
    xyz = rng.normal(size=(40, 3))
    tets = np.array([rng.choice(40, 4, replace=False) for _ in range(25)])
    V, b = fem.tet_geometry(xyz, tets)
    for t in range(len(tets)):
        vb, gb = _tet_brute(xyz[tets[t]])
        assert V[t] == pytest.approx(vb, rel=1e-12)
        np.testing.assert_allclose(b[t], gb, rtol=1e-8, atol=1e-8 * np.abs(gb).max())


def test_gradients_reproduce_affine_functions():
    wl = synth.small_cube(n_mag=3, h=1e-9, jitter=0.07, seed=5)
    xyz = wl.mesh.xyz / 1e-9
    V, b = fem.tet_geometry(xyz, wl.mesh.tets)
    np.testing.assert_allclose(b.sum(axis=1), 0.0, atol=1e-12)
    a = np.array([0.3, -1.7, 2.2])
    f = xyz @ a + 0.5
    grad = np.einsum("ti,tic->tc", f[wl.mesh.tets], b)
    np.testing.assert_allclose(grad, np.broadcast_to(a, grad.shape), rtol=1e-10, atol=1e-10)
    # Kuhn tets of an unjittered voxel all have volume h^3/6
    wl0 = synth.small_cube(n_mag=3, h=1e-9)
    V0, _ = fem.tet_geometry(wl0.mesh.xyz / 1e-9, wl0.mesh.tets)
    np.testing.assert_allclose(V0, 1.0 / 6.0, rtol=1e-12)


def test_exchange_zero_for_uniform_m():
    wl = synth.small_cube(n_mag=4, h=1.5e-9, jitter=0.07, seed=7)
    P = fem.assemble_workload(wl)
    np.testing.assert_allclose(P.KA @ np.ones(P.n_mag), 0.0, atol=1e-10 * abs(P.KA).max())
    m = energy.normalize(np.tile([0.3, -0.2, 0.9], (P.n_mag, 1)))
    ex = energy.energy_terms(P, m, np.zeros(P.n_phi), np.zeros(3))["exchange"]
    assert abs(ex) < 1e-10 * abs(P.KA).sum()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_exchange_helix_exact_on_kuhn_lattice(axis):
    """m = (cos kx, sin kx, 0): every Kuhn tet spans exactly one lattice step
    along x, so the P1 exchange energy is A V (2 - 2 cos kh) / h^2 exactly."""
    n, h_m, A = 5, 1.0e-9, 1.3e-11
    wl = synth.small_cube(n_mag=n, h=h_m, A=A)
    P = fem.assemble_workload(wl)
    xyz = wl.mesh.xyz[P.mag_nodes] / 1e-9
    k = 0.7
    s = xyz[:, axis]
    m = np.zeros((P.n_mag, 3))
    o = [(axis + 1) % 3, (axis + 2) % 3]
    m[:, o[0]] = np.cos(k * s)
    m[:, o[1]] = np.sin(k * s)
    ex = energy.energy_terms(P, m, np.zeros(P.n_phi), np.zeros(3))["exchange"]
    A_int = A / (MU0 * P.units.Mref ** 2 * 1e-18)
    vol = (n * 1.0) ** 3
    h = 1.0
    assert ex == pytest.approx(A_int * vol * (2 - 2 * np.cos(k * h)) / h ** 2, rel=1e-12)


def test_anisotropy_and_zeeman_uniform():
    K, Ms = 4.3e6, 1.28e6
    ax = np.array([0.2, 0.1, 1.0]) / np.linalg.norm([0.2, 0.1, 1.0])
    wl = synth.small_cube(n_mag=3, h=1e-9, Ms=Ms, K1=K, axis=ax, jitter=0.05, seed=2)
    P = fem.assemble_workload(wl)
    u = np.array([0.6, -0.64, 0.48])
    m = np.tile(u, (P.n_mag, 1))
    b = np.array([0.1, -0.3, 0.5])
    t = energy.energy_terms(P, m, np.zeros(P.n_phi), P.units.field_int(b))
    V = 27.0
    K_int = K / (MU0 * P.units.Mref ** 2)
    assert t["anisotropy"] == pytest.approx(-K_int * V * (u @ ax) ** 2, rel=1e-12)
    # Zeeman in joules: -Ms V (mu0 H . m)
    assert t["zeeman"] * P.units.energy_J == pytest.approx(-Ms * V * 1e-27 * (b @ u), rel=1e-12)
    assert P.w.sum() == pytest.approx(V, rel=1e-12)


def test_potential_stiffness_annihilates_affine_at_interior_nodes():
    wl = synth.small_cube(n_mag=3, h=1e-9, jitter=0.07, seed=11)
    P = fem.assemble_workload(wl)
    xyz = wl.mesh.xyz / 1e-9
    f = xyz @ np.array([1.0, -2.0, 0.5]) + 3.0
    r = P.Kfull @ f
    interior = np.setdiff1d(np.arange(P.n_nodes), P.dirichlet_nodes)
    np.testing.assert_allclose(r[interior], 0.0, atol=1e-10 * np.abs(f).max())
    # symmetric positive definite after Dirichlet removal
    assert abs(P.Kphi - P.Kphi.T).max() < 1e-14 * abs(P.Kphi).max()
    lo = np.linalg.eigvalsh(P.Kphi.toarray()).min()
    assert lo > 0


def test_outer_surface_nodes_of_box():
    wl = synth.small_cube(n_mag=2, h=1e-9, box_factor=3.0)
    P = fem.assemble_workload(wl)
    n = wl.mesh.shape[0]
    assert P.dirichlet_nodes.size == n ** 3 - (n - 2) ** 3
    assert P.n_phi == (n - 2) ** 3


def test_divergence_of_uniform_m_is_surface_charge():
    """(D m)_j = int Ms m . grad N_j = surface integral of Ms (m.n) N_j: zero
    off the magnet surface, summing to +-Ms*area over the two faces normal
    to m."""
    n, h = 4, 1e-9
    wl = synth.small_cube(n_mag=n, h=h, box_factor=2.0)
    P = fem.assemble_workload(wl)
    m = np.tile([0.0, 0.0, 1.0], (P.n_mag, 1))
    q = energy.poisson_rhs(P, m)
    z = wl.mesh.xyz[P.free_nodes, 2] / 1e-9
    top, bot = z == n / 2.0, z == -n / 2.0
    area = float(n * n)
    assert q[top].sum() == pytest.approx(area, rel=1e-12)
    assert q[bot].sum() == pytest.approx(-area, rel=1e-12)
    assert np.abs(q[~(top | bot)]).max() < 1e-12
    assert abs(q.sum()) < 1e-12
