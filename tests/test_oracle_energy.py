"""Pins of the oracle's energy, gradient, projection and magnetostatics
(Sec. 2.2, Eqs. energy, proj, nablaLF, opt2)."""
import numpy as np
import pytest

import synth
from oracle import fem, energy


def _problem(**kw):
    t = np.radians(20.0)
    args = dict(n_mag=3, h=1.5e-9, Ms=1.0e6, A=1.0e-11, K1=2.0e6,
                axis=(np.sin(t), 0.0, np.cos(t)), jitter=0.07, seed=4)
    args.update(kw)
    wl = synth.small_cube(**args)
    return wl, fem.assemble_workload(wl)


def _F_raw(P, m, h):
    """F for arbitrary (not unit) vectors m, exact potential."""
    phi, _ = energy.solve_potential(P, m)
    return energy.energy_terms(P, m, phi, h)["total"]


def test_gradient_equals_central_differences():
    """F is a quadratic form in m, so central differences are exact up to
    round-off for any step."""
    wl, P = _problem()
    rng = np.random.default_rng(1)
    m = rng.normal(size=(P.n_mag, 3))
    h = P.units.field_int([0.2, -0.1, 0.4])
    phi, _ = energy.solve_potential(P, m)
    grad = energy.gradient(P, m, phi, h)
    step = 0.5
    for _ in range(12):
        i, c = rng.integers(P.n_mag), rng.integers(3)
        mp, mm = m.copy(), m.copy()
        mp[i, c] += step
        mm[i, c] -= step
        fd = (_F_raw(P, mp, h) - _F_raw(P, mm, h)) / (2 * step)
        assert fd == pytest.approx(grad[i, c], rel=1e-8, abs=1e-9 * np.abs(grad).max())


def test_normalised_objective_derivative():
    """d/da F(N(x + a d)) equals Eq. (opt2) contracted with d."""
    wl, P = _problem()
    rng = np.random.default_rng(2)
    x = energy.normalize(rng.normal(size=(P.n_mag, 3)))
    d = energy.project(x, rng.normal(size=(P.n_mag, 3)))
    h = P.units.field_int([0.0, 0.0, 0.3])
    a, da = 0.05, 1e-5
    e = energy.evaluate(P, energy.normalize(x + a * d), h)
    an = energy.ftilde_derivative(e["g"], x + a * d, d)

    def phi(al):
        return energy.evaluate(P, energy.normalize(x + al * d), h)["F"]
    fd = (phi(a + da) - phi(a - da)) / (2 * da)
    assert an == pytest.approx(fd, rel=1e-6)


def test_projection_properties():
    rng = np.random.default_rng(3)
    m = energy.normalize(rng.normal(size=(50, 3)))
    v = rng.normal(size=(50, 3))
    p = energy.project(m, v)
    np.testing.assert_allclose(np.sum(p * m, axis=1), 0.0, atol=1e-14)
    np.testing.assert_allclose(energy.project(m, p), p, atol=1e-14)
    np.testing.assert_allclose(energy.normalize(3.0 * m), m, atol=1e-15)


def test_kkt_multiplier_and_projected_gradient():
    """g = grad F - lambda m with lambda = m . grad F (Eqs. nablaLF1, nablaLF)."""
    wl, P = _problem()
    m = energy.normalize(wl.m0[P.mag_nodes])
    e = energy.evaluate(P, m, P.units.field_int([0.1, 0.2, 0.3]))
    lam = np.sum(m * e["grad"], axis=1)
    np.testing.assert_allclose(e["g"], e["grad"] - lam[:, None] * m, atol=1e-12)


def test_demag_energy_positive_and_solvers_agree():
    wl, P = _problem(jitter=0.05)
    m = energy.normalize(wl.m0[P.mag_nodes])
    ed = energy.evaluate(P, m, np.zeros(3), poisson="direct")
    ec = energy.evaluate(P, m, np.zeros(3), poisson="cg", tol=1e-13)
    assert ed["terms"]["demag"] > 0
    assert ec["terms"]["demag"] == pytest.approx(ed["terms"]["demag"], rel=1e-12)
    np.testing.assert_allclose(ec["phi"], ed["phi"], rtol=0, atol=1e-10 * np.abs(ed["phi"]).max())
    # at the exact potential the variational form equals 1/2 phi^T D m
    b = energy.poisson_rhs(P, m)
    assert ed["terms"]["demag"] == pytest.approx(0.5 * ed["phi"] @ b, rel=1e-12)


def test_demag_factor_of_cube_tends_to_one_third():
    """A uniformly magnetised cube has demagnetising factor 1/3 along every
    axis.  On the Kuhn lattice the three axes agree exactly (the lattice is
    invariant under axis permutations); the grounded air box truncates the
    stray field by O(L^-3), removed by Richardson extrapolation in L."""
    n = 4
    res = {}
    for bf in (3.0, 6.0):
        wl = synth.small_cube(n_mag=n, h=1e-9, box_factor=bf, m0=(0, 0, 1))
        P = fem.assemble_workload(wl)
        Ns = []
        for ax in np.eye(3):
            m = np.tile(ax, (P.n_mag, 1))
            phi, _ = energy.solve_potential(P, m)
            Ns.append(energy.energy_terms(P, m, phi, np.zeros(3))["demag"] / (0.5 * n ** 3))
        assert Ns[0] == pytest.approx(Ns[1], rel=1e-10)
        assert Ns[0] == pytest.approx(Ns[2], rel=1e-10)
        res[bf] = Ns[0]
    assert res[3.0] < res[6.0] < 1.0 / 3.0
    Linf = res[6.0] + (res[6.0] - res[3.0]) / (2.0 ** 3 - 1.0)
    assert Linf == pytest.approx(1.0 / 3.0, rel=0.15)
    assert Linf > res[6.0]


def test_sphere_interior_field_is_uniform_one_third():
    """A uniformly magnetised sphere has a uniform interior field H = -M/3,
    i.e. the potential of K_phi phi = D m is phi = z/3 (reduced units,
    lengths in nm) inside it.  On a staircase sphere of radius 6 h the
    potential at the nodes within half the radius is fitted by a linear
    function: it is linear to 0.1% of its range, its gradient points along
    m (the x and y slopes vanish to 1e-3), and the slope along m, after
    Richardson extrapolation of the grounded box's O(L^-3) truncation, is
    1/3 within 1% (the staircase surface leaves 0.4%)."""
    slopes = {}
    for bf in (3.0, 6.0):
        wl = synth.sphere_in_box(n_rad=6, h=1e-9, box_factor=bf, ratio=1.15)
        P = fem.assemble_workload(wl)
        phi, _ = energy.solve_potential(P, np.tile([0.0, 0.0, 1.0], (P.n_mag, 1)))
        xyz = wl.mesh.xyz[P.free_nodes] * 1e9
        sel = np.linalg.norm(xyz, axis=1) < 3.0
        A = np.c_[xyz[sel], np.ones(sel.sum())]
        coef, *_ = np.linalg.lstsq(A, phi[sel], rcond=None)
        rms = np.sqrt(np.mean((A @ coef - phi[sel]) ** 2))
        assert sel.sum() > 50
        assert rms < 1e-3 * (2.0 * 3.0 * coef[2])              # 0.1% of the range of phi there
        assert abs(coef[0]) < 1e-3 and abs(coef[1]) < 1e-3
        slopes[bf] = coef[2]
    assert slopes[3.0] < slopes[6.0] < 1.0 / 3.0
    s_inf = slopes[6.0] + (slopes[6.0] - slopes[3.0]) / (2.0 ** 3 - 1.0)
    assert s_inf == pytest.approx(1.0 / 3.0, rel=0.01)


def test_variational_demag_energy_error_is_quadratic():
    """The magnetostatic energy is evaluated in the variational form
    phi.b - 1/2 phi.K phi, whose value at phi* + e v (phi* the exact
    potential) is the exact energy 1/2 phi*.b minus 1/2 e^2 v.K v: no term
    linear in the potential error, so an inexact potential solve costs only
    its square."""
    wl, P = _problem()
    m = energy.normalize(wl.m0[P.mag_nodes])
    phi, _ = energy.solve_potential(P, m)
    exact = 0.5 * float(phi @ energy.poisson_rhs(P, m))
    e0 = energy.energy_terms(P, m, phi, np.zeros(3))["demag"]
    assert e0 == pytest.approx(exact, rel=1e-12)
    v = np.random.default_rng(8).normal(size=P.n_phi)
    vKv = float(v @ (P.Kphi @ v))
    for eps in (1e-2, 1e-3):
        e = energy.energy_terms(P, m, phi + eps * v * np.abs(phi).max(), np.zeros(3))["demag"]
        want = exact - 0.5 * (eps * np.abs(phi).max()) ** 2 * vKv
        assert e == pytest.approx(want, rel=1e-9, abs=1e-12 * abs(exact))
