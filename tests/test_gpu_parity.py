"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Tolerances: operator applications (K_phi v, H v) 1e-12 relative; the
energy 1e-10 relative and the gradient 1e-9 relative to its max norm against
the exact (direct-solve) potential, with the GPU potential solved to a
relative residual of 1e-13; minimisations: energy 1e-8 relative, max nodal
|dm| 1e-5, coercive field 0.5%.
"""
import numpy as np
import pytest

import synth
from oracle import fem, energy, ncg, precond, curve

pytestmark = pytest.mark.gpu

TIGHT = dict(poisson_tol=1e-13)


@pytest.fixture(scope="module")
def lib():
    from paper_1801_03690_gb300 import Magnet, Params
    return Magnet, Params


def _setup(lib, wl):
    Magnet, Params = lib
    mag = Magnet(device=0)
    mag.upload_workload(wl)
    P = fem.assemble_workload(wl)
    return mag, P


def _hard(n_mag=6, jitter=0.07, seed=4, box=2.0):
    t = np.radians(25.0)
    return synth.small_cube(n_mag=n_mag, h=1.5e-9, box_factor=box, Ms=1.28e6, A=7.7e-12,
                            K1=4.3e6, axis=(np.sin(t), 0.2, np.cos(t)), jitter=jitter, seed=seed)


PATH_COUNTERS = ("nli", "evals", "li", "ls_extra", "li2", "li2_first", "restarts", "steepest")


def _same_path(st, r):
    """Parity along the same path: every counter of Algorithm 4's branches
    (iterations, evaluations, inner steps, backtracking evaluations, li2
    exits, safeguard restarts and steepest-descent fallbacks) equals the
    oracle's."""
    for k in PATH_COUNTERS:
        assert st[k] == r.stats[k], (k, st[k], r.stats[k])


def test_sizes_match_oracle(lib):
    wl = _hard()
    mag, P = _setup(lib, wl)
    s = mag.sizes()
    assert s["n_mag"] == P.n_mag
    assert s["n_phi"] == P.n_phi
    assert s["nnz_mag"] == P.KA.nnz
    assert s["nnz_phi"] == P.Kphi.nnz


@pytest.mark.parametrize("n_mag,box", [(6, 2.0), (5, 3.0)])
def test_potential_matvec(lib, n_mag, box):
    wl = _hard(n_mag=n_mag, box=box)
    mag, P = _setup(lib, wl)
    rng = np.random.default_rng(0)
    v = rng.normal(size=wl.mesh.n_nodes)
    out = mag.potential_matvec(v)
    ref = np.zeros(wl.mesh.n_nodes)
    ref[P.free_nodes] = P.Kphi @ v[P.free_nodes]
    scale = np.abs(ref).max()
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * scale)
    assert np.all(out[P.dirichlet_nodes] == 0.0)


def test_energy_terms_and_gradient(lib):
    Magnet, Params = lib
    wl = _hard()
    mag, P = _setup(lib, wl)
    b = np.array([0.3, -0.2, -1.5])
    mag.set_field(b)
    m = wl.m0
    F, terms = mag.energy(m, Params(**TIGHT))
    mo = energy.normalize(m[P.mag_nodes])
    h = P.units.field_int(b)
    e = energy.evaluate(P, mo, h)
    EJ = P.units.energy_J
    for k, name in enumerate(["exchange", "anisotropy", "demag", "zeeman"]):
        assert terms[k] == pytest.approx(e["terms"][name] * EJ, rel=1e-10), name
    assert F == pytest.approx(e["F"] * EJ, rel=1e-10)
    g = mag.gradient(None, projected=False, params=Params(**TIGHT))
    gp = mag.gradient(None, projected=True, params=Params(**TIGHT))
    sc = np.abs(e["grad"]).max()
    np.testing.assert_allclose(g[P.mag_nodes], e["grad"], rtol=0, atol=1e-9 * sc)
    np.testing.assert_allclose(gp[P.mag_nodes], e["g"], rtol=0, atol=1e-9 * sc)
    nonmag = np.setdiff1d(np.arange(wl.mesh.n_nodes), P.mag_nodes)
    assert np.all(g[nonmag] == 0.0)
    phi = mag.potential()
    ref = np.zeros(wl.mesh.n_nodes)
    ref[P.free_nodes] = e["phi"]
    np.testing.assert_allclose(phi, ref, rtol=0, atol=1e-9 * np.abs(ref).max())


def test_potential_solve_matches_same_algorithm(lib):
    """With equal tolerance and zero start the GPU potential solve and the
    oracle's Algorithm 1 take the same steps."""
    Magnet, Params = lib
    wl = _hard(n_mag=5)
    mag, P = _setup(lib, wl)
    mo = energy.normalize(wl.m0[P.mag_nodes])
    mag.set_magnetization(wl.m0)
    F, terms = mag.energy(None, Params(poisson_tol=1e-8))
    phi_or, steps = energy.solve_potential(P, mo, method="cg", tol=1e-8)
    phi = mag.potential()[P.free_nodes]
    np.testing.assert_allclose(phi, phi_or, rtol=0, atol=1e-11 * np.abs(phi_or).max())


def test_hessian_apply(lib):
    Magnet, Params = lib
    for keep in (False, True):
        wl = _hard()
        mag, P = _setup(lib, wl)
        mag.set_field([0.1, 0.0, 0.7])
        grad = mag.gradient(wl.m0, projected=False, params=Params(**TIGHT))[P.mag_nodes]
        rng = np.random.default_rng(1)
        v = rng.normal(size=(wl.mesh.n_nodes, 3))
        out = mag.hessian_apply(v, Params(keep_last_term=keep))[P.mag_nodes]
        mo = energy.normalize(wl.m0[P.mag_nodes])
        ref = precond.apply_H(P, mo, grad, v[P.mag_nodes], keep_last=keep)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("jmax", [0, 1, 4, 12])
def test_precond_solve(lib, jmax):
    Magnet, Params = lib
    wl = _hard()
    mag, P = _setup(lib, wl)
    mag.set_field([0.0, 0.0, 2.0])
    grad = mag.gradient(wl.m0, projected=False, params=Params(**TIGHT))[P.mag_nodes]
    mo = energy.normalize(wl.m0[P.mag_nodes])
    g = energy.project(mo, grad)
    y, steps = mag.precond_solve(Params(jmax=jmax))
    y_or, steps_or = precond.precond_solve(P, mo, grad, g, jmax)
    assert steps == steps_or
    np.testing.assert_allclose(y[P.mag_nodes], y_or, rtol=0, atol=1e-10 * np.abs(y_or).max())


@pytest.mark.parametrize("jmax", [1, 4, 12])
def test_precond_solve_fp32(lib, jmax):
    """The precision form's preconditioner apply (H products and the inner
    CG's vectors in FP32; sums, step lengths and the solution in FP64)
    against the oracle's FP64 Algorithm 1 on H: the same number of steps
    (one more or less where an li3 test sits at the FP32 rounding level) and
    y within 1e-3 of its largest entry."""
    Magnet, Params = lib
    wl = _hard()
    mag, P = _setup(lib, wl)
    mag.set_field([0.0, 0.0, 2.0])
    grad = mag.gradient(wl.m0, projected=False, params=Params(**TIGHT))[P.mag_nodes]
    mo = energy.normalize(wl.m0[P.mag_nodes])
    g = energy.project(mo, grad)
    y, steps = mag.precond_solve(Params(jmax=jmax, precision=1))
    y_or, steps_or = precond.precond_solve(P, mo, grad, g, jmax)
    dev = np.abs(y[P.mag_nodes] - y_or).max() / np.abs(y_or).max()
    print(f"FP32 preconditioner, j_max {jmax}: steps {steps} (oracle {steps_or}), deviation {dev:.2e}")
    assert abs(steps - steps_or) <= 1
    assert dev < 1e-3


@pytest.mark.parametrize("jmax", [0, 4])
def test_minimize_parity_soft(lib, jmax):
    Magnet, Params = lib
    wl = synth.small_cube(n_mag=4, h=2e-9, jitter=0.05, seed=3)
    mag, P = _setup(lib, wl)
    b = np.array([0.02, 0.0, 0.05])
    mag.set_magnetization(wl.m0)
    mag.set_field(b)
    st = mag.minimize(Params(jmax=jmax, **TIGHT))
    m = mag.get_magnetization()[P.mag_nodes]
    r = ncg.minimize(P, energy.normalize(wl.m0[P.mag_nodes]), P.units.field_int(b),
                     ncg.Params(jmax=jmax))
    assert st["status"] == "ok" and r.status == "converged"
    assert st["F"] == pytest.approx(r.F * P.units.energy_J, rel=1e-8)
    assert np.abs(m - r.m).max() < 1e-5
    _same_path(st, r)
    np.testing.assert_allclose(np.linalg.norm(m, axis=1), 1.0, atol=1e-14)
    assert st["evals"] == 2 * st["nli"] + 1 + st["ls_extra"]
    assert st["li"] <= jmax * (st["nli"] + 1)


def test_coercive_field_parity(lib):
    """A small hard-magnetic cube swept through switching: the GPU curve's
    coercive field agrees with the oracle's within 0.5%."""
    Magnet, Params = lib
    t = np.radians(1.0)
    wl = synth.small_cube(n_mag=3, h=1e-9, box_factor=2.0, Ms=1.28e6, A=7.7e-12, K1=4.3e6,
                          axis=(np.sin(t), 0.0, np.cos(t)), m0=(0, 0, 1))
    mag, P = _setup(lib, wl)
    bz = -np.linspace(5.0, 7.0, 21)
    fields = np.stack([np.zeros_like(bz), np.zeros_like(bz), bz], axis=1)
    mag.set_magnetization(wl.m0)
    sts = mag.demag_curve(fields, Params(jmax=4, **TIGHT))
    M = np.array([s["M"] for s in sts])
    from paper_1801_03690_gb300 import coercive_field
    hc_gpu = coercive_field(fields, M)                # the library's H_c (mm_coercive_field)
    res = curve.demag_curve(P, fields, wl.m0, ncg.Params(jmax=4))
    assert hc_gpu is not None and res["Hc_T"] is not None
    assert abs(hc_gpu - res["Hc_T"]) <= 0.005 * res["Hc_T"]
    np.testing.assert_allclose(M, res["M"], atol=1e-5)


def test_magnet_touching_outer_boundary(lib):
    """No air box: magnetic nodes on the outer surface carry phi = 0."""
    Magnet, Params = lib
    wl = synth.small_cube(n_mag=4, h=2e-9, box_factor=1.0, jitter=0.0, seed=2)
    mag, P = _setup(lib, wl)
    b = np.array([0.0, 0.1, 0.0])
    mag.set_field(b)
    F, terms = mag.energy(wl.m0, Params(**TIGHT))
    e = energy.evaluate(P, energy.normalize(wl.m0[P.mag_nodes]), P.units.field_int(b))
    assert F == pytest.approx(e["F"] * P.units.energy_J, rel=1e-10)


def test_invalid_inputs(lib):
    Magnet, Params = lib
    from paper_1801_03690_gb300 import MMError
    wl = synth.small_cube(n_mag=2, h=1e-9)
    mag = Magnet(device=0)
    bad = wl.mesh.tets.copy()
    bad[0, 0] = wl.mesh.n_nodes + 5
    with pytest.raises(MMError) as ei:
        mag.upload_mesh(wl.mesh.xyz, bad, wl.mesh.region, wl.materials)
    assert ei.value.status == -2
    flat = wl.mesh.xyz.copy()
    t0 = wl.mesh.tets[0]
    flat[t0[3]] = flat[t0[0]] + 0.5 * (flat[t0[1]] - flat[t0[0]])  # collapse a tet
    with pytest.raises(MMError):
        mag.upload_mesh(flat, wl.mesh.tets, wl.mesh.region, wl.materials)
    mag.upload_workload(wl)
    m = wl.m0.copy()
    P = fem.assemble_workload(wl)
    m[P.mag_nodes[0]] = np.nan
    with pytest.raises(MMError):
        mag.set_magnetization(m)
    with pytest.raises(MMError):
        mag.minimize(Params(tau_F=-1.0))
    air = wl.materials.copy()
    air[:, 0] = 0.0
    with pytest.raises(MMError):
        mag.upload_mesh(wl.mesh.xyz, wl.mesh.tets, wl.mesh.region, air)


@pytest.mark.parametrize("prec,amg", [(0, 0), (1, 0), (1, 1)])
def test_soft_cube_first_field_step(lib, prec, amg):
    """Config 1 at full size (40 nm permalloy cube, 16^3 voxels, 29,791
    potential unknowns) from its seeded random start at +100 mT: the GPU
    minimisation (plain FP64, precision form with Jacobi and with the
    multigrid preconditioner) against the oracle's."""
    Magnet, Params = lib
    wl = synth.soft_cube()
    mag, P = _setup(lib, wl)
    b = wl.fields[0]
    mag.set_magnetization(wl.m0)
    mag.set_field(b)
    if amg:
        assert mag.amg_levels()
    st = mag.minimize(Params(jmax=4, poisson_tol=1e-12, precision=prec, amg=amg,
                             inner_tol=1e-3 if amg else 0.1))
    m = mag.get_magnetization()[P.mag_nodes]
    r = ncg.minimize(P, energy.normalize(wl.m0[P.mag_nodes]), P.units.field_int(b), ncg.Params(jmax=4))
    assert st["status"] == "ok" and r.status == "converged"
    assert st["F"] == pytest.approx(r.F * P.units.energy_J, rel=1e-8)
    assert np.abs(m - r.m).max() < 1e-5
    if prec == 0:
        _same_path(st, r)


@pytest.mark.parametrize("psi_deg", [20.0, 45.0, 70.0])
def test_stoner_wohlfarth_astroid_on_gpu(lib, psi_deg):
    """The GPU minimiser on a single-domain particle (2 nm edge, far below
    the exchange length; a cube has no shape anisotropy, so the stray field
    of the uniform state does not move the switching field): the metastable
    state from m = +z survives at 0.98 and is gone at 1.02 of the astroid
    field 2K/(mu0 Ms) (cos^2/3 psi + sin^2/3 psi)^-3/2."""
    Magnet, Params = lib[0], lib[1]
    wl = synth.small_cube(n_mag=2, h=1e-9, Ms=1.28e6, A=7.7e-12, K1=4.3e6, axis=(0.0, 0.0, 1.0),
                          m0=(0, 0, 1), box_factor=3.0)
    psi = np.radians(psi_deg)
    hsw = 2 * 4.3e6 / 1.28e6 * (np.cos(psi) ** (2 / 3) + np.sin(psi) ** (2 / 3)) ** -1.5
    u = np.array([np.sin(psi), 0.0, -np.cos(psi)])
    mag = Magnet(device=0)
    mag.upload_workload(wl)
    for f, switched in ((0.98, False), (1.02, True)):
        mag.set_magnetization(wl.m0)
        mag.set_field(f * hsw * u)
        st = mag.minimize(Params(jmax=4))
        assert st["status"] == "ok"
        m = mag.get_magnetization()
        mz = m[np.linalg.norm(m, axis=1) > 0, 2]
        assert (mz.mean() < 0) == switched
    mag.close()


def _anti(n_mag, b, seed=0):
    """A hard cube magnetised against a strong field (m ~ -z, field +z): the
    approximate Hessian is indefinite there, so the preconditioner solve
    exits by negative curvature (li2), on its first step too (y = g), and
    the descent safeguard restarts the direction and falls back to -g."""
    wl = _hard(n_mag=n_mag)
    rng = np.random.default_rng(seed)
    m0 = -np.tile([0.0, 0.0, 1.0], (wl.mesh.n_nodes, 1)) + 0.05 * rng.standard_normal((wl.mesh.n_nodes, 3))
    return wl, m0, np.asarray(b, dtype=np.float64)


@pytest.mark.parametrize("case", ["negative_curvature_and_safeguard", "backtracking"])
def test_rare_branches_fire_and_match_oracle(lib, case):
    """The rare branches of Algorithm 4 fire on the GPU and the path equals
    the oracle's: 16 iterations of the anti-parallel cube (li2 on the first
    and later inner steps, a safeguard restart and a steepest-descent
    fallback), and 12 iterations with the sufficient-decrease constant
    c1 = 0.99, under which the cubic step fails the test and the line search
    backtracks."""
    Magnet, Params = lib
    if case == "backtracking":
        wl = _hard(n_mag=4)
        m0, b, it, extra = wl.m0, np.array([0.1, 0.0, 0.5]), 12, dict(c1=0.99)
    else:
        wl, m0, b = _anti(3, [0.0, 0.0, 6.0])
        it, extra = 16, {}
    mag, P = _setup(lib, wl)
    mag.set_magnetization(m0)
    mag.set_field(b)
    st = mag.minimize(Params(jmax=4, max_iter=it, **TIGHT, **extra))
    r = ncg.minimize(P, energy.normalize(m0[P.mag_nodes]), P.units.field_int(b),
                     ncg.Params(jmax=4, max_iter=it, **extra))
    assert st["status"] == "not_converged" and r.status == "max_iter"
    _same_path(st, r)
    if case == "backtracking":
        assert st["ls_extra"] > 0
    else:
        assert st["li2"] > 0 and st["li2_first"] > 0 and st["restarts"] > 0 and st["steepest"] > 0
    assert st["F"] == pytest.approx(r.F * P.units.energy_J, rel=1e-8)
    assert np.abs(mag.get_magnetization()[P.mag_nodes] - r.m).max() < 1e-5
    mag.close()


@pytest.mark.parametrize("rule", [1, 2])
def test_beta_rules_match_oracle(lib, rule):
    """beta*FR (1) and beta*PRP (2) of Sec. 2.1 / Algorithm 3 selected in
    place of beta*ZA: the GPU minimisation follows the oracle's path with
    the same rule and reaches the same minimum."""
    Magnet, Params = lib
    wl = _hard(n_mag=5)
    mag, P = _setup(lib, wl)
    b = np.array([0.2, 0.0, -1.0])
    mag.set_magnetization(wl.m0)
    mag.set_field(b)
    st = mag.minimize(Params(jmax=4, beta_rule=rule, **TIGHT))
    r = ncg.minimize(P, energy.normalize(wl.m0[P.mag_nodes]), P.units.field_int(b),
                     ncg.Params(jmax=4, beta_rule={1: "FR", 2: "PRP"}[rule]))
    assert st["status"] == "ok" and r.status == "converged"
    _same_path(st, r)
    assert st["F"] == pytest.approx(r.F * P.units.energy_J, rel=1e-8)
    assert np.abs(mag.get_magnetization()[P.mag_nodes] - r.m).max() < 1e-5
    mag.close()


@pytest.mark.parametrize("prec,amg", [(0, 0), (1, 1)])
def test_poisson_schedule_keeps_the_minimum(lib, prec, amg):
    """The potential tolerance tied to t1 (poisson_sched): the same minimum
    as the oracle's (energy 1e-8, max nodal |dm| 1e-5) and as the GPU
    without the schedule, with fewer potential steps; the plain FP64 form
    along the same path as the oracle with the same schedule."""
    Magnet, Params = lib
    wl = synth.hard_cube(n_mag=16)
    mag, P = _setup(lib, wl)
    b = wl.fields[3]
    base = dict(jmax=4, precision=prec, amg=amg, inner_tol=1e-3 if amg else 0.1)
    out = []
    for sched in (0, 1):
        mag.set_magnetization(wl.m0)
        mag.set_field(b)
        out.append((mag.minimize(Params(poisson_sched=sched, **base)), mag.get_magnetization()[P.mag_nodes]))
    (s0, m0), (s1, m1) = out
    r = ncg.minimize(P, energy.normalize(wl.m0[P.mag_nodes]), P.units.field_int(b),
                     ncg.Params(jmax=4, poisson="cg", poisson_sched=True))
    assert s1["status"] == "ok" and r.status == "converged"
    assert s1["F"] == pytest.approx(r.F * P.units.energy_J, rel=1e-8)
    assert np.abs(m1 - r.m).max() < 1e-5
    assert s1["F"] == pytest.approx(s0["F"], rel=1e-8)
    assert np.abs(m1 - m0).max() < 1e-5
    assert s1["mi"] < s0["mi"]
    if prec == 0:
        for k in ("nli", "evals", "li", "ls_extra"):
            assert s1[k] == r.stats[k], (k, s1[k], r.stats[k])
    mag.close()


def test_jmax_autotune_restores_the_state(lib):
    """mm_autotune_jmax times the candidates on the given field steps from
    the current state and leaves that state unchanged; the minimisation
    afterwards is the same as without the autotuning."""
    Magnet, Params = lib
    wl = synth.hard_cube(n_mag=10)
    mag = Magnet(device=0)
    mag.upload_workload(wl)
    mag.set_magnetization(wl.m0)
    mag.set_field(wl.fields[2])
    mag.minimize(Params())
    m_before = mag.get_magnetization()
    best, ms = mag.autotune_jmax(wl.fields[3:6], candidates=(0, 2, 4, 8))
    assert best in (0, 2, 4, 8) and all(t > 0 for t in ms.values())
    assert ms[best] == min(ms.values())
    np.testing.assert_array_equal(mag.get_magnetization(), m_before)
    mag.set_field(wl.fields[3])
    st_a = mag.minimize(Params())
    m_a = mag.get_magnetization()
    mag2 = Magnet(device=0)
    mag2.upload_workload(wl)
    mag2.set_magnetization(m_before)
    mag2.set_field(wl.fields[3])
    st_b = mag2.minimize(Params())
    assert st_a["F"] == pytest.approx(st_b["F"], rel=1e-9)          # (different potential warm starts)
    assert np.abs(m_a - mag2.get_magnetization()).max() < 1e-6
    mag.close()
    mag2.close()
