"""Pins of Algorithm 4 (projected preconditioned NCG), beta*ZA, the descent
safeguard, the line search and the field loop."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import fem, energy, ncg, curve

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_iteration_counts.txt")


def test_beta_za_branches():
    g_old = np.array([[1.0, 0.0, 0.0]])
    g_new = np.array([[0.0, 2.0, 0.0]])
    d_old = np.array([[-1.0, -1.0, 0.0]])
    y_new = np.array([[0.0, 1.0, 0.0]])          # y.g_new = 2 > y.g_old = 0
    # (g+ - g).y+ = 2, (g+ - g).d = 1 - 2 = -1
    assert ncg.beta_za(g_new, g_old, y_new, d_old) == pytest.approx(-2.0)
    y_bad = np.array([[1.0, 0.0, 0.0]])          # y.g_new = 0 < y.g_old = 1 -> restart
    assert ncg.beta_za(g_new, g_old, y_bad, d_old) == 0.0
    # tie -> restart
    assert ncg.beta_za(g_new, g_new, y_new, d_old) == 0.0


def test_direction_safeguard():
    g_old = np.array([[1.0, 0.0, 0.0]])
    g_new = np.array([[0.0, 1.0, 0.0]])
    d_old = np.array([[0.0, 10.0, 0.0]])
    # y pointing against g: -y is ascent, beta = 0 -> replaced by y = g
    y_new = np.array([[0.0, -1.0, 0.0]])
    d, gy = ncg.direction(g_new, g_old, y_new, d_old)
    assert float(np.sum(g_new * d)) < 0
    assert gy == pytest.approx(1.0)                      # y was replaced by g
    # a regular case keeps d = -y + beta d_old
    y_ok = np.array([[0.0, 0.5, 0.0]])
    d_prev = np.array([[-1.0, 0.0, 0.0]])
    beta = ncg.beta_za(g_new, g_old, y_ok, d_prev)
    assert beta == pytest.approx(0.5)
    d, gy = ncg.direction(g_new, g_old, y_ok, d_prev)
    np.testing.assert_allclose(d, [[-0.5, -0.5, 0.0]])
    assert gy == pytest.approx(0.5)


def test_cubic_step_exact_for_cubics():
    # phi(a) = a^3 - 3a has its local minimum at a = 1
    assert ncg.cubic_step(0.0, -3.0, 2.0, 2.0, 9.0) == pytest.approx(1.0)
    # phi(a) = (a - 0.3)^2
    f = lambda a: (a - 0.3) ** 2
    df = lambda a: 2 * (a - 0.3)
    assert ncg.cubic_step(f(0), df(0), 1.0, f(1.0), df(1.0)) == pytest.approx(0.3)
    # phi(a) = -a^3: no minimiser
    assert ncg.cubic_step(0.0, 0.0, 1.0, -1.0, -3.0) is None


def _sw_problem():
    t = np.radians(1.0)
    wl = synth.small_cube(n_mag=2, h=1e-9, Ms=1.28e6, A=7.7e-12, K1=4.3e6,
                          axis=(np.sin(t), 0.0, np.cos(t)), m0=(0, 0, 1))
    P = fem.assemble_workload(wl)
    P.D = sp.csr_matrix(P.D.shape)          # magnetostatics off: pure SW particle
    bK = 2 * 4.3e6 / 1.28e6
    hsw = (np.sin(t) ** (2 / 3) + np.cos(t) ** (2 / 3)) ** -1.5
    return P, bK * hsw


@pytest.mark.parametrize("jmax", [0, 4])
def test_stoner_wohlfarth_switching_field(jmax):
    """A 2 nm Nd2Fe14B cube (far below the exchange length) rotates
    coherently; with the field 1 degree off the easy axis it must switch
    between 0.995 and 1.005 of h_sw = 2K/(mu0 Ms) (cos^2/3 + sin^2/3)^-3/2."""
    P, bsw = _sw_problem()
    for f, switched in ((0.995, False), (1.005, True)):
        m = np.tile([0.0, 0.0, 1.0], (P.n_mag, 1))
        r = ncg.minimize(P, m, P.units.field_int([0, 0, -f * bsw]), ncg.Params(jmax=jmax))
        assert r.status == "converged"
        assert (r.m[:, 2].mean() < 0) == switched
        assert r.m[:, 2].std() < 1e-5


@pytest.mark.parametrize("psi_deg", [15.0, 30.0, 45.0, 60.0, 75.0])
def test_stoner_wohlfarth_astroid(psi_deg):
    """The same single-domain particle with its easy axis along z and the
    field reversed at angle psi from the axis: the metastable state reached
    from m = +z must survive at 0.98 and be gone at 1.02 of the astroid
    field h_sw(psi) = 2K/(mu0 Ms) (cos^2/3 psi + sin^2/3 psi)^-3/2."""
    wl = synth.small_cube(n_mag=2, h=1e-9, Ms=1.28e6, A=7.7e-12, K1=4.3e6, axis=(0.0, 0.0, 1.0),
                          m0=(0, 0, 1))
    P = fem.assemble_workload(wl)
    P.D = sp.csr_matrix(P.D.shape)          # magnetostatics off
    psi = np.radians(psi_deg)
    hsw = 2 * 4.3e6 / 1.28e6 * (np.cos(psi) ** (2 / 3) + np.sin(psi) ** (2 / 3)) ** -1.5
    u = np.array([np.sin(psi), 0.0, -np.cos(psi)])
    for f, switched in ((0.98, False), (1.02, True)):
        m = np.tile([0.0, 0.0, 1.0], (P.n_mag, 1))
        r = ncg.minimize(P, m, P.units.field_int(f * hsw * u), ncg.Params(jmax=4))
        assert r.status == "converged"
        assert (r.m[:, 2].mean() < 0) == switched
        assert r.m[:, 2].std() < 1e-5


def _soft_problem():
    wl = synth.small_cube(n_mag=3, h=2e-9, jitter=0.05, seed=9)
    return wl, fem.assemble_workload(wl)


def test_iteration_identities_and_invariants():
    wl, P = _soft_problem()
    m0 = energy.normalize(wl.m0[P.mag_nodes])
    h = P.units.field_int([0.05, 0.0, 0.02])
    jmax = 3
    r = ncg.minimize(P, m0, h, ncg.Params(jmax=jmax))
    st = r.stats
    assert r.status == "converged"
    assert st["evals"] == 2 * st["nli"] + 1 + st["ls_extra"]
    assert st["li"] <= jmax * (st["nli"] + 1)
    np.testing.assert_allclose(np.linalg.norm(r.m, axis=1), 1.0, atol=1e-14)
    # energy never increases along the iterates
    Fs = []
    for k in range(1, 8):
        rk = ncg.minimize(P, m0, h, ncg.Params(jmax=jmax, max_iter=k))
        Fs.append(rk.F)
    assert all(Fs[i + 1] <= Fs[i] for i in range(len(Fs) - 1))
    # t3 holds at the returned state
    assert np.abs(r.g).max() < 1e-10 ** (1 / 3) * (1 + abs(r.F))


def test_preconditioning_reduces_evaluations():
    """Sec. 3.2: a few inner steps cut the number of evaluations relative to
    j_max = 0 (no preconditioning)."""
    wl, P = _soft_problem()
    m0 = energy.normalize(wl.m0[P.mag_nodes])
    h = P.units.field_int([0.05, 0.0, 0.02])
    r0 = ncg.minimize(P, m0, h, ncg.Params(jmax=0))
    r4 = ncg.minimize(P, m0, h, ncg.Params(jmax=4))
    assert r4.stats["evals"] < r0.stats["evals"]
    assert r4.F == pytest.approx(r0.F, rel=1e-6)


def test_paper_printed_tables_satisfy_iteration_identities():
    """A check of the paper's printed data only (no oracle function runs
    here): the rows of Tables 1, 2 and 4 copied into the golden file satisfy
    evals = 2 nli + n_fields up to a small excess (the rare extra line-search
    evaluations) and li <= j_max (nli + n_fields), with equality when every
    inner solve runs to j_max (Table 1 j_max = 2, Table 2 j_max = 4).  Table 4
    j_max = 2 prints li 0.3% above that bound, so the bound is checked to
    within 0.5%.  These identities are what the line-search reading of the
    oracle (two evaluations per iteration) and its li1 reading reproduce;
    the oracle itself is held to them in
    test_iteration_identities_and_invariants."""
    rows = np.loadtxt(GOLDEN, comments="#", dtype=np.int64)
    for tab, jm, evals, nli, li, nf in rows:
        extra = evals - (2 * nli + nf)
        assert 0 <= extra <= 0.005 * evals, (tab, jm)
        assert li <= 1.005 * jm * (nli + nf), (tab, jm)
    exact = {(1, 2), (2, 4)}
    for tab, jm, evals, nli, li, nf in rows:
        if (tab, jm) in exact:
            assert li == jm * (nli + nf)


def test_coercive_field_interpolation():
    fields = np.array([[0, 0, 0.0], [0, 0, -1.0], [0, 0, -2.0], [0, 0, -3.0]])
    M = np.array([[0, 0, 1.0], [0, 0, 0.5], [0, 0, -0.5], [0, 0, -1.0]])
    assert curve.coercive_field(fields, M) == pytest.approx(1.5)
    assert curve.coercive_field(fields, np.abs(M)) is None


def test_stoner_wohlfarth_curve():
    P, bsw = _sw_problem()
    fields = np.stack([np.zeros(9), np.zeros(9), -bsw * np.linspace(0.96, 1.04, 9)], axis=1)
    m0 = np.tile([0.0, 0.0, 1.0], (P.n_nodes, 1))
    res = curve.demag_curve(P, fields, m0, ncg.Params(jmax=4))
    assert abs(res["Hc_T"] - bsw) <= 0.01 * bsw
    assert all(rec["status"] == "converged" for rec in res["records"])


@pytest.mark.parametrize("rule", ["ZA", "FR", "PRP"])
def test_preconditioned_rules_are_linear_pcg_on_a_quadratic(rule):
    """On F = 1/2 x^T A x - b^T x with exact line searches and y = M^-1 g
    (M = diag A), beta*ZA, beta*FR and beta*PRP (Sec. 2.1, Algorithm 3) all
    reproduce preconditioned linear CG: the directions are A-conjugate and
    the minimiser is reached in n steps (in exact arithmetic)."""
    rng = np.random.default_rng(5)
    n = 12
    Q = rng.standard_normal((n, n))
    A = Q @ Q.T + n * np.eye(n)
    b = rng.standard_normal(n)
    Minv = 1.0 / np.diag(A)
    x = np.zeros(n)
    g = A @ x - b
    y = Minv * g
    d = -y
    gy = float(g @ y)
    dirs = []
    for _ in range(n):
        dirs.append(d.copy())
        a = -float(g @ d) / float(d @ A @ d)            # exact line search
        x = x + a * d
        g_new = A @ x - b
        if np.linalg.norm(g_new) < 1e-12 * np.linalg.norm(b):
            break
        y_new = Minv * g_new
        dn, gy = ncg.direction(g_new.reshape(-1, 3), g.reshape(-1, 3), y_new.reshape(-1, 3),
                               d.reshape(-1, 3), rule=rule, gy_old=gy)
        d = dn.reshape(-1)
        g = g_new
    np.testing.assert_allclose(A @ x, b, rtol=0, atol=1e-9 * np.abs(b).max())
    D = np.array(dirs)
    C = D @ A @ D.T
    off = C - np.diag(np.diag(C))
    assert np.abs(off).max() <= 1e-8 * np.abs(np.diag(C)).max()


def test_tolerance_schedule_values():
    p = ncg.Params(poisson_sched=True, tau_F=1e-10, poisson_tol=1e-10, poisson_tol_max=1e-6)
    F0 = 99.0                                             # threshold tau_F (1 + |F|) = 1e-8
    assert ncg.scheduled_tolerance(p, None, F0) == 1e-10            # first iteration
    assert ncg.scheduled_tolerance(p, 1e-6, F0) == 1e-10            # q = 100: not loosened
    assert ncg.scheduled_tolerance(p, 1e-2, F0) == pytest.approx(1e-10 * 1e3 / 10)   # q = 1e6
    assert ncg.scheduled_tolerance(p, 1e8, F0) == 1e-6               # capped
    assert ncg.scheduled_tolerance(ncg.Params(), 1e8, F0) == 1e-10   # schedule off


def test_tolerance_schedule_keeps_the_minimum():
    """The scheduled potential tolerance reaches the same minimum (energy
    1e-9 relative, m 1e-6) with fewer potential CG steps."""
    wl = synth.small_cube(n_mag=5, h=2e-9, jitter=0.05, seed=3)
    P = fem.assemble_workload(wl)
    m0 = energy.normalize(wl.m0[P.mag_nodes])
    h = P.units.field_int(np.array([0.02, 0.0, 0.05]))
    r0 = ncg.minimize(P, m0, h, ncg.Params(jmax=4, poisson="cg"))
    r1 = ncg.minimize(P, m0, h, ncg.Params(jmax=4, poisson="cg", poisson_sched=True))
    assert r0.status == "converged" and r1.status == "converged"
    assert r1.F == pytest.approx(r0.F, rel=1e-9)
    assert np.abs(r1.m - r0.m).max() < 1e-6
    assert r1.stats["mi"] < r0.stats["mi"]


def test_stops_at_the_first_iteration_where_t1_t2_t3_hold():
    """Sec. 3.1: Algorithm 4 stops once t1 (energy decrease below
    tau_F (1 + |F|)), t2 (largest component step below sqrt(tau_F)
    (1 + |m|_inf)) and t3 (largest projected-gradient component below
    tau_F^(1/3) (1 + |F|)) hold together.  The three conditions are
    evaluated here from the iterates themselves (the same run capped by
    max_iter): all hold for the last iteration, not all for the one before."""
    wl, P = _soft_problem()
    m0 = energy.normalize(wl.m0[P.mag_nodes])
    h = P.units.field_int([0.05, 0.0, 0.02])
    tau = 1e-10
    r = ncg.minimize(P, m0, h, ncg.Params(jmax=3, tau_F=tau))
    n = r.stats["nli"]
    assert r.status == "converged" and n >= 3
    it = {k: ncg.minimize(P, m0, h, ncg.Params(jmax=3, tau_F=tau, max_iter=k)) for k in (n - 2, n - 1)}
    it[n] = r

    def rules(a, b):
        t1 = a.F - b.F < tau * (1.0 + abs(b.F))
        t2 = np.abs(a.m - b.m).max() < np.sqrt(tau) * (1.0 + np.abs(b.m).max())
        t3 = np.abs(b.g).max() < tau ** (1.0 / 3.0) * (1.0 + abs(b.F))
        return t1, t2, t3

    assert all(rules(it[n - 1], it[n]))
    assert not all(rules(it[n - 2], it[n - 1]))
    assert it[n - 1].status == "max_iter"
