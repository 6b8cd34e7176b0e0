"""The batched form: many independent problems in one persistent launch,
against the same problems solved one by one and against the oracle."""
import numpy as np
import pytest

import synth
from oracle import fem, energy, ncg

pytestmark = pytest.mark.gpu


def _members():
    t = np.radians(20.0)
    return [
        synth.small_cube(n_mag=4, h=2e-9, jitter=0.05, seed=3),
        synth.small_cube(n_mag=6, h=1.5e-9, Ms=1.28e6, A=7.7e-12, K1=4.3e6,
                         axis=(np.sin(t), 0.0, np.cos(t)), jitter=0.07, seed=5),
        synth.small_cube(n_mag=3, h=2.5e-9, box_factor=3.0, seed=7),
        synth.platelet("ellipse", 20e-9, 10e-9, thickness=5e-9, h=2.5e-9),
    ]


FIELDS = np.array([[0.02, 0.0, 0.05], [0.0, 0.0, -1.0], [0.05, 0.05, 0.0], [0.01, 0.0, 0.0]])


def _magnets(wls, prec=0):
    from paper_1801_03690_gb300 import Magnet
    mags = []
    for wl, b in zip(wls, FIELDS):
        m = Magnet(device=0)
        m.upload_workload(wl)
        m.set_magnetization(wl.m0)
        m.set_field(b)
        mags.append(m)
    return mags


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_minimize_matches_single_problem_runs(prec):
    from paper_1801_03690_gb300 import Batch, Params
    wls = _members()
    prm = Params(jmax=4, poisson_tol=1e-12, precision=prec)
    single = []
    for mag in _magnets(wls):
        st = mag.minimize(prm)
        single.append((st, mag.get_magnetization()))
        mag.close()
    mags = _magnets(wls)
    batch = Batch(mags)
    sts = batch.minimize(prm)
    for (s1, m1), s2, mag in zip(single, sts, mags):
        assert s1["status"] == "ok" and s2["status"] == "ok"
        assert s2["F"] == pytest.approx(s1["F"], rel=1e-8)
        assert np.abs(mag.get_magnetization() - m1).max() < 1e-5
    batch.close()


def test_batch_member_matches_oracle():
    from paper_1801_03690_gb300 import Batch, Params
    wls = _members()
    mags = _magnets(wls)
    batch = Batch(mags)
    batch.config(blocks_per_sm=4, gamma=0.5)
    sts = batch.minimize(Params(jmax=4, poisson_tol=1e-12))
    wl, b = wls[0], FIELDS[0]
    P = fem.assemble_workload(wl)
    r = ncg.minimize(P, energy.normalize(wl.m0[P.mag_nodes]), P.units.field_int(b), ncg.Params(jmax=4))
    assert sts[0]["F"] == pytest.approx(r.F * P.units.energy_J, rel=1e-8)
    assert np.abs(mags[0].get_magnetization()[P.mag_nodes] - r.m).max() < 1e-5


def test_batch_demag_curve_graph_matches_single_curves():
    from paper_1801_03690_gb300 import Batch, Params
    wls = _members()
    n_steps = 5
    scale = np.linspace(1.0, -1.0, n_steps)
    fields = scale[:, None, None] * FIELDS[None, :, :]          # [steps, members, 3]
    prm = Params(jmax=4, poisson_tol=1e-12)
    ref = []
    for t, mag in enumerate(_magnets(wls)):
        ref.append([s["M"] for s in mag.demag_curve(fields[:, t, :], prm)])
        mag.close()
    mags = _magnets(wls)
    batch = Batch(mags)
    out = batch.demag_curve(fields, prm)
    assert len(out) == n_steps and len(out[0]) == len(wls)
    for t in range(len(wls)):
        M = np.array([out[s][t]["M"] for s in range(n_steps)])
        np.testing.assert_allclose(M, np.array(ref[t]), atol=1e-5)
        assert all(out[s][t]["status"] == "ok" for s in range(n_steps))
    assert batch.last_ms() > 0
    batch.close()


def test_batch_autotune_keeps_results():
    from paper_1801_03690_gb300 import Batch, Params
    wls = _members()
    prm = Params(jmax=4, poisson_tol=1e-12)
    mags = _magnets(wls)
    before = [m.get_magnetization() for m in mags]
    batch = Batch(mags)
    bps, gamma, ms = batch.autotune(prm)
    assert bps in (2, 3, 4) and gamma in (0.5, 0.75, 1.0) and ms > 0
    cfg = batch.get_config()
    assert cfg["blocks_per_sm"] == bps and cfg["gamma"] == gamma
    assert cfg["rows_per_thread"] in (1, 2) and cfg["restrict_lanes"] in (4, 8, 16)
    for m, b0 in zip(mags, before):                  # states restored
        np.testing.assert_array_equal(m.get_magnetization(), b0)
    sts = batch.minimize(prm)
    assert all(s["status"] == "ok" for s in sts)
    batch.close()


def test_batch_multigrid_form_matches_single_problem_runs():
    """Members with and without a multigrid hierarchy in one launch, with the
    multigrid precision form: each team runs its own problem's V-cycle."""
    from paper_1801_03690_gb300 import Batch, Magnet, Params
    t = np.radians(25.0)
    wls = [synth.small_cube(n_mag=8, h=1.5e-9, Ms=1.28e6, A=7.7e-12, K1=4.3e6,
                            axis=(np.sin(t), 0.2, np.cos(t)), jitter=0.07, seed=3),
           synth.hard_cube(n_mag=12, jitter=0.07, seed=6),
           synth.small_cube(n_mag=4, h=2e-9, jitter=0.05, seed=3)]
    fields = FIELDS[:3]
    prm = Params(jmax=4, poisson_tol=1e-12, precision=1, amg=1, inner_tol=1e-3)

    def mags():
        out = []
        for wl, b in zip(wls, fields):
            m = Magnet(device=0)
            m.upload_workload(wl)
            m.set_magnetization(wl.m0)
            m.set_field(b)
            out.append(m)
        return out

    single = []
    for mag in mags():
        st = mag.minimize(prm)
        single.append((st, mag.get_magnetization(), len(mag.amg_levels())))
        mag.close()
    assert [s[2] > 0 for s in single] == [True, True, False]
    ms = mags()
    batch = Batch(ms)
    sts = batch.minimize(prm)
    for (s1, m1, _), s2, mag in zip(single, sts, ms):
        assert s1["status"] == "ok" and s2["status"] == "ok"
        assert s2["F"] == pytest.approx(s1["F"], rel=1e-8)
        assert np.abs(mag.get_magnetization() - m1).max() < 1e-5
    batch.close()
