"""The no-allocation energy/gradient entry point (mm_energy_gradient_noalloc).

It serves callers that cannot call cudaMalloc (device memory handed in full
to their own pool allocator or held to a quota, or loops that cannot afford
cudaFree's device-wide synchronisation): all of its work space is one fixed
device array of the library.  This test calls it through the C-ABI twice in
a row and checks it against the allocating entry points mm_energy and
mm_gradient, at the tolerances of the other GPU parity tests.  It lives in a
file of its own, collected last.
"""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _hard(n_mag, seed=4):
    t = np.radians(25.0)
    return synth.small_cube(n_mag=n_mag, h=1.5e-9, Ms=1.28e6, A=7.7e-12, K1=4.3e6,
                            axis=(np.sin(t), 0.2, np.cos(t)), jitter=0.07, seed=seed)


def test_noalloc_matches_allocating_entry_points():
    import torch
    from paper_1801_03690_gb300 import Magnet, Params
    from paper_1801_03690_gb300 import _lib

    lib = _lib.load()
    wl = _hard(6)
    mag = Magnet(device=0)
    mag.upload_workload(wl)
    b = np.array([0.3, -0.2, -1.5])
    mag.set_field(b)
    prm = Params(poisson_tol=1e-13)
    pc = prm.to_c()
    rng = np.random.default_rng(5)
    for call in range(2):
        m = wl.m0 if call == 0 else rng.normal(size=wl.m0.shape)
        m_dev = torch.tensor(m, dtype=torch.float64, device="cuda")
        grad_dev = torch.full_like(m_dev, np.nan)
        energy_dev = torch.zeros(5, dtype=torch.float64, device="cuda")
        projected = call
        rc = lib.mm_energy_gradient_noalloc(mag._h, C.c_void_p(m_dev.data_ptr()), C.byref(pc),
                                            C.c_void_p(grad_dev.data_ptr()), projected,
                                            C.c_void_p(energy_dev.data_ptr()))
        assert rc == 0, lib.mm_last_error(mag._h).decode()
        torch.cuda.synchronize()
        F_ref, terms_ref = mag.energy(m, prm)
        g_ref = mag.gradient(None, projected=bool(projected), params=prm)
        e = energy_dev.cpu().numpy()
        assert e[0] == pytest.approx(F_ref, rel=1e-10)
        for k in range(4):
            assert e[1 + k] == pytest.approx(terms_ref[k], rel=1e-10, abs=1e-12 * abs(F_ref))
        g = grad_dev.cpu().numpy()
        np.testing.assert_allclose(g, g_ref, rtol=0, atol=1e-9 * np.abs(g_ref).max())
    mag.close()


def test_noalloc_rejects_problems_beyond_its_array():
    import torch
    from paper_1801_03690_gb300 import Magnet
    from paper_1801_03690_gb300 import _lib

    lib = _lib.load()
    wl = synth.small_cube(n_mag=28, h=2e-9)          # 55^3 potential unknowns: > 8 MiB
    mag = Magnet(device=0)
    mag.upload_workload(wl)
    m_dev = torch.tensor(wl.m0, dtype=torch.float64, device="cuda")
    energy_dev = torch.zeros(5, dtype=torch.float64, device="cuda")
    rc = lib.mm_energy_gradient_noalloc(mag._h, C.c_void_p(m_dev.data_ptr()), None, None, 0,
                                        C.c_void_p(energy_dev.data_ptr()))
    assert rc == -1
    assert "MiB" in lib.mm_last_error(mag._h).decode()
    mag.close()


def test_noalloc_rejects_zero_and_nonfinite_vectors():
    """A zero vector or a NaN on one of the last magnetic nodes is reported
    as MM_ERR_NONFINITE on every call (the flag is cleared on the stream
    before the launch that may set it), and a valid call after them works."""
    import torch
    from paper_1801_03690_gb300 import Magnet, Params
    from paper_1801_03690_gb300 import _lib

    lib = _lib.load()
    wl = _hard(6)
    mag = Magnet(device=0)
    mag.upload_workload(wl)
    mag.set_field([0.1, 0.0, -0.5])
    pc = Params(poisson_tol=1e-12).to_c()
    mag_nodes = np.nonzero(np.isin(np.arange(wl.mesh.n_nodes),
                                   np.unique(wl.mesh.tets[wl.mesh.region == 1])))[0]
    energy_dev = torch.zeros(5, dtype=torch.float64, device="cuda")
    for bad in ("zero", "nan"):
        m = wl.m0.copy()
        node = mag_nodes[-1] if bad == "zero" else mag_nodes[-2]
        m[node] = 0.0 if bad == "zero" else np.nan
        m_dev = torch.tensor(m, dtype=torch.float64, device="cuda")
        for _ in range(4):
            rc = lib.mm_energy_gradient_noalloc(mag._h, C.c_void_p(m_dev.data_ptr()), C.byref(pc), None, 0,
                                                C.c_void_p(energy_dev.data_ptr()))
            assert rc == -5, (bad, rc)
    m_dev = torch.tensor(wl.m0, dtype=torch.float64, device="cuda")
    rc = lib.mm_energy_gradient_noalloc(mag._h, C.c_void_p(m_dev.data_ptr()), C.byref(pc), None, 0,
                                        C.c_void_p(energy_dev.data_ptr()))
    assert rc == 0, lib.mm_last_error(mag._h).decode()
    F_ref, _ = mag.energy(wl.m0, Params(poisson_tol=1e-12))
    assert float(energy_dev[0].item()) == pytest.approx(F_ref, rel=1e-10)
    mag.close()
