"""Each operator of Eq. (energy) applied once by the CUDA path (through the
C-ABI mm_operator_apply and mm_potential_matvec, the device code the
minimiser runs) against the oracle's assembled matrices, element by
element at 1e-12 relative to the largest entry of the result:

  D v        the right-hand side of the potential equation (Sec. 3.1)
  D^T phi    the magnetostatic part of the gradient
  (C_A + C_K) v   the exchange and anisotropy part of the gradient
  K_phi v    the potential stiffness

on a jittered cube (every coupling genuine), on the cube whose potential
solve has a two-level multigrid hierarchy, and on an unjittered graded
polycrystal, whose potential stiffness the upload stores without its
rounding residues (the operator must still agree at 1e-12)."""
import numpy as np
import pytest

import synth
from oracle import fem, precond

pytestmark = pytest.mark.gpu


def _hard(n_mag=6, jitter=0.07, seed=4):
    t = np.radians(25.0)
    return synth.small_cube(n_mag=n_mag, h=1.5e-9, Ms=1.28e6, A=7.7e-12, K1=4.3e6,
                            axis=(np.sin(t), 0.2, np.cos(t)), jitter=jitter, seed=seed)


MESHES = {
    "jittered_cube": lambda: _hard(),
    "two_level_cube": lambda: synth.hard_cube(n_mag=24),
    "graded_polycrystal": lambda: synth.large_polycrystal(n_mag=16, edge=32e-9, n_grains=5),
}


@pytest.fixture(scope="module", params=list(MESHES))
def case(request):
    from paper_1801_03690_gb300 import Magnet
    wl = MESHES[request.param]()
    mag = Magnet(device=0)
    mag.upload_workload(wl)
    P = fem.assemble_workload(wl)
    yield request.param, wl, mag, P
    mag.close()


def _close(out, ref):
    scale = np.abs(ref).max()
    assert scale > 0
    err = np.abs(out - ref).max()
    assert err <= 1e-12 * scale, err / scale


def test_divergence(case):
    name, wl, mag, P = case
    rng = np.random.default_rng(1)
    v = rng.normal(size=(wl.mesh.n_nodes, 3))
    out = mag.divergence(v)
    ref = np.zeros(wl.mesh.n_nodes)
    ref[P.free_nodes] = P.D @ v[P.mag_nodes].reshape(-1)
    _close(out, ref)


def test_divergence_transpose(case):
    name, wl, mag, P = case
    rng = np.random.default_rng(2)
    phi = rng.normal(size=wl.mesh.n_nodes)
    out = mag.divergence_t(phi)
    ref = np.zeros((wl.mesh.n_nodes, 3))
    ref[P.mag_nodes] = (P.D.T @ phi[P.free_nodes]).reshape(-1, 3)
    _close(out, ref)


def test_local_operators(case):
    name, wl, mag, P = case
    rng = np.random.default_rng(3)
    v = rng.normal(size=(wl.mesh.n_nodes, 3))
    out = mag.local_apply(v)
    ref = np.zeros((wl.mesh.n_nodes, 3))
    ref[P.mag_nodes] = precond.apply_C_local(P, v[P.mag_nodes])
    _close(out, ref)


def test_potential_stiffness(case):
    name, wl, mag, P = case
    rng = np.random.default_rng(4)
    v = rng.normal(size=wl.mesh.n_nodes)
    out = mag.potential_matvec(v)
    ref = np.zeros(wl.mesh.n_nodes)
    ref[P.free_nodes] = P.Kphi @ v[P.free_nodes]
    _close(out, ref)
    if name == "graded_polycrystal":
        # the stored operator dropped the rounding residues of the lattice
        assert mag.sizes()["nnz_phi"] < 0.75 * P.Kphi.nnz
    if name == "two_level_cube":
        assert len(mag.amg_levels()) == 3          # two smoothed levels + the dense one


def test_operator_rejects_unknown_op(case):
    import ctypes as C
    from paper_1801_03690_gb300 import _lib
    name, wl, mag, P = case
    lib = _lib.load()
    v = np.zeros((wl.mesh.n_nodes, 3))
    out = np.zeros((wl.mesh.n_nodes, 3))
    rc = lib.mm_operator_apply(mag._h, 7, v.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p))
    assert rc == -1
