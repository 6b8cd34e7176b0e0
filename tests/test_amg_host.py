"""Host logic of the potential solve's multigrid preconditioner (no GPU):
the hierarchy that mm_upload_mesh builds and the V-cycle the solver kernel
runs, applied in FP64 on the host by mm_amg_host_apply to the oracle's
potential stiffness matrices.  Pins: an independent scipy restatement of the
same smoothed aggregation and cycle (agreement to rounding), symmetry and
positive definiteness of the cycle (what CG needs), and its effect as a CG
preconditioner."""
import numpy as np
import pytest
import scipy.sparse as sp

import synth
from oracle import fem


def _K(wl):
    A = fem.assemble_workload(wl).Kphi.tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    return A


@pytest.fixture(scope="module")
def lib():
    from paper_1801_03690_gb300 import amg_host_apply, MMError
    return amg_host_apply, MMError


@pytest.fixture(scope="module")
def K16():
    return _K(synth.hard_cube(n_mag=16))


@pytest.fixture(scope="module")
def Kgraded():
    """Potential stiffness of an unjittered polycrystal in a graded air box:
    its face- and body-diagonal couplings are rounding residues."""
    return _K(synth.large_polycrystal(n_mag=20, edge=40e-9, n_grains=6))


def _apply(lib, A, R):
    return lib[0](A.indptr, A.indices, A.data, R)


# ---- an independent restatement of the set-up and the cycle -------------
def _aggregate(A):
    """Greedy distance-one aggregation: a node whose neighbours are all free
    roots an aggregate with them; leftovers join their first aggregated
    neighbour (of the first pass); the rest are singletons."""
    n = A.shape[0]
    agg = -np.ones(n, dtype=np.int64)
    na = 0
    for i in range(n):
        if agg[i] >= 0:
            continue
        cols = A.indices[A.indptr[i]:A.indptr[i + 1]]
        nb = cols[cols != i]
        if np.any(agg[nb] >= 0):
            continue
        agg[i] = na
        agg[cols] = na
        na += 1
    first = agg.copy()
    for i in range(n):
        if first[i] >= 0:
            continue
        for j in A.indices[A.indptr[i]:A.indptr[i + 1]]:
            if j != i and first[j] >= 0:
                agg[i] = first[j]
                break
    for i in range(n):
        if agg[i] < 0:
            agg[i] = na
            na += 1
    return agg, na


def _prune(A, rel=1e-12):
    """A without the off-diagonal entries |a_ij| <= rel sqrt(|a_ii a_jj|):
    couplings that vanish in exact arithmetic (the face and body diagonals
    of a rectilinear Kuhn lattice) but were assembled as rounding residues."""
    C = A.tocoo()
    d = np.abs(A.diagonal())
    keep = (C.row == C.col) | (np.abs(C.data) > rel * np.sqrt(d[C.row] * d[C.col]))
    return sp.csr_matrix((C.data[keep], (C.row[keep], C.col[keep])), shape=A.shape)


def _hierarchy(A, n_dense=1536):
    levels = []
    while A.shape[0] > n_dense:
        agg, nc = _aggregate(A)            # on the stored pattern
        if nc > A.shape[0] // 2:
            break
        if not levels:
            A = _prune(A)                  # level 0: numerics without the residues
        d = A.diagonal()
        rho = (abs(A).sum(axis=1).A1 / d).max()
        Dinv = sp.diags(1.0 / d)
        Pt = sp.csr_matrix((np.ones(A.shape[0]), (np.arange(A.shape[0]), agg)), shape=(A.shape[0], nc))
        P = (Pt - (2.0 / rho) * (Dinv @ (A @ Pt))).tocsr()
        omega = min(0.9, 1.95 / rho)
        levels.append((A, P, 1.0 / d, omega))
        A = _prune((P.T @ A @ P).tocsr())  # coarse operator without residues
    return levels, np.linalg.inv(A.toarray())


def _vcycle(levels, Ainv, b, l=0):
    if l == len(levels):
        return Ainv @ b
    A, P, dinv, om = levels[l]
    x = om * dinv * b                       # pre-smoothing from zero
    r = b - A @ x
    x = x + P @ _vcycle(levels, Ainv, P.T @ r, l + 1)   # coarse correction
    return x + om * dinv * (b - A @ x)      # post-smoothing


# ---- tests ----------------------------------------------------------------
def test_small_matrix_gets_no_hierarchy(lib):
    A = _K(synth.small_cube(n_mag=4, h=2e-9))
    assert A.shape[0] <= 1536
    Z, levels = _apply(lib, A, np.ones((1, A.shape[0])))
    assert Z is None and levels == []


def test_levels(lib, K16):
    _, levels = _apply(lib, K16, np.ones((1, K16.shape[0])))
    assert levels[0] == K16.shape[0] == 29791
    assert len(levels) >= 2 and 0 < levels[-1] <= 1536
    assert all(a > 2 * b for a, b in zip(levels[:-1], levels[1:]))


def test_cycle_matches_independent_restatement(lib, K16):
    rng = np.random.default_rng(3)
    R = rng.standard_normal((3, K16.shape[0]))
    Z, levels = _apply(lib, K16, R)
    lv, Ainv = _hierarchy(K16)
    assert [L[0].shape[0] for L in lv] + [Ainv.shape[0]] == levels
    for r, z in zip(R, Z):
        ref = _vcycle(lv, Ainv, r)
        assert np.abs(z - ref).max() <= 1e-10 * np.abs(ref).max()


def test_cycle_is_symmetric_positive_definite(lib, K16):
    rng = np.random.default_rng(4)
    R = rng.standard_normal((8, K16.shape[0]))
    Z, _ = _apply(lib, K16, R)
    S = R @ Z.T                               # r_i^T M r_j
    assert np.abs(S - S.T).max() <= 1e-11 * np.abs(S).max()
    assert np.linalg.eigvalsh(0.5 * (S + S.T)).min() > 0.0


def _pcg_steps(A, b, prec, tol=1e-8, maxit=2000):
    x = np.zeros_like(b)
    r = b.copy()
    z = prec(r)
    p = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    for k in range(1, maxit + 1):
        q = A @ p
        a = rz / (p @ q)
        x += a * p
        r -= a * q
        if np.linalg.norm(r) < tol * nb:
            return k, x
        z = prec(r)
        rzn = r @ z
        p = z + (rzn / rz) * p
        rz = rzn
    return maxit, x


def test_cycle_preconditions_cg(lib, K16):
    rng = np.random.default_rng(5)
    b = rng.standard_normal(K16.shape[0])
    k_mg, x = _pcg_steps(K16, b, lambda r: _apply(lib, K16, r[None, :])[0][0])
    k_jac, _ = _pcg_steps(K16, b, lambda r: r / K16.diagonal())
    assert np.linalg.norm(K16 @ x - b) < 1e-8 * np.linalg.norm(b)
    assert k_mg <= 30 and 3 * k_mg < k_jac


def test_rejects_bad_csr(lib):
    A = sp.identity(2000, format="csr")
    bad = A.indices.copy()
    bad[5] = 2000
    with pytest.raises(lib[1]):
        lib[0](A.indptr, bad, A.data, np.ones((1, 2000)))


def test_residues_are_pruned_and_cycle_matches(lib, Kgraded):
    """On a rectilinear Kuhn lattice about half of the stored couplings are
    rounding residues (below 1e-15 of the diagonal); the hierarchy's
    numerics drop them (the aggregates still come from the stored pattern)
    and the cycle agrees with the restatement that does the same."""
    P = _prune(Kgraded)
    d = np.abs(Kgraded.diagonal())
    C = Kgraded.tocoo()
    off = C.row != C.col
    rel = np.abs(C.data[off]) / np.sqrt(d[C.row[off]] * d[C.col[off]])
    assert (rel <= 1e-12).sum() > 0.3 * off.sum()
    assert rel[rel <= 1e-12].max() < 1e-15 and rel[rel > 1e-12].min() > 1e-3
    rng = np.random.default_rng(6)
    R = rng.standard_normal((2, Kgraded.shape[0]))
    Z, levels = _apply(lib, Kgraded, R)
    lv, Ainv = _hierarchy(Kgraded)
    assert [L[0].shape[0] for L in lv] + [Ainv.shape[0]] == levels
    assert lv[0][0].nnz == P.nnz < 0.7 * Kgraded.nnz
    for r, z in zip(R, Z):
        ref = _vcycle(lv, Ainv, r)
        assert np.abs(z - ref).max() <= 1e-10 * np.abs(ref).max()
