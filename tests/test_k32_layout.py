"""Host logic of the FP32 potential stiffness layout the precision form
streams (no GPU): mm_k32_host_apply builds the layout mm_upload_mesh
uploads and applies it in FP32 in the solver kernel's entry order.  Pins: the
product against scipy's FP64 product of the same matrix (FP32 rounding
only); an independent count of the slices that get an offset table and of the
matrix bytes; both kinds of slice (a lattice stencil, a jittered mesh), ragged
last slices; argument checks."""
import numpy as np
import pytest

import synth
from oracle import fem


def _K(wl):
    A = fem.assemble_workload(wl).Kphi.tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    return A


def _pruned(A):
    """A without its rounding residues (off-diagonal |a_ij| <= 1e-12
    sqrt(a_ii a_jj)), the matrix the upload stores."""
    C = A.tocoo()
    d = np.abs(A.diagonal())
    keep = (C.row == C.col) | (np.abs(C.data) > 1e-12 * np.sqrt(d[C.row] * d[C.col]))
    B = type(A)((C.data[keep], (C.row[keep], C.col[keep])), shape=A.shape).tocsr()
    B.sort_indices()
    return B


def _expected_layout(B):
    """Slices of 32 rows; a slice gets a table when its rows' offsets c - r
    number at most 8 and r + offset stays in [0, n) for all of its rows and
    offsets; matrix bytes 4 per stored value (32 x table size per slice,
    real rows only) + 32 per table, 8 per nonzero elsewhere + 32."""
    n = B.shape[0]
    tables, nbytes = 0, 0
    for s in range((n + 31) // 32):
        r0, r1 = 32 * s, min(n, 32 * s + 32)
        offs = set()
        for r in range(r0, r1):
            offs.update((B.indices[B.indptr[r]:B.indptr[r + 1]] - r).tolist())
        ok = len(offs) <= 8 and all(0 <= r + d < n for r in range(r0, r1) for d in offs)
        if ok:
            tables += 1
            nbytes += 4 * len(offs) * (r1 - r0) + 32
        else:
            nbytes += 8 * (B.indptr[r1] - B.indptr[r0]) + 32
    return tables, nbytes


@pytest.fixture(scope="module")
def k32():
    from paper_1801_03690_gb300 import k32_host_apply, MMError
    return k32_host_apply, MMError


@pytest.mark.parametrize("case", ["lattice", "graded", "jittered"])
def test_layout_product_and_counts(k32, case):
    wl = {"lattice": lambda: synth.hard_cube(n_mag=12, jitter=0.0),
          "graded": lambda: synth.large_polycrystal(n_mag=14, edge=30e-9, n_grains=4),
          "jittered": lambda: synth.hard_cube(n_mag=10, jitter=0.07, seed=2)}[case]()
    A = _K(wl)
    n = A.shape[0]
    x = np.random.default_rng(3).standard_normal(n).astype(np.float32)
    y, tables, nbytes = k32[0](A.indptr, A.indices, A.data, x)
    B = _pruned(A)
    ref = B @ x.astype(np.float64)
    scale = np.abs(B) @ np.abs(x.astype(np.float64))
    assert np.all(np.abs(y - ref) <= 1e-5 * scale + 1e-30)
    want_tables, want_bytes = _expected_layout(B)
    assert (tables, nbytes) == (want_tables, want_bytes)
    slices = (n + 31) // 32
    if case == "jittered":
        assert tables == 0                                    # 15 couplings per row: no tables
    else:
        assert tables > 0.95 * slices                         # the 7-point lattice stencil
        assert nbytes < 0.6 * 8 * B.nnz


def test_layout_small_and_bad_arguments(k32):
    apply, MMError = k32
    # 5 x 5 tridiagonal: one ragged slice, offsets {-1, 0, 1}; row 0 + (-1)
    # and row 4 + 1 leave [0, n), so the slice keeps its columns
    n = 5
    A = (np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1))
    import scipy.sparse as sp
    S = sp.csr_matrix(A)
    x = np.arange(1, n + 1, dtype=np.float32)
    y, tables, nbytes = apply(S.indptr, S.indices, S.data, x)
    np.testing.assert_array_equal(y, (A @ x).astype(np.float32))
    assert tables == 0 and nbytes == 8 * S.nnz + 32
    with pytest.raises(MMError):
        apply(S.indptr, np.where(S.indices == 4, 7, S.indices).astype(np.int32), S.data, x)
    with pytest.raises(MMError):
        apply(S.indptr[::-1].copy(), S.indices, S.data, x)
