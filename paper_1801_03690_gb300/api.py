"""Python binding of the mmncg C-ABI (include/mmncg.h).

Argument marshalling only: numpy arrays (host) or torch CUDA tensors (device
pointers) are handed to the CUDA library, which runs every step of the
method.  There is no CPU fallback: if the library is missing or no GPU is
present, construction raises.
"""
import ctypes as C
from dataclasses import dataclass, fields as dc_fields

import numpy as np

from . import _lib as L


class MMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{L.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


@dataclass
class Params:
    """Parameters of Algorithm 4 (see mm_params in include/mmncg.h)."""
    tau_F: float = 1e-10
    jmax: int = 4
    max_iter: int = 10000
    theta_max: float = 0.1
    c1: float = 1e-4
    max_backtrack: int = 10
    keep_last_term: bool = False
    poisson_tol: float = 1e-10
    poisson_max_iter: int = 20000
    precision: int = 0           # 1 = FP32 potential solve with FP64 refinement
    inner_tol: float = 0.1
    max_refine: int = 64
    amg: int = 0                 # 1 = multigrid-preconditioned FP32 solve
    beta_rule: int = 0           # 0 = beta*ZA, 1 = beta*FR, 2 = beta*PRP (Sec. 2.1)
    poisson_sched: int = 0       # 1 = potential tolerance tied to t1
    poisson_tol_max: float = 1e-6

    def to_c(self):
        p = L.mm_params()
        for f in dc_fields(self):
            v = getattr(self, f.name)
            setattr(p, f.name, int(v) if isinstance(v, (bool, int)) else float(v))
        return p


def _stats_dict(s):
    return {"evals": s.evals, "nli": s.nli, "li": s.li, "mi": s.mi, "ls_extra": s.ls_extra, "mr": s.mr,
            "status": L.STATUS_NAMES.get(s.status, s.status), "status_code": s.status,
            "F": s.F, "terms": list(s.terms), "F_internal": s.F_internal, "M": list(s.M),
            "li2": s.li2, "li2_first": s.li2_first, "restarts": s.restarts, "steepest": s.steepest}


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Magnet:
    """One micromagnetic problem on one GPU."""

    def __init__(self, device=0, blocks_per_sm=0, stream=None):
        self._lib = L.load()
        opt = L.mm_options(device=device, blocks_per_sm=blocks_per_sm,
                           stream=C.c_void_p(stream) if stream else None)
        h = C.c_void_p()
        rc = self._lib.mm_create(C.byref(h), C.byref(opt))
        if rc != 0:
            raise MMError(rc, "mm_create failed (no CUDA device, or no cooperative launch)")
        self._h = h
        self.n_nodes = 0

    # ------------------------------------------------------------------ util
    def _check(self, rc, soft_ok=False):
        if rc < 0 or (rc > 0 and not soft_ok):
            raise MMError(rc, self._lib.mm_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def stream(self):
        return self._lib.mm_stream(self._h)

    # ------------------------------------------------------------------ mesh
    def upload_mesh(self, xyz, tets, region, materials):
        xyz = _f64(xyz)
        tets = np.ascontiguousarray(tets, dtype=np.int32)
        region = np.ascontiguousarray(region, dtype=np.int32)
        mats = np.asarray(materials, dtype=np.float64).reshape(-1, 6)
        marr = (L.mm_material * len(mats))()
        for r, row in enumerate(mats):
            marr[r].Ms, marr[r].A, marr[r].K1 = row[0], row[1], row[2]
            marr[r].axis[0], marr[r].axis[1], marr[r].axis[2] = row[3], row[4], row[5]
        self._check(self._lib.mm_upload_mesh(self._h, xyz.shape[0], _ptr(xyz), tets.shape[0],
                                             _ptr(tets), _ptr(region), len(mats), marr))
        self.n_nodes = int(xyz.shape[0])
        return self

    def upload_workload(self, wl):
        return self.upload_mesh(wl.mesh.xyz, wl.mesh.tets, wl.mesh.region, wl.materials)

    def sizes(self):
        v = [C.c_int64() for _ in range(4)]
        self._check(self._lib.mm_sizes(self._h, *[C.byref(x) for x in v]))
        return {"n_mag": v[0].value, "n_phi": v[1].value, "nnz_mag": v[2].value, "nnz_phi": v[3].value}

    def k32_layout(self):
        """Layout of the FP32 K_phi the precision form streams: SELL-32
        slices, slices with an offset table (values only) and the matrix
        bytes of one product."""
        v = [C.c_int64() for _ in range(3)]
        self._check(self._lib.mm_k32_layout_info(self._h, *[C.byref(x) for x in v]))
        return {"slices": v[0].value, "table_slices": v[1].value, "matrix_bytes": v[2].value}

    def amg_levels(self):
        """Rows of every level of the potential solve's multigrid hierarchy,
        finest first, coarsest (dense) last; [] when there is none."""
        return [lv["rows"] for lv in self.amg_info()]

    def amg_info(self):
        """Per level of the multigrid hierarchy: rows, nonzeros of the
        operator (nnz_a; the coarsest: entries of its dense inverse), of U
        (nnz_u, the up phase's prolongation) and of the smoothed prolongation
        P (nnz_p, whose transpose restricts); None at the coarsest."""
        n = C.c_int32()
        rows, na, nu, npp = [(C.c_int64 * 64)() for _ in range(4)]
        self._check(self._lib.mm_amg_info(self._h, C.byref(n), rows, na, nu, npp, 64))
        L = n.value
        return [{"rows": int(rows[l]), "nnz_a": int(na[l]), "nnz_u": int(nu[l]) if l < L else None,
                 "nnz_p": int(npp[l]) if l < L else None}
                for l in range(L + 1)] if L > 0 else []

    # ----------------------------------------------------------------- state
    def set_magnetization(self, m):
        m = _f64(m, (self.n_nodes, 3))
        self._check(self._lib.mm_set_magnetization(self._h, _ptr(m)))

    def get_magnetization(self):
        out = np.zeros((self.n_nodes, 3))
        self._check(self._lib.mm_get_magnetization(self._h, _ptr(out)))
        return out

    def set_magnetization_dev(self, t):
        """t: contiguous float64 CUDA tensor [n_nodes, 3]."""
        assert t.is_cuda and t.dtype.is_floating_point and t.is_contiguous()
        self._check(self._lib.mm_set_magnetization_dev(self._h, C.c_void_p(t.data_ptr())))

    def get_magnetization_dev(self, t):
        assert t.is_cuda and t.is_contiguous()
        self._check(self._lib.mm_get_magnetization_dev(self._h, C.c_void_p(t.data_ptr())))

    def set_field(self, mu0h):
        b = (C.c_double * 3)(*[float(x) for x in mu0h])
        self._check(self._lib.mm_set_field(self._h, b))

    def set_tiles(self, rows_per_thread=0, restrict_lanes=0):
        """Tile shape of the FP32 potential-solve products (0 = default:
        two rows per thread, eight lanes per restriction row)."""
        self._check(self._lib.mm_set_tiles(self._h, int(rows_per_thread), int(restrict_lanes)))

    # ------------------------------------------------------------ operations
    def minimize(self, params=None):
        p = (params or Params()).to_c()
        s = L.mm_stats()
        rc = self._lib.mm_minimize(self._h, C.byref(p), C.byref(s))
        self._check(rc, soft_ok=True)
        return _stats_dict(s)

    def minimize_async(self, params=None):
        p = (params or Params()).to_c()
        self._check(self._lib.mm_minimize_async(self._h, C.byref(p)))

    def get_stats(self):
        s = L.mm_stats()
        rc = self._lib.mm_get_stats(self._h, C.byref(s))
        self._check(rc, soft_ok=True)
        return _stats_dict(s)

    def energy(self, m=None, params=None):
        p = (params or Params()).to_c()
        F = C.c_double()
        terms = (C.c_double * 4)()
        mm = None if m is None else _f64(m, (self.n_nodes, 3))
        self._check(self._lib.mm_energy(self._h, None if mm is None else _ptr(mm), C.byref(p),
                                        C.byref(F), terms))
        return F.value, list(terms)

    def gradient(self, m=None, projected=False, params=None):
        p = (params or Params()).to_c()
        out = np.zeros((self.n_nodes, 3))
        mm = None if m is None else _f64(m, (self.n_nodes, 3))
        self._check(self._lib.mm_gradient(self._h, None if mm is None else _ptr(mm), C.byref(p),
                                          _ptr(out), int(projected)))
        return out

    def potential(self):
        out = np.zeros(self.n_nodes)
        self._check(self._lib.mm_get_potential(self._h, _ptr(out)))
        return out

    def precond_solve(self, params=None):
        p = (params or Params()).to_c()
        out = np.zeros((self.n_nodes, 3))
        steps = C.c_int64()
        self._check(self._lib.mm_precond_solve(self._h, C.byref(p), _ptr(out), C.byref(steps)))
        return out, steps.value

    def hessian_apply(self, v, params=None):
        p = (params or Params()).to_c()
        v = _f64(v, (self.n_nodes, 3))
        out = np.zeros((self.n_nodes, 3))
        self._check(self._lib.mm_hessian_apply(self._h, C.byref(p), _ptr(v), _ptr(out)))
        return out

    def potential_matvec(self, v):
        v = _f64(v, (self.n_nodes,))
        out = np.zeros(self.n_nodes)
        self._check(self._lib.mm_potential_matvec(self._h, _ptr(v), _ptr(out)))
        return out

    def divergence(self, v):
        """D v (mm_operator_apply MM_OP_DIV): v [n_nodes, 3] -> [n_nodes]."""
        v = _f64(v, (self.n_nodes, 3))
        out = np.zeros(self.n_nodes)
        self._check(self._lib.mm_operator_apply(self._h, L.MM_OP_DIV, _ptr(v), _ptr(out)))
        return out

    def divergence_t(self, phi):
        """D^T phi (MM_OP_DIVT): phi [n_nodes] -> [n_nodes, 3]."""
        v = _f64(phi, (self.n_nodes,))
        out = np.zeros((self.n_nodes, 3))
        self._check(self._lib.mm_operator_apply(self._h, L.MM_OP_DIVT, _ptr(v), _ptr(out)))
        return out

    def local_apply(self, v):
        """(C_A + C_K) v (MM_OP_LOCAL): [n_nodes, 3] -> [n_nodes, 3]."""
        v = _f64(v, (self.n_nodes, 3))
        out = np.zeros((self.n_nodes, 3))
        self._check(self._lib.mm_operator_apply(self._h, L.MM_OP_LOCAL, _ptr(v), _ptr(out)))
        return out

    def demag_curve(self, fields, params=None):
        f = _f64(fields).reshape(-1, 3)
        p = (params or Params()).to_c()
        st = (L.mm_stats * len(f))()
        rc = self._lib.mm_demag_curve(self._h, len(f), _ptr(f), C.byref(p), st)
        self._check(rc, soft_ok=True)
        return [_stats_dict(s) for s in st]

    def autotune_jmax(self, fields, candidates=(0, 2, 4, 6, 8, 10, 12), params=None):
        """(best j_max, {j_max: device ms}) over the given field steps from the
        current state (mm_autotune_jmax); the state is restored."""
        f = _f64(fields).reshape(-1, 3)
        c = np.ascontiguousarray(candidates, dtype=np.int32)
        ms = np.zeros(len(c))
        best = C.c_int32()
        p = (params or Params()).to_c()
        self._check(self._lib.mm_autotune_jmax(self._h, C.byref(p), len(f), _ptr(f), _ptr(c), len(c),
                                               C.byref(best), _ptr(ms)))
        return best.value, {int(j): float(t) for j, t in zip(c, ms)}

    def last_kernel_ms(self):
        ms = C.c_double()
        self._check(self._lib.mm_last_kernel_ms(self._h, C.byref(ms)))
        return ms.value


def coercive_field(fields, M):
    """Coercive field (tesla) of a demagnetisation curve from the applied
    fields [n, 3] and the reduced magnetisation per step [n, 3]
    (mm_coercive_field); None if M never changes sign along the sweep."""
    lib = L.load()
    f = _f64(fields).reshape(-1, 3)
    m = _f64(M).reshape(-1, 3)
    if f.shape != m.shape:
        raise ValueError("fields and M must have the same shape [n, 3]")
    hc = C.c_double()
    found = C.c_int32()
    rc = lib.mm_coercive_field(len(f), _ptr(f), _ptr(m), C.byref(hc), C.byref(found))
    if rc != 0:
        raise MMError(rc, "mm_coercive_field rejected its arguments")
    return hc.value if found.value else None


def batch_plan(work, total_blocks, gamma=1.0):
    """Team sizes for a batch (pure host computation, no GPU needed)."""
    lib = L.load()
    w = np.ascontiguousarray(work, dtype=np.int64)
    out = np.zeros(len(w), dtype=np.int32)
    rc = lib.mm_batch_plan(len(w), w.ctypes.data_as(C.POINTER(C.c_int64)), int(total_blocks),
                           float(gamma), out.ctypes.data_as(C.POINTER(C.c_int32)))
    if rc != 0:
        raise MMError(rc, "mm_batch_plan rejected its arguments")
    return out


def amg_host_apply(indptr, indices, data, R):
    """The potential solve's multigrid V-cycle applied on the host (FP64, no
    GPU needed) to the rows of R, for the SPD matrix in CSR form (indptr,
    indices, data).  Returns (Z, level rows); ([], ...) when the matrix gets
    no hierarchy, Z is then None."""
    lib = L.load()
    ip = np.ascontiguousarray(indptr, dtype=np.int64)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    dv = np.ascontiguousarray(data, dtype=np.float64)
    n = len(ip) - 1
    R = np.ascontiguousarray(np.atleast_2d(R), dtype=np.float64)
    if R.shape[1] != n:
        raise ValueError("R must have n columns")
    Z = np.zeros_like(R)
    nl = C.c_int32()
    rows = (C.c_int64 * 64)()
    rc = lib.mm_amg_host_apply(n, ip.ctypes.data_as(C.POINTER(C.c_int64)), ix.ctypes.data_as(C.POINTER(C.c_int32)),
                               dv.ctypes.data_as(C.POINTER(C.c_double)), R.shape[0],
                               R.ctypes.data_as(C.POINTER(C.c_double)), Z.ctypes.data_as(C.POINTER(C.c_double)),
                               C.byref(nl), rows, 64)
    if rc != 0:
        raise MMError(rc, "mm_amg_host_apply rejected its arguments")
    if nl.value == 0:
        return None, []
    return Z, [int(rows[l]) for l in range(nl.value + 1)]


def k32_host_apply(indptr, indices, data, x):
    """The FP32 layout of K_phi that mm_upload_mesh builds, built on the host
    (no GPU needed) for the matrix in CSR form and applied in FP32 to x.
    Returns (y, slices with an offset table, matrix bytes of one product)."""
    lib = L.load()
    ip = np.ascontiguousarray(indptr, dtype=np.int64)
    ix = np.ascontiguousarray(indices, dtype=np.int32)
    dv = np.ascontiguousarray(data, dtype=np.float64)
    n = len(ip) - 1
    xv = np.ascontiguousarray(x, dtype=np.float32)
    if xv.shape != (n,):
        raise ValueError("x must have n entries")
    y = np.zeros(n, dtype=np.float32)
    tabs, nbytes = C.c_int64(), C.c_int64()
    rc = lib.mm_k32_host_apply(n, ip.ctypes.data_as(C.POINTER(C.c_int64)), ix.ctypes.data_as(C.POINTER(C.c_int32)),
                               dv.ctypes.data_as(C.POINTER(C.c_double)), xv.ctypes.data_as(C.POINTER(C.c_float)),
                               y.ctypes.data_as(C.POINTER(C.c_float)), C.byref(tabs), C.byref(nbytes))
    if rc != 0:
        raise MMError(rc, "mm_k32_host_apply rejected its arguments")
    return y, tabs.value, nbytes.value


class Batch:
    """Many independent magnets minimised in one persistent launch."""

    def __init__(self, magnets):
        self._lib = L.load()
        self.magnets = list(magnets)
        arr = (C.c_void_p * len(self.magnets))(*[m._h.value for m in self.magnets])
        h = C.c_void_p()
        rc = self._lib.mm_batch_create(C.byref(h), len(self.magnets), arr)
        if rc != 0:
            raise MMError(rc, "mm_batch_create failed (every member needs a mesh, one device)")
        self._h = h

    def _check(self, rc, soft_ok=False):
        if rc < 0 or (rc > 0 and not soft_ok):
            raise MMError(rc, self._lib.mm_batch_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def config(self, blocks_per_sm=3, gamma=1.0):
        self._check(self._lib.mm_batch_config(self._h, int(blocks_per_sm), float(gamma)))

    def set_tiles(self, rows_per_thread=0, restrict_lanes=0):
        self._check(self._lib.mm_batch_set_tiles(self._h, int(rows_per_thread), int(restrict_lanes)))

    def get_config(self):
        """The configuration batch launches use (after autotune: the chosen one)."""
        bps, rows, lanes = C.c_int32(), C.c_int32(), C.c_int32()
        gamma = C.c_double()
        self._check(self._lib.mm_batch_get_config(self._h, C.byref(bps), C.byref(gamma), C.byref(rows),
                                                  C.byref(lanes)))
        return {"blocks_per_sm": bps.value, "gamma": gamma.value, "rows_per_thread": rows.value,
                "restrict_lanes": lanes.value}

    def minimize(self, params=None):
        p = (params or Params()).to_c()
        st = (L.mm_stats * len(self.magnets))()
        self._check(self._lib.mm_batch_minimize(self._h, C.byref(p), st), soft_ok=True)
        return [_stats_dict(s) for s in st]

    def demag_curve(self, fields, params=None):
        """fields: [n_steps, n_members, 3] mu0*H in tesla."""
        f = _f64(fields)
        n = len(self.magnets)
        f = f.reshape(-1, n, 3)
        p = (params or Params()).to_c()
        st = (L.mm_stats * (f.shape[0] * n))()
        self._check(self._lib.mm_batch_demag_curve(self._h, f.shape[0], _ptr(f), C.byref(p), st),
                    soft_ok=True)
        return [[_stats_dict(st[s * n + t]) for t in range(n)] for s in range(f.shape[0])]

    def autotune(self, params=None):
        p = (params or Params()).to_c()
        bps = C.c_int()
        gamma = C.c_double()
        ms = C.c_double()
        self._check(self._lib.mm_batch_autotune(self._h, C.byref(p), C.byref(bps), C.byref(gamma),
                                                C.byref(ms)))
        return bps.value, gamma.value, ms.value

    def last_ms(self):
        ms = C.c_double()
        self._check(self._lib.mm_batch_last_ms(self._h, C.byref(ms)))
        return ms.value


class MLP:
    """The warm-start network (16 -> 128 -> 128 -> 128 -> 4), trained and
    evaluated by the library's tensor-core kernels."""

    def __init__(self, device=0, seed=0):
        self._lib = L.load()
        h = C.c_void_p()
        rc = self._lib.mm_mlp_create(C.byref(h), int(device), C.c_uint64(seed))
        if rc != 0:
            raise MMError(rc, "mm_mlp_create failed")
        self._h = h
        self.device = device
        self.n_params = int(self._lib.mm_mlp_param_count())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat):
        f = np.ascontiguousarray(flat, dtype=np.float32)
        rc = self._lib.mm_mlp_set_params(self._h, f.ctypes.data_as(C.c_void_p), f.size)
        if rc:
            raise MMError(rc, "mm_mlp_set_params")

    def set_input_norm(self, mean, stdev):
        m = np.ascontiguousarray(mean, dtype=np.float32)
        s = np.ascontiguousarray(stdev, dtype=np.float32)
        rc = self._lib.mm_mlp_set_input_norm(self._h, m.ctypes.data_as(C.c_void_p), s.ctypes.data_as(C.c_void_p))
        if rc:
            raise MMError(rc, "mm_mlp_set_input_norm")

    def set_tensor_path(self, path):
        """0: tcgen05 forward pass (default); 1: mma.sync (comparison)."""
        rc = self._lib.mm_mlp_set_tensor_path(self._h, int(path))
        if rc:
            raise MMError(rc, "mm_mlp_set_tensor_path")

    def fit_input_norm(self, X):
        """Input standardisation from the data X [n, 16] (float32, device)."""
        assert X.is_cuda and X.is_contiguous() and X.shape[1] == 16
        rc = self._lib.mm_mlp_fit_input_norm(self._h, C.c_void_p(X.data_ptr()), X.shape[0])
        if rc:
            raise MMError(rc, "mm_mlp_fit_input_norm")

    def input_norm(self):
        """(mean, 1/std) in use, float32 arrays of 16."""
        m = np.zeros(16, dtype=np.float32)
        s = np.zeros(16, dtype=np.float32)
        rc = self._lib.mm_mlp_get_input_norm(self._h, m.ctypes.data_as(C.c_void_p), s.ctypes.data_as(C.c_void_p))
        if rc:
            raise MMError(rc, "mm_mlp_get_input_norm")
        return m, s

    def fit_target_scales(self, T):
        """(Tn, scale_m, scale_phi): T [n, 4] (float32, device) with its m and
        potential columns divided by their standard deviations."""
        import torch
        assert T.is_cuda and T.is_contiguous() and T.shape[1] == 4
        Tn = torch.empty_like(T)
        sm = C.c_double()
        sp = C.c_double()
        rc = self._lib.mm_mlp_fit_target_scales(self._h, C.c_void_p(T.data_ptr()), T.shape[0],
                                                C.c_void_p(Tn.data_ptr()), C.byref(sm), C.byref(sp))
        if rc:
            raise MMError(rc, "mm_mlp_fit_target_scales")
        return Tn, sm.value, sp.value

    def step_targets(self, X0, X1):
        """(T, |dh|, largest nodal change) of one field step from the
        features before and after it (mm_warmstart_targets); T is None when
        the field did not change."""
        import torch
        assert X0.shape == X1.shape and X0.shape[1] == 16 and X0.is_contiguous() and X1.is_contiguous()
        T = torch.empty((X0.shape[0], 4), dtype=torch.float32, device=X0.device)
        dh = C.c_double()
        mx = C.c_double()
        rc = self._lib.mm_warmstart_targets(self._h, C.c_void_p(X0.data_ptr()), C.c_void_p(X1.data_ptr()),
                                            X0.shape[0], C.c_void_p(T.data_ptr()), C.byref(dh), C.byref(mx))
        if rc:
            raise MMError(rc, "mm_warmstart_targets")
        return (T if dh.value > 0 else None), dh.value, mx.value

    def get_params(self):
        f = np.zeros(self.n_params, dtype=np.float32)
        rc = self._lib.mm_mlp_get_params(self._h, f.ctypes.data_as(C.c_void_p), f.size)
        if rc:
            raise MMError(rc, "mm_mlp_get_params")
        return f

    def forward(self, X):
        import torch
        assert X.is_cuda and X.dtype == torch.float32 and X.shape[1] == 16 and X.is_contiguous()
        Y = torch.empty((X.shape[0], 4), dtype=torch.float32, device=X.device)
        torch.cuda.synchronize()
        rc = self._lib.mm_mlp_forward(self._h, C.c_void_p(X.data_ptr()), X.shape[0], C.c_void_p(Y.data_ptr()))
        if rc:
            raise MMError(rc, "mm_mlp_forward")
        return Y

    def gradient(self, X, T):
        import torch
        torch.cuda.synchronize()
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = C.c_float()
        rc = self._lib.mm_mlp_gradient(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                       X.shape[0], g.ctypes.data_as(C.c_void_p), C.byref(loss))
        if rc:
            raise MMError(rc, "mm_mlp_gradient")
        return g, loss.value

    def train_step(self, X, T, lr, want_loss=False):
        loss = C.c_float()
        rc = self._lib.mm_mlp_train_step(self._h, C.c_void_p(X.data_ptr()), C.c_void_p(T.data_ptr()),
                                         X.shape[0], C.c_float(lr), C.byref(loss) if want_loss else None)
        if rc:
            raise MMError(rc, "mm_mlp_train_step")
        return loss.value if want_loss else None


def warmstart_features(mag, mu0h_next, n_mag):
    """Features [n_mag, 16] (float32, device) of the current state of `mag`
    for the step to mu0h_next."""
    import torch
    X = torch.empty((n_mag, 16), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    b = (C.c_double * 3)(*[float(v) for v in mu0h_next])
    mag._check(mag._lib.mm_warmstart_features(mag._h, b, C.c_void_p(X.data_ptr())))
    return X


def warmstart_apply(mag, mlp, mu0h_next, scale_m, scale_phi, max_change=0.02):
    b = (C.c_double * 3)(*[float(v) for v in mu0h_next])
    mag._check(mag._lib.mm_warmstart_apply(mag._h, mlp._h, b, float(scale_m), float(scale_phi),
                                           float(max_change)))
