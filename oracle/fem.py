"""P1 finite-element assembly of the quadratic micromagnetic energy.

Sec. 2.2, Eq. (energy): F(m) = 1/2 m^T C m - 1/2 h_d^T M m - h_ext^T M m
with C = C_A + C_K.  The paper leaves the discretisation to its references;
this oracle uses the standard P1 (linear tetrahedral) form, written out
element by element:

  exchange    A |grad m|^2 :  K_A[i,j] = sum_e A_e V_e b_i^e . b_j^e,
                              C_A = 2 K_A (x) I_3, so 1/2 m^T C_A m = int A|grad m|^2
  anisotropy  -K (m.k)^2, lumped to the nodes:
                              C_K[i] = -2 sum_{e ni i} K_e V_e/4 k_e k_e^T   (3x3 per node)
  Ms weights  w_i = sum_{e ni i} Ms_e V_e/4       (lumped M; Zeeman = -sum_i w_i h.m_i)
  potential   K_phi[i,j] = sum_e V_e b_i^e . b_j^e over ALL tets (magnet + air box),
              phi = 0 on the outer surface of the mesh (Sec. 3.1: air box)
  divergence  (D m)_j = sum_e Ms_e V_e/4 sum_{i in e} m_i . b_j^e   (magnetic tets)

b_i^e = grad of the barycentric hat function of local vertex i on tet e.
With these, K_phi phi = D m is the weak form of lap(phi) = div(M), the stray
field is -grad(phi), and E_demag = 1/2 phi^T D m (= -1/2 h_d^T M m).

Pins (tests/test_oracle_fem.py): zero exchange for uniform m, the exact
Kuhn-lattice helix energy A V (2 - 2 cos kh)/h^2, total anisotropy -K V cos^2,
total Zeeman -Ms V mu0H.m, K_phi annihilating linear functions at interior
nodes, D m for uniform m equal to the surface charge Ms m.n times area, the
gradients b summing to zero and reproducing linear functions.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

MU0 = 4e-7 * np.pi
NM = 1e-9


@dataclass
class Units:
    """Internal units: x_int = x / 1 nm, Ms_int = Ms / M_ref,
    A_int = A / (mu0 M_ref^2 nm^2), K_int = K / (mu0 M_ref^2),
    h_int = mu0 H / (mu0 M_ref), F_int = F / (mu0 M_ref^2 nm^3)."""
    Mref: float

    @property
    def energy_J(self):
        return MU0 * self.Mref ** 2 * NM ** 3

    def field_int(self, b_tesla):
        return np.asarray(b_tesla, dtype=np.float64) / (MU0 * self.Mref)


@dataclass
class Problem:
    n_nodes: int
    units: Units
    mag_nodes: np.ndarray        # (Nm,) node ids carrying m, ascending
    free_nodes: np.ndarray       # (Nphi,) node ids carrying an unknown potential
    dirichlet_nodes: np.ndarray  # outer-surface node ids (phi = 0)
    KA: sp.csr_matrix            # (Nm, Nm) scalar exchange stiffness
    CK: np.ndarray               # (Nm, 3, 3) lumped anisotropy blocks
    w: np.ndarray                # (Nm,) lumped Ms weights
    Kphi: sp.csr_matrix          # (Nphi, Nphi) potential stiffness, Dirichlet removed
    Kfull: sp.csr_matrix         # (N, N) potential stiffness before Dirichlet removal
    D: sp.csr_matrix             # (Nphi, 3 Nm) divergence coupling, m flattened as [i*3+c]
    diag_CA: np.ndarray          # (Nm,) diagonal of C_A (same for all 3 components)
    volume: np.ndarray           # (T,) tet volumes (nm^3)
    magnetic_tet: np.ndarray     # (T,) bool
    cache: dict = field(default_factory=dict)

    @property
    def n_mag(self):
        return int(self.mag_nodes.size)

    @property
    def n_phi(self):
        return int(self.free_nodes.size)


def tet_geometry(xyz, tets):
    """Signed volume and barycentric gradients of every tetrahedron.

    With E the matrix whose rows are the edges x_k - x_0 (k = 1..3), a point
    is x = x_0 + E^T lam, so grad(lam_k) is row k of E^{-T}, i.e. column k
    of E^{-1}; grad(lam_0) = -sum_k grad(lam_k).  Returns (V, b) with V (T,)
    the unsigned volume and b (T, 4, 3)."""
    X = xyz[tets]                          # (T, 4, 3)
    E = X[:, 1:, :] - X[:, :1, :]          # (T, 3, 3) rows = edges
    det = np.linalg.det(E)
    if np.any(np.abs(det) <= 0.0):
        raise ValueError("degenerate tetrahedron")
    Einv = np.linalg.inv(E)                # (T, 3, 3)
    b = np.empty((tets.shape[0], 4, 3))
    b[:, 1:, :] = np.transpose(Einv, (0, 2, 1))   # row k = column k of E^{-1}
    b[:, 0, :] = -b[:, 1:, :].sum(axis=1)
    return np.abs(det) / 6.0, b


def surface_nodes(tets, n_nodes):
    """Nodes on faces that belong to exactly one tetrahedron."""
    faces = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]],
                            tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]], axis=0).astype(np.int64)
    faces.sort(axis=1)
    key = (faces[:, 0] * n_nodes + faces[:, 1]) * n_nodes + faces[:, 2]
    uniq, cnt = np.unique(key, return_counts=True)
    once = uniq[cnt == 1]
    a = once // (n_nodes * n_nodes)
    b = (once // n_nodes) % n_nodes
    c = once % n_nodes
    return np.unique(np.concatenate([a, b, c]))


def assemble(xyz_m, tets, region, materials):
    """Assemble every matrix of Eq. (energy) for a mesh in metres with a
    per-region material table (Ms, A, K1, axis_x, axis_y, axis_z)."""
    tets = np.asarray(tets, dtype=np.int64)
    region = np.asarray(region, dtype=np.int64)
    materials = np.asarray(materials, dtype=np.float64)
    n = xyz_m.shape[0]
    Mref = materials[:, 0].max()
    if not Mref > 0:
        raise ValueError("no magnetic material")
    units = Units(Mref=Mref)
    xyz = np.asarray(xyz_m, dtype=np.float64) / NM

    V, b = tet_geometry(xyz, tets)
    mat = materials[region]
    Ms = mat[:, 0] / Mref
    A = mat[:, 1] / (MU0 * Mref ** 2 * NM ** 2)
    K = mat[:, 2] / (MU0 * Mref ** 2)
    k = mat[:, 3:6] / np.linalg.norm(mat[:, 3:6], axis=1, keepdims=True)
    magnetic = Ms > 0

    # magnetic nodes, ascending node id; index map node -> magnet row
    mag_nodes = np.unique(tets[magnetic].ravel())
    mag_of = -np.ones(n, dtype=np.int64)
    mag_of[mag_nodes] = np.arange(mag_nodes.size)
    nm = mag_nodes.size

    # b_i . b_j per tet
    bb = np.einsum("tic,tjc->tij", b, b)

    # exchange stiffness on magnetic tets
    tm = tets[magnetic]
    rows = mag_of[np.repeat(tm, 4, axis=1)]            # (Tm, 16): i repeated
    cols = mag_of[np.tile(tm, (1, 4))]                 # (Tm, 16): j tiled
    vals = (A[magnetic] * V[magnetic])[:, None] * bb[magnetic].reshape(-1, 16)
    KA = sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(nm, nm)).tocsr()

    # lumped anisotropy blocks and Ms weights
    CK = np.zeros((nm, 3, 3))
    kk = np.einsum("ta,tb->tab", k, k)
    w = np.zeros(nm)
    for c in range(4):
        idx = mag_of[tm[:, c]]
        np.add.at(CK, idx, (-2.0 * K[magnetic] * V[magnetic] / 4.0)[:, None, None] * kk[magnetic])
        np.add.at(w, idx, Ms[magnetic] * V[magnetic] / 4.0)

    # scalar-potential stiffness on all tets, Dirichlet on the outer surface
    rows = np.repeat(tets, 4, axis=1)
    cols = np.tile(tets, (1, 4))
    vals = V[:, None] * bb.reshape(-1, 16)
    Kfull = sp.coo_matrix((vals.ravel(), (rows.ravel(), cols.ravel())), shape=(n, n)).tocsr()
    dnodes = surface_nodes(tets, n)
    free = np.setdiff1d(np.arange(n), dnodes)
    free_of = -np.ones(n, dtype=np.int64)
    free_of[free] = np.arange(free.size)
    Kphi = Kfull[free][:, free].tocsr()

    # divergence coupling D: row j (free node of a magnetic tet), column 3*i + c
    d_rows, d_cols, d_vals = [], [], []
    scale = Ms[magnetic] * V[magnetic] / 4.0
    bm = b[magnetic]
    for jl in range(4):
        for il in range(4):
            for c in range(3):
                d_rows.append(free_of[tm[:, jl]])
                d_cols.append(3 * mag_of[tm[:, il]] + c)
                d_vals.append(scale * bm[:, jl, c])
    d_rows = np.concatenate(d_rows)
    d_cols = np.concatenate(d_cols)
    d_vals = np.concatenate(d_vals)
    keep = d_rows >= 0
    D = sp.coo_matrix((d_vals[keep], (d_rows[keep], d_cols[keep])),
                      shape=(free.size, 3 * nm)).tocsr()

    diag_CA = 2.0 * KA.diagonal()
    return Problem(n_nodes=n, units=units, mag_nodes=mag_nodes, free_nodes=free,
                   dirichlet_nodes=dnodes, KA=KA, CK=CK, w=w, Kphi=Kphi, Kfull=Kfull, D=D,
                   diag_CA=diag_CA, volume=V, magnetic_tet=magnetic)


def assemble_workload(wl):
    """Assemble a synth.Workload."""
    return assemble(wl.mesh.xyz, wl.mesh.tets, wl.mesh.region, wl.materials)
