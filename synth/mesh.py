"""Structured tetrahedral meshes (Kuhn / Freudenthal split of a box lattice).

Coordinates are in metres.  A mesh is a set of nodes, tetrahedra (4 node
indices each, positively oriented on the unjittered lattice) and one region
label per tetrahedron.  Region 0 is conventionally the non-magnetic air box;
the material table that gives meaning to the labels lives with the workload.
"""
from dataclasses import dataclass, field
from itertools import permutations

import numpy as np


@dataclass
class Mesh:
    xyz: np.ndarray          # (N, 3) float64, metres
    tets: np.ndarray         # (T, 4) int32
    region: np.ndarray       # (T,)   int32
    shape: tuple = ()        # lattice node counts (nx, ny, nz) if structured
    spacing: float = 0.0     # nominal lattice spacing h (m)
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self):
        return int(self.xyz.shape[0])

    @property
    def n_tets(self):
        return int(self.tets.shape[0])


def _perm_parity(p):
    p = list(p)
    s = 1
    for i in range(len(p)):
        for j in range(i + 1, len(p)):
            if p[i] > p[j]:
                s = -s
    return s


def kuhn_lattice(xs, ys, zs):
    """Nodes on the tensor lattice xs x ys x zs (node id = i + nx*(j + ny*k))
    and 6 tetrahedra per voxel, one per monotone corner path from (0,0,0) to
    (1,1,1).  Returns (xyz, tets, voxel_of_tet)."""
    xs, ys, zs = (np.asarray(a, dtype=np.float64) for a in (xs, ys, zs))
    nx, ny, nz = len(xs), len(ys), len(zs)
    X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
    # node id = i + nx*(j + ny*k): order with i fastest
    xyz = np.stack([X.transpose(2, 1, 0).ravel(),
                    Y.transpose(2, 1, 0).ravel(),
                    Z.transpose(2, 1, 0).ravel()], axis=1)

    I, J, K = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1),
                          np.arange(nz - 1), indexing="ij")
    I = I.transpose(2, 1, 0).ravel()
    J = J.transpose(2, 1, 0).ravel()
    K = K.transpose(2, 1, 0).ravel()

    def nid(di, dj, dk):
        return (I + di) + nx * ((J + dj) + ny * (K + dk))

    tets = []
    for p in permutations(range(3)):
        corner = [0, 0, 0]
        path = [nid(0, 0, 0)]
        for ax in p:
            corner[ax] = 1
            path.append(nid(*corner))
        if _perm_parity(p) < 0:          # keep every tet positively oriented
            path[2], path[3] = path[3], path[2]
        tets.append(np.stack(path, axis=1))
    # interleave so the 6 tets of a voxel are contiguous
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    vox = np.repeat(np.arange(I.size), 6)
    return xyz, tets, vox


def cube_in_box(n_mag, h, box_factor=2.0, center=(0.0, 0.0, 0.0)):
    """A cube magnet of n_mag voxels per edge (spacing h) centred in a cubic
    air box whose edge is about box_factor times the magnet edge, on one
    uniform lattice.  Region 1 = magnet, region 0 = air."""
    n_box = int(round(n_mag * box_factor))
    if (n_box - n_mag) % 2:
        n_box += 1
    pad = (n_box - n_mag) // 2
    coords = (np.arange(n_box + 1) - n_box / 2.0) * h
    xs = coords + center[0]
    ys = coords + center[1]
    zs = coords + center[2]
    xyz, tets, vox = kuhn_lattice(xs, ys, zs)
    nv = n_box
    vi = vox % nv
    vj = (vox // nv) % nv
    vk = vox // (nv * nv)
    inside = ((vi >= pad) & (vi < pad + n_mag) & (vj >= pad) & (vj < pad + n_mag)
              & (vk >= pad) & (vk < pad + n_mag))
    region = inside.astype(np.int32)
    mesh = Mesh(xyz=xyz, tets=tets, region=region, shape=(nv + 1,) * 3,
                spacing=h, meta={"n_mag": n_mag, "n_box": n_box, "pad": pad})
    return mesh


def _node_region_range(mesh):
    n = mesh.n_nodes
    lo = np.full(n, np.iinfo(np.int32).max, dtype=np.int64)
    hi = np.full(n, -1, dtype=np.int64)
    for c in range(4):
        np.minimum.at(lo, mesh.tets[:, c], mesh.region)
        np.maximum.at(hi, mesh.tets[:, c], mesh.region)
    return lo, hi


def jitter_nodes(mesh, amp, seed):
    """Displace every node whose incident tetrahedra all carry one region
    label and that is not on the outer lattice boundary by independent
    uniform offsets in [-amp*h, amp*h] per coordinate.  Region interfaces and
    the outer box stay planar.  For amp <= 0.07 every Kuhn tetrahedron keeps a
    positive volume: its unperturbed edge matrix is h*L*P with L the 3x3
    lower-triangular matrix of ones (smallest singular value 0.555) and P a
    permutation, the perturbation has entries |E_ij| <= 2*amp*h and hence
    spectral norm <= 6*amp*h, so the smallest singular value stays
    >= h*(0.555 - 6*amp) > 0."""
    if amp > 0.07:
        raise ValueError("jitter amplitude above 0.07 h can invert tetrahedra")
    nx, ny, nz = mesh.shape
    ids = np.arange(mesh.n_nodes)
    i = ids % nx
    j = (ids // nx) % ny
    k = ids // (nx * ny)
    boundary = (i == 0) | (i == nx - 1) | (j == 0) | (j == ny - 1) | (k == 0) | (k == nz - 1)
    lo, hi = _node_region_range(mesh)
    movable = (~boundary) & (lo == hi)
    rng = np.random.default_rng(seed)
    d = rng.uniform(-amp * mesh.spacing, amp * mesh.spacing, size=(mesh.n_nodes, 3))
    xyz = mesh.xyz.copy()
    xyz[movable] += d[movable]
    return Mesh(xyz=xyz, tets=mesh.tets, region=mesh.region, shape=mesh.shape,
                spacing=mesh.spacing, meta=dict(mesh.meta, jitter=amp, jitter_seed=seed))


def _two_nearest(points, seeds):
    """Indices of the nearest and second-nearest seed of every point (a k-d
    tree query) and the squared distances to them."""
    from scipy.spatial import cKDTree
    _, idx = cKDTree(seeds).query(points, k=2, workers=-1)
    a = idx[:, 0].astype(np.int64)
    b = idx[:, 1].astype(np.int64)
    da = ((points - seeds[a]) ** 2).sum(-1)
    db = ((points - seeds[b]) ** 2).sum(-1)
    return a, b, da, db


def voronoi_regions(mesh, n_grains, lo, hi, gb_thickness, seed, magnet_region=1):
    """Split the tetrahedra labelled `magnet_region` into Voronoi grains around
    n_grains seeds uniform in the box [lo, hi]^3.  A tetrahedron whose
    centroid lies within gb_thickness/2 of the bisector plane of its two
    nearest seeds is labelled as grain-boundary phase.  Labels: grains
    1..n_grains, boundary phase n_grains+1, others unchanged."""
    rng = np.random.default_rng(seed)
    seeds = rng.uniform(lo, hi, size=(n_grains, 3))
    sel = np.nonzero(mesh.region == magnet_region)[0]
    c = mesh.xyz[mesh.tets[sel]].mean(axis=1)
    a, b, da, db = _two_nearest(c, seeds)
    sep = np.linalg.norm(seeds[a] - seeds[b], axis=1)
    dist_plane = (db - da) / (2.0 * sep)
    lab = (a + 1).astype(np.int32)
    lab[dist_plane < 0.5 * gb_thickness] = n_grains + 1
    region = mesh.region.copy()
    region[sel] = lab
    return Mesh(xyz=mesh.xyz, tets=mesh.tets, region=region, shape=mesh.shape,
                spacing=mesh.spacing, meta=dict(mesh.meta, grains=n_grains, grain_seed=seed)), seeds


def grain_patches(mesh, n_grains, patches_per_grain, seed):
    """Divide every grain (labels 1..n_grains) into patches_per_grain
    sub-regions: patch centres are the centroids of tetrahedra of the grain
    drawn without replacement (seeded), and every tetrahedron of the grain
    joins its nearest centre.  Returns (patch index in [0, patches) per
    tetrahedron, -1 outside the grains)."""
    rng = np.random.default_rng(seed)
    patch = np.full(mesh.n_tets, -1, dtype=np.int32)
    order = np.argsort(mesh.region, kind="stable")
    bounds = np.searchsorted(mesh.region[order], np.arange(1, n_grains + 2))
    for g in range(n_grains):
        idx = order[bounds[g]:bounds[g + 1]]
        if idx.size == 0:
            continue
        k = min(patches_per_grain, idx.size)
        cen = mesh.xyz[mesh.tets[idx]].mean(axis=1)
        centres = cen[rng.choice(idx.size, size=k, replace=False)]
        if k == 1:
            patch[idx] = 0
            continue
        from scipy.spatial import cKDTree
        _, nearest = cKDTree(centres).query(cen, k=1, workers=-1)
        patch[idx] = nearest.astype(np.int32)
    return patch
