"""Seeded synthetic workloads shaped like the paper's soft- and hard-magnetic
test cases (Sec. 3.2-3.4): a permalloy cube, a hard-magnetic Nd2Fe14B cube
and a polycrystalline cube with a grain-boundary phase, each inside an air
box for the magnetostatic potential.

A material table has one row per region label: (Ms [A/m], A [J/m],
K1 [J/m^3], easy-axis x, y, z).  Row 0 is air (Ms = 0).  Fields are applied
flux densities mu0*H in tesla, one row per field step.
"""
from dataclasses import dataclass, field

import numpy as np

from .mesh import Mesh, cube_in_box, jitter_nodes, voronoi_regions, grain_patches, kuhn_lattice

MU0 = 4e-7 * np.pi

PERMALLOY = dict(Ms=8.0e5, A=1.3e-11, K1=0.0)
ND2FE14B = dict(Ms=1.28e6, A=7.7e-12, K1=4.3e6)


@dataclass
class Workload:
    name: str
    mesh: Mesh
    materials: np.ndarray      # (R, 6)
    fields: np.ndarray         # (F, 3) mu0*H in T
    m0: np.ndarray             # (N, 3) unit vectors (only magnetic nodes matter)
    meta: dict = field(default_factory=dict)


def random_unit_vectors(n, seed):
    """n independent unit vectors uniform on the sphere (normalised Gaussians)."""
    rng = np.random.default_rng(seed)
    v = rng.standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def cone_axes(n, max_angle_deg, seed):
    """n unit vectors uniform within a cone of half-angle max_angle about +z
    (cos(theta) ~ U[cos max, 1], azimuth ~ U[0, 2 pi))."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(np.cos(np.radians(max_angle_deg)), 1.0, size=n)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n)
    s = np.sqrt(1.0 - c * c)
    return np.stack([s * np.cos(phi), s * np.sin(phi), c], axis=1)


def _material_table(rows):
    t = np.zeros((len(rows), 6))
    for r, row in enumerate(rows):
        t[r] = row
    return t


def small_cube(n_mag=4, h=2.0e-9, box_factor=2.0, Ms=8.0e5, A=1.3e-11, K1=0.0,
               axis=(0.0, 0.0, 1.0), jitter=0.0, seed=0, m0=None,
               fields=((0.0, 0.0, 0.0),)):
    """A small cube magnet in an air box for tests."""
    mesh = cube_in_box(n_mag, h, box_factor)
    if jitter > 0:
        mesh = jitter_nodes(mesh, jitter, seed)
    ax = np.asarray(axis, dtype=np.float64)
    ax = ax / np.linalg.norm(ax)
    mats = _material_table([(0, 0, 0, 0, 0, 1), (Ms, A, K1, *ax)])
    if m0 is None:
        m0 = random_unit_vectors(mesh.n_nodes, seed + 1)
    else:
        m0 = np.broadcast_to(np.asarray(m0, dtype=np.float64), (mesh.n_nodes, 3)).copy()
        m0 /= np.linalg.norm(m0, axis=1, keepdims=True)
    return Workload(name=f"small_cube_{n_mag}", mesh=mesh, materials=mats,
                    fields=np.asarray(fields, dtype=np.float64).reshape(-1, 3), m0=m0,
                    meta={"n_mag": n_mag, "h": h, "box_factor": box_factor})


def soft_cube(n_mag=16, edge=40e-9, box_factor=2.0, seed=1, n_fields=21):
    """Permalloy cube (40 nm, Ms 8.0e5 A/m, A 1.3e-11 J/m, K 0) of n_mag^3
    voxels (6 tets each) in an air box of box_factor x edge with a grounded
    outer boundary; random initial magnetisation; field along x swept from
    +100 mT to -100 mT."""
    h = edge / n_mag
    mesh = cube_in_box(n_mag, h, box_factor)
    mats = _material_table([(0, 0, 0, 0, 0, 1),
                            (PERMALLOY["Ms"], PERMALLOY["A"], PERMALLOY["K1"], 1, 0, 0)])
    b = np.linspace(0.1, -0.1, n_fields)
    fields = np.stack([b, np.zeros_like(b), np.zeros_like(b)], axis=1)
    m0 = random_unit_vectors(mesh.n_nodes, seed)
    return Workload(name=f"soft_cube_{n_mag}", mesh=mesh, materials=mats, fields=fields,
                    m0=m0, meta={"edge": edge, "h": h, "seed": seed})


def hard_cube(n_mag=48, edge=80e-9, box_factor=2.0, seed=2, n_fields=40,
              b_stop=-8.0, jitter=0.07, tilt_deg=1.0):
    """Nd2Fe14B cube (80 nm, Ms 1.28e6 A/m, A 7.7e-12 J/m, K1 4.3e6 J/m^3),
    easy axis tilted tilt_deg from z towards x, n_mag^3 voxels with jittered
    interior nodes, air box of box_factor x edge; m0 = +z; field along -z from
    0 to b_stop tesla in n_fields values."""
    h = edge / n_mag
    mesh = cube_in_box(n_mag, h, box_factor)
    if jitter > 0:
        mesh = jitter_nodes(mesh, jitter, seed)
    t = np.radians(tilt_deg)
    mats = _material_table([(0, 0, 0, 0, 0, 1),
                            (ND2FE14B["Ms"], ND2FE14B["A"], ND2FE14B["K1"],
                             np.sin(t), 0.0, np.cos(t))])
    b = np.linspace(0.0, b_stop, n_fields)
    fields = np.stack([np.zeros_like(b), np.zeros_like(b), b], axis=1)
    m0 = np.tile([0.0, 0.0, 1.0], (mesh.n_nodes, 1))
    return Workload(name=f"hard_cube_{n_mag}", mesh=mesh, materials=mats, fields=fields,
                    m0=m0, meta={"edge": edge, "h": h, "seed": seed, "jitter": jitter})


def polycrystal_cube(n_mag=114, edge=200e-9, box_factor=2.0, n_grains=27, seed=3,
                     gb_thickness=2e-9, cone_deg=15.0, n_fields=60, b_stop=-8.0,
                     gb_factor=0.4):
    """Polycrystalline Nd2Fe14B cube: n_grains Voronoi grains with easy axes
    uniform in a cone about +z, a grain-boundary phase of thickness
    gb_thickness whose Ms and K1 are scaled by gb_factor (A unchanged),
    air box of box_factor x edge; m0 = +z; field along -z."""
    h = edge / n_mag
    mesh = cube_in_box(n_mag, h, box_factor)
    half = edge / 2.0
    mesh, seeds = voronoi_regions(mesh, n_grains, -half, half, gb_thickness, seed)
    axes = cone_axes(n_grains, cone_deg, seed + 1000)
    rows = [(0, 0, 0, 0, 0, 1)]
    for g in range(n_grains):
        rows.append((ND2FE14B["Ms"], ND2FE14B["A"], ND2FE14B["K1"], *axes[g]))
    rows.append((gb_factor * ND2FE14B["Ms"], ND2FE14B["A"], gb_factor * ND2FE14B["K1"], 0, 0, 1))
    mats = _material_table(rows)
    b = np.linspace(0.0, b_stop, n_fields)
    fields = np.stack([np.zeros_like(b), np.zeros_like(b), b], axis=1)
    m0 = np.tile([0.0, 0.0, 1.0], (mesh.n_nodes, 1))
    return Workload(name=f"polycrystal_{n_grains}g_{n_mag}", mesh=mesh, materials=mats,
                    fields=fields, m0=m0,
                    meta={"edge": edge, "h": h, "seed": seed, "grain_seeds": seeds})


def graded_cube_in_box(n_mag, edge, box_factor=2.0, ratio=1.06):
    """A cube magnet of n_mag voxels per edge (spacing h = edge / n_mag)
    centred in a cubic air box of box_factor x edge, on a tensor lattice that
    is uniform over the magnet and graded outside it (each air cell `ratio`
    times the previous one).  Region 1 = magnet, region 0 = air."""
    h = edge / n_mag
    ax = _graded_axis(edge / 2.0, h, box_factor * edge / 2.0, ratio)
    xyz, tets, vox = kuhn_lattice(ax, ax, ax)
    nv = len(ax) - 1
    lo = (nv - n_mag) // 2
    vi = vox % nv
    vj = (vox // nv) % nv
    vk = vox // (nv * nv)
    inside = ((vi >= lo) & (vi < lo + n_mag) & (vj >= lo) & (vj < lo + n_mag)
              & (vk >= lo) & (vk < lo + n_mag))
    return Mesh(xyz=xyz, tets=tets, region=inside.astype(np.int32), shape=(nv + 1,) * 3, spacing=h,
                meta={"n_mag": n_mag, "graded_ratio": ratio, "n_box": nv})


def large_polycrystal(n_mag=149, edge=250e-9, box_factor=2.0, ratio=1.06, n_grains=125, seed=5,
                      gb_thickness=2e-9, cone_deg=15.0, n_fields=60, b_stop=-8.0, gb_factor=0.4,
                      patches_per_grain=0, k1_sigma=0.05):
    """Large polycrystalline Nd2Fe14B cube: n_mag^3 voxels (6 tets each;
    149^3 voxels = 19.8 M magnet tets, 150^3 = 3.375 M magnetic nodes),
    n_grains Voronoi grains with easy axes uniform in a cone about +z, a
    grain-boundary phase of thickness gb_thickness with Ms and K1 at
    gb_factor, in a graded air box of box_factor x edge; m0 = +z; field along
    -z from 0 to b_stop tesla in n_fields values.  With patches_per_grain > 0
    every grain is split into that many patches whose K1 is drawn from a
    Gaussian of mean K1 and relative standard deviation k1_sigma (the
    nanocrystalline magnet of Sec. 3.4: local changes of the composition)."""
    mesh = graded_cube_in_box(n_mag, edge, box_factor, ratio)
    half = edge / 2.0
    mesh, seeds = voronoi_regions(mesh, n_grains, -half, half, gb_thickness, seed)
    axes = cone_axes(n_grains, cone_deg, seed + 1000)
    rows = [(0, 0, 0, 0, 0, 1)]
    Ms, A, K1 = ND2FE14B["Ms"], ND2FE14B["A"], ND2FE14B["K1"]
    if patches_per_grain > 0:
        patch = grain_patches(mesh, n_grains, patches_per_grain, seed + 2000)
        rng = np.random.default_rng(seed + 3000)
        k1 = K1 * (1.0 + k1_sigma * rng.standard_normal((n_grains, patches_per_grain)))
        region = mesh.region.copy()
        g = region - 1
        isg = (region >= 1) & (region <= n_grains)
        region[isg] = 1 + g[isg] * patches_per_grain + patch[isg]
        region[mesh.region == n_grains + 1] = 1 + n_grains * patches_per_grain
        for gi in range(n_grains):
            for q in range(patches_per_grain):
                rows.append((Ms, A, k1[gi, q], *axes[gi]))
        mesh = Mesh(xyz=mesh.xyz, tets=mesh.tets, region=region, shape=mesh.shape, spacing=mesh.spacing,
                    meta=dict(mesh.meta, patches_per_grain=patches_per_grain, k1_sigma=k1_sigma))
    else:
        for gi in range(n_grains):
            rows.append((Ms, A, K1, *axes[gi]))
    rows.append((gb_factor * Ms, A, gb_factor * K1, 0, 0, 1))
    mats = _material_table(rows)
    b = np.linspace(0.0, b_stop, n_fields)
    fields = np.stack([np.zeros_like(b), np.zeros_like(b), b], axis=1)
    m0 = np.tile([0.0, 0.0, 1.0], (mesh.n_nodes, 1))
    tag = f"_p{patches_per_grain}" if patches_per_grain else ""
    return Workload(name=f"large_polycrystal_{n_grains}g_{n_mag}{tag}", mesh=mesh, materials=mats,
                    fields=fields, m0=m0,
                    meta={"edge": edge, "h": edge / n_mag, "seed": seed, "grain_seeds": seeds,
                          "graded_ratio": ratio, "n_mag": n_mag})


def sp3_cube(L_lex, n_mag=24, box_factor=4.0, ratio=1.15, Ms=8.0e5, A=1.3e-11, start="flower"):
    """The cube of the muMAG standard problem 3 (Sec. 3.3): edge L = L_lex
    exchange lengths l_ex = sqrt(A / Km), Km = mu0 Ms^2 / 2, uniaxial
    anisotropy K = 0.1 Km along z, n_mag^3 voxels (h = L / n_mag; 24 voxels
    give h = 0.35 l_ex at L = 8.4 l_ex), in an air box of box_factor x L
    graded by `ratio` per cell, zero applied field.  start = "flower": the
    saturated state m = +z; start = "vortex": two domains m = +z (x < 0) and
    m = -z (x > 0) with a sharp transition."""
    km = 0.5 * MU0 * Ms ** 2
    lex = np.sqrt(A / km)
    L = L_lex * lex
    mesh = graded_cube_in_box(n_mag, L, box_factor, ratio)
    mats = _material_table([(0, 0, 0, 0, 0, 1), (Ms, A, 0.1 * km, 0.0, 0.0, 1.0)])
    m0 = np.tile([0.0, 0.0, 1.0], (mesh.n_nodes, 1))
    if start == "vortex":
        m0[mesh.xyz[:, 0] > 0.0, 2] = -1.0
    elif start != "flower":
        raise ValueError(start)
    return Workload(name=f"sp3_{L_lex:.2f}lex_{start}", mesh=mesh, materials=mats, fields=np.zeros((1, 3)), m0=m0,
                    meta={"L": L, "lex": lex, "Km": km, "n_mag": n_mag, "h_lex": L_lex / n_mag})


def _graded_axis(half_mag, h, half_box, ratio):
    """Coordinates covering [-half_box, half_box]: uniform spacing h over
    [-half_mag, half_mag], then spacing growing by `ratio` per cell outward."""
    n = max(1, int(np.ceil(2 * half_mag / h - 1e-9)))
    inner = np.linspace(-half_mag, half_mag, n + 1)
    out = []
    x, step = half_mag, h
    while x < half_box - 1e-15:
        step *= ratio
        x = min(x + step, half_box)
        out.append(x)
    out = np.array(out)
    return np.concatenate([-out[::-1], inner, out])


def platelet(shape, a, b, thickness=5e-9, h=2.5e-9, hz=2.5e-9, air=1.3, ratio=2.0,
             seed=0, n_fields=51, b_max=0.05):
    """A permalloy platelet (Sec. 3.2 material class) of the given in-plane
    shape ('ellipse', 'rectangle' or 'disc'; semi-axes a >= b in x and y)
    and thickness, on a lattice that is uniform (h in-plane, hz across)
    over the platelet and graded (growth `ratio`) out to an air box of
    `air` times the platelet's extent in every direction.  Field along the
    long axis (x) from +b_max to -b_max tesla in n_fields values."""
    if shape == "disc":
        b = a
    xs = _graded_axis(a, h, air * a, ratio)
    ys = _graded_axis(b, h, air * a, ratio)
    zs = _graded_axis(thickness / 2, hz, max(air * a * 0.5, 3 * thickness), ratio)
    from .mesh import kuhn_lattice
    xyz, tets, _ = kuhn_lattice(xs, ys, zs)
    c = xyz[tets].mean(axis=1)
    inz = np.abs(c[:, 2]) < thickness / 2
    if shape == "rectangle":
        inxy = (np.abs(c[:, 0]) < a) & (np.abs(c[:, 1]) < b)
    else:
        inxy = (c[:, 0] / a) ** 2 + (c[:, 1] / b) ** 2 < 1.0
    region = (inz & inxy).astype(np.int32)
    mesh = Mesh(xyz=xyz, tets=tets, region=region, shape=(len(xs), len(ys), len(zs)),
                spacing=h, meta={"shape": shape, "a": a, "b": b})
    mats = _material_table([(0, 0, 0, 0, 0, 1),
                            (PERMALLOY["Ms"], PERMALLOY["A"], PERMALLOY["K1"], 1, 0, 0)])
    bx = np.linspace(b_max, -b_max, n_fields)
    fields = np.stack([bx, np.zeros_like(bx), np.zeros_like(bx)], axis=1)
    m0 = np.tile([1.0, 0.0, 0.0], (mesh.n_nodes, 1))
    return Workload(name=f"platelet_{shape}_{2 * a * 1e9:.0f}x{2 * b * 1e9:.0f}", mesh=mesh,
                    materials=mats, fields=fields, m0=m0, meta={"seed": seed})


def platelet_batch(n=64, seed=4, lateral=(100e-9, 500e-9), thickness=5e-9, n_fields=51,
                   max_cells=160):
    """n seeded platelets: shape uniform over ellipse/rectangle/disc, long
    side uniform in `lateral`, aspect ratio U[1, 3] (discs round), in-plane
    spacing max(2.5 nm, long side / max_cells), 5 nm thick (3 node layers)."""
    rng = np.random.default_rng(seed)
    shapes = ["ellipse", "rectangle", "disc"]
    out = []
    for k in range(n):
        shape = shapes[int(rng.integers(0, 3))]
        L = rng.uniform(*lateral)
        asp = 1.0 if shape == "disc" else rng.uniform(1.0, 3.0)
        a, b = L / 2, L / 2 / asp
        h = max(2.5e-9, L / max_cells)
        out.append(platelet(shape, a, b, thickness=thickness, h=h, seed=seed * 1000 + k,
                            n_fields=n_fields))
    return out


def sphere_in_box(n_rad=8, h=1e-9, box_factor=6.0, ratio=1.15, Ms=8.0e5, A=1.3e-11):
    """A sphere magnet of radius n_rad * h on a Kuhn lattice (the tets whose
    centroid lies inside the sphere; a staircase surface) in a cubic air box
    of box_factor x the radius per half-edge, uniform spacing h over the
    sphere's bounding cube and graded by `ratio` per cell outside it; m0 =
    +z, no anisotropy, zero field."""
    R = n_rad * h
    ax = _graded_axis(R, h, box_factor * R, ratio)
    xyz, tets, _ = kuhn_lattice(ax, ax, ax)
    c = xyz[tets].mean(axis=1)
    inside = (np.einsum("ij,ij->i", c, c) < R * R).astype(np.int32)
    nv = len(ax) - 1
    mesh = Mesh(xyz=xyz, tets=tets, region=inside, shape=(nv + 1,) * 3, spacing=h,
                meta={"radius": R, "box_factor": box_factor, "graded_ratio": ratio})
    mats = _material_table([(0, 0, 0, 0, 0, 1), (Ms, A, 0.0, 0.0, 0.0, 1.0)])
    m0 = np.tile([0.0, 0.0, 1.0], (mesh.n_nodes, 1))
    return Workload(name=f"sphere_{n_rad}h", mesh=mesh, materials=mats, fields=np.zeros((1, 3)), m0=m0,
                    meta={"radius": R, "h": h})
