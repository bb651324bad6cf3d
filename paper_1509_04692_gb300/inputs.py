"""Seeded synthetic inputs for the checkerboard hard-particle MC sweep.

This module is shared by the tests, the benchmark, the oracle checks and the
CUDA path.  It holds none of the method's arithmetic: no overlap test, no
cell list, no random stream of the sweep.  It only builds shapes, boxes and
overlap-free starting configurations by construction:

* 2D, random orientations: a (slightly stretched) triangular lattice whose
  nearest-site distance is at least the circumdiameter 2R, so no two shapes
  can touch whatever their orientations.
* 2D, aligned: the same lattice with every shape at the same orientation and a
  nearest-site distance of at least the shape's diameter (largest vertex
  distance).  Translates K and K+t overlap only if t lies in the difference
  body K-K, which sits inside the disk of that radius.
* 3D, aligned: a simple cubic lattice with spacing at least the largest
  axis-aligned extent of the shape; two aligned translates whose centres
  differ by at least that much along some axis have disjoint bounding boxes.

Numbers follow the benchmark systems (Sec. 3: pentagon fluids) and the
workload list this library is measured on (regular pentagons of circumradius
0.5; unit cubes; replicas with N in [256, 8192] and packing fraction in
[0.40, 0.70]).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def regular_polygon(n: int, R: float = 0.5) -> np.ndarray:
    """Counter-clockwise regular n-gon of circumradius R, first vertex at +y."""
    k = np.arange(n)
    th = 0.5 * math.pi + 2.0 * math.pi * k / n
    return np.stack([R * np.cos(th), R * np.sin(th)], axis=1)


def cube(edge: float = 1.0) -> np.ndarray:
    h = 0.5 * edge
    return np.array([[sx * h, sy * h, sz * h]
                     for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)], dtype=np.float64)


def polygon_area(v: np.ndarray) -> float:
    x, y = v[:, 0], v[:, 1]
    return 0.5 * float(np.sum(x * np.roll(y, -1) - np.roll(x, -1) * y))


def dodecahedron(volume: float = 1.0) -> np.ndarray:
    """Regular dodecahedron (20 vertices) of the given volume, centred, in the
    standard orientation: the cube (+-1, +-1, +-1) and the cyclic
    permutations of (0, +-1/g, +-g), g the golden ratio, scaled."""
    g = (1.0 + math.sqrt(5.0)) / 2.0
    v = [(x, y, z) for x in (-1.0, 1.0) for y in (-1.0, 1.0) for z in (-1.0, 1.0)]
    for a in (-1.0, 1.0):
        for b in (-1.0, 1.0):
            v += [(0.0, a / g, b * g), (a / g, b * g, 0.0), (a * g, 0.0, b / g)]
    v = np.array(v)
    edge = 2.0 / g                                   # of the coordinates above
    vol = (15.0 + 7.0 * math.sqrt(5.0)) / 4.0 * edge ** 3
    return v * (volume / vol) ** (1.0 / 3.0)


def cube_volume(edge: float) -> float:
    return edge ** 3


def diameter(v: np.ndarray) -> float:
    d = v[:, None, :] - v[None, :, :]
    return float(np.sqrt((d * d).sum(-1)).max())


def circumradius(v: np.ndarray) -> float:
    return float(np.sqrt((v * v).sum(1)).max())


def box_length(N: int, particle_measure: float, phi: float, dim: int) -> float:
    """Side of a square/cubic box holding N shapes at packing fraction phi."""
    return (N * particle_measure / phi) ** (1.0 / dim)


def _tri_lattice_dims(N: int, L: float):
    """Columns/rows (rows even) of a triangular lattice in an L x L box with at
    least N sites and the largest nearest-site distance."""
    best = None
    ny0 = max(2, int(round(math.sqrt(N * 2.0 / math.sqrt(3.0)))))
    for ny in range(max(2, ny0 - 12), ny0 + 13):
        if ny % 2:
            continue
        nx = -(-N // ny)
        ax, ay = L / nx, L / ny
        # neighbours along a row, in the next row (offset by half a column)
        # and two rows apart (same column)
        dmin = min(ax, math.hypot(0.5 * ax, ay), 2.0 * ay)
        if best is None or dmin > best[0]:
            best = (dmin, nx, ny)
    return best


def triangular_lattice(N: int, L: float, rng: np.random.Generator, aligned: bool = False):
    """N sites of a periodic triangular lattice in [0,L)^2 (vacancies random).

    Returns (pos[N,2], orient[N,2], nearest_site_distance)."""
    dmin, nx, ny = _tri_lattice_dims(N, L)
    ax, ay = L / nx, L / ny
    j, i = np.divmod(np.arange(nx * ny, dtype=np.int64), nx)
    sites = np.stack([(i + 0.5 * (j % 2)) * ax, j * ay], axis=1)
    keep = np.sort(rng.permutation(sites.shape[0])[:N])
    pos = sites[keep]
    pos += rng.uniform(0.0, L, size=2)[None, :]          # random global offset
    pos = np.mod(pos, L)
    pos[pos >= L] = 0.0
    if aligned:
        ori = np.tile(np.array([1.0, 0.0]), (N, 1))
    else:
        th = rng.uniform(0.0, 2.0 * math.pi, size=N)
        ori = np.stack([np.cos(th), np.sin(th)], axis=1)
    return pos, ori, dmin


def cubic_lattice(N: int, L: float, rng: np.random.Generator):
    """N sites of a periodic simple cubic lattice in [0,L)^3, identity
    orientations.  Returns (pos[N,3], quat[N,4], spacing)."""
    n = -(-int(round(N ** (1.0 / 3.0))) // 1)
    while n ** 3 < N:
        n += 1
    a = L / n
    g = np.arange(n) * a
    sites = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    keep = np.sort(rng.permutation(sites.shape[0])[:N])
    pos = np.mod(sites[keep] + rng.uniform(0.0, L, size=3)[None, :], L)
    pos[pos >= L] = 0.0
    q = np.tile(np.array([1.0, 0.0, 0.0, 0.0]), (N, 1))
    return pos, q, a


def fcc_lattice(n: int, a: float, rng: np.random.Generator):
    """4 n^3 sites of a periodic face-centred cubic lattice of cubic cell a in
    [0, n a)^3 (random global offset), identity orientations.
    Returns (pos[4n^3, 3], quat[4n^3, 4])."""
    g = np.arange(n) * a
    corner = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    basis = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]]) * a
    sites = (corner[:, None, :] + basis[None, :, :]).reshape(-1, 3)
    L = n * a
    pos = np.mod(sites + rng.uniform(0.0, L, size=3)[None, :], L)
    pos[pos >= L] = 0.0
    q = np.tile(np.array([1.0, 0.0, 0.0, 0.0]), (pos.shape[0], 1))
    return pos, q


@dataclass
class System:
    """One replica: shape, box and a starting configuration."""
    name: str
    dim: int
    verts: np.ndarray
    L: np.ndarray
    pos: np.ndarray
    orient: np.ndarray
    phi: float
    seed: int
    d: float = 0.1
    a: float = 0.1
    nselect: int = 4
    w_min: float = 0.0
    notes: dict = field(default_factory=dict)

    @property
    def N(self):
        return self.pos.shape[0]


def pentagon_system(N: int, phi: float, seed: int, name: str = "pentagons",
                    d: float = 0.1, a: float = 0.1, nselect: int = 4, w_min: float = 0.0,
                    gen_seed: int | None = None) -> System:
    """Regular pentagons (circumradius 0.5) on an overlap-free lattice.

    Random orientations while the lattice spacing allows 2R; aligned shapes up
    to the diameter bound otherwise; raises if phi is beyond both."""
    v = regular_polygon(5, 0.5)
    A = polygon_area(v)
    L = box_length(N, A, phi, 2)
    rng = np.random.default_rng(seed if gen_seed is None else gen_seed)
    dmin, _, _ = _tri_lattice_dims(N, L)
    R = circumradius(v)
    if dmin >= 2.0 * R:
        pos, ori, dmin = triangular_lattice(N, L, rng, aligned=False)
        kind = "triangular lattice, random orientations (site distance >= 2R)"
    elif dmin >= diameter(v):
        pos, ori, dmin = triangular_lattice(N, L, rng, aligned=True)
        kind = "triangular lattice, aligned (site distance >= shape diameter)"
    else:
        raise ValueError(f"phi={phi} too dense for an overlap-free lattice start")
    return System(name=name, dim=2, verts=v, L=np.array([L, L]), pos=pos, orient=ori,
                  phi=phi, seed=seed, d=d, a=a, nselect=nselect, w_min=w_min,
                  notes={"init": kind, "site_distance": dmin})


def cube_system(N: int, phi: float, seed: int, name: str = "cubes", d: float = 0.1,
                a: float = 0.1, nselect: int = 4) -> System:
    v = cube(1.0)
    L = box_length(N, 1.0, phi, 3)
    rng = np.random.default_rng(seed)
    pos, q, a_sp = cubic_lattice(N, L, rng)
    if a_sp < 1.0:
        raise ValueError("cubic lattice spacing below the cube edge")
    return System(name=name, dim=3, verts=v, L=np.array([L, L, L]), pos=pos, orient=q,
                  phi=phi, seed=seed, d=d, a=a, nselect=nselect,
                  notes={"init": "simple cubic lattice, aligned (spacing >= edge)",
                         "spacing": a_sp})


# The 4096-pentagon fluid at area fraction 0.60: d = a = 0.165 gives a 30%
# acceptance ratio.  Found with tune.tune_scale (d/a fixed at 1, bisection on
# 100-sweep pilots) after a 3000-sweep melt from the lattice start at
# d = a = 0.2; the chain is implementation independent, so any sweep
# implementation reproduces it.
FLUID4096_D = 0.165
FLUID4096_A = 0.165


def fluid4096(seed: int = 42) -> System:
    """4096 regular pentagons, area fraction 0.60, moves sized for ~30% acceptance."""
    return pentagon_system(4096, 0.60, seed, name="pentagon fluid N=4096 phi=0.60",
                           d=FLUID4096_D, a=FLUID4096_A, nselect=4)


def replica_params(n_replicas: int = 512, gen_seed: int = 2024, n_lo: int = 256,
                   n_hi: int = 8192, phi_lo: float = 0.40, phi_hi: float = 0.70):
    """(N_r, phi_r, seed_r = 42 + r) for a batch of independent replicas.
    All N are drawn before all densities, so the densities of the first k
    replicas depend on the batch size (a shorter batch is not a prefix)."""
    rng = np.random.default_rng(gen_seed)
    Ns = rng.integers(n_lo, n_hi + 1, size=n_replicas)
    phis = rng.uniform(phi_lo, phi_hi, size=n_replicas)
    return [(int(Ns[r]), float(phis[r]), 42 + r) for r in range(n_replicas)]


def replica_systems(n_replicas: int = 512, gen_seed: int = 2024, **kw):
    return [pentagon_system(N, phi, seed, name=f"replica{r}", gen_seed=gen_seed * 100003 + r)
            for r, (N, phi, seed) in enumerate(replica_params(n_replicas, gen_seed, **kw))]


# 32768 cubes (edge 1) at volume fraction 0.50: d = a = 0.0817 gives a 30%
# acceptance ratio, found with tune.tune_scale (d/a fixed at 1, 100-sweep
# pilots) after a 1000-sweep melt from the simple cubic start at d = a = 0.1.
CUBES32768_D = 0.0817
CUBES32768_A = 0.0817


def cubes32768(seed: int = 42) -> System:
    """32768 cubes, volume fraction 0.50, moves sized for ~30% acceptance."""
    return cube_system(32768, 0.50, seed, name="cube fluid N=32768 phi=0.50",
                       d=CUBES32768_D, a=CUBES32768_A, nselect=4)


def cube_replica_params(n_replicas: int = 32, gen_seed: int = 2025, n_lo: int = 2048, n_hi: int = 16384,
                        phi_lo: float = 0.40, phi_hi: float = 0.55):
    """(N_r, phi_r, seed_r = 1000 + r) for a batch of independent cube
    replicas of uneven size and density (all N drawn before all densities)."""
    rng = np.random.default_rng(gen_seed)
    Ns = rng.integers(n_lo, n_hi + 1, size=n_replicas)
    phis = rng.uniform(phi_lo, phi_hi, size=n_replicas)
    return [(int(Ns[r]), float(phis[r]), 1000 + r) for r in range(n_replicas)]


def cube_replica_systems(n_replicas: int = 32, gen_seed: int = 2025, **kw):
    """Independent replicas of unit cubes on their simple cubic lattices, with
    the 32768-cube system's move sizes (acceptance then varies with density)."""
    return [cube_system(N, phi, seed, name=f"cube replica{r}", d=CUBES32768_D, a=CUBES32768_A, nselect=4)
            for r, (N, phi, seed) in enumerate(cube_replica_params(n_replicas, gen_seed, **kw))]


# The large 2D system: 2^24 pentagons at area fraction 0.60 with cells no
# narrower than 1.99, i.e. a 2048 x 2048 cell list (about 4 shapes per cell).
# Same shape and density as the 4096-pentagon fluid, so the same move sizes
# give the same ~30% acceptance.
LARGE2D_N = 1 << 24
LARGE2D_W_MIN = 1.99


def large2d(seed: int = 42, N: int = LARGE2D_N) -> System:
    """2^24 regular pentagons, area fraction 0.60, 2048^2 cells of width >= 1.99."""
    return pentagon_system(N, 0.60, seed, name=f"pentagon fluid N={N} phi=0.60 w_min=1.99",
                           d=FLUID4096_D, a=FLUID4096_A, nselect=4, w_min=LARGE2D_W_MIN)


def dodecahedron_system(n: int = 20, phi: float = 0.50, seed: int = 42, d: float = 0.1, a: float = 0.1,
                        nselect: int = 4) -> System:
    """4 n^3 unit-volume regular dodecahedra at volume fraction phi, aligned in
    the standard orientation on an FCC lattice (cubic cell (4 / phi)^(1/3);
    at phi = 0.5 its nearest-site distance 1.414 keeps aligned shapes apart,
    which tests check with the oracle)."""
    v = dodecahedron(1.0)
    cell = (4.0 / phi) ** (1.0 / 3.0)
    rng = np.random.default_rng(seed)
    pos, q = fcc_lattice(n, cell, rng)
    L = n * cell
    return System(name=f"dodecahedra N={pos.shape[0]} phi={phi}", dim=3, verts=v, L=np.array([L, L, L]),
                  pos=pos, orient=q, phi=phi, seed=seed, d=d, a=a, nselect=nselect,
                  notes={"init": "FCC lattice, aligned (standard orientation)"})


# 32000 unit-volume dodecahedra at volume fraction 0.50 (the paper's 3D
# benchmark shape and density): d = a = 0.087 gives a 30% acceptance ratio,
# found with tune.tune_scale (d/a fixed at 1, 100-sweep pilots) after a
# 1000-sweep melt from the FCC start at d = a = 0.1.
DODECA_D = 0.087
DODECA_A = 0.087


def dodecahedra32000(seed: int = 42) -> System:
    """32000 unit-volume regular dodecahedra, volume fraction 0.50."""
    return dodecahedron_system(20, 0.50, seed, d=DODECA_D, a=DODECA_A, nselect=4)


def disk_system(N: int, phi: float, seed: int, sigma: float = 1.0, d: float = 0.1, nselect: int = 4,
                w_min: float = 0.0) -> System:
    """N hard disks of diameter sigma at area fraction phi on a triangular
    lattice (site distance >= sigma up to phi = 0.9069); orientations (1, 0)
    (carried, irrelevant to the overlap).  verts is the radius (a scalar)."""
    area = math.pi * 0.25 * sigma * sigma
    L = box_length(N, area, phi, 2)
    rng = np.random.default_rng(seed)
    pos, ori, dmin = triangular_lattice(N, L, rng, aligned=True)
    if dmin < sigma:
        raise ValueError(f"phi={phi} too dense for an overlap-free lattice start")
    return System(name=f"disks N={N} phi={phi}", dim=2, verts=np.array(0.5 * sigma), L=np.array([L, L]),
                  pos=pos, orient=ori, phi=phi, seed=seed, d=d, a=0.0, nselect=nselect, w_min=w_min,
                  notes={"init": "triangular lattice", "site_distance": dmin})


def sphere_system(n: int, phi: float, seed: int, sigma: float = 1.0, d: float = 0.1, nselect: int = 4,
                  w_min: float = 0.0) -> System:
    """4 n^3 hard spheres of diameter sigma at volume fraction phi on an FCC
    lattice (nearest-site distance >= sigma up to phi = 0.7405)."""
    vol = math.pi / 6.0 * sigma ** 3
    cell = (4.0 * vol / phi) ** (1.0 / 3.0)
    if cell / math.sqrt(2.0) < sigma:
        raise ValueError(f"phi={phi} too dense for an overlap-free FCC start")
    rng = np.random.default_rng(seed)
    pos, q = fcc_lattice(n, cell, rng)
    L = n * cell
    return System(name=f"spheres N={pos.shape[0]} phi={phi}", dim=3, verts=np.array(0.5 * sigma),
                  L=np.array([L, L, L]), pos=pos, orient=q, phi=phi, seed=seed, d=d, a=0.0,
                  nselect=nselect, w_min=w_min, notes={"init": "FCC lattice"})
