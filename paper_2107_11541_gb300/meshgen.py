"""Seeded synthetic meshes and fields shaped like the paper's combustion workloads.

This module only generates inputs (node coordinates, connectivity, nodal fields).
It contains none of the finite-element arithmetic, so both the FP64 oracle and the
CUDA path can consume its output without sharing any method code.

Meshes
------
* Unit cube split into an ``n^3`` grid of cells, node id ``i + M*j + M^2*k``
  (``M`` nodes per axis).
* Tet4: Kuhn split of each cube into 6 tetrahedra.  Cube ``(i,j,k)`` with corner
  ``c`` gives, for each axis permutation ``sigma`` (lexicographic order), the
  tet ``c, c+e_s0, c+e_s0+e_s1, c+(1,1,1)``; odd permutations swap the 2nd and
  3rd vertex so every tet is positively oriented.  Element id = ``6*cube + p``.
* Hex8: node ``a = i + 2j + 4k`` of an element is the grid node at offset
  ``(i,j,k)``.
* Hex27: element ``(ex,ey,ez)`` owns grid nodes ``(2ex+i, 2ey+j, 2ez+k)``,
  local node ``a = i + 3j + 9k``.
* Pen6: each cube is split into two prisms whose triangles lie in x = const planes
  (cut along the diagonal from (y1, z0) to (y0, z1)) and are extruded along x;
  local nodes 0-2 on the face x0, 3-5 the same vertices on x1.
* Pyr5: each cube gets a centre node (ids after the grid nodes) and is split into
  six pyramids, one per face, base corners counter-clockwise seen from the centre
  (the apex, local node 4).
* Mixed: the cells with k < n/3 are Hex8, n/3 <= k < 2n/3 Pyr5, the rest Pen6; the
  interfaces between the layers are the quads of all three types.

Fields
------
velocity ``u = (sin(pi x) cos(pi y), -cos(pi x) sin(pi y), 0.1)`` at the nodes,
diffusivity ``k ~ lognormal(-4, 0.5)``, reaction ``s ~ U[0, s_max]``, previous
step ``phi ~ U[0, 1]``, per node and per equation; ``dt = 1e-3``.

Random draws use ``numpy.random.default_rng(11541 + config_index)`` in this
order: interior perturbation (N x 3), node permutation, element permutation,
then for each equation k, s, phi.
"""
from __future__ import annotations

import dataclasses
import itertools

import numpy as np

TET4, HEX8, HEX27, PEN6, PYR5 = 0, 1, 2, 3, 4
NEN = {TET4: 4, HEX8: 8, HEX27: 27, PEN6: 6, PYR5: 5}
NAMES = {TET4: "tet4", HEX8: "hex8", HEX27: "hex27", PEN6: "pen6", PYR5: "pyr5"}
SEED_BASE = 11541
DT = 1e-3


@dataclasses.dataclass
class Mesh:
    elem_type: int
    coords: np.ndarray   # (N, 3) float64
    conn: np.ndarray     # (E, nen) int32, 0-based
    n_cells: int         # cells per axis of the generating grid
    h: float             # grid cell width

    @property
    def n_node(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elem(self) -> int:
        return int(self.conn.shape[0])


@dataclasses.dataclass
class Fields:
    velocity: np.ndarray     # (3, N)   SoA
    diffusivity: np.ndarray  # (n_eq, N)
    reaction: np.ndarray     # (n_eq, N)
    phi_old: np.ndarray      # (n_eq, N)
    dt: float = DT

    @property
    def n_eq(self) -> int:
        return int(self.diffusivity.shape[0])

    def astype(self, dtype) -> "Fields":
        return Fields(self.velocity.astype(dtype), self.diffusivity.astype(dtype),
                      self.reaction.astype(dtype), self.phi_old.astype(dtype), self.dt)


def grid_nodes(m: int, z_faces: np.ndarray | None = None) -> np.ndarray:
    """(m^3, 3) coordinates of a uniform grid with m nodes per axis on [0,1]^3."""
    t = np.linspace(0.0, 1.0, m)
    tz = t if z_faces is None else z_faces
    z, y, x = np.meshgrid(tz, t, t, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def _cell_origins(n: int, m: int, stride: int) -> np.ndarray:
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return (stride * i + stride * m * j + stride * m * m * k).ravel().astype(np.int64)


def kuhn_tets(n: int) -> np.ndarray:
    m = n + 1
    base = _cell_origins(n, m, 1)
    off = [1, m, m * m]
    conn = np.empty((n ** 3, 6, 4), dtype=np.int64)
    for p, sigma in enumerate(itertools.permutations(range(3))):
        v0 = np.zeros_like(base)
        v1 = v0 + off[sigma[0]]
        v2 = v1 + off[sigma[1]]
        v3 = np.full_like(base, 1 + m + m * m)
        # parity of the permutation: number of inversions
        inv = sum(1 for a in range(3) for b in range(a + 1, 3) if sigma[a] > sigma[b])
        if inv % 2 == 1:
            v1, v2 = v2, v1
        conn[:, p, 0] = base + v0
        conn[:, p, 1] = base + v1
        conn[:, p, 2] = base + v2
        conn[:, p, 3] = base + v3
    return conn.reshape(-1, 4).astype(np.int32)


def hex_conn(n: int, order: int) -> np.ndarray:
    m = order * n + 1
    base = _cell_origins(n, m, order)
    q = order + 1
    offs = [i + m * j + m * m * k for k in range(q) for j in range(q) for i in range(q)]
    return (base[:, None] + np.asarray(offs, dtype=np.int64)[None, :]).astype(np.int32)


# grid offsets (dx, dy, dz) of the two prisms of a cube and of the six pyramid bases
PRISMS = (((0, 0, 0), (0, 1, 0), (0, 0, 1), (1, 0, 0), (1, 1, 0), (1, 0, 1)),
          ((0, 1, 0), (0, 1, 1), (0, 0, 1), (1, 1, 0), (1, 1, 1), (1, 0, 1)))
PYRAMID_BASES = (((0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0)),   # z0, inward normal +z
                 ((0, 0, 1), (0, 1, 1), (1, 1, 1), (1, 0, 1)),   # z1
                 ((0, 0, 0), (0, 0, 1), (1, 0, 1), (1, 0, 0)),   # y0
                 ((0, 1, 0), (1, 1, 0), (1, 1, 1), (0, 1, 1)),   # y1
                 ((0, 0, 0), (0, 1, 0), (0, 1, 1), (0, 0, 1)),   # x0
                 ((1, 0, 0), (1, 0, 1), (1, 1, 1), (1, 1, 0)))   # x1


def _offsets(m: int, pts) -> np.ndarray:
    return np.asarray([dx + m * dy + m * m * dz for dx, dy, dz in pts], dtype=np.int64)


def prism_conn(base: np.ndarray, m: int) -> np.ndarray:
    conn = np.stack([base[:, None] + _offsets(m, p)[None, :] for p in PRISMS], axis=1)
    return conn.reshape(-1, 6).astype(np.int32)


def pyramid_conn(base: np.ndarray, m: int, centre: np.ndarray) -> np.ndarray:
    conn = np.empty((base.size, 6, 5), dtype=np.int64)
    for f, quad in enumerate(PYRAMID_BASES):
        conn[:, f, :4] = base[:, None] + _offsets(m, quad)[None, :]
        conn[:, f, 4] = centre
    return conn.reshape(-1, 5).astype(np.int32)


def cell_centres(n: int, cells: np.ndarray) -> np.ndarray:
    """Centres of the cells with the given indices (k slowest) of the n^3 grid on [0,1]^3."""
    k, rem = np.divmod(cells, n * n)
    j, i = np.divmod(rem, n)
    return (np.stack([i, j, k], axis=1) + 0.5) / n


def structured_mesh(elem_type: int, n: int, z_faces: np.ndarray | None = None) -> Mesh:
    order = 2 if elem_type == HEX27 else 1
    m = order * n + 1
    coords = grid_nodes(m, z_faces)
    if elem_type == TET4:
        conn = kuhn_tets(n)
    elif elem_type == PEN6:
        conn = prism_conn(_cell_origins(n, m, 1), m)
    elif elem_type == PYR5:
        cells = np.arange(n ** 3)
        conn = pyramid_conn(_cell_origins(n, m, 1), m, m ** 3 + cells)
        centres = cell_centres(n, cells)
        if z_faces is not None:  # the centre of each cell between its own z faces
            k = cells // (n * n)
            centres[:, 2] = 0.5 * (np.asarray(z_faces)[k] + np.asarray(z_faces)[k + 1])
        coords = np.concatenate([coords, centres])
    else:
        conn = hex_conn(n, order)
    return Mesh(elem_type, coords, conn, n, 1.0 / n)


@dataclasses.dataclass
class MixedMesh:
    """A mesh of element blocks of different types sharing one node set."""
    coords: np.ndarray   # (N, 3) float64
    blocks: list         # [(elem_type, conn (E_b, nen_b) int32)]
    n_cells: int
    h: float

    @property
    def n_node(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elem(self) -> int:
        return int(sum(c.shape[0] for _, c in self.blocks))


def mixed_mesh(n: int) -> MixedMesh:
    """Unit cube, n^3 cells: Hex8 cells below z = 1/3, Pyr5 cells (six pyramids around a
    centre node) up to z = 2/3, Pen6 cells (two prisms) above; n >= 3."""
    if n < 3:
        raise ValueError("a mixed mesh needs n >= 3 cells per axis")
    m = n + 1
    base = _cell_origins(n, m, 1)
    k1, k2 = n // 3, (2 * n) // 3
    hexes = base[: k1 * n * n]
    pyr_cells = np.arange(k1 * n * n, k2 * n * n)
    prisms = base[k2 * n * n:]
    centres = cell_centres(n, pyr_cells)
    coords = np.concatenate([grid_nodes(m), centres])
    blocks = [(HEX8, (hexes[:, None] + _offsets(m, [(i, j, k) for k in range(2) for j in range(2)
                                                    for i in range(2)])[None, :]).astype(np.int32)),
              (PYR5, pyramid_conn(base[pyr_cells], m, m ** 3 + np.arange(pyr_cells.size))),
              (PEN6, prism_conn(prisms, m))]
    return MixedMesh(coords, blocks, n, 1.0 / n)


def interior_mask(mesh: Mesh) -> np.ndarray:
    c = mesh.coords
    return np.all((c > 0.0) & (c < 1.0), axis=1)


def perturb_interior(mesh: Mesh, rng: np.random.Generator, frac: float, move_z: bool = True) -> None:
    """Move interior nodes by U[-frac*h, frac*h] per coordinate (boundary stays planar);
    with move_z False the z displacement is drawn but not applied (meshes whose z spacing
    is not uniform, where h-sized moves in z would invert the thin cells)."""
    d = rng.uniform(-frac * mesh.h, frac * mesh.h, size=mesh.coords.shape)
    if not move_z:
        d[:, 2] = 0.0
    mask = interior_mask(mesh)
    if frac > 0.0:
        mesh.coords[mask] += d[mask]


def permute_nodes(mesh: Mesh, perm: np.ndarray) -> None:
    """Relabel node ``i`` as ``perm[i]``."""
    new = np.empty_like(mesh.coords)
    new[perm] = mesh.coords
    mesh.coords = new
    mesh.conn = perm[mesh.conn].astype(np.int32)


def permute_elements(mesh: Mesh, perm: np.ndarray) -> None:
    """Element ``e`` moves to position ``perm[e]``."""
    new = np.empty_like(mesh.conn)
    new[perm] = mesh.conn
    mesh.conn = new


def velocity_field(coords: np.ndarray) -> np.ndarray:
    x, y = coords[:, 0], coords[:, 1]
    u = np.empty((3, coords.shape[0]))
    u[0] = np.sin(np.pi * x) * np.cos(np.pi * y)
    u[1] = -np.cos(np.pi * x) * np.sin(np.pi * y)
    u[2] = 0.1
    return u


def draw_fields(rng: np.random.Generator, coords: np.ndarray, n_eq: int, s_max: float,
                dt: float = DT, dtype=np.float64) -> Fields:
    """The seeded nodal fields; dtype=float32 rounds each draw as it is made (the same values as
    drawing in float64 and rounding afterwards, without the float64 arrays)."""
    n = coords.shape[0]
    k = np.empty((n_eq, n), dtype=dtype)
    s = np.empty((n_eq, n), dtype=dtype)
    p = np.empty((n_eq, n), dtype=dtype)
    for q in range(n_eq):
        k[q] = rng.lognormal(-4.0, 0.5, size=n)
        s[q] = rng.uniform(0.0, s_max, size=n)
        p[q] = rng.uniform(0.0, 1.0, size=n)
    return Fields(velocity_field(coords).astype(dtype), k, s, p, dt)


def step_params(n_steps: int, n_eq: int, seed: int = SEED_BASE + 1000) -> np.ndarray:
    """Parameters of the per-step field perturbation, float32 [n_steps][n_eq][5]:
    amplitude A ~ U[0.01, 0.05], wave vector k = 2 pi f d with f ~ U[0.5, 2] and d a
    uniformly random unit direction, phase psi ~ U[0, 2 pi)."""
    rng = np.random.default_rng(seed)
    out = np.empty((n_steps, n_eq, 5))
    for s in range(n_steps):
        for q in range(n_eq):
            d = rng.normal(size=3)
            d /= np.linalg.norm(d)
            f = rng.uniform(0.5, 2.0)
            out[s, q, 0] = rng.uniform(0.01, 0.05)
            out[s, q, 1:4] = 2.0 * np.pi * f * d
            out[s, q, 4] = rng.uniform(0.0, 2.0 * np.pi)
    return out.astype(np.float32)


@dataclasses.dataclass
class Workload:
    name: str
    mesh: Mesh
    fields: Fields
    precision: str  # "f64" or "f32"


# Workloads shaped like the paper's: (type, cells/axis, perturbation, permute, n_eq, s_max, precision)
CONFIGS = {
    0: dict(name="tet4_10_f64_1eq", elem_type=TET4, n=10, frac=0.0, permute=False, n_eq=1, s_max=10.0, precision="f64"),
    1: dict(name="tet4_100_perm_1eq", elem_type=TET4, n=100, frac=0.2, permute=True, n_eq=1, s_max=10.0, precision="f32"),
    2: dict(name="hex8_128_21eq", elem_type=HEX8, n=128, frac=0.15, permute=False, n_eq=21, s_max=50.0, precision="f32"),
    3: dict(name="hex27_48_11eq", elem_type=HEX27, n=48, frac=0.0, permute=False, n_eq=11, s_max=50.0, precision="f32"),
    4: dict(name="hex8_256_32eq", elem_type=HEX8, n=256, frac=0.15, permute=False, n_eq=32, s_max=50.0, precision="f32"),
}


def make_workload(index: int, n: int | None = None, n_eq: int | None = None, seed: int | None = None,
                  stretched_slab: bool = False, dtype=np.float64) -> Workload:
    """Build workload ``index`` (optionally shrunk: ``n`` cells per axis, ``n_eq`` equations).

    ``stretched_slab`` compresses the middle layer of cells in z to 1e-4 of its width
    (aspect ratio 1e4), which makes the Jacobians of that layer badly conditioned.
    ``dtype`` is the dtype of the fields (float32: the values the FP32 path consumes).
    """
    cfg = dict(CONFIGS[index])
    if n is not None:
        cfg["n"] = n
    if n_eq is not None:
        cfg["n_eq"] = n_eq
    mesh, rng = _workload_mesh(index, cfg, seed, stretched_slab)
    fields = draw_fields(rng, mesh.coords, cfg["n_eq"], cfg["s_max"], dtype=dtype)
    return Workload(cfg["name"] if n is None and n_eq is None else f"{cfg['name']}_n{mesh.n_cells}_q{cfg['n_eq']}",
                    mesh, fields, cfg["precision"])


def make_mesh(index: int, n: int | None = None) -> Mesh:
    """The mesh of workload ``index`` alone (the same draws as ``make_workload``, no fields)."""
    cfg = dict(CONFIGS[index])
    if n is not None:
        cfg["n"] = n
    return _workload_mesh(index, cfg, None, False)[0]


def _workload_mesh(index: int, cfg: dict, seed: int | None, stretched_slab: bool):
    rng = np.random.default_rng(SEED_BASE + index if seed is None else seed)
    z_faces = None
    et, nc = cfg["elem_type"], cfg["n"]
    if stretched_slab:
        order = 2 if et == HEX27 else 1
        widths = np.ones(nc)
        widths[nc // 2] = 1e-4
        widths /= widths.sum()
        faces = np.concatenate([[0.0], np.cumsum(widths)])
        faces[-1] = 1.0
        if order == 2:
            mids = 0.5 * (faces[:-1] + faces[1:])
            zf = np.empty(2 * nc + 1)
            zf[0::2] = faces
            zf[1::2] = mids
            faces = zf
        z_faces = faces
    mesh = structured_mesh(et, nc, z_faces)
    if cfg["frac"] > 0.0:
        perturb_interior(mesh, rng, cfg["frac"], move_z=not stretched_slab)
    else:
        rng.uniform(size=mesh.coords.shape)  # keep the draw order fixed
    if cfg["permute"]:
        permute_nodes(mesh, rng.permutation(mesh.n_node).astype(np.int64))
        permute_elements(mesh, rng.permutation(mesh.n_elem).astype(np.int64))
    return mesh, rng


def single_element(elem_type: int, rng: np.random.Generator | None = None, distort: float = 0.0,
                   scale: float = 1.0) -> Mesh:
    """One element on [0, scale]^3 (Tet4: the first Kuhn tet), optionally distorted."""
    mesh = structured_mesh(elem_type, 1)
    if elem_type == TET4:
        mesh.conn = mesh.conn[:1]
    mesh.coords *= scale
    if distort > 0.0 and rng is not None:
        mesh.coords += rng.uniform(-distort * scale, distort * scale, size=mesh.coords.shape)
    return mesh

