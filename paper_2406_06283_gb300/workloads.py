"""Seeded synthetic inputs for the Helmholtz solver: meshes, coefficient fields,
element partitions and right-hand sides.

This module holds none of the method's arithmetic (no assembly, no
decomposition, no eigen or Krylov work).  It only lays out the problems the
solver is run on, so that the CPU oracle and the CUDA library receive the
same bytes.  It imports nothing from the rest of the package.

Random numbers come from one counter-based generator, SplitMix64 (Steele,
Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
draw i of stream s is mix(s + (i + 1) * 0x9E3779B97F4A7C15), where mix is the
SplitMix64 finaliser.  Uniforms on [0, 1) take the top 53 bits; normals use
the Box-Muller transform on two uniforms.  A stream seed is derived from
integers (config id, instance, purpose, index) by chained mixing.

Meshes (the paper allows any shape-regular simplicial mesh, Sec. 2.1):
  * 2D: the unit square cut into C x C cells, each cell split by the diagonal
    from its lower-left to its upper-right corner into two right triangles.
  * 3D: the unit cube cut into C^3 cubes, each split into the 6 Kuhn
    tetrahedra that share the cube's main diagonal.
Nodes on the boundary carry the homogeneous Dirichlet condition of Eq. (1.1)
and are flagged; they are not degrees of freedom.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def stream_seed(*keys: int) -> int:
    """Fold integer keys into one 64-bit stream seed."""
    s = np.array([0x243F6A8885A308D3], dtype=np.uint64)
    for k in keys:
        with np.errstate(over="ignore"):
            s = _mix(s ^ np.uint64(int(k) & 0xFFFFFFFFFFFFFFFF)) + _GOLDEN
    return int(s[0])


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the SplitMix64 stream `seed`."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(seed) + idx * _GOLDEN
    return _mix(state)


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int) -> np.ndarray:
    """Box-Muller: pairs (u1, u2) -> sqrt(-2 ln(1 - u1)) cos(2 pi u2)."""
    u = uniform(seed, 2 * count)
    u1, u2 = u[0::2], u[1::2]
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)


@dataclass
class Mesh:
    """Simplicial mesh: `dim`-dimensional node coordinates, (dim+1)-node elements."""
    dim: int
    xyz: np.ndarray            # (n_nodes, dim) float64
    elems: np.ndarray          # (n_elems, dim+1) int32, 0-based
    is_boundary: np.ndarray    # (n_nodes,) uint8, 1 = Dirichlet node
    cells: int                 # cells per side of the structured generator
    elem_cell: np.ndarray      # (n_elems, dim) int32 cell coordinates of each element

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.elems.shape[0])

    @property
    def n_dofs(self) -> int:
        return int(self.n_nodes - int(self.is_boundary.sum()))


def square_mesh(cells: int) -> Mesh:
    """Unit square, `cells` x `cells` cells, each split along its '/' diagonal."""
    C = int(cells)
    j, i = np.meshgrid(np.arange(C + 1), np.arange(C + 1), indexing="ij")
    xyz = np.stack([i.ravel() / C, j.ravel() / C], axis=1).astype(np.float64)
    nid = lambda a, b: b * (C + 1) + a  # noqa: E731
    cy, cx = np.meshgrid(np.arange(C), np.arange(C), indexing="ij")
    cx, cy = cx.ravel(), cy.ravel()
    n00, n10, n11, n01 = nid(cx, cy), nid(cx + 1, cy), nid(cx + 1, cy + 1), nid(cx, cy + 1)
    lower = np.stack([n00, n10, n11], axis=1)
    upper = np.stack([n00, n11, n01], axis=1)
    elems = np.stack([lower, upper], axis=1).reshape(-1, 3).astype(np.int32)
    cell = np.stack([cx, cy], axis=1)
    elem_cell = np.repeat(cell, 2, axis=0).astype(np.int32)
    ii, jj = i.ravel(), j.ravel()
    bnd = ((ii == 0) | (ii == C) | (jj == 0) | (jj == C)).astype(np.uint8)
    return Mesh(2, xyz, elems, bnd, C, elem_cell)


def cube_mesh(cells: int) -> Mesh:
    """Unit cube, `cells`^3 cubes, each split into 6 Kuhn tetrahedra."""
    C = int(cells)
    k, j, i = np.meshgrid(np.arange(C + 1), np.arange(C + 1), np.arange(C + 1), indexing="ij")
    xyz = np.stack([i.ravel() / C, j.ravel() / C, k.ravel() / C], axis=1).astype(np.float64)
    nid = lambda a, b, c: (c * (C + 1) + b) * (C + 1) + a  # noqa: E731
    cz, cy, cx = np.meshgrid(np.arange(C), np.arange(C), np.arange(C), indexing="ij")
    cx, cy, cz = cx.ravel(), cy.ravel(), cz.ravel()
    tets = []
    for perm in itertools.permutations(range(3)):
        off = np.zeros(3, dtype=np.int64)
        path = [nid(cx, cy, cz)]
        for ax in perm:
            off[ax] += 1
            path.append(nid(cx + off[0], cy + off[1], cz + off[2]))
        tets.append(np.stack(path, axis=1))
    elems = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    cell = np.stack([cx, cy, cz], axis=1)
    elem_cell = np.repeat(cell, 6, axis=0).astype(np.int32)
    ii, jj, kk = i.ravel(), j.ravel(), k.ravel()
    bnd = ((ii == 0) | (ii == C) | (jj == 0) | (jj == C) | (kk == 0) | (kk == C)).astype(np.uint8)
    return Mesh(3, xyz, elems, bnd, C, elem_cell)


def box_partition(mesh: Mesh, parts: int) -> np.ndarray:
    """Non-overlapping element partition into parts^dim boxes of cells.

    Cell coordinate c maps to box floor(c * parts / cells) along each axis
    (uneven when parts does not divide cells).  Box ids are lexicographic
    with the first axis fastest.
    """
    P, C = int(parts), mesh.cells
    b = (mesh.elem_cell.astype(np.int64) * P) // C
    sub = np.zeros(mesh.n_elems, dtype=np.int64)
    for ax in reversed(range(mesh.dim)):
        sub = sub * P + b[:, ax]
    return sub.astype(np.int32)


def checkerboard(mesh: Mesh, blocks: int, seed: int, lo_exp: float = 0.0, hi_exp: float = 2.0) -> np.ndarray:
    """Per-element scalar coefficient 10^U[lo_exp, hi_exp], constant on each
    of blocks^dim blocks of cells (each block drawn independently)."""
    B, C = int(blocks), mesh.cells
    bc = (mesh.elem_cell.astype(np.int64) * B) // C
    bid = np.zeros(mesh.n_elems, dtype=np.int64)
    for ax in reversed(range(mesh.dim)):
        bid = bid * B + bc[:, ax]
    vals = 10.0 ** (lo_exp + (hi_exp - lo_exp) * uniform(seed, B ** mesh.dim))
    return vals[bid]


def layered(mesh: Mesh, layers: int, seed: int, lo: float = 0.5, hi: float = 2.0) -> np.ndarray:
    """Per-element scalar coefficient, constant on `layers` horizontal layers
    of cell rows (along the last axis), each U[lo, hi]."""
    L, C = int(layers), mesh.cells
    lid = (mesh.elem_cell[:, mesh.dim - 1].astype(np.int64) * L) // C
    vals = lo + (hi - lo) * uniform(seed, L)
    return vals[lid]


@dataclass
class Problem:
    """One Helmholtz instance: mesh, coefficient a_T per element, wavenumber,
    partition, and the solver parameters that go with it."""
    name: str
    mesh: Mesh
    coeff: np.ndarray
    k: float
    parts: int
    elem_to_sub: np.ndarray
    overlap: int = 2
    tau: float = 0.5
    restart: int = 50
    max_iters: int = 1000
    tol: float = 1e-8
    rhs: np.ndarray = field(default=None)          # (n_rhs, n_dofs) load vectors, or None
    f_nodal: np.ndarray = field(default=None)      # (n_nodes,) nodal source when the load vector is assembled

    @property
    def n_sub(self) -> int:
        return int(self.parts ** self.mesh.dim)


def config_c1() -> Problem:
    """h = 1/64 '/' mesh (3,969 dofs), a = 1, k = 20, f = 1, 4x4 boxes, overlap 2, tau 0.5."""
    m = square_mesh(64)
    return Problem("c1_h64_k20_p4", m, np.ones(m.n_elems), 20.0, 4, box_partition(m, 4),
                   f_nodal=np.ones(m.n_nodes))


def config_c2() -> Problem:
    """h = 1/256 (65,025 dofs), k = 50, 8x8 checkerboard a in 10^U[0,2], 8x8 boxes, N(0,1) rhs."""
    m = square_mesh(256)
    a = checkerboard(m, 8, stream_seed(2, 0, 1))
    rhs = normal(stream_seed(2, 0, 2, 0), m.n_dofs)[None, :]
    return Problem("c2_h256_k50_p8", m, a, 50.0, 8, box_partition(m, 8), rhs=rhs)


def config_c3(n_rhs: int = 16) -> Problem:
    """h = 1/512 (261,121 dofs), k = 100, 16 layers a in U[0.5,2], 16x16 boxes, 16 N(0,1) rhs."""
    m = square_mesh(512)
    a = layered(m, 16, stream_seed(3, 0, 1))
    rhs = np.stack([normal(stream_seed(3, 0, 2, r), m.n_dofs) for r in range(n_rhs)])
    return Problem("c3_h512_k100_p16", m, a, 100.0, 16, box_partition(m, 16), rhs=rhs)


def config_c4(seed: int = 4, n_instances: int = 64):
    """Batched workload: 64 independent 2D instances.  h = 1/cells with cells uniform in
    {128, 192, 256, 384}, k ~ U[20, 80], 8x8 checkerboard a in 10^U[0,2], P x P boxes with P uniform in
    [4, 12], overlap 2, s ~ U{1..8} seeded N(0,1) right-hand sides each."""
    out, meshes = [], {}
    choices = [128, 192, 256, 384]
    for i in range(n_instances):
        u = uniform(stream_seed(seed, i, 0), 4)
        cells = choices[min(int(u[0] * len(choices)), len(choices) - 1)]
        k = 20.0 + 60.0 * float(u[1])
        P = 4 + min(int(u[2] * 9), 8)
        s = 1 + min(int(u[3] * 8), 7)
        m = meshes.setdefault(cells, square_mesh(cells))
        a = checkerboard(m, 8, stream_seed(seed, i, 1))
        rhs = np.stack([normal(stream_seed(seed, i, 2, r), m.n_dofs) for r in range(s)])
        out.append(Problem(f"c4_{i:02d}_h{cells}_k{k:.1f}_p{P}_s{s}", m, a, k, P, box_partition(m, P), rhs=rhs))
    return out


def config_c5(seed: int = 5, pool: int = 8):
    """Serving workload: 24 operators and a request-stream recipe.

    16 operators in 2D: h = 1/cells with cells uniform in {128, 192, 256, 384, 512}, k ~ U[20, 100],
    an 8x8 checkerboard a in 10^U[0,2], P x P boxes with P = ceil(k / 6), so that H k <= 6, overlap 2.
    8 operators in 3D: unit cube, Kuhn tetrahedra, h = 1/32 (29,791 dofs), k = 20, 4x4x4 boxes,
    a from a 4x4x4 checkerboard.  Each operator carries `pool` seeded N(0,1) right-hand sides that
    the requests of serving_stream draw from.
    """
    ops, meshes = [], {}
    choices = [128, 192, 256, 384, 512]
    for i in range(16):
        u = uniform(stream_seed(seed, i, 0), 2)
        cells = choices[min(int(u[0] * len(choices)), len(choices) - 1)]
        k = 20.0 + 80.0 * float(u[1])
        P = int(math.ceil(k / 6.0))
        m = meshes.setdefault(cells, square_mesh(cells))
        a = checkerboard(m, 8, stream_seed(seed, i, 1))
        rhs = np.stack([normal(stream_seed(seed, i, 2, r), m.n_dofs) for r in range(pool)])
        ops.append(Problem(f"c5_op{i:02d}_2d_h{cells}_k{k:.1f}_p{P}", m, a, k, P, box_partition(m, P), rhs=rhs))
    cube = cube_mesh(32)
    for i in range(16, 24):
        a = checkerboard(cube, 4, stream_seed(seed, i, 1))
        rhs = np.stack([normal(stream_seed(seed, i, 2, r), cube.n_dofs) for r in range(pool)])
        ops.append(Problem(f"c5_op{i:02d}_3d_h32_k20_p4", cube, a, 20.0, 4, box_partition(cube, 4), rhs=rhs))
    return ops


def serving_stream(n_ops: int, n_requests: int, rate: float, seed: int = 5, pool: int = 8, max_rhs: int = 4):
    """Poisson arrivals: exponential inter-arrival times of mean 1/rate seconds, operator uniform,
    s ~ U{1..max_rhs} right-hand sides drawn (seeded) from the operator's pool.
    Returns a list of (arrival_s, op_index, rhs_indices)."""
    u = uniform(stream_seed(seed, 1000, int(rate * 1000)), 3 * n_requests + pool * max_rhs * n_requests)
    t, out = 0.0, []
    for q in range(n_requests):
        t += -math.log(max(1.0 - float(u[3 * q]), 1e-300)) / rate
        op = min(int(u[3 * q + 1] * n_ops), n_ops - 1)
        s = 1 + min(int(u[3 * q + 2] * max_rhs), max_rhs - 1)
        base = 3 * n_requests + q * max_rhs
        idx = [min(int(u[base + r] * pool), pool - 1) for r in range(s)]
        out.append((t, op, idx))
    return out


def small_problem(cells: int = 16, parts: int = 2, k: float = 6.0, overlap: int = 1,
                  seed: int = 7, n_rhs: int = 1, checker: int = 0, tau: float = 0.5) -> Problem:
    """A small seeded 2D case for parity tests that the oracle finishes in seconds."""
    m = square_mesh(cells)
    a = np.ones(m.n_elems) if checker == 0 else checkerboard(m, checker, stream_seed(seed, 0, 1))
    rhs = np.stack([normal(stream_seed(seed, 0, 2, r), m.n_dofs) for r in range(n_rhs)])
    return Problem(f"small_h{cells}_k{k:g}_p{parts}_ov{overlap}", m, a, float(k), parts,
                   box_partition(m, parts), overlap=overlap, tau=tau, rhs=rhs)


def small_problem_3d(cells: int = 8, parts: int = 2, k: float = 4.0, overlap: int = 1,
                     seed: int = 9, n_rhs: int = 1, tau: float = 0.5) -> Problem:
    """A small seeded 3D tetrahedral case."""
    m = cube_mesh(cells)
    a = checkerboard(m, 2, stream_seed(seed, 0, 1))
    rhs = np.stack([normal(stream_seed(seed, 0, 2, r), m.n_dofs) for r in range(n_rhs)])
    return Problem(f"small3d_h{cells}_k{k:g}_p{parts}_ov{overlap}", m, a, float(k), parts,
                   box_partition(m, parts), overlap=overlap, tau=tau, rhs=rhs)


def dof_numbering(mesh: Mesh) -> np.ndarray:
    """Global dof id of each node (-1 on Dirichlet nodes): interior nodes in
    increasing node order.  This is the layout convention of rhs and u."""
    d = np.full(mesh.n_nodes, -1, dtype=np.int64)
    inner = np.flatnonzero(mesh.is_boundary == 0)
    d[inner] = np.arange(inner.size)
    return d


def uniform_h(mesh: Mesh) -> float:
    return 1.0 / mesh.cells


def _isclose(a: float, b: float) -> bool:
    return math.isclose(a, b, rel_tol=0, abs_tol=1e-12)
