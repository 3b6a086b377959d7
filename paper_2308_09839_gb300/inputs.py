"""Seeded synthetic inputs: meshes, cell-wise material fields, Dirichlet masks and vectors.

This module is shared by the CUDA path's tests and benchmark and by the CPU oracle. It holds no
finite-element arithmetic (no Jacobians, no quadrature, no element matrices): only the geometry and
random fields the workloads are built from, so that both sides receive identical inputs.

Conventions (used by every caller):

* Domain: the unit cube [0, 1]^3 split into nx x ny x nz hexahedra.
* Node (i, j, k), 0 <= i <= nx etc., has id ``i + (nx + 1) * (j + (ny + 1) * k)``.
* Element (ex, ey, ez) has id ``ex + nx * (ey + ny * ez)``.
* Corner ``a`` of an element (a = 0..7) sits at offset ``(a & 1, (a >> 1) & 1, (a >> 2) & 1)``:
  bit 0 runs along x (reference xi), bit 1 along y (eta), bit 2 along z (zeta).  The paper numbers
  the nodes of a hexahedron 1..8 without fixing an order (Sec. 2); this lexicographic order is the
  one used throughout.
* Degree of freedom ``3 * node + k`` for vector problems (xyz interleaved, the ``3(i-1)+k`` index of
  Eqs. 2-3), ``node`` for the scalar problem.

Every generator takes an explicit integer seed.  Independent fields draw from independent streams
``numpy.random.default_rng([seed, stream_id])`` so that, e.g., the coefficient field does not change
when the mesh jitter is switched on.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# stream ids for numpy.random.default_rng([seed, stream])
_S_JITTER, _S_KAPPA, _S_LAYER, _S_NU, _S_X, _S_B, _S_PERM, _S_GRF, _S_SIZES = range(1, 10)


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


# --------------------------------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------------------------------

def node_id(i, j, k, nx, ny):
    return i + (nx + 1) * (j + (ny + 1) * k)


def box_coords(nx: int, ny: int, nz: int, jitter: float = 0.0, seed: int = 0) -> np.ndarray:
    """Node coordinates of the nx x ny x nz box mesh of the unit cube, float64 [N][3].

    With ``jitter = c > 0`` every node strictly inside the cube moves by an independent
    U[-c*h, c*h] offset in each coordinate (h = 1/n along that axis).  Boundary nodes stay put, so
    the union of the cells is still exactly the unit cube.
    """
    xs = np.linspace(0.0, 1.0, nx + 1)
    ys = np.linspace(0.0, 1.0, ny + 1)
    zs = np.linspace(0.0, 1.0, nz + 1)
    n = (nx + 1) * (ny + 1) * (nz + 1)
    X = np.empty((n, 3), dtype=np.float64)
    # node id runs x fastest: reshape as [k][j][i]
    Xv = X.reshape(nz + 1, ny + 1, nx + 1, 3)
    Xv[..., 0] = xs[None, None, :]
    Xv[..., 1] = ys[None, :, None]
    Xv[..., 2] = zs[:, None, None]
    if jitter > 0.0:
        h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        rng = _rng(seed, _S_JITTER)
        inner = Xv[1:nz, 1:ny, 1:nx, :]
        d = rng.uniform(-1.0, 1.0, size=inner.shape) * (jitter * h)
        inner += d
    return X


def tensor_coords(nx: int, ny: int, nz: int, seed: int = 0, spread: float = 0.5) -> np.ndarray:
    """Node coordinates of a non-uniform tensor-product grid of the unit cube: along each axis the
    cell widths are (1 + U[-spread, spread]) times uniform, renormalised to sum to one."""
    rng = _rng(seed, _S_JITTER)
    axes = []
    for n in (nx, ny, nz):
        w = 1.0 + rng.uniform(-spread, spread, size=n)
        t = np.concatenate([[0.0], np.cumsum(w)])
        t /= t[-1]
        t[-1] = 1.0
        axes.append(t)
    X = np.empty(((nx + 1) * (ny + 1) * (nz + 1), 3))
    Xv = X.reshape(nz + 1, ny + 1, nx + 1, 3)
    Xv[..., 0] = axes[0][None, None, :]
    Xv[..., 1] = axes[1][None, :, None]
    Xv[..., 2] = axes[2][:, None, None]
    return X


def box_cells(nx: int, ny: int, nz: int) -> np.ndarray:
    """Element -> node map of the box mesh, int32 [E][8], corners in the lexicographic order above."""
    ex = np.arange(nx, dtype=np.int64)
    ey = np.arange(ny, dtype=np.int64)
    ez = np.arange(nz, dtype=np.int64)
    EZ, EY, EX = np.meshgrid(ez, ey, ex, indexing="ij")  # element id runs ex fastest
    base = node_id(EX, EY, EZ, nx, ny).reshape(-1)
    cells = np.empty((base.size, 8), dtype=np.int64)
    for a in range(8):
        di, dj, dk = a & 1, (a >> 1) & 1, (a >> 2) & 1
        cells[:, a] = base + node_id(di, dj, dk, nx, ny)
    if cells.max(initial=0) >= 2**31:
        raise ValueError("mesh too large for int32 node ids")
    return cells.astype(np.int32)


# The 6 tetrahedra of a hexahedron that share its diagonal from corner 0 to corner 7 (Kuhn's
# subdivision): one per order in which a path from corner 0 to corner 7 steps along x (corner bit
# 1), y (bit 2) and z (bit 4), with the parity of that order.
_KUHN = ((1, 2, 4, 0), (1, 4, 2, 1), (2, 1, 4, 1), (2, 4, 1, 0), (4, 1, 2, 0), (4, 2, 1, 1))


def tet_cells(nx: int, ny: int, nz: int) -> np.ndarray:
    """Tetrahedral connectivity of the box, int32 [6E][4]: hexahedron e of ``box_cells`` becomes
    tetrahedra 6e..6e+5 with nodes (c0, c_a, c_{a+b}, c7).  Every hexahedron face is cut along its
    diagonal through the face's lowest corner, so neighbouring hexahedra cut a shared face the same
    way (the mesh is conforming).  Paths of odd parity swap their two middle nodes, which makes every
    tetrahedron positively oriented on the undistorted box."""
    hexes = box_cells(nx, ny, nz)
    out = np.empty((hexes.shape[0], 6, 4), dtype=np.int32)
    for t, (a, b, _c, odd) in enumerate(_KUHN):
        mid = [a + b, a] if odd else [a, a + b]
        out[:, t] = hexes[:, [0, mid[0], mid[1], 7]]
    return out.reshape(-1, 4)


def dirichlet_z0(nx: int, ny: int, nz: int) -> np.ndarray:
    """uint8 [N] mask, 1 on the nodes of the face z = 0."""
    m = np.zeros((nz + 1, ny + 1, nx + 1), dtype=np.uint8)
    m[0] = 1
    return m.reshape(-1)


# --------------------------------------------------------------------------------------------------
# material fields (cell-wise)
# --------------------------------------------------------------------------------------------------

def lognormal_cells(n_cells: int, sigma: float, seed: int, stream: int = _S_KAPPA) -> np.ndarray:
    """exp(N(0, sigma^2)) per cell."""
    return np.exp(_rng(seed, stream).normal(0.0, sigma, size=n_cells))


def layer_multiplier(nx: int, ny: int, nz: int, n_layers: int, seed: int) -> np.ndarray:
    """Per-cell multiplier 10**s_l of ``n_layers`` equal z-slabs, s_l ~ U[-1, 1] (seeded)."""
    s = _rng(seed, _S_LAYER).uniform(-1.0, 1.0, size=n_layers)
    ez = np.arange(nz)
    layer = np.minimum((ez * n_layers) // nz, n_layers - 1)
    per_z = 10.0 ** s[layer]
    return np.broadcast_to(per_z[:, None, None], (nz, ny, nx)).reshape(-1).copy()


def layered_lognormal(nx, ny, nz, sigma, seed, n_layers=8) -> np.ndarray:
    return layer_multiplier(nx, ny, nz, n_layers, seed) * lognormal_cells(nx * ny * nz, sigma, seed)


def poisson_ratio(n_cells: int, seed: int, lo=0.15, hi=0.35) -> np.ndarray:
    return _rng(seed, _S_NU).uniform(lo, hi, size=n_cells)


def gaussian_random_field(nx, ny, nz, corr_cells: float, sigma: float, seed: int) -> np.ndarray:
    """Cell-wise zero-mean field: white noise smoothed by a periodic separable Gaussian of standard
    deviation ``corr_cells`` cells, rescaled to standard deviation ``sigma``."""
    w = _rng(seed, _S_GRF).normal(size=(nz, ny, nx))
    f = np.fft.fftn(w)
    for axis, n in enumerate((nz, ny, nx)):
        k = np.fft.fftfreq(n)  # cycles per cell
        g = np.exp(-2.0 * (math.pi * corr_cells * k) ** 2)  # FT of a unit-mass Gaussian
        shape = [1, 1, 1]
        shape[axis] = n
        f = f * g.reshape(shape)
    field_ = np.real(np.fft.ifftn(f))
    field_ -= field_.mean()
    sd = field_.std()
    if sd > 0:
        field_ *= sigma / sd
    return field_.reshape(-1)


# --------------------------------------------------------------------------------------------------
# vectors
# --------------------------------------------------------------------------------------------------

def uniform_vector(n: int, seed: int, stream: int = _S_X, dirichlet_dofs: np.ndarray | None = None) -> np.ndarray:
    v = _rng(seed, stream).uniform(-1.0, 1.0, size=n)
    if dirichlet_dofs is not None:
        v[dirichlet_dofs] = 0.0
    return v


def dof_mask(node_mask: np.ndarray, ndof_per_node: int) -> np.ndarray:
    """Boolean DoF mask from a node mask (xyz interleaved)."""
    return np.repeat(node_mask.astype(bool), ndof_per_node)


# --------------------------------------------------------------------------------------------------
# renumbering (exercises the general, unstructured code path on box meshes)
# --------------------------------------------------------------------------------------------------

def renumber(coords, cells, dirichlet, seed: int):
    """Randomly permute node and element numbering.  Returns (coords, cells, dirichlet, node_perm,
    elem_perm) with ``new_coords[node_perm[i]] = coords[i]`` and ``new_cells = cells[elem_perm]``
    relabelled."""
    rng = _rng(seed, _S_PERM)
    n = coords.shape[0]
    node_perm = rng.permutation(n)  # old -> new
    elem_perm = rng.permutation(cells.shape[0])  # new position -> old element
    new_coords = np.empty_like(coords)
    new_coords[node_perm] = coords
    new_dir = np.empty_like(dirichlet)
    new_dir[node_perm] = dirichlet
    new_cells = node_perm[cells[elem_perm]].astype(np.int32)
    return new_coords, new_cells, new_dir, node_perm, elem_perm


# --------------------------------------------------------------------------------------------------
# workload recipes
# --------------------------------------------------------------------------------------------------

@dataclass
class Problem:
    """One seeded FE problem on a box mesh.  ``cells`` is None when the caller asked for the
    implicit (structured) connectivity; ``structured()`` recreates it on demand."""
    name: str
    physics: str            # "laplace" | "elasticity"
    nx: int
    ny: int
    nz: int
    coords: np.ndarray      # float64 [N][3]
    mat: np.ndarray         # float64 [E] (kappa) or [E][2] (Young's modulus, Poisson ratio)
    dirichlet: np.ndarray   # uint8 [N]
    seed: int = 0
    cells: np.ndarray | None = None
    meta: dict = field(default_factory=dict)
    element: str = "hex8"   # "hex8" (Q1) | "tet4" (P1 tetrahedra) | "hex27" (Q2); the last two with explicit cells

    @property
    def n_nodes(self) -> int:
        return self.coords.shape[0]

    @property
    def n_cells(self) -> int:
        return self.cells.shape[0] if self.cells is not None else self.nx * self.ny * self.nz

    @property
    def ndpn(self) -> int:
        return 1 if self.physics == "laplace" else 3

    @property
    def n_dof(self) -> int:
        return self.n_nodes * self.ndpn

    @property
    def n_free(self) -> int:
        return int(self.n_dof - self.ndpn * int(self.dirichlet.sum()))

    def cell_array(self) -> np.ndarray:
        if self.cells is None:
            return box_cells(self.nx, self.ny, self.nz)
        return self.cells

    def dirichlet_dofs(self) -> np.ndarray:
        return np.nonzero(dof_mask(self.dirichlet, self.ndpn))[0]

    def x(self, seed: int | None = None) -> np.ndarray:
        """Input vector x ~ U[-1, 1] with Dirichlet entries zeroed."""
        s = self.seed if seed is None else seed
        return uniform_vector(self.n_dof, s, _S_X, self.dirichlet_dofs())

    def b(self, seed: int | None = None) -> np.ndarray:
        """Right-hand side b ~ U[-1, 1] with Dirichlet entries zeroed."""
        s = self.seed if seed is None else seed
        return uniform_vector(self.n_dof, s, _S_B, self.dirichlet_dofs())


def laplace_box(n, jitter=0.0, sigma=1.0, layered=False, seed=0, name=None, ny=None, nz=None, graded=0.0) -> Problem:
    """Laplace on an n x ny x nz box; ``graded > 0`` gives a non-uniform tensor-product grid."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    coords = tensor_coords(n, ny, nz, seed, graded) if graded > 0 else box_coords(n, ny, nz, jitter, seed)
    if layered:
        kappa = layered_lognormal(n, ny, nz, sigma, seed)
    else:
        kappa = lognormal_cells(n * ny * nz, sigma, seed)
    return Problem(name or f"laplace_{n}x{ny}x{nz}", "laplace", n, ny, nz, coords, kappa,
                   dirichlet_z0(n, ny, nz), seed, meta=dict(jitter=jitter, sigma=sigma, layered=layered))


def elasticity_box(n, jitter=0.0, sigma=0.5, layered=True, seed=0, name=None, ny=None, nz=None,
                   graded=0.0) -> Problem:
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    coords = tensor_coords(n, ny, nz, seed, graded) if graded > 0 else box_coords(n, ny, nz, jitter, seed)
    E = layered_lognormal(n, ny, nz, sigma, seed) if layered else lognormal_cells(n * ny * nz, sigma, seed)
    nu = poisson_ratio(n * ny * nz, seed)
    mat = np.stack([E, nu], axis=1)
    return Problem(name or f"elasticity_{n}x{ny}x{nz}", "elasticity", n, ny, nz, coords, mat,
                   dirichlet_z0(n, ny, nz), seed, meta=dict(jitter=jitter, sigma=sigma, layered=layered))


def vector_laplace_box(n, jitter=0.0, sigma=1.0, layered=False, seed=0, name=None, ny=None, nz=None,
                       graded=0.0) -> Problem:
    """Vector Laplace (three components, one coefficient kappa per cell) on the same boxes as
    ``laplace_box``."""
    p = laplace_box(n, jitter=jitter, sigma=sigma, layered=layered, seed=seed, ny=ny, nz=nz, graded=graded)
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    return Problem(name or f"vector_laplace_{n}x{ny}x{nz}", "vector_laplace", n, ny, nz, p.coords, p.mat,
                   p.dirichlet, seed, meta=p.meta)


def tet_box(physics: str, n, jitter=0.0, sigma=0.5, layered=True, seed=0, name=None, ny=None,
            nz=None) -> Problem:
    """P1 tetrahedra: the n x ny x nz box (node jitter as ``box_coords``) with every hexahedron split
    into 6 tetrahedra (``tet_cells``).  Each tetrahedron takes the cell constants of its hexahedron:
    the recipe of ``laplace_box`` / ``elasticity_box`` / ``vector_laplace_box``, repeated 6 times.
    Dirichlet on z = 0."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    maker = {"laplace": laplace_box, "elasticity": elasticity_box, "vector_laplace": vector_laplace_box}[physics]
    h = maker(n, jitter=jitter, sigma=sigma, layered=layered, seed=seed, ny=ny, nz=nz)
    mat = np.repeat(h.mat, 6, axis=0)
    return Problem(name or f"tet_{physics}_{n}x{ny}x{nz}", physics, n, ny, nz, h.coords, mat, h.dirichlet, seed,
                   cells=tet_cells(n, ny, nz), meta=dict(h.meta, element="tet4"), element="tet4")


def q2_cells(nx: int, ny: int, nz: int) -> np.ndarray:
    """Triquadratic (27-node) connectivity of the box, int32 [E][27].  Nodes form the
    (2nx+1) x (2ny+1) x (2nz+1) lattice with id I + (2nx+1)(J + (2ny+1)K); node a = i + 3j + 9k of
    element (ex, ey, ez) is lattice node (2ex + i, 2ey + j, 2ez + k)."""
    NX, NY = 2 * nx + 1, 2 * ny + 1
    ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ex, ey, ez = (v.transpose(2, 1, 0).reshape(-1) for v in (ex, ey, ez))  # element id runs ex fastest
    a = np.arange(27)
    I = 2 * ex[:, None] + (a % 3)[None]
    J = 2 * ey[:, None] + ((a // 3) % 3)[None]
    K = 2 * ez[:, None] + (a // 9)[None]
    ids = I + NX * (J + NY * K)
    if ids.max(initial=0) >= 2**31:
        raise ValueError("mesh too large for int32 node ids")
    return ids.astype(np.int32)


def q2_coords(nx: int, ny: int, nz: int, jitter: float = 0.0, curve: float = 0.0, seed: int = 0) -> np.ndarray:
    """Lattice coordinates of the triquadratic box mesh, float64 [(2nx+1)(2ny+1)(2nz+1)][3].  The
    element vertices are the nodes of ``box_coords(nx, ny, nz, jitter, seed)``; every other lattice
    node is the mean of the vertices around it (the trilinear midpoint, so edges stay straight).
    ``curve = c > 0`` then moves every non-vertex node strictly inside the cube by U[-c h, c h] per
    coordinate (curved elements)."""
    V = box_coords(nx, ny, nz, jitter, seed).reshape(nz + 1, ny + 1, nx + 1, 3)
    L = np.empty((2 * nz + 1, 2 * ny + 1, 2 * nx + 1, 3))
    L[::2, ::2, ::2] = V
    L[::2, ::2, 1::2] = 0.5 * (V[:, :, :-1] + V[:, :, 1:])
    L[::2, 1::2, :] = 0.5 * (L[::2, :-1:2, :] + L[::2, 2::2, :])
    L[1::2] = 0.5 * (L[:-1:2] + L[2::2])
    X = L.reshape(-1, 3)
    if curve > 0.0:
        NX, NY, NZ = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
        K, J, I = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
        I, J, K = I.reshape(-1), J.reshape(-1), K.reshape(-1)
        vertex = (I % 2 == 0) & (J % 2 == 0) & (K % 2 == 0)
        inner = (I > 0) & (I < NX - 1) & (J > 0) & (J < NY - 1) & (K > 0) & (K < NZ - 1)
        sel = inner & ~vertex
        h = np.array([1.0 / nx, 1.0 / ny, 1.0 / nz])
        X[sel] += _rng(seed, _S_JITTER + 100).uniform(-curve, curve, size=(int(sel.sum()), 3)) * h
    return X


def q2_box(physics: str, n, jitter=0.0, curve=0.0, sigma=0.5, layered=True, seed=0, name=None, ny=None,
           nz=None) -> Problem:
    """Q2 hexahedra on the n x ny x nz box (``q2_coords``, ``q2_cells``); cell constants as the Q1
    recipe of the same physics; Dirichlet on z = 0 (lattice plane K = 0)."""
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    maker = {"laplace": laplace_box, "elasticity": elasticity_box, "vector_laplace": vector_laplace_box}[physics]
    h = maker(n, jitter=jitter, sigma=sigma, layered=layered, seed=seed, ny=ny, nz=nz)
    coords = q2_coords(n, ny, nz, jitter, curve, seed)
    NX, NY = 2 * n + 1, 2 * ny + 1
    dirichlet = np.zeros(coords.shape[0], dtype=np.uint8)
    dirichlet[: NX * NY] = 1
    return Problem(name or f"q2_{physics}_{n}x{ny}x{nz}", physics, n, ny, nz, coords, h.mat, dirichlet, seed,
                   cells=q2_cells(n, ny, nz), meta=dict(h.meta, element="hex27", curve=curve), element="hex27")


def small_laplace_16(seed=0) -> Problem:
    """16^3 cells, interior nodes jittered by U[-0.2h, 0.2h], kappa ~ lognormal(0, 1) per cell,
    Dirichlet u = 0 on z = 0."""
    return laplace_box(16, jitter=0.2, sigma=1.0, layered=False, seed=seed, name="laplace_16_jitter")


def cartesian_laplace_256(seed=0, n=256) -> Problem:
    """256^3 Cartesian cells, 8 z-layers times lognormal(0, 0.5) noise, Dirichlet on z = 0."""
    return laplace_box(n, jitter=0.0, sigma=0.5, layered=True, seed=seed, name=f"laplace_{n}_cartesian")


def cartesian_elasticity_160(seed=0, n=160) -> Problem:
    """160^3 Cartesian cells, E = 8 z-layers times lognormal(0, 0.5), nu ~ U[0.15, 0.35]."""
    return elasticity_box(n, jitter=0.0, sigma=0.5, layered=True, seed=seed, name=f"elasticity_{n}_cartesian")


def jittered_elasticity_192(seed=0, n=192) -> Problem:
    """192^3 cells, interior node jitter U[-0.1h, 0.1h], material as the Cartesian elasticity case."""
    return elasticity_box(n, jitter=0.1, sigma=0.5, layered=True, seed=seed, name=f"elasticity_{n}_jitter")


def batch_sizes(n_problems=64, lo=8, hi=96, seed=0) -> np.ndarray:
    """Elements per side, log-uniform in [lo, hi] (seeded)."""
    u = _rng(seed, _S_SIZES).uniform(math.log(lo), math.log(hi), size=n_problems)
    return np.clip(np.rint(np.exp(u)).astype(np.int64), lo, hi)


def grf_laplace_128(seed=0, n=128) -> Problem:
    """Laplace with log kappa a Gaussian random field (correlation 8 cells, sigma 1.5) plus 8 z-layer
    offsets (log10 offsets U[-1, 1])."""
    logk = gaussian_random_field(n, n, n, 8.0, 1.5, seed)
    logk = logk + np.log(layer_multiplier(n, n, n, 8, seed))
    coords = box_coords(n, n, n, 0.0, seed)
    return Problem(f"laplace_{n}_grf", "laplace", n, n, n, coords, np.exp(logk), dirichlet_z0(n, n, n), seed,
                   meta=dict(jitter=0.0, grf=True))
