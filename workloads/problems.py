"""Seeded synthetic transport problems (inputs only, no method arithmetic).

Grid convention (shared by every consumer, stated once here):

* The transition region is an ``Nx x Ny x Nz`` grid with spacing ``h``; ``z``
  is the transport direction.  A grid point ``(x, y, z)`` has the linear index
  ``(z * Ny + y) * Nx + x`` (x fastest).
* Transverse walls are Dirichlet: the grid point ``i`` sits at ``(i + 1) h`` so
  that the walls are at ``0`` and ``(N + 1) h``.  Along ``z`` the plane ``k``
  sits at ``k h``.
* A Gaussian well is ``-D exp(-|r - c|^2 / (2 w^2))``; "width" is read as the
  standard deviation ``w``.
* A Kleinman-Bylander projector is ``p(r) = exp(-|r - R|^2 / (2 s^2))`` on the
  grid points with ``|r - R| <= r_cut`` (clipped at the walls), scaled so that
  ``sum_j p_j^2 h^3 = 1``; it enters the Hamiltonian as
  ``E_a p (p^T psi) h^3``.

Every random draw uses ``numpy.random.Generator(PCG64(1000 + index))`` where
``index`` is the configuration's position in the workload list below.
"""

from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence, Tuple

import numpy as np

CONFIG_NAMES = (
    "tiny_wire_fp64",          # 8x8x12, 2nd order, 3 wells, all 128 plane columns, 8 energies
    "sampled_columns_mixed",   # 64x64x128, 4th order, 200 wells, 256 sampled columns, 128 energies
    "full_boundary",           # 48x48x160, 4th order, every boundary column, 64 energies
    "uneven_regions",          # six regions of different sizes in one batch
    "peapod",                  # 72x72x256, 4th order, 460 atoms with KB projectors, 100 energies
)


@dataclass
class Projectors:
    """Separable nonlocal projectors in CSR form (one row per atom)."""

    E: np.ndarray      # [n_atoms] float64, projector energies (Hartree)
    ptr: np.ndarray    # [n_atoms + 1] int64, row pointers into idx/val
    idx: np.ndarray    # [nnz] int64, linear grid indices, ascending within an atom
    val: np.ndarray    # [nnz] float64, projector values, sum(val^2) h^3 = 1 per atom

    @property
    def n_atoms(self) -> int:
        return int(self.E.shape[0])

    @property
    def nnz(self) -> int:
        return int(self.idx.shape[0])


@dataclass
class Problem:
    """One transition region plus the solve parameters applied to it."""

    name: str
    grid: Tuple[int, int, int]           # (Nx, Ny, Nz)
    h: float                             # grid spacing (bohr)
    fd_order: int                        # 2 (7-point) or 4 (13-point)
    V: np.ndarray                        # local potential, float64, shape (Nz, Ny, Nx)
    energies: np.ndarray                 # real energies E_k (Hartree), float64 [K]
    eta: float                           # imaginary part of Z_k = E_k + i eta
    tol: float                           # relative residual tolerance
    cols: np.ndarray                     # right-hand-side columns: linear grid indices, int64
    n_face: int                          # planes per side in the boundary row set
    precision: str                       # "fp64" or "mixed"
    seed: int
    proj: Optional[Projectors] = None
    maxit: int = 100000
    notes: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        nx, ny, nz = self.grid
        return nx * ny * nz

    @property
    def Nxy(self) -> int:
        return self.grid[0] * self.grid[1]

    @property
    def K(self) -> int:
        return int(self.energies.shape[0])


def grid_coordinates(grid: Sequence[int], h: float):
    """Return the 1D coordinate arrays (x, y, z) of the grid points."""
    nx, ny, nz = grid
    x = (np.arange(nx) + 1.0) * h
    y = (np.arange(ny) + 1.0) * h
    z = np.arange(nz) * h
    return x, y, z


def boundary_plane_points(grid: Sequence[int], planes: Sequence[int]) -> np.ndarray:
    """Linear indices of every point of the given z-planes, plane by plane, x fastest."""
    nx, ny, _ = grid
    nxy = nx * ny
    return np.concatenate([np.arange(nxy, dtype=np.int64) + p * nxy for p in planes])


def _box(grid, h):
    nx, ny, nz = grid
    return np.array([(nx + 1) * h, (ny + 1) * h, (nz - 1) * h])


def _gaussian_wells(grid, h, centres, depths, widths, cut_sigmas=10.0) -> np.ndarray:
    """Sum of -D exp(-|r-c|^2/(2w^2)) on the grid (terms beyond cut_sigmas*w dropped, < 1e-21)."""
    nx, ny, nz = grid
    x, y, z = grid_coordinates(grid, h)
    V = np.zeros((nz, ny, nx))
    for c, D, w in zip(centres, depths, widths):
        rc = cut_sigmas * w
        ix = np.nonzero(np.abs(x - c[0]) <= rc)[0]
        iy = np.nonzero(np.abs(y - c[1]) <= rc)[0]
        iz = np.nonzero(np.abs(z - c[2]) <= rc)[0]
        if ix.size == 0 or iy.size == 0 or iz.size == 0:
            continue
        dx2 = (x[ix] - c[0]) ** 2
        dy2 = (y[iy] - c[1]) ** 2
        dz2 = (z[iz] - c[2]) ** 2
        d2 = dz2[:, None, None] + dy2[None, :, None] + dx2[None, None, :]
        V[iz[0]:iz[-1] + 1, iy[0]:iy[-1] + 1, ix[0]:ix[-1] + 1] -= D * np.exp(-d2 / (2.0 * w * w))
    return V


def _kb_projectors(grid, h, atoms, sigma=1.2, r_cut=3.0, energy=0.5) -> Projectors:
    nx, ny, nz = grid
    x, y, z = grid_coordinates(grid, h)
    ptr = [0]
    idx_all, val_all = [], []
    for R in atoms:
        ix = np.nonzero(np.abs(x - R[0]) <= r_cut)[0]
        iy = np.nonzero(np.abs(y - R[1]) <= r_cut)[0]
        iz = np.nonzero(np.abs(z - R[2]) <= r_cut)[0]
        if ix.size and iy.size and iz.size:
            Z, Y, X = np.meshgrid(iz, iy, ix, indexing="ij")
            d2 = (x[X] - R[0]) ** 2 + (y[Y] - R[1]) ** 2 + (z[Z] - R[2]) ** 2
            inside = d2 <= r_cut * r_cut
            lin = ((Z * ny + Y) * nx + X)[inside].astype(np.int64)
            p = np.exp(-d2[inside] / (2.0 * sigma * sigma))
            order = np.argsort(lin)
            lin, p = lin[order], p[order]
            p = p / np.sqrt(np.sum(p * p) * h ** 3)
        else:
            lin, p = np.zeros(0, np.int64), np.zeros(0)
        idx_all.append(lin)
        val_all.append(p)
        ptr.append(ptr[-1] + lin.size)
    return Projectors(
        E=np.full(len(atoms), float(energy)),
        ptr=np.asarray(ptr, dtype=np.int64),
        idx=np.concatenate(idx_all) if idx_all else np.zeros(0, np.int64),
        val=np.concatenate(val_all) if val_all else np.zeros(0),
    )


def _random_wells(rng, grid, h, n, depth=(0.5, 1.5), width=1.0):
    box = _box(grid, h)
    centres = rng.uniform(0.0, 1.0, size=(n, 3)) * box
    depths = rng.uniform(depth[0], depth[1], size=n)
    widths = np.full(n, width)
    return centres, depths, widths


def _peapod_sites(rng, grid, h):
    """(10,10)-tube-like cylinder (20 rings of 20 sites) plus a 60-site sphere at mid-length."""
    box = _box(grid, h)
    cx, cy, zmid = box[0] / 2.0, box[1] / 2.0, box[2] / 2.0
    sites = []
    n_rings, per_ring, radius, spacing = 20, 20, 12.8, 2.3
    for r in range(n_rings):
        zr = zmid + (r - (n_rings - 1) / 2.0) * spacing
        phase = np.deg2rad(9.0) if (r % 2) else 0.0
        for s in range(per_ring):
            a = 2.0 * np.pi * s / per_ring + phase
            sites.append((cx + radius * np.cos(a), cy + radius * np.sin(a), zr))
    # near-uniform sphere: a golden-angle spiral, randomly rotated (seeded)
    n_s, rad_s = 60, 6.7
    k = np.arange(n_s) + 0.5
    polar = np.arccos(1.0 - 2.0 * k / n_s)
    azim = np.pi * (1.0 + 5 ** 0.5) * k
    pts = np.stack([np.sin(polar) * np.cos(azim), np.sin(polar) * np.sin(azim), np.cos(polar)], 1)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    pts = pts @ q.T * rad_s
    for p in pts:
        sites.append((cx + p[0], cy + p[1], zmid + p[2]))
    return np.asarray(sites)


def sample_plane_columns(grid, n_cols, seed):
    """n_cols distinct points drawn uniformly from the planes z=0 and z=Nz-1 (sorted), seeded."""
    return _sample_plane_columns(np.random.Generator(np.random.PCG64(seed)), grid, n_cols)


def _sample_plane_columns(rng, grid, n_cols):
    nx, ny, nz = grid
    pool = boundary_plane_points(grid, [0, nz - 1])
    if n_cols >= pool.size:
        return pool
    pick = np.sort(rng.choice(pool.size, size=n_cols, replace=False))
    return pool[pick]


def make_problem(name_or_index, **overrides):
    """Build one of the five named workloads (a list of Problems for the uneven batch).

    ``overrides`` replaces fields after construction (e.g. ``precision="fp64"`` or
    ``cols=...``) without changing any random draw.
    """
    index = name_or_index if isinstance(name_or_index, int) else CONFIG_NAMES.index(name_or_index)
    name = CONFIG_NAMES[index]
    seed = 1000 + index
    rng = np.random.Generator(np.random.PCG64(seed))

    if name == "tiny_wire_fp64":
        grid, h = (8, 8, 12), 0.5
        c, d, w = _random_wells(rng, grid, h, 3)
        p = Problem(name, grid, h, 2, _gaussian_wells(grid, h, c, d, w),
                    np.linspace(0.1, 0.8, 8), 1e-3, 1e-12,
                    boundary_plane_points(grid, [0, grid[2] - 1]), 1, "fp64", seed, maxit=20000)
    elif name == "sampled_columns_mixed":
        grid, h = (64, 64, 128), 0.4
        c, d, w = _random_wells(rng, grid, h, 200)
        V = _gaussian_wells(grid, h, c, d, w)
        cols = _sample_plane_columns(rng, grid, 256)
        p = Problem(name, grid, h, 4, V, np.linspace(-0.5, 0.5, 128), 1e-3, 1e-6,
                    cols, 1, "mixed", seed, maxit=40000)
    elif name == "full_boundary":
        grid, h = (48, 48, 160), 0.4
        c, d, w = _random_wells(rng, grid, h, 140)
        V = _gaussian_wells(grid, h, c, d, w)
        nz = grid[2]
        cols = boundary_plane_points(grid, [0, 1, nz - 2, nz - 1])
        p = Problem(name, grid, h, 4, V, np.linspace(-0.5, 0.5, 64), 5e-4, 1e-6,
                    cols, 2, "mixed", seed, maxit=60000)
    elif name == "uneven_regions":
        grids = [(32, 32, 64), (40, 40, 96), (48, 48, 128), (56, 56, 80), (64, 64, 160), (72, 72, 112)]
        out = []
        for r, grid in enumerate(grids):
            h = 0.4
            nx, ny, nz = grid
            n_wells = max(8, int(round(200 * nx * ny * nz / (64 * 64 * 128))))
            c, d, w = _random_wells(rng, grid, h, n_wells)
            V = _gaussian_wells(grid, h, c, d, w)
            K = int(rng.integers(32, 201))
            eta = float(rng.choice([1e-3, 5e-4]))
            if 2 * nx * ny <= 4096:
                cols = boundary_plane_points(grid, [0, nz - 1])
            else:
                cols = _sample_plane_columns(rng, grid, 512)
            out.append(Problem(f"{name}[{r}]", grid, h, 4, V, np.linspace(-0.5, 0.5, K), eta, 1e-6,
                               cols, 1, "mixed", seed, maxit=60000))
        for q in out:
            for k, v in overrides.items():
                setattr(q, k, v)
        return out
    elif name == "peapod":
        grid, h = (72, 72, 256), 0.4
        atoms = _peapod_sites(rng, grid, h)
        V = _gaussian_wells(grid, h, atoms, np.ones(len(atoms)), np.full(len(atoms), 0.8))
        proj = _kb_projectors(grid, h, atoms)
        nz = grid[2]
        cols = boundary_plane_points(grid, [0, 1, nz - 2, nz - 1])
        p = Problem(name, grid, h, 4, V, np.linspace(-0.3, 0.3, 100), 1e-3, 1e-6,
                    cols, 2, "mixed", seed, proj=proj, maxit=60000)
    else:  # pragma: no cover
        raise ValueError(name)
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def small_problem(grid=(6, 5, 8), h=0.5, fd_order=2, n_wells=2, n_energies=6,
                  e_range=(0.2, 1.2), eta=1e-2, tol=1e-12, projectors=0, cols="planes",
                  n_face=None, precision="fp64", seed=7, depth=(0.5, 1.5), width=1.0):
    """A small problem built with the same recipe as the named workloads, for tests.

    ``cols`` is "planes" (every point of the outer ``n_face`` planes on each side,
    in boundary order), "first_plane_pair" (planes z=0 and z=Nz-1 only), an int
    (that many plane points sampled) or an explicit index array.
    ``projectors`` > 0 adds that many KB projectors centred at random points.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_face = (fd_order // 2) if n_face is None else n_face
    c, d, w = _random_wells(rng, grid, h, n_wells, depth, width)
    V = _gaussian_wells(grid, h, c, d, w) if n_wells else np.zeros(grid[::-1])
    proj = None
    if projectors:
        atoms = rng.uniform(0.0, 1.0, size=(projectors, 3)) * _box(grid, h)
        proj = _kb_projectors(grid, h, atoms, sigma=1.2 * h / 0.4, r_cut=3.0 * h / 0.4)
    nz = grid[2]
    if isinstance(cols, str) and cols == "planes":
        planes = list(range(n_face)) + list(range(nz - n_face, nz))
        colv = boundary_plane_points(grid, planes)
    elif isinstance(cols, str) and cols == "first_plane_pair":
        colv = boundary_plane_points(grid, [0, nz - 1])
    elif isinstance(cols, (int, np.integer)):
        colv = _sample_plane_columns(rng, grid, int(cols))
    else:
        colv = np.asarray(cols, dtype=np.int64)
    energies = np.linspace(e_range[0], e_range[1], n_energies)
    return Problem(f"small{grid}o{fd_order}", tuple(grid), h, fd_order, V, energies, eta, tol,
                   colv, n_face, precision, seed, proj=proj, maxit=20000)


def random_complex_matrices(n: int, K: int, seed: int, scale: float = 1.0, symmetric: bool = True,
                            imag_sign: float = 0.0) -> np.ndarray:
    """K random complex n x n matrices (complex128), optionally complex symmetric.

    ``imag_sign`` < 0 adds ``-i*|scale|*I`` so the imaginary part is negative definite
    (the sign a retarded self-energy has); > 0 adds the opposite.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    A = (rng.normal(size=(K, n, n)) + 1j * rng.normal(size=(K, n, n))) * (scale / np.sqrt(n))
    if symmetric:
        A = 0.5 * (A + np.transpose(A, (0, 2, 1)))
    if imag_sign:
        A = A + np.sign(imag_sign) * 1j * abs(scale) * np.eye(n)[None]
    return A
