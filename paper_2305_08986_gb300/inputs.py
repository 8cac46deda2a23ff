"""Seeded synthetic workloads for the generalized Stokes solve.

This module only describes problems: mesh extents, the per-cell viscosity
field, the reaction coefficient, obstacle cells, Dirichlet faces, and nodal
load / boundary data evaluated at node coordinates.  It contains none of the
discretisation or solver arithmetic, so both the CUDA path and the CPU oracle
can draw their inputs from it.

Vector layout used for nodal data (shared convention of the whole library):
velocity nodes live on the (2 n_x + 1) x (2 n_y + 1) [x (2 n_z + 1)] grid of a
Q2 field, numbered lexicographically with x fastest; pressure nodes live on the
(n_x + 1) x (n_y + 1) [x (n_z + 1)] Q1 grid.  A full vector is
[u_x | u_y | (u_z) | p].

Workload shapes follow the paper's test problems: the 2D channel with an
obstacle and an attached stiff bar mirrors the FSI2i geometry (Sec. 5,
Table "turek_geometry", L = 2.5, H = 0.41, bar 0.35 x 0.02 behind the
obstacle), the viscosity contrast comes from the viscosity splitting
eta = eta_f in the fluid and gamma*tau*mu_s in the solid (Sec. 3.1.2,
Eq. "viscosity-splitting"), and alpha = rho / (gamma tau) is the BDF reaction
coefficient (Sec. 3.1, Eq. "stencil").
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

FACE_XM, FACE_XP, FACE_YM, FACE_YP, FACE_ZM, FACE_ZP = (1 << i for i in range(6))


def all_faces(dim: int) -> int:
    return (1 << (2 * dim)) - 1


@dataclasses.dataclass
class Problem:
    """One generalized Stokes instance on a structured Cartesian mesh."""

    name: str
    dim: int
    n: tuple            # cells per axis on the finest level
    length: tuple       # domain extent per axis (origin at 0)
    levels: int         # multigrid levels (finest has n, level l has n / 2^(levels-1-l))
    eta: np.ndarray     # float64, one value per cell, cell-lexicographic (x fastest)
    alpha: float
    dirichlet_faces: int
    void: Optional[np.ndarray] = None   # uint8 per cell, 1 = obstacle cell (excluded)
    f: Optional[np.ndarray] = None      # nodal load, full vector layout
    g: Optional[np.ndarray] = None      # Dirichlet data, full vector layout

    @property
    def n_cells(self) -> int:
        return int(np.prod(self.n))

    @property
    def n_vnodes(self) -> int:
        return int(np.prod([2 * k + 1 for k in self.n]))

    @property
    def n_pnodes(self) -> int:
        return int(np.prod([k + 1 for k in self.n]))

    @property
    def n_u(self) -> int:
        return self.dim * self.n_vnodes

    @property
    def n_total(self) -> int:
        return self.n_u + self.n_pnodes


# --------------------------------------------------------------------------
# coordinates (geometry only)
# --------------------------------------------------------------------------

def cell_centroids(dim: int, n: Sequence[int], length: Sequence[float]) -> np.ndarray:
    """(N_c, dim) centroids, cell-lexicographic with x fastest."""
    axes = [(np.arange(n[a]) + 0.5) * (length[a] / n[a]) for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")  # slowest axis first
    return np.stack([g.ravel() for g in grids[::-1]], axis=1)


def vnode_coords(dim: int, n: Sequence[int], length: Sequence[float]) -> np.ndarray:
    """(N_v, dim) coordinates of Q2 velocity nodes, x fastest."""
    axes = [np.arange(2 * n[a] + 1) * (length[a] / (2 * n[a])) for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([g.ravel() for g in grids[::-1]], axis=1)


def pnode_coords(dim: int, n: Sequence[int], length: Sequence[float]) -> np.ndarray:
    axes = [np.arange(n[a] + 1) * (length[a] / n[a]) for a in range(dim)]
    grids = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([g.ravel() for g in grids[::-1]], axis=1)


def _full(dim, n, u_nodal: Optional[np.ndarray] = None) -> np.ndarray:
    nv = int(np.prod([2 * k + 1 for k in n]))
    npn = int(np.prod([k + 1 for k in n]))
    v = np.zeros(dim * nv + npn)
    if u_nodal is not None:
        for a in range(dim):
            v[a * nv:(a + 1) * nv] = u_nodal[:, a]
    return v


# --------------------------------------------------------------------------
# config 1: unit square, disc inclusion, manufactured smooth field
# --------------------------------------------------------------------------

def mms_velocity(x: np.ndarray, y: np.ndarray):
    """u = curl psi with psi = sin^2(pi x) sin^2(pi y): zero on the boundary, div-free."""
    ux = math.pi * np.sin(math.pi * x) ** 2 * np.sin(2 * math.pi * y)
    uy = -math.pi * np.sin(2 * math.pi * x) * np.sin(math.pi * y) ** 2
    return ux, uy


def mms_velocity_grad(x, y):
    """Gradient d u_a / d x_b of mms_velocity, returned as (dux_dx, dux_dy, duy_dx, duy_dy)."""
    pi = math.pi
    dux_dx = pi * pi * np.sin(2 * pi * x) * np.sin(2 * pi * y)
    dux_dy = 2 * pi * pi * np.sin(pi * x) ** 2 * np.cos(2 * pi * y)
    duy_dx = -2 * pi * pi * np.cos(2 * pi * x) * np.sin(pi * y) ** 2
    duy_dy = -pi * pi * np.sin(2 * pi * x) * np.sin(2 * pi * y)
    return dux_dx, dux_dy, duy_dx, duy_dy


def mms_pressure(x, y):
    return np.cos(math.pi * x) * np.cos(math.pi * y)


def mms_forcing(x, y, eta, alpha):
    """Strong-form load alpha u - eta Laplace(u) + grad p for piecewise-constant eta."""
    pi = math.pi
    ux, uy = mms_velocity(x, y)
    lap_ux = 2 * pi ** 3 * np.sin(2 * pi * y) * (2 * np.cos(2 * pi * x) - 1)
    lap_uy = -2 * pi ** 3 * np.sin(2 * pi * x) * (2 * np.cos(2 * pi * y) - 1)
    dpx = -pi * np.sin(pi * x) * np.cos(pi * y)
    dpy = -pi * np.cos(pi * x) * np.sin(pi * y)
    return alpha * ux - eta * lap_ux + dpx, alpha * uy - eta * lap_uy + dpy


def config_disc(n: int = 16, levels: int = 3, eta_in: float = 1e3, alpha: float = 1.0,
                radius: float = 0.25) -> Problem:
    """2D unit square, n x n cells, eta = eta_in on cells whose centroid lies in the centred disc."""
    dim = 2
    nn = (n, n)
    L = (1.0, 1.0)
    c = cell_centroids(dim, nn, L)
    inside = (c[:, 0] - 0.5) ** 2 + (c[:, 1] - 0.5) ** 2 <= radius ** 2
    eta = np.where(inside, eta_in, 1.0)
    xv = vnode_coords(dim, nn, L)
    inside_v = (xv[:, 0] - 0.5) ** 2 + (xv[:, 1] - 0.5) ** 2 <= radius ** 2
    fx, fy = mms_forcing(xv[:, 0], xv[:, 1], np.where(inside_v, eta_in, 1.0), alpha)
    f = _full(dim, nn, np.stack([fx, fy], axis=1))
    g = _full(dim, nn)  # u = 0 on the whole boundary
    return Problem("disc16", dim, nn, L, levels, eta, alpha, all_faces(dim), None, f, g)


# --------------------------------------------------------------------------
# config 2: 2D channel with obstacle and stiff bar (FSI2i-like)
# --------------------------------------------------------------------------

CHANNEL_L, CHANNEL_H = 2.5, 0.41


def config_channel(nx: int = 1280, ny: int = 224, levels: int = 6, eta_solid: float = 1e4,
                   alpha: float = 1000.0, v_in: float = 1.0, rho_ratio: Optional[float] = None) -> Problem:
    """Channel 2.5 x 0.41; square obstacle [0.15,0.25]^2 (void cells); bar [0.25,0.60]x[0.19,0.21]
    with eta = eta_solid; parabolic inflow on x = 0, no-slip walls, do-nothing outflow on x = L.
    rho_ratio: alpha per cell, alpha * rho_ratio on the bar (rho_s / rho_f; 10 in FSI2i)."""
    dim = 2
    nn = (nx, ny)
    L = (CHANNEL_L, CHANNEL_H)
    c = cell_centroids(dim, nn, L)
    void = ((c[:, 0] >= 0.15) & (c[:, 0] <= 0.25) & (c[:, 1] >= 0.15) & (c[:, 1] <= 0.25))
    bar = ((c[:, 0] >= 0.25) & (c[:, 0] <= 0.60) & (c[:, 1] >= 0.19) & (c[:, 1] <= 0.21))
    eta = np.where(bar & ~void, eta_solid, 1.0)
    xv = vnode_coords(dim, nn, L)
    ux = np.where(xv[:, 0] == 0.0, 6.0 * v_in * xv[:, 1] * (CHANNEL_H - xv[:, 1]) / CHANNEL_H ** 2, 0.0)
    g = _full(dim, nn, np.stack([ux, np.zeros_like(ux)], axis=1))
    f = _full(dim, nn)
    faces = FACE_XM | FACE_YM | FACE_YP
    al = alpha if rho_ratio is None else np.where(bar & ~void, alpha * rho_ratio, alpha)
    return Problem(f"channel{nx}x{ny}", dim, nn, L, levels, eta, al, faces,
                   void.astype(np.uint8), f, g)


def config_extension(nx: int = 1280, ny: int = 224, levels: int = 6, tip: float = 0.02,
                     point_a=(0.6, 0.2)) -> Problem:
    """Mesh-extension problem on the channel geometry (Eq. "extenstion"): the solid (square obstacle
    [0.15,0.25]^2 and bar [0.25,0.60]x[0.19,0.21]) is made of obstacle cells whose nodes carry the
    solid displacement u_s; every outer face is Dirichlet (u = 0).  u_s: the obstacle is at rest,
    the bar bends, u_y = tip ((x - 0.25) / 0.35)^2.  eta per cell = mu_A / 2 with
    mu_A = 1 + 50 exp(-800 ((x - A_x)^2 + (y - A_y)^2)) (Eq. "mu_distribution") at the cell
    centroid, A = point_a (the bar's tip); alpha = 0; no load."""
    dim = 2
    nn = (nx, ny)
    L = (CHANNEL_L, CHANNEL_H)
    c = cell_centroids(dim, nn, L)
    obst = (c[:, 0] >= 0.15) & (c[:, 0] <= 0.25) & (c[:, 1] >= 0.15) & (c[:, 1] <= 0.25)
    bar = (c[:, 0] >= 0.25) & (c[:, 0] <= 0.60) & (c[:, 1] >= 0.19) & (c[:, 1] <= 0.21)
    solid = obst | bar
    mu = 1.0 + 50.0 * np.exp(-800.0 * ((c[:, 0] - point_a[0]) ** 2 + (c[:, 1] - point_a[1]) ** 2))
    xv = vnode_coords(dim, nn, L)
    s = np.clip((xv[:, 0] - 0.25) / 0.35, 0.0, None)
    on_bar = ((xv[:, 0] >= 0.25) & (xv[:, 0] <= 0.60 + 1e-12) & (xv[:, 1] >= 0.19 - 1e-12)
              & (xv[:, 1] <= 0.21 + 1e-12))
    uy = np.where(on_bar, tip * s * s, 0.0)
    g = _full(dim, nn, np.stack([np.zeros_like(uy), uy], axis=1))
    f = _full(dim, nn)
    return Problem(f"extension{nx}x{ny}", dim, nn, L, levels, 0.5 * mu, 0.0, all_faces(dim),
                   solid.astype(np.uint8), f, g)


# --------------------------------------------------------------------------
# config 3: 3D cube with random stiff spheres
# --------------------------------------------------------------------------

def config_spheres(n: int = 64, levels: int = 5, n_spheres: int = 64, eta_in: float = 1e6,
                   alpha: float = 100.0, seed: int = 0, rmin: float = 0.03, rmax: float = 0.08) -> Problem:
    """Unit cube, n^3 cells; eta = eta_in on cells whose centroid is inside any of the seeded
    spheres (centres U(0,1)^3, radius U(rmin, rmax)); nodal load i.i.d. N(0,1); no-slip faces."""
    dim = 3
    nn = (n, n, n)
    L = (1.0, 1.0, 1.0)
    rng = np.random.Generator(np.random.Philox(seed))
    centres = rng.uniform(0.0, 1.0, size=(n_spheres, 3))
    radii = rng.uniform(rmin, rmax, size=n_spheres)
    c = cell_centroids(dim, nn, L)
    inside = np.zeros(len(c), dtype=bool)
    for s in range(n_spheres):
        inside |= ((c - centres[s]) ** 2).sum(axis=1) <= radii[s] ** 2
    eta = np.where(inside, eta_in, 1.0)
    nv = int(np.prod([2 * k + 1 for k in nn]))
    u = rng.standard_normal(size=(nv, dim))
    f = _full(dim, nn, u)
    g = _full(dim, nn)
    return Problem(f"spheres{n}", dim, nn, L, levels, eta, alpha, all_faces(dim), None, f, g)


def config_discs(n: int = 64, levels: int = 4, n_discs: int = 8, eta_in: float = 1e6, alpha: float = 100.0,
                 seed: int = 0, rmin: float = 0.015, rmax: float = 0.04) -> Problem:
    """2D analog of the spheres workload: unit square, n^2 cells, eta = eta_in on cells whose
    centroid lies in one of the seeded discs (centres U(0,1)^2, radius U(rmin, rmax)), 1 outside;
    nodal load N(0, 1); no-slip."""
    dim = 2
    nn = (n, n)
    L = (1.0, 1.0)
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(n_discs, 2))
    radii = rng.uniform(rmin, rmax, size=n_discs)
    c = cell_centroids(dim, nn, L)
    inside = np.zeros(len(c), dtype=bool)
    for k in range(n_discs):
        inside |= ((c - centres[k]) ** 2).sum(axis=1) <= radii[k] ** 2
    eta = np.where(inside, eta_in, 1.0)
    nv = (2 * n + 1) ** 2
    f = _full(dim, nn, rng.standard_normal(size=(nv, dim)))
    g = _full(dim, nn)
    return Problem(f"discs{n}_s{seed}", dim, nn, L, levels, eta, float(alpha), all_faces(dim), None, f, g)


# --------------------------------------------------------------------------
# generic random instances (tests, batching, serving)
# --------------------------------------------------------------------------

def config_box_inclusion(dim: int, n: Sequence[int], levels: int, contrast: float, alpha: float,
                         seed: int, length: Optional[Sequence[float]] = None,
                         faces: Optional[int] = None, align_coarse: bool = False) -> Problem:
    """Random axis-aligned box inclusion with eta = contrast inside, 1 outside; random N(0,1) load.

    align_coarse: snap the box to cell boundaries of the coarsest level (n / 2^(levels-1) cells per
    axis), so that every level resolves the interface, as the coarse meshes of the paper's FSI
    benchmarks do (Sec. 4: the coarsest mesh is aligned with the solid-fluid interface)."""
    nn = tuple(int(k) for k in n)
    L = tuple(length) if length is not None else (1.0,) * dim
    rng = np.random.default_rng(seed)
    corner = rng.uniform(0.0, 0.6, size=dim) * np.array(L)
    side = rng.uniform(0.1, 0.4, size=dim) * np.array(L)
    if align_coarse:
        for a in range(dim):
            nc = nn[a] >> (levels - 1)
            h0 = L[a] / nc
            i0 = min(int(corner[a] / h0), nc - 1)
            i1 = min(max(i0 + 1, int(round((corner[a] + side[a]) / h0))), nc)
            corner[a], side[a] = i0 * h0, (i1 - i0) * h0
    c = cell_centroids(dim, nn, L)
    inside = np.all((c >= corner) & (c <= np.minimum(corner + side, L)), axis=1)
    eta = np.where(inside, contrast, 1.0)
    nv = int(np.prod([2 * k + 1 for k in nn]))
    f = _full(dim, nn, rng.standard_normal(size=(nv, dim)))
    g = _full(dim, nn)
    return Problem(f"box{dim}d_" + "x".join(map(str, nn)) + f"_s{seed}", dim, nn, L, levels, eta,
                   float(alpha), all_faces(dim) if faces is None else faces, None, f, g)


def config_random_field(dim: int, n: Sequence[int], levels: int = 1, seed: int = 0,
                        contrast: float = 1e6, alpha: float = 10.0,
                        length: Optional[Sequence[float]] = None, faces: Optional[int] = None,
                        void_fraction: float = 0.0) -> Problem:
    """Log-uniform per-cell eta in [1, contrast], random load and Dirichlet data; optional random
    void cells (parity tests of the operators on ragged, obstacle-carrying meshes)."""
    nn = tuple(int(k) for k in n)
    L = tuple(length) if length is not None else tuple(0.5 + 0.25 * a for a in range(dim))
    rng = np.random.default_rng(seed)
    nc = int(np.prod(nn))
    eta = np.exp(rng.uniform(0.0, math.log(contrast), size=nc))
    void = None
    if void_fraction > 0:
        void = (rng.uniform(size=nc) < void_fraction).astype(np.uint8)
    nv = int(np.prod([2 * k + 1 for k in nn]))
    npn = int(np.prod([k + 1 for k in nn]))
    f = rng.standard_normal(size=dim * nv + npn)
    g = rng.standard_normal(size=dim * nv + npn)
    return Problem(f"rand{dim}d_" + "x".join(map(str, nn)) + f"_s{seed}", dim, nn, L, levels, eta,
                   float(alpha), all_faces(dim) if faces is None else faces, void, f, g)


def batch_instances(count: int = 256, seed: int = 0, max2d: int = 256, max3d: int = 32,
                    align_coarse: bool = True) -> List[Problem]:
    """Batched workload: sizes drawn from 2D {16..256}^2 and 3D {8..32}^3 (coarsest level at most
    7 cells (2D) or 4 cells (3D) per axis), contrast U(1e2, 1e6) in a random box, alpha U(1, 1e3).
    align_coarse: snap each box to the coarsest mesh (default); False keeps the box as drawn.  The
    random draws do not depend on align_coarse, so both forms hold the same instances."""
    sizes2 = [s for s in (16, 24, 32, 40, 48, 56, 64, 80, 96, 112, 128, 160, 192, 224, 256) if s <= max2d]
    sizes3 = [s for s in (8, 12, 16, 24, 32) if s <= max3d]
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dim = 2 if rng.uniform() < 0.5 else 3
        s = int(rng.choice(sizes2 if dim == 2 else sizes3))
        contrast = float(rng.uniform(1e2, 1e6))
        alpha = float(rng.uniform(1.0, 1e3))
        out.append(config_box_inclusion(dim, (s,) * dim, levels_for(s, dim), contrast, alpha,
                                        seed=int(rng.integers(1 << 31)), align_coarse=align_coarse))
    return out


def levels_for(n: int, dim: int) -> int:
    """Number of levels that halves n while the coarse mesh keeps more than the limit
    (7 cells per axis in 2D, 4 in 3D)."""
    lim = 7 if dim == 2 else 4
    lv = 1
    while n % 2 == 0 and n // 2 >= 2 and n > lim:
        n //= 2
        lv += 1
    return lv


def serving_stream(rate: float, count: int, seed: int = 0, n2=(32, 512), n3=(8, 48)):
    """Poisson arrivals at `rate` req/s; sizes log-uniform in n2 (2D) and n3 (3D) rounded to
    c * 2^k with a small coarse c; random-inclusion contrast log-uniform up to 1e6."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for i in range(count):
        t += rng.exponential(1.0 / rate)
        dim = 2 if rng.uniform() < 0.5 else 3
        lo, hi = n2 if dim == 2 else n3
        s = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        s = _round_pow2_mult(s, 7 if dim == 2 else 4)
        contrast = float(math.exp(rng.uniform(0.0, math.log(1e6))))
        alpha = float(rng.uniform(1.0, 1e3))
        p = config_box_inclusion(dim, (s,) * dim, levels_for(s, dim), contrast, alpha,
                                 seed=int(rng.integers(1 << 31)), align_coarse=True)
        reqs.append((t, p))
    return reqs


@dataclasses.dataclass
class ProblemSpec:
    """A box-inclusion instance described by its draws alone (no arrays): the serving workload
    holds thousands of these and builds each one's arrays only when its setup starts."""

    dim: int
    n: tuple
    levels: int
    contrast: float
    alpha: float
    seed: int
    length: tuple = ()
    dirichlet_faces: int = -1
    void: None = None

    def __post_init__(self):
        if not self.length:
            self.length = (1.0,) * self.dim
        if self.dirichlet_faces < 0:
            self.dirichlet_faces = all_faces(self.dim)

    @property
    def n_total(self) -> int:
        return self.dim * int(np.prod([2 * k + 1 for k in self.n])) + int(np.prod([k + 1 for k in self.n]))

    def build(self) -> Problem:
        return config_box_inclusion(self.dim, self.n, self.levels, self.contrast, self.alpha, seed=self.seed,
                                    length=self.length, faces=self.dirichlet_faces, align_coarse=True)


def serving_specs(count: int, seed: int = 0, n2=(32, 1536), n3=(8, 96)) -> List[ProblemSpec]:
    """Request mix of the serving workload: dimension 2 or 3 with probability 1/2, size
    log-uniform in n2 (2D) or n3 (3D) rounded to c * 2^k with a small coarse c, box inclusion
    aligned with the coarsest mesh with contrast log-uniform in [1, 1e6], alpha U(1, 1e3).  The
    default ranges put the mean device footprint near 2.5 GB (largest ~20 GB), so that at high
    request rates a 150 GB admission cap binds."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        dim = 2 if rng.uniform() < 0.5 else 3
        lo, hi = n2 if dim == 2 else n3
        s = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        s = _round_pow2_mult(s, 7 if dim == 2 else 4)
        contrast = float(math.exp(rng.uniform(0.0, math.log(1e6))))
        alpha = float(rng.uniform(1.0, 1e3))
        out.append(ProblemSpec(dim, (s,) * dim, levels_for(s, dim), contrast, alpha, int(rng.integers(1 << 31))))
    return out


def _round_pow2_mult(s: int, cmax: int) -> int:
    best = None
    for c in range(2, cmax + 1):
        k = 0
        while c * (2 ** (k + 1)) <= s * 1.5:
            k += 1
        for kk in (k - 1, k):
            if kk < 0:
                continue
            v = c * 2 ** kk
            if best is None or abs(v - s) < abs(best - s):
                best = v
    return int(best)
