"""Seeded synthetic mesh and boundary-condition generators.

This module only produces inputs: vertex coordinates, cell connectivity,
tagged boundary edges and the boundary-condition table for each tag.  It holds
none of the finite-volume lattice Boltzmann arithmetic (no areas, normals,
gradients or equilibria), so both the CUDA path and the CPU oracle can be fed
from it.

The paper builds its meshes with Salome (Sec. 3); those meshes are not
available, so every case here is a seeded stand-in with the same structure:

* plate-driven Couette flow (Sec. 3.1): a periodic channel of right
  triangles whose interior vertices are jittered;
* lid-driven cavity (Sec. 3.2): a non-uniform Cartesian quad mesh with
  tanh wall clustering;
* flow past a cylinder (Sec. 3.3): a hybrid mesh, an O-grid of quads at
  the wall and triangles out to a circular far field;
* fully periodic and inlet/outlet channels used by the invariant tests.

All cells are listed counter-clockwise.  Boundary-condition kinds follow the
paper's ghost-cell section (Sec. 2.4.1, 2.4.2); periodic pairs follow the
Couette set-up of Sec. 3.1.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

# Boundary-condition kinds (same numbering as the C headers use).
BC_WALL = 0
BC_INLET = 1
BC_OUTLET = 2
BC_SYMMETRY = 3
BC_PERIODIC = 4


@dataclasses.dataclass
class BC:
    """One boundary-condition tag.

    kind      -- BC_WALL / BC_INLET / BC_OUTLET / BC_SYMMETRY / BC_PERIODIC
    external  -- 1: external-flow rules (inlet rho* = rho_inf, outlet ghost =
                 interior value); 0: internal-flow rules (inlet rho* = rho_i,
                 pressure outlet)
    u_w       -- wall velocity (walls)
    rho_inf   -- free-stream density (inlet / outlet)
    u_inf     -- free-stream velocity (inlet / outlet)
    partner   -- tag of the matching periodic boundary (periodic only)
    shift     -- vector that, added to the partner edge's points, gives this
                 edge's points (periodic only)
    """

    kind: int
    external: int = 1
    u_w: tuple = (0.0, 0.0)
    rho_inf: float = 1.0
    u_inf: tuple = (0.0, 0.0)
    partner: int = -1
    shift: tuple = (0.0, 0.0)


@dataclasses.dataclass
class Mesh:
    """Polygonal 2-D mesh in plain arrays.

    xy        -- float64 [n_vert, 2]
    cell_ptr  -- int64   [n_cell + 1], CSR offsets into cell_vert
    cell_vert -- int32   [cell_ptr[-1]], vertices of each cell, CCW
    bedge     -- int32   [n_bedge, 2], boundary edges as vertex pairs
    btag      -- int32   [n_bedge], index into bcs
    bcs       -- list of BC, one per tag
    name      -- short description of the case
    """

    xy: np.ndarray
    cell_ptr: np.ndarray
    cell_vert: np.ndarray
    bedge: np.ndarray
    btag: np.ndarray
    bcs: List[BC]
    name: str = ""

    @property
    def n_vert(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_cell(self) -> int:
        return int(self.cell_ptr.shape[0] - 1)

    @property
    def n_bedge(self) -> int:
        return int(self.bedge.shape[0])

    def permuted(self, perm: np.ndarray) -> "Mesh":
        """Same mesh with cells listed in the order perm (new k = old perm[k])."""
        cells = [self.cell_vert[self.cell_ptr[c]:self.cell_ptr[c + 1]] for c in perm]
        ptr = np.zeros(len(cells) + 1, np.int64)
        ptr[1:] = np.cumsum([len(c) for c in cells])
        return Mesh(self.xy.copy(), ptr, np.concatenate(cells).astype(np.int32),
                    self.bedge.copy(), self.btag.copy(), list(self.bcs), self.name)

    def bc_arrays(self):
        """BC table as plain arrays (kind, external, u_w, rho_inf, u_inf, partner, shift)."""
        n = len(self.bcs)
        kind = np.array([b.kind for b in self.bcs], np.int32)
        ext = np.array([b.external for b in self.bcs], np.int32)
        uw = np.array([b.u_w for b in self.bcs], np.float64).reshape(n, 2)
        rinf = np.array([b.rho_inf for b in self.bcs], np.float64)
        uinf = np.array([b.u_inf for b in self.bcs], np.float64).reshape(n, 2)
        partner = np.array([b.partner for b in self.bcs], np.int32)
        shift = np.array([b.shift for b in self.bcs], np.float64).reshape(n, 2)
        return kind, ext, uw, rinf, uinf, partner, shift


def _pack(xy, cells: Sequence[Sequence[int]], bedges, btags, bcs, name) -> Mesh:
    ptr = np.zeros(len(cells) + 1, np.int64)
    ptr[1:] = np.cumsum([len(c) for c in cells])
    cv = np.fromiter((v for c in cells for v in c), np.int32, count=int(ptr[-1]))
    return Mesh(np.ascontiguousarray(xy, np.float64), ptr, cv,
                np.asarray(bedges, np.int32).reshape(-1, 2),
                np.asarray(btags, np.int32).reshape(-1), list(bcs), name)


def _grid_vertices(xs: np.ndarray, ys: np.ndarray) -> np.ndarray:
    X, Y = np.meshgrid(xs, ys, indexing="xy")  # [ny+1, nx+1]
    return np.stack([X.ravel(), Y.ravel()], axis=1)


def _rect_boundary(nx: int, ny: int, vid, tags):
    """Boundary edges of a structured (nx x ny) rectangle, CCW around the domain.

    tags = (bottom, right, top, left)."""
    be, bt = [], []
    for i in range(nx):                      # bottom, left to right
        be.append((vid(i, 0), vid(i + 1, 0))); bt.append(tags[0])
    for j in range(ny):                      # right, bottom to top
        be.append((vid(nx, j), vid(nx, j + 1))); bt.append(tags[1])
    for i in range(nx, 0, -1):               # top, right to left
        be.append((vid(i, ny), vid(i - 1, ny))); bt.append(tags[2])
    for j in range(ny, 0, -1):               # left, top to bottom
        be.append((vid(0, j), vid(0, j - 1))); bt.append(tags[3])
    return be, bt


def _jitter_interior(xy, nx, ny, hx, hy, amp, rng):
    """Move strictly interior vertices of a structured grid by U(-amp, amp) x spacing."""
    xy = xy.copy()
    for j in range(1, ny):
        for i in range(1, nx):
            k = j * (nx + 1) + i
            xy[k, 0] += rng.uniform(-amp, amp) * hx
            xy[k, 1] += rng.uniform(-amp, amp) * hy
    return xy


def _split_tris(nx, ny, vid, alternate=False):
    cells = []
    for j in range(ny):
        for i in range(nx):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            if alternate and (i + j) % 2 == 1:
                cells.append((a, b, d)); cells.append((b, c, d))
            else:
                cells.append((a, b, c)); cells.append((a, c, d))
    return cells


def couette(nx: int = 32, ny: int = 8, h: float = 1.0, U: float = 0.1,
            jitter: float = 0.1, seed: int = 1812) -> Mesh:
    """Plate-driven Couette channel (Sec. 3.1).

    An nx x ny grid of squares of side h, each split into two right triangles
    along the same diagonal; interior vertices jittered by U(-jitter, jitter) x h
    on both axes (seeded).  Bottom wall at rest, top wall moving at (U, 0),
    periodic in x."""
    rng = np.random.default_rng(seed)
    xy = _grid_vertices(np.arange(nx + 1) * h, np.arange(ny + 1) * h)
    xy = _jitter_interior(xy, nx, ny, h, h, jitter, rng)
    vid = lambda i, j: j * (nx + 1) + i
    cells = _split_tris(nx, ny, vid)
    L = nx * h
    # tags: 0 bottom wall, 1 right periodic, 2 top wall, 3 left periodic
    be, bt = _rect_boundary(nx, ny, vid, (0, 1, 2, 3))
    bcs = [BC(BC_WALL, u_w=(0.0, 0.0)),
           BC(BC_PERIODIC, partner=3, shift=(L, 0.0)),
           BC(BC_WALL, u_w=(U, 0.0)),
           BC(BC_PERIODIC, partner=1, shift=(-L, 0.0))]
    return _pack(xy, cells, be, bt, bcs, f"couette{nx}x{ny}")


def periodic_tri(nx: int = 16, ny: int = 12, lx: float = 1.0, ly: float = 1.0,
                 jitter: float = 0.15, seed: int = 7, alternate: bool = True) -> Mesh:
    """Fully periodic rectangle [0,lx] x [0,ly] of triangles, interior vertices jittered."""
    rng = np.random.default_rng(seed)
    hx, hy = lx / nx, ly / ny
    xy = _grid_vertices(np.arange(nx + 1) * hx, np.arange(ny + 1) * hy)
    xy = _jitter_interior(xy, nx, ny, hx, hy, jitter, rng)
    vid = lambda i, j: j * (nx + 1) + i
    cells = _split_tris(nx, ny, vid, alternate)
    be, bt = _rect_boundary(nx, ny, vid, (0, 1, 2, 3))
    bcs = [BC(BC_PERIODIC, partner=2, shift=(0.0, -ly)),
           BC(BC_PERIODIC, partner=3, shift=(lx, 0.0)),
           BC(BC_PERIODIC, partner=0, shift=(0.0, ly)),
           BC(BC_PERIODIC, partner=1, shift=(-lx, 0.0))]
    return _pack(xy, cells, be, bt, bcs, f"periodic{nx}x{ny}")


def periodic_quad(nx: int = 12, ny: int = 10, lx: float = 1.0, ly: float = 1.0,
                  jitter: float = 0.1, seed: int = 11) -> Mesh:
    """Fully periodic rectangle of jittered quadrilaterals."""
    rng = np.random.default_rng(seed)
    hx, hy = lx / nx, ly / ny
    xy = _grid_vertices(np.arange(nx + 1) * hx, np.arange(ny + 1) * hy)
    xy = _jitter_interior(xy, nx, ny, hx, hy, jitter, rng)
    vid = lambda i, j: j * (nx + 1) + i
    cells = [(vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1))
             for j in range(ny) for i in range(nx)]
    be, bt = _rect_boundary(nx, ny, vid, (0, 1, 2, 3))
    bcs = [BC(BC_PERIODIC, partner=2, shift=(0.0, -ly)),
           BC(BC_PERIODIC, partner=3, shift=(lx, 0.0)),
           BC(BC_PERIODIC, partner=0, shift=(0.0, ly)),
           BC(BC_PERIODIC, partner=1, shift=(-lx, 0.0))]
    return _pack(xy, cells, be, bt, bcs, f"pquad{nx}x{ny}")


def tanh_nodes(n: int, ratio: float) -> np.ndarray:
    """n+1 nodes on [0,1] clustered at both ends: x_i = (1 + tanh(b(2i/n-1))/tanh b)/2,
    with b chosen so that (smallest cell)/(largest cell) = 1/ratio."""
    def cell_ratio(b):
        x = 0.5 * (1.0 + np.tanh(b * (2.0 * np.arange(n + 1) / n - 1.0)) / np.tanh(b))
        d = np.diff(x)
        return d.max() / d.min()
    if ratio <= 1.0:
        return np.linspace(0.0, 1.0, n + 1)
    lo, hi = 1e-6, 20.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if cell_ratio(mid) < ratio:
            lo = mid
        else:
            hi = mid
    b = 0.5 * (lo + hi)
    x = 0.5 * (1.0 + np.tanh(b * (2.0 * np.arange(n + 1) / n - 1.0)) / np.tanh(b))
    x[0], x[-1] = 0.0, 1.0
    return x


def cavity(n: int = 128, ratio: float = 20.0, U: float = 0.1, L: float = 1.0,
           triangles: bool = False) -> Mesh:
    """Lid-driven square cavity (Sec. 3.2) on a tanh-stretched Cartesian grid.

    Quads by default (the paper's non-uniform Cartesian mesh of its timing
    study); triangles=True splits each quad in two.  Lid (top) moves at (U, 0);
    the other three walls are at rest."""
    xs = tanh_nodes(n, ratio) * L
    xy = _grid_vertices(xs, xs)
    vid = lambda i, j: j * (n + 1) + i
    if triangles:
        cells = _split_tris(n, n, vid, alternate=True)
    else:
        cells = [(vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1))
                 for j in range(n) for i in range(n)]
    be, bt = _rect_boundary(n, n, vid, (0, 0, 1, 0))
    bcs = [BC(BC_WALL, u_w=(0.0, 0.0)), BC(BC_WALL, u_w=(U, 0.0))]
    return _pack(xy, cells, be, bt, bcs, f"cavity{n}")


def channel(nx: int = 16, ny: int = 8, lx: float = 2.0, ly: float = 1.0,
            u_inf=(0.05, 0.0), rho_inf: float = 1.0, jitter: float = 0.1,
            seed: int = 3, top_bottom: str = "inlet", external: int = 1) -> Mesh:
    """Rectangular far-field box of triangles: left inlet, right outlet, top and
    bottom either inlet (the paper's external-flow set-up, Sec. 3.3) or
    symmetry planes."""
    rng = np.random.default_rng(seed)
    hx, hy = lx / nx, ly / ny
    xy = _grid_vertices(np.arange(nx + 1) * hx, np.arange(ny + 1) * hy)
    xy = _jitter_interior(xy, nx, ny, hx, hy, jitter, rng)
    vid = lambda i, j: j * (nx + 1) + i
    cells = _split_tris(nx, ny, vid, alternate=True)
    tb = {"inlet": 0, "symmetry": 2, "outlet": 1}[top_bottom]
    be, bt = _rect_boundary(nx, ny, vid, (tb, 1, tb, 0))
    bcs = [BC(BC_INLET, external=external, rho_inf=rho_inf, u_inf=tuple(u_inf)),
           BC(BC_OUTLET, external=external, rho_inf=rho_inf, u_inf=tuple(u_inf)),
           BC(BC_SYMMETRY)]
    return _pack(xy, cells, be, bt, bcs, f"channel{nx}x{ny}")


def two_triangles(lid: float = 0.1, periodic: bool = False) -> Mesh:
    """Unit square split into two triangles: walls (lid moving) or fully periodic."""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    cells = [(0, 1, 2), (0, 2, 3)]
    be = [(0, 1), (1, 2), (2, 3), (3, 0)]
    if periodic:
        bt = [0, 1, 2, 3]
        bcs = [BC(BC_PERIODIC, partner=2, shift=(0.0, -1.0)),
               BC(BC_PERIODIC, partner=3, shift=(1.0, 0.0)),
               BC(BC_PERIODIC, partner=0, shift=(0.0, 1.0)),
               BC(BC_PERIODIC, partner=1, shift=(-1.0, 0.0))]
    else:
        bt = [0, 0, 1, 0]
        bcs = [BC(BC_WALL), BC(BC_WALL, u_w=(lid, 0.0))]
    return _pack(xy, cells, be, bt, bcs, "two_triangles")


def cylinder_hybrid(n_rad: int = 100, n_circ: int = 200, D: float = 1.0,
                    first: float = 0.0015, growth: float = 1.05,
                    r_far: float = 30.0, n_tri_rings: int = 100,
                    u_inf: float = 0.05, rho_inf: float = 1.0,
                    jitter: float = 0.1, seed: int = 100,
                    center=(0.0, 0.0)) -> Mesh:
    """Hybrid mesh around a circular cylinder (Sec. 3.3 style).

    An O-grid of n_rad x n_circ quads with first radial spacing first*D and
    geometric growth, then n_tri_rings rings of triangles (each ring quad split
    in two, interior vertices jittered) out to radius r_far*D.  Tag 0 is the
    cylinder wall, tag 1 the far-field inlet (edge midpoint upstream of the
    centre, x < x_c), tag 2 the far-field outlet (x >= x_c), both with the
    external-flow rules."""
    rng = np.random.default_rng(seed)
    R = 0.5 * D
    radii = [R]
    dr = first * D
    for _ in range(n_rad):
        radii.append(radii[-1] + dr)
        dr *= growth
    r0 = radii[-1]
    q = (r_far * D / r0) ** (1.0 / n_tri_rings)
    for _ in range(n_tri_rings):
        radii.append(radii[-1] * q)
    radii[-1] = r_far * D
    radii = np.array(radii)
    nr = len(radii) - 1
    th = 2.0 * np.pi * np.arange(n_circ) / n_circ
    cx, cy = center
    xy = np.zeros(((nr + 1) * n_circ, 2))
    vid = lambda k, j: k * n_circ + (j % n_circ)
    for k in range(nr + 1):
        xy[k * n_circ:(k + 1) * n_circ, 0] = cx + radii[k] * np.cos(th)
        xy[k * n_circ:(k + 1) * n_circ, 1] = cy + radii[k] * np.sin(th)
    # jitter triangle-region interior rings
    for k in range(n_rad + 1, nr):
        drr = min(radii[k + 1] - radii[k], radii[k] - radii[k - 1])
        for j in range(n_circ):
            v = vid(k, j)
            ds = radii[k] * 2.0 * np.pi / n_circ
            t = th[j] + rng.uniform(-jitter, jitter) * ds / radii[k]
            r = radii[k] + rng.uniform(-jitter, jitter) * drr
            xy[v] = (cx + r * math.cos(t), cy + r * math.sin(t))
    cells = []
    for k in range(nr):
        for j in range(n_circ):
            # radial index k first, then angle: (k,j) -> (k+1,j) -> (k+1,j+1) -> (k,j+1) is CCW
            a, b, c, d = vid(k, j), vid(k + 1, j), vid(k + 1, j + 1), vid(k, j + 1)
            if k < n_rad:
                cells.append((a, b, c, d))
            elif (j + k) % 2 == 0:
                cells.append((a, b, c)); cells.append((a, c, d))
            else:
                cells.append((a, b, d)); cells.append((b, c, d))
    be, bt = [], []
    for j in range(n_circ):   # wall: the cylinder, domain lies outside -> edge runs clockwise
        be.append((vid(0, j + 1), vid(0, j))); bt.append(0)
    for j in range(n_circ):   # far field, CCW
        a, b = vid(nr, j), vid(nr, j + 1)
        xm = 0.5 * (xy[a, 0] + xy[b, 0])
        be.append((a, b)); bt.append(1 if xm < cx else 2)
    bcs = [BC(BC_WALL),
           BC(BC_INLET, external=1, rho_inf=rho_inf, u_inf=(u_inf, 0.0)),
           BC(BC_OUTLET, external=1, rho_inf=rho_inf, u_inf=(u_inf, 0.0))]
    return _pack(xy, cells, be, bt, bcs, f"cylinder{len(cells)}")


def random_state(n_cell: int, seed: int, rho_amp: float = 0.02, u_amp: float = 0.05,
                 noise: float = 1e-3):
    """Seeded random macroscopic fields and a positive non-equilibrium perturbation.

    Returns (rho [n], u [n,2], dev [n,9]): dev is a zero-mean-per-cell noise
    the callers add on top of an equilibrium they compute themselves."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + rho_amp * rng.uniform(-1.0, 1.0, n_cell)
    u = u_amp * rng.uniform(-1.0, 1.0, (n_cell, 2))
    dev = noise * rng.uniform(-1.0, 1.0, (n_cell, 9))
    return rho, u, dev


def batch_specs(n: int = 256, seed: int = 2018, re_lo: float = 10.0, re_hi: float = 1000.0):
    """Instance list for the batched solve: thirds of Couette (64x16 -> 2048 cells),
    stretched cavities (128^2) and cylinder hybrids (~60k cells), Reynolds number
    log-uniform in [re_lo, re_hi]."""
    rng = np.random.default_rng(seed)
    kinds = ["couette", "cavity", "cylinder"]
    out = []
    for k in range(n):
        re = float(np.exp(rng.uniform(np.log(re_lo), np.log(re_hi))))
        out.append({"kind": kinds[k % 3], "re": re, "seed": int(rng.integers(1 << 30))})
    return out


def bricks(nx: int = 8, ny: int = 6, U: float = 0.1, lx: float = 1.0, ly: float = 1.0) -> Mesh:
    """Running-bond brick mesh of a walled box: most cells are hexagons (two grid
    squares merged, with a straight-through vertex in the middle of each long
    side), row ends are single squares.  Exercises cells with up to 6 faces.
    Lid (top) moves at (U, 0)."""
    if nx % 2:
        raise ValueError("nx must be even")
    hx, hy = lx / nx, ly / ny
    xy = _grid_vertices(np.arange(nx + 1) * hx, np.arange(ny + 1) * hy)
    vid = lambda i, j: j * (nx + 1) + i
    cells = []
    for j in range(ny):
        i = 0
        if j % 2 == 1:
            cells.append((vid(0, j), vid(1, j), vid(1, j + 1), vid(0, j + 1)))
            i = 1
        while i + 2 <= nx:
            cells.append((vid(i, j), vid(i + 1, j), vid(i + 2, j), vid(i + 2, j + 1),
                          vid(i + 1, j + 1), vid(i, j + 1)))
            i += 2
        if i < nx:
            cells.append((vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)))
    be, bt = _rect_boundary(nx, ny, vid, (0, 0, 1, 0))
    bcs = [BC(BC_WALL), BC(BC_WALL, u_w=(U, 0.0))]
    return _pack(xy, cells, be, bt, bcs, f"bricks{nx}x{ny}")


def tandem_cylinders(gap_ratio: float = 3.0, D: float = 1.0, n_circ: int = 160,
                     first: float = 0.0015, growth: float = 1.1, r_far: float = 30.0,
                     grade: float = 0.12, u_inf: float = 0.05, rho_inf: float = 1.0,
                     seed: int = 0) -> Mesh:
    """Two cylinders of diameter D in tandem, centres (0, 0) and (gap_ratio*D, 0)
    (the tandem arrangement of Sec. 3.4).  Each has an O-grid of quads (first
    radial spacing first*D, geometric growth) as thick as the gap allows; the
    rest of the disc of radius r_far*D around the midpoint is filled with
    triangles whose size grows with the distance from the cylinders (rate
    `grade`), from a Delaunay triangulation of graded jittered points.  Walls on
    both cylinders, far-field inlet / outlet as in cylinder_hybrid."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    R = 0.5 * D
    L = gap_ratio * D
    centers = [(0.0, 0.0), (L, 0.0)]
    thick = min(0.35 * (L - D), 1.0 * D)
    radii = [R]
    dr = first * D
    while radii[-1] - R < thick:
        radii.append(radii[-1] + dr)
        dr *= growth
    radii[-1] = R + thick
    n_rad = len(radii) - 1
    Ro = radii[-1]
    th = 2.0 * np.pi * np.arange(n_circ) / n_circ
    xy = []
    cells = []
    be, bt = [], []
    for (cx, cy) in centers:
        off = len(xy)
        for r in radii:
            for t in th:
                xy.append((cx + r * math.cos(t), cy + r * math.sin(t)))
        vid = lambda k, j, off=off: off + k * n_circ + (j % n_circ)
        for k in range(n_rad):
            for j in range(n_circ):
                cells.append((vid(k, j), vid(k + 1, j), vid(k + 1, j + 1), vid(k, j + 1)))
        for j in range(n_circ):
            be.append((vid(0, j + 1), vid(0, j))); bt.append(0)
    n_og = len(xy)
    outer_ids = [[c * (n_rad + 1) * n_circ + n_rad * n_circ + j for j in range(n_circ)] for c in range(2)]
    s_o = 2.0 * np.pi * Ro / n_circ
    xm = 0.5 * L
    Rf = r_far * D

    def size(p):
        d = min(math.hypot(p[0] - cx, p[1] - cy) for cx, cy in centers) - Ro
        return s_o + grade * max(d, 0.0)

    # far-field ring
    h_far = size((xm + Rf, 0.0))
    n_far = max(16, int(round(2 * np.pi * Rf / h_far)))
    far_ids = []
    for j in range(n_far):
        t = 2 * np.pi * j / n_far
        far_ids.append(len(xy))
        xy.append((xm + Rf * math.cos(t), Rf * math.sin(t)))
    # graded interior points: level l has spacing s_o * 2^l where size() falls in it
    pts = []
    h = s_o
    while h < 2 * Rf:
        nx = int(math.ceil(2 * Rf / h))
        xs = xm - Rf + (np.arange(nx) + 0.5) * h
        ys = -Rf + (np.arange(nx) + 0.5) * h
        X, Y = np.meshgrid(xs, ys)
        P = np.stack([X.ravel(), Y.ravel()], 1)
        P = P + rng.uniform(-0.2, 0.2, P.shape) * h
        d = np.min(np.stack([np.hypot(P[:, 0] - cx, P[:, 1] - cy) for cx, cy in centers]), 0) - Ro
        sz = s_o + grade * np.maximum(d, 0.0)
        keep = (sz >= h) & (sz < 2 * h) & (d > 0.6 * sz) & (np.hypot(P[:, 0] - xm, P[:, 1]) < Rf - 0.6 * sz)
        if h == s_o:
            keep = (sz < 2 * h) & (d > 0.6 * sz) & (np.hypot(P[:, 0] - xm, P[:, 1]) < Rf - 0.6 * sz)
        pts.append(P[keep])
        h *= 2
    base = len(xy)
    xy = np.array(xy + [tuple(p) for p in np.concatenate(pts)], dtype=np.float64)
    # triangulate O-grid outer rings, far ring and field points
    tri_ids = np.array(sum(outer_ids, []) + far_ids + list(range(base, len(xy))))
    tri = Delaunay(xy[tri_ids])
    simp = tri_ids[tri.simplices]
    cen = xy[simp].mean(1)
    inside = np.zeros(len(simp), bool)
    for cx, cy in centers:
        inside |= np.hypot(cen[:, 0] - cx, cen[:, 1] - cy) < Ro
    inside |= np.hypot(cen[:, 0] - xm, cen[:, 1]) > Rf
    simp = simp[~inside]
    # CCW
    a, b, c = xy[simp[:, 0]], xy[simp[:, 1]], xy[simp[:, 2]]
    cr = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    simp[cr < 0] = simp[cr < 0][:, [0, 2, 1]]
    # every O-grid outer edge and far-field edge must be a triangle edge
    edges = set()
    for t3 in simp:
        for k in range(3):
            edges.add(tuple(sorted((int(t3[k]), int(t3[(k + 1) % 3])))))
    for ring in outer_ids:
        for j in range(n_circ):
            if tuple(sorted((ring[j], ring[(j + 1) % n_circ]))) not in edges:
                raise ValueError("triangulation missed an O-grid edge; change grade or n_circ")
    for j in range(n_far):
        e = (far_ids[j], far_ids[(j + 1) % n_far])
        if tuple(sorted(e)) not in edges:
            raise ValueError("triangulation missed a far-field edge")
        xmid = 0.5 * (xy[e[0], 0] + xy[e[1], 0])
        be.append(e); bt.append(1 if xmid < xm else 2)
    cells += [tuple(int(v) for v in t3) for t3 in simp]
    # drop field points that ended up unused (none expected)
    used = np.zeros(len(xy), bool)
    for cl in cells:
        used[list(cl)] = True
    remap = -np.ones(len(xy), np.int64)
    remap[used] = np.arange(used.sum())
    xy = xy[used]
    cells = [tuple(int(remap[v]) for v in cl) for cl in cells]
    be = [(int(remap[a_]), int(remap[b_])) for a_, b_ in be]
    bcs = [BC(BC_WALL),
           BC(BC_INLET, external=1, rho_inf=rho_inf, u_inf=(u_inf, 0.0)),
           BC(BC_OUTLET, external=1, rho_inf=rho_inf, u_inf=(u_inf, 0.0))]
    return _pack(xy, cells, be, bt, bcs, f"tandem{gap_ratio:.2f}_{len(cells)}")
