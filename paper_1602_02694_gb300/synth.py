"""Seeded synthetic inputs for the WLS-ENO hot path.

This module is shared by the oracle tests, the GPU parity tests and the
benchmark.  It holds none of the method's arithmetic (no stencils, moments,
weights, least squares, fluxes or time stepping): only

* jittered simplex meshes shaped like the paper's test meshes (Sec. 5.2 and
  Sec. 5.3 use unstructured triangle and tetrahedral meshes of a square or a
  cube; here they are rescaled to the unit square / cube),
* cell averages of analytic initial fields (the method's input, Eq. (4)'s
  "given the cell averages"), integrated with a high-degree product rule, and
* seeded random draws (loss weights, directions).

Jitter recipe: every vertex of a regular lattice with spacing h = 1/n moves
by independent U(-j*h, j*h) offsets per coordinate, drawn with numpy's PCG64
``default_rng(seed)`` in vertex-index order, x then y (then z).  On a
periodic mesh every unique vertex is jittered once; on a transmissive mesh
boundary vertices move only tangentially and corners stay fixed.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Mesh:
    """A conforming simplex mesh.

    vertices: float64 [n_vertices][dim] (periodic meshes: in [0,1)^dim + jitter)
    cells:    int64 [n_cells][dim+1], positively oriented simplices
    period:   float64 [dim]; 0 along an axis means transmissive (no wrap)
    cell_coords: float64 [n_cells][dim+1][dim] the cells' vertex coordinates
        with periodic wrap removed (each cell as one connected simplex).  It is
        only used here to integrate initial data; the method's two
        implementations unwrap cells themselves from ``vertices``/``period``.
    """

    vertices: np.ndarray
    cells: np.ndarray
    period: np.ndarray
    cell_coords: np.ndarray
    n: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def dim(self) -> int:
        return self.vertices.shape[1]

    @property
    def n_cells(self) -> int:
        return self.cells.shape[0]


def tri_mesh(n: int, jitter: float = 0.2, seed: int = 1, periodic: bool = True) -> Mesh:
    """n x n squares on the unit square, each split along its "/" diagonal
    into two counter-clockwise triangles (2 n^2 cells)."""
    if n < 4:
        raise ValueError("n must be >= 4")
    h = 1.0 / n
    rng = np.random.default_rng(seed)
    nv1 = n if periodic else n + 1
    jj, ii = np.meshgrid(np.arange(nv1), np.arange(nv1), indexing="ij")
    base = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1)  # vertex v = j*nv1 + i
    jit = rng.uniform(-jitter * h, jitter * h, size=base.shape)
    if not periodic:
        bi = ii.ravel()
        bj = jj.ravel()
        on_x = (bi == 0) | (bi == n)  # vertical boundary: keep x
        on_y = (bj == 0) | (bj == n)  # horizontal boundary: keep y
        jit[on_x, 0] = 0.0
        jit[on_y, 1] = 0.0
    verts = base + jit
    lattice_jit = jit  # jitter per lattice vertex, reused for unwrapped coords

    def vid(i, j):
        if periodic:
            return (j % n) * n + (i % n)
        return j * nv1 + i

    cells = []
    coords = []
    for j in range(n):
        for i in range(n):
            v00, v10, v11, v01 = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            p = {}
            for (di, dj), v in (((0, 0), v00), ((1, 0), v10), ((1, 1), v11), ((0, 1), v01)):
                p[(di, dj)] = np.array([(i + di) * h, (j + dj) * h]) + lattice_jit[v]
            cells.append((v00, v10, v11))
            coords.append((p[(0, 0)], p[(1, 0)], p[(1, 1)]))
            cells.append((v00, v11, v01))
            coords.append((p[(0, 0)], p[(1, 1)], p[(0, 1)]))
    period = np.array([1.0, 1.0]) if periodic else np.zeros(2)
    return Mesh(verts, np.asarray(cells, dtype=np.int64), period,
                np.asarray(coords, dtype=np.float64), n=n,
                meta={"kind": "tri", "jitter": jitter, "seed": seed, "periodic": periodic})


def tet_mesh(n: int, jitter: float = 0.15, seed: int = 1, periodic: bool = True) -> Mesh:
    """n^3 hexahedra on the unit cube, each split into the 6 Kuhn tetrahedra
    along its main diagonal (6 n^3 cells), periodic or transmissive."""
    if n < 3:
        raise ValueError("n must be >= 3")
    h = 1.0 / n
    rng = np.random.default_rng(seed)
    nv1 = n if periodic else n + 1
    kk, jj, ii = np.meshgrid(np.arange(nv1), np.arange(nv1), np.arange(nv1), indexing="ij")
    lat = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)  # v = (k*nv1 + j)*nv1 + i
    jit = rng.uniform(-jitter * h, jitter * h, size=lat.shape)
    if not periodic:
        jit[(lat == 0) | (lat == n)] = 0.0  # boundary vertices move tangentially only
    verts = lat * h + jit

    def vid(ijk):
        if periodic:
            ijk = ijk % n
        return (ijk[:, 2] * nv1 + ijk[:, 1]) * nv1 + ijk[:, 0]

    ck, cj, ci = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    cube = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], axis=1)
    cells = np.zeros((cube.shape[0], 6, 4), dtype=np.int64)
    coords = np.zeros((cube.shape[0], 6, 4, 3))
    for t, perm in enumerate(itertools.permutations(range(3))):
        path = [np.zeros(3, dtype=np.int64)]
        for ax in perm:
            nxt = path[-1].copy()
            nxt[ax] += 1
            path.append(nxt)
        # orientation of the unjittered tet = sign of the axis permutation
        if np.linalg.det(np.eye(3)[list(perm)]) < 0:
            path[2], path[3] = path[3], path[2]
        for a, o in enumerate(path):
            v = vid(cube + o)
            cells[:, t, a] = v
            coords[:, t, a, :] = (cube + o) * h + jit[v]
    return Mesh(verts, cells.reshape(-1, 4), np.ones(3) if periodic else np.zeros(3),
                coords.reshape(-1, 4, 3), n=n,
                meta={"kind": "tet", "jitter": jitter, "seed": seed, "periodic": periodic})


def line_mesh(nodes: np.ndarray) -> Mesh:
    """A 1-D mesh of the intervals between consecutive ``nodes`` (transmissive)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    cells = np.stack([np.arange(len(nodes) - 1), np.arange(1, len(nodes))], axis=1)
    coords = nodes[cells][:, :, None]
    return Mesh(nodes[:, None].copy(), cells.astype(np.int64), np.zeros(1), coords,
                n=len(nodes) - 1, meta={"kind": "line"})


def periodic_line_mesh(n: int, jitter: float = 0.0, seed: int = 0) -> Mesh:
    """n intervals on the periodic unit interval: nodes k/n jittered by
    U(-jitter, jitter)/n (PCG64 seed), the last interval wrapping to node 0."""
    rng = np.random.default_rng(seed)
    nodes = (np.arange(n) + (rng.uniform(-jitter, jitter, n) if jitter > 0 else 0.0)) / n
    cells = np.stack([np.arange(n), (np.arange(n) + 1) % n], axis=1)
    right = nodes[cells[:, 1]] + (cells[:, 1] == 0)  # unwrap the last interval
    coords = np.stack([nodes[cells[:, 0]], right], axis=1)[:, :, None]
    return Mesh(nodes[:, None].copy(), cells.astype(np.int64), np.ones(1), coords,
                n=n, meta={"kind": "periodic line"})


# --------------------------------------------------------------------------
# cell averages of analytic fields
# --------------------------------------------------------------------------

def _gauss_legendre01(k: int):
    x, w = np.polynomial.legendre.leggauss(k)
    return 0.5 * (x + 1.0), 0.5 * w


def simplex_rule(dim: int, k: int = 6):
    """Collapsed (Duffy) Gauss-Legendre product rule on the reference simplex:
    returns barycentric points [Q][dim+1] and weights [Q] summing to 1.
    Exact for polynomials of degree <= 2k-1-dim+1 on the simplex."""
    x, w = _gauss_legendre01(k)
    pts, wts = [], []
    if dim == 1:
        for a, wa in zip(x, w):
            pts.append((1 - a, a))
            wts.append(wa)
    elif dim == 2:
        for s, ws in zip(x, w):
            for t, wt in zip(x, w):
                # y = s*(1-t, t) on the unit triangle; Jacobian s
                l1, l2 = s * (1 - t), s * t
                pts.append((1 - l1 - l2, l1, l2))
                wts.append(2.0 * ws * wt * s)
    elif dim == 3:
        for r, wr in zip(x, w):
            for s, ws in zip(x, w):
                for t, wt in zip(x, w):
                    l1 = r * (1 - s)
                    l2 = r * s * (1 - t)
                    l3 = r * s * t
                    pts.append((1 - l1 - l2 - l3, l1, l2, l3))
                    wts.append(6.0 * wr * ws * wt * r * r * s)
    else:
        raise ValueError(dim)
    return np.asarray(pts), np.asarray(wts)


def cell_averages(mesh: Mesh, f, k: int = 6) -> np.ndarray:
    """Average of f(x) (vectorised over points [P][dim]) over each cell."""
    lam, wq = simplex_rule(mesh.dim, k)
    pts = np.einsum("qv,cvd->cqd", lam, mesh.cell_coords)
    vals = f(pts.reshape(-1, mesh.dim)).reshape(pts.shape[0], pts.shape[1])
    return vals @ wq


def _clip_polygon(poly, axis, bound, keep_greater):
    out = []
    nq = len(poly)
    for a in range(nq):
        p, q = poly[a], poly[(a + 1) % nq]
        pin = (p[axis] >= bound) if keep_greater else (p[axis] <= bound)
        qin = (q[axis] >= bound) if keep_greater else (q[axis] <= bound)
        if pin:
            out.append(p)
        if pin != qin:
            t = (bound - p[axis]) / (q[axis] - p[axis])
            out.append(p + t * (q - p))
    return out


def _polygon_area(poly):
    if len(poly) < 3:
        return 0.0
    a = 0.0
    for k in range(len(poly)):
        x0, y0 = poly[k]
        x1, y1 = poly[(k + 1) % len(poly)]
        a += x0 * y1 - x1 * y0
    return 0.5 * abs(a)


def box_fraction_2d(mesh: Mesh, lo, hi) -> np.ndarray:
    """Exact area fraction of each triangle inside the box [lo, hi] (polygon clipping)."""
    out = np.zeros(mesh.n_cells)
    for c in range(mesh.n_cells):
        tri = [np.asarray(p) for p in mesh.cell_coords[c]]
        area = _polygon_area(tri)
        poly = tri
        for axis in range(2):
            poly = _clip_polygon(poly, axis, lo[axis], True)
            if not poly:
                break
            poly = _clip_polygon(poly, axis, hi[axis], False)
            if not poly:
                break
        out[c] = _polygon_area(poly) / area if poly else 0.0
    return out


def advection_2d_initial(mesh: Mesh) -> np.ndarray:
    """sin(2 pi x) sin(2 pi y) plus the unit indicator of [0.3,0.6]^2."""
    smooth = cell_averages(mesh, lambda p: np.sin(2 * np.pi * p[:, 0]) * np.sin(2 * np.pi * p[:, 1]))
    return smooth + box_fraction_2d(mesh, (0.3, 0.3), (0.6, 0.6))


def burgers_2d_initial(mesh: Mesh) -> np.ndarray:
    """0.5 + sin(2 pi (x + y))."""
    return cell_averages(mesh, lambda p: 0.5 + np.sin(2 * np.pi * (p[:, 0] + p[:, 1])))


def smooth_random_initial(mesh: Mesh, seed: int, kmax: int = 3, std: float = 0.2) -> np.ndarray:
    """0.5 + sum_k a_k sin(2 pi k.x) over the half-plane lattice vectors with
    0 < |k| <= kmax, a_k ~ N(0, std^2)."""
    rng = np.random.default_rng(seed)
    ks = [(kx, ky) for kx in range(-kmax, kmax + 1) for ky in range(-kmax, kmax + 1)
          if (kx > 0 or (kx == 0 and ky > 0)) and kx * kx + ky * ky <= kmax * kmax]
    ks = np.asarray(ks, dtype=np.float64)
    a = rng.normal(0.0, std, size=len(ks))

    def f(p):
        return 0.5 + np.sin(2 * np.pi * (p @ ks.T)) @ a

    return cell_averages(mesh, f)


def gaussian_ball_3d_initial(mesh: Mesh, sub: int = 2) -> np.ndarray:
    """exp(-50 |x-c|^2) plus the indicator of the ball |x-c| <= 0.15, c = (1/2,1/2,1/2),
    min-image distance; the indicator is averaged on the cell's 8^sub sub-tets."""
    c = np.array([0.5, 0.5, 0.5])

    def dist2(p):
        d = p - c
        d -= np.round(d)
        return np.sum(d * d, axis=1)

    smooth = cell_averages(mesh, lambda p: np.exp(-50.0 * dist2(p)))
    lam, wq = simplex_rule(3, 3 + 2 * sub)
    pts = np.einsum("qv,cvd->cqd", lam, mesh.cell_coords)
    ind = (dist2(pts.reshape(-1, 3)) <= 0.15 ** 2).astype(np.float64).reshape(pts.shape[0], -1)
    return smooth + ind @ wq


def quadrant_fractions(mesh: Mesh, x0: float = 0.5, y0: float = 0.5) -> np.ndarray:
    """Exact area fraction of each triangle in the four quadrants around
    (x0, y0), ordered (x<x0,y<y0), (x>x0,y<y0), (x<x0,y>y0), (x>x0,y>y0);
    only cells straddling x = x0 or y = y0 are clipped."""
    X = mesh.cell_coords
    lo = X.min(axis=1)
    hi = X.max(axis=1)
    qx = (lo[:, 0] >= x0).astype(int)
    qy = (lo[:, 1] >= y0).astype(int)
    out = np.zeros((mesh.n_cells, 4))
    out[np.arange(mesh.n_cells), qx + 2 * qy] = 1.0
    straddle = np.nonzero((lo[:, 0] < x0) & (hi[:, 0] > x0) | (lo[:, 1] < y0) & (hi[:, 1] > y0))[0]
    big = 1e9
    boxes = [((-big, -big), (x0, y0)), ((x0, -big), (big, y0)), ((-big, y0), (x0, big)), ((x0, y0), (big, big))]
    for c in straddle:
        tri = [np.asarray(p) for p in X[c]]
        area = _polygon_area(tri)
        for k, (blo, bhi) in enumerate(boxes):
            poly = tri
            for axis in range(2):
                poly = _clip_polygon(poly, axis, blo[axis], True) if poly else poly
                poly = _clip_polygon(poly, axis, bhi[axis], False) if poly else poly
            out[c, k] = _polygon_area(poly) / area if poly else 0.0
    return out


def euler_quadrant_initial(mesh: Mesh, seed: int, gamma: float = 1.4):
    """Four piecewise-constant states around (1/2, 1/2): density U[0.1, 1.5],
    velocity components U[-0.8, 0.8], pressure U[0.03, 1.5], drawn per
    quadrant from ``default_rng(seed)``.  Returns conserved cell averages
    [4][n_cells] (rho, rho u, rho v, E) and the primitive states [4][4]."""
    rng = np.random.default_rng(seed)
    prim = np.stack([rng.uniform(0.1, 1.5, 4), rng.uniform(-0.8, 0.8, 4), rng.uniform(-0.8, 0.8, 4),
                     rng.uniform(0.03, 1.5, 4)], axis=1)  # [quadrant][rho, u, v, p]
    rho, u, v, p = prim.T
    cons = np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)], axis=0)
    frac = quadrant_fractions(mesh)
    return cons @ frac.T, prim


def shock_tube_initial(mesh: Mesh, x0: float = 0.5, left=(1.0, 0.0, 1.0), right=(0.125, 0.0, 0.1),
                       gamma: float = 1.4) -> np.ndarray:
    """1-D Riemann data (density, velocity, pressure) on each side of x0 --
    by default the textbook shock-tube states -- as exact conserved cell
    averages [3][n_cells] (rho, rho u, E) of a 1-D mesh."""
    assert mesh.dim == 1
    a = np.minimum(mesh.cell_coords[:, 0, 0], mesh.cell_coords[:, 1, 0])
    b = np.maximum(mesh.cell_coords[:, 0, 0], mesh.cell_coords[:, 1, 0])
    frac = np.clip((x0 - a) / (b - a), 0.0, 1.0)  # share of the cell left of x0

    def cons(state):
        rho, u, p = state
        return np.array([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])

    return cons(left)[:, None] * frac[None, :] + cons(right)[:, None] * (1.0 - frac)[None, :]


def isentropic_vortex(points: np.ndarray, t: float, gamma: float = 1.4, strength: float = 5.0,
                      core: float = 0.1, center=(0.5, 0.5), velocity=(1.0, 1.0)) -> np.ndarray:
    """Conserved variables [4][P] of the isentropic vortex of the 2-D Euler
    equations (the classic test of Shu's 1998 lecture notes), an exact
    solution: a free stream rho = p = 1 with `velocity`, carrying a vortex
    of temperature drop (gamma-1) s^2/(8 gamma pi^2) exp(1 - r^2) and swirl
    s/(2 pi) exp((1 - r^2)/2) (r in units of `core`), translated with the
    stream (periodic unit square: minimum-image distance).  Spatial units
    scaled by `core` leave the equations unchanged; core 0.1 puts the
    standard [-5, 5]^2 box on the unit square."""
    x = points[:, 0] - center[0] - velocity[0] * t
    y = points[:, 1] - center[1] - velocity[1] * t
    x = (x - np.round(x)) / core
    y = (y - np.round(y)) / core
    r2 = x * x + y * y
    temp = 1.0 - (gamma - 1.0) * strength ** 2 / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = temp ** (1.0 / (gamma - 1.0))
    swirl = strength / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    u = velocity[0] - swirl * y
    v = velocity[1] + swirl * x
    p = rho ** gamma
    return np.stack([rho, rho * u, rho * v, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v)])


def isentropic_vortex_averages(mesh: Mesh, t: float, k: int = 10, **kw) -> np.ndarray:
    """Cell averages [4][n_cells] of `isentropic_vortex` at time t."""
    return np.stack([cell_averages(mesh, lambda P, c=c: isentropic_vortex(P, t, **kw)[c], k=k)
                     for c in range(4)])


def random_unit_directions(n_cells: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(count, n_cells))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def loss_weights(n_cells: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=n_cells)
