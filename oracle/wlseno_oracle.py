"""Plain, slow FP64 CPU oracle of the WLS-ENO finite-volume hot path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or
executes this file: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` do.  It shares no
code with the CUDA library (paper_1602_02694_gb300/csrc) and imports nothing
from the package; its inputs are plain numpy arrays.

Everything is FP64 and written cell by cell, in the paper's order and
notation, from:

  Liu & Jiao, "WLS-ENO: Weighted-Least-Squares Based Essentially
  Non-Oscillatory Schemes for Finite Volume Methods on Unstructured Meshes"
  (arXiv 1602.02694).

  Sec. 1, Eq. (fvm) and Eq. (flux) ....... finite-volume update, LF flux
  Sec. 3.1.1, Eq. (average_eq), Eq. (WLS)  Taylor-moment system, weighted LS
  Sec. 3.1.2, Eqs. (smoothness indicator), (weight)   beta_j, omega_j
  Sec. 3.2 ............................... 2-D/3-D moments about the centroid,
                                           k-ring stencils (1/2- and 1/3-ring)
  Sec. 3.3.1 ............................. half-facet sibling adjacency
  Sec. 3.3.2, Eq. (scaled_WLS) ........... column scaling, QR with column
                                           pivoting, rank-truncated solve
  Sec. 4.2.1, Eq. (3rd-order-Runge-Kutta)  TVD-RK3 (Shu-Osher)

Readings where the paper is silent, garbled or ambiguous (each is listed in
the design notes of the repository):
  * Eq. (fvm) prints the boundary integral multiplied by |tau_i|; it is
    divided by |tau_i| here (the definition of the cell average above it).
  * moments are divided by |tau_j| (the stencil cell), factorials per term.
  * h in eps*h^2 is the mean edge length of the centre cell tau_i.
  * beta_i of the centre cell is the minimum of beta_j over the stencil cells
    that share a facet with tau_i (1-D: tau_{i-1}, tau_{i+1}).
  * rows of the least-squares system are multiplied by omega_j (not sqrt).
  * the expansion point is the centroid of tau_i in every dimension; the
    unknowns are h-normalised, d_kappa = h_i^|kappa| d^kappa u(x_i).
  * numerical rank r = #{k : |R_kk| > rank_tol * |R_11|}; coefficients of
    dropped columns are 0 (basic solution).
  * column pivoting: at each step the lowest-index remaining column whose
    squared trailing norm is within a relative 1e-6 of the largest (after
    the column scaling all norms are 1, so the paper's rule alone leaves the
    first pivot to rounding); trailing norms recomputed at every step.
  * facet quadrature: Gauss-Legendre with 2 points per edge in 2-D, the
    degree-2 three-point rule at barycentric (2/3,1/6,1/6) in 3-D.
  * Lax-Friedrichs alpha: |velocity| for advection; per facet the maximum
    over its quadrature points and both sides of |F'(u).n| for Burgers and
    of |u.n| + c for Euler.
  * time step dt = CFL * min_i r_i / lambda_max with r_i = d|tau_i|/|d tau_i|.
  * periodic meshes: each stencil cell is taken at its minimum-image copy.
  * transmissive boundary facets use u+ = u-.

Parity of every function here is pinned: the scheme in tests/test_oracle_pins.py,
Euler in tests/test_oracle_euler.py, the geometry, facet rules, adjacency,
radius-cut stencils and CFL wave speeds in tests/test_oracle_geometry.py, the
reverse mode (residual_vjp, rk3_step_vjp) against central differences of
the forward in tests/test_oracle_adjoint.py.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np
import scipy.linalg

ADVECTION, BURGERS, EULER = 0, 1, 2


# ----------------------------------------------------------------------------
# geometry (Sec. 1: cells tau_i, volumes |tau_i|, centroids; Sec. 3.2)
# ----------------------------------------------------------------------------

def min_image(delta, period):
    """Wrap a coordinate difference into the nearest periodic image."""
    delta = np.array(delta, dtype=np.float64)
    for c in range(delta.shape[-1]):
        if period[c] > 0:
            delta[..., c] -= period[c] * np.round(delta[..., c] / period[c])
    return delta


def unwrap_cell(vertices, cell, period):
    """Vertex coordinates of one cell as a connected simplex (minimum image
    relative to its first vertex)."""
    x0 = vertices[cell[0]]
    return np.array([x0 + min_image(vertices[v] - x0, period) for v in cell])


def simplex_volume(X):
    d = X.shape[1]
    return abs(np.linalg.det((X[1:] - X[0]).reshape(d, d))) / math.factorial(d)


def facet_measure(F):
    """(d-1)-measure of a facet given by d points in R^d."""
    d = F.shape[1]
    if d == 1:
        return 1.0
    E = (F[1:] - F[0])
    G = E @ E.T
    return math.sqrt(max(np.linalg.det(G), 0.0)) / math.factorial(d - 1)


@dataclass
class Geometry:
    coords: np.ndarray      # [N][d+1][d] unwrapped vertex coordinates
    centroid: np.ndarray    # [N][d]
    volume: np.ndarray      # [N]
    h: np.ndarray           # [N] mean edge length
    inradius: np.ndarray    # [N] d*|tau| / |d tau|


def geometry(vertices, cells, period):
    N, dp1 = cells.shape
    d = dp1 - 1
    coords = np.array([unwrap_cell(vertices, cells[c], period) for c in range(N)])
    centroid = coords.mean(axis=1)
    volume = np.array([simplex_volume(coords[c]) for c in range(N)])
    h = np.zeros(N)
    inr = np.zeros(N)
    for c in range(N):
        edges = [np.linalg.norm(coords[c][a] - coords[c][b])
                 for a, b in itertools.combinations(range(dp1), 2)]
        h[c] = float(np.mean(edges))
        bnd = sum(facet_measure(np.delete(coords[c], f, axis=0)) for f in range(dp1))
        inr[c] = d * volume[c] / bnd
    return Geometry(coords, centroid, volume, h, inr)


# ----------------------------------------------------------------------------
# half-facet adjacency (Sec. 3.3.1) and k-ring stencils (Sec. 3.2)
# ----------------------------------------------------------------------------

def sibling_half_facets(cells):
    """For each half-facet (cell c, local facet f = the facet opposite local
    vertex f) the sibling (c', f'), or (-1, -1) on the boundary."""
    N, dp1 = cells.shape
    owner = {}
    sib = -np.ones((N, dp1, 2), dtype=np.int64)
    for c in range(N):
        for f in range(dp1):
            key = tuple(sorted(int(v) for k, v in enumerate(cells[c]) if k != f))
            if key in owner:
                c2, f2 = owner.pop(key)
                sib[c, f] = (c2, f2)
                sib[c2, f2] = (c, f)
            else:
                owner[key] = (c, f)
    return sib


def sharing_neighbours(cells, min_shared):
    """Cells sharing at least ``min_shared`` vertices with each cell
    (d vertices: facet neighbours; 1 vertex: the 1-ring)."""
    N = cells.shape[0]
    v2c = {}
    for c in range(N):
        for v in cells[c]:
            v2c.setdefault(int(v), []).append(c)
    out = []
    for c in range(N):
        count = {}
        for v in cells[c]:
            for c2 in v2c[int(v)]:
                if c2 != c:
                    count[c2] = count.get(c2, 0) + 1
        out.append(sorted(c2 for c2, k in count.items() if k >= min_shared))
    return out


def ring_levels(d, ring):
    """Decompose a ring size into increments: 2-D uses 1/2-ring steps
    (edge-sharing) and 1-ring steps (vertex-sharing); 3-D uses 1/3 (face),
    2/3 (edge) and 1 (vertex) steps, as in Sec. 3.2."""
    k = int(math.floor(ring + 1e-9))
    frac = ring - k
    steps = ["vertex"] * k
    if abs(frac) < 1e-6:
        return steps
    if d == 2 and abs(frac - 0.5) < 1e-6:
        return steps + ["facet"]
    if d == 3 and abs(frac - 1.0 / 3.0) < 1e-3:
        return steps + ["facet"]
    if d == 3 and abs(frac - 2.0 / 3.0) < 1e-3:
        return steps + ["edge"]
    raise ValueError(f"ring {ring} is not a valid increment in {d}-D")


def k_ring(c, steps, nbr):
    """The k-ring neighbourhood of cell c: start from {c}; each step adds the
    neighbours (of the step's kind) of every cell collected so far."""
    ring = {c}
    for kind in steps:
        grown = set(ring)
        for c2 in ring:
            grown.update(nbr[kind][c2])
        ring = grown
    return ring


def neighbour_tables(cells, dim):
    nbr = {"facet": sharing_neighbours(cells, dim),
           "vertex": sharing_neighbours(cells, 1)}
    if dim == 3:
        nbr["edge"] = sharing_neighbours(cells, 2)
    return nbr


def stencil_of(c, nbr, ring, dim, radius_cut=0.0, centroid=None, h=None, period=None,
               min_rows=0):
    """Stencil S(c): the centre cell first, then the others in increasing cell
    index.  With radius_cut > 0, cells of the next whole vertex-sharing ring
    (ceil(ring) rings) whose centroid lies within radius_cut * h_c of x_c are
    added too.  With min_rows > 0 (transmissive boundaries) a short stencil
    then grows by facet-neighbour increments until it has min_rows cells."""
    S = k_ring(c, ring_levels(dim, ring), nbr)
    if radius_cut > 0:
        outer = k_ring(c, ["vertex"] * (int(math.floor(ring + 1e-9)) + 1), nbr) - S
        for c2 in outer:
            dx = min_image(centroid[c2] - centroid[c], period)
            if np.linalg.norm(dx) <= radius_cut * h[c]:
                S.add(c2)
    while len(S) < min_rows:
        grown = set(S)
        for c2 in S:
            grown.update(nbr["facet"][c2])
        if grown == S:
            break
        S = grown
    return [c] + sorted(S - {c})


def build_stencils(cells, ring, dim, radius_cut=0.0, centroid=None, h=None, period=None,
                   min_rows=0):
    """Stencils of every cell (see stencil_of) and the facet-neighbour lists."""
    nbr = neighbour_tables(cells, dim)
    out = [stencil_of(c, nbr, ring, dim, radius_cut, centroid, h, period, min_rows)
           for c in range(cells.shape[0])]
    return out, nbr["facet"]


class LazyStencils:
    """Stencils computed on first use (large meshes are only sampled)."""

    def __init__(self, prob):
        self.prob = prob
        self.cache = {}

    def __getitem__(self, c):
        if c not in self.cache:
            P = self.prob
            self.cache[c] = stencil_of(c, P.nbr, P.ring, P.dim, P.radius_cut, P.geo.centroid,
                                       P.geo.h, P.period, P.min_rows)
        return self.cache[c]

    def __len__(self):
        return self.prob.N


# ----------------------------------------------------------------------------
# Taylor moments (Sec. 3.1.1, Sec. 3.2)
# ----------------------------------------------------------------------------

def multi_indices(d, p):
    """Exponents kappa with |kappa| <= p-1: degree-major, then descending
    powers of x, then y (1, x, y, x^2, xy, y^2, ...)."""
    out = []
    for q in range(p):
        for kappa in itertools.product(range(q, -1, -1), repeat=d):
            if sum(kappa) == q:
                out.append(kappa)
    # itertools.product with descending ranges already lists x-major first
    return out


def compositions(k, parts):
    """All tuples of ``parts`` non-negative integers summing to k."""
    if parts == 1:
        yield (k,)
        return
    for a in range(k, -1, -1):
        for rest in compositions(k - a, parts - 1):
            yield (a,) + rest


def simplex_monomial_integral(Y, kappa):
    """Exact integral over the simplex with vertices Y [d+1][d] of
    prod_c y_c^kappa_c, from y = sum_v lambda_v Y_v, the multinomial theorem
    and int_T lambda^alpha = d! |T| alpha! / (|alpha| + d)!."""
    dp1, d = Y.shape
    vol = simplex_volume(Y)
    per_axis = [list(compositions(kappa[c], dp1)) for c in range(d)]
    total = 0.0
    for choice in itertools.product(*per_axis):
        coef = 1.0
        alpha = [0] * dp1
        for c in range(d):
            beta = choice[c]
            coef *= math.factorial(kappa[c])
            for v in range(dp1):
                coef /= math.factorial(beta[v])
                coef *= Y[v, c] ** beta[v]
                alpha[v] += beta[v]
        a_fact = 1.0
        for v in range(dp1):
            a_fact *= math.factorial(alpha[v])
        total += coef * math.factorial(d) * vol * a_fact / math.factorial(sum(alpha) + d)
    return total


def moment_row(Yj, xi, hi, kappas):
    """Row of A for stencil cell tau_j: (1/|tau_j|) int_{tau_j}
    prod_c ((x_c - x_i,c)/h_i)^kappa_c / kappa_c!  for every kappa."""
    Y = (Yj - xi) / hi
    volY = simplex_volume(Y)
    row = np.empty(len(kappas))
    for k, kappa in enumerate(kappas):
        fact = 1.0
        for e in kappa:
            fact *= math.factorial(e)
        row[k] = simplex_monomial_integral(Y, kappa) / (volY * fact)
    return row


def stencil_coords(geo, S, i, period):
    """Vertex coordinates of every stencil cell at its minimum-image copy
    nearest to tau_i."""
    out = []
    for j in S:
        shift = min_image(geo.centroid[j] - geo.centroid[i], period) - (geo.centroid[j] - geo.centroid[i])
        out.append(geo.coords[j] + shift)
    return out


def moment_matrix(geo, S, i, p, period):
    """The n x m matrix A of Eq. (average_eq) for cell i on stencil S, in
    h_i-normalised unknowns."""
    d = geo.coords.shape[2]
    kappas = multi_indices(d, p)
    Ys = stencil_coords(geo, S, i, period)
    return np.array([moment_row(Yj, geo.centroid[i], geo.h[i], kappas) for Yj in Ys])


# ----------------------------------------------------------------------------
# weights (Sec. 3.1.2) and the scaled weighted least squares (Sec. 3.3.2)
# ----------------------------------------------------------------------------

def wls_eno_weights(ubar_S, face_mask, h, eps=1e-2, alpha_c=1.5):
    """omega_j of Eq. (weight) from beta_j of Eq. (smoothness indicator).

    ubar_S[0] is the centre cell; face_mask marks the stencil cells that share
    a facet with it (the centre's beta is their minimum)."""
    ubar_S = np.asarray(ubar_S, dtype=np.float64)
    n = len(ubar_S)
    beta = np.empty(n)
    for j in range(1, n):
        beta[j] = (ubar_S[j] - ubar_S[0]) ** 2 + eps * h * h
    beta[0] = min(beta[j] for j in range(1, n) if face_mask[j])
    omega = 1.0 / beta
    omega[0] = alpha_c / beta[0]
    return omega


PIVOT_TOL = 1e-6


def qr_column_pivoting(B, tau_piv=PIVOT_TOL):
    """Householder QR with column pivoting, B[:, piv] = Q R (Sec. 3.3.2).
    Pivot rule (reading R6; the paper does not break ties, and after the
    column scaling every column has norm 1): at step k the pivot is the
    lowest-index remaining column whose squared trailing norm is at least
    (1 - tau_piv) times the largest one, the trailing norms recomputed from
    the partly reduced matrix at every step.  Returns (R [min(n,m)][m], piv,
    the Householder vectors v_k with Q_k = I - 2 v v^T / v^T v)."""
    n, m = B.shape
    W = np.array(B, dtype=np.float64)
    piv = list(range(m))
    vs = []
    for k in range(min(n, m)):
        T = W[k:, k:]
        norms = np.einsum("ij,ij->j", T, T)
        p = k + int(np.argmax(norms >= (1.0 - tau_piv) * norms.max()))  # first such column
        if p != k:
            W[:, [k, p]] = W[:, [p, k]]
            piv[k], piv[p] = piv[p], piv[k]
        v = W[k:, k].copy()
        nrm = math.sqrt(float(norms[p - k]))
        alpha = -nrm if v[0] >= 0.0 else nrm
        v[0] -= alpha
        vtv = float(np.dot(v, v))
        if vtv > 0.0:
            T -= v[:, None] * ((2.0 / vtv) * (v @ T))[None, :]
        vs.append(v)
    return np.triu(W[:min(n, m)]), piv, vs


def apply_qt(vs, y):
    """Q^T y with the Householder vectors of qr_column_pivoting."""
    z = np.array(y, dtype=np.float64)
    for k, v in enumerate(vs):
        vtv = float(np.dot(v, v))
        if vtv > 0.0:
            z[k:] -= (2.0 / vtv) * float(np.dot(v, z[k:])) * v
    return z


def scaled_wls_solve(A, omega, rhs, rank_tol=1e-10):
    """Minimise ||W A S d - W rhs||_2 (Eq. (scaled_WLS)) with W = diag(omega),
    S = diag(1/||column of W A||), by QR with column pivoting
    (W A S E = Q R); the solution is v = S E R^-1 Q^T W rhs restricted to the
    numerical rank r (dropped coefficients are 0).  Returns (v, rank, R)."""
    WA = omega[:, None] * A
    s = 1.0 / np.linalg.norm(WA, axis=0)
    B = WA * s[None, :]
    R, piv, vs = qr_column_pivoting(B)
    diag = np.abs(np.diag(R))
    r = int(np.sum(diag > rank_tol * diag[0]))
    c = apply_qt(vs, omega * rhs)[:r]
    y = scipy.linalg.solve_triangular(R[:r, :r], c, lower=False)
    dvec = np.zeros(A.shape[1])
    dvec[np.asarray(piv[:r], dtype=int)] = y
    return s * dvec, r, R


# ----------------------------------------------------------------------------
# the reconstruction of every cell
# ----------------------------------------------------------------------------

@dataclass
class Problem:
    vertices: np.ndarray
    cells: np.ndarray
    period: np.ndarray
    p: int
    ring: float
    pde: int = ADVECTION
    velocity: tuple = (1.0, 1.0, 0.0)
    gamma: float = 1.4
    eps: float = 1e-2
    alpha_c: float = 1.5
    rank_tol: float = 1e-10
    radius_cut: float = 0.0
    min_rows: int = 0
    characteristic: bool = False  # Euler: characteristic-wise reconstruction
    balanced: bool = False        # scalar: balanced-stencil re-selection (Sec. 3.2)
    balance_margin: float = 2e-2  # out of range: beyond [min, max] by this share of the data's range

    def __post_init__(self):
        self.vertices = np.asarray(self.vertices, dtype=np.float64)
        self.cells = np.asarray(self.cells, dtype=np.int64)
        self.period = np.asarray(self.period, dtype=np.float64)
        self.dim = self.cells.shape[1] - 1
        self.geo = geometry(self.vertices, self.cells, self.period)
        self.nbr = neighbour_tables(self.cells, self.dim)
        self.face_nbrs = self.nbr["facet"]
        self.stencils = LazyStencils(self)
        self.kappas = multi_indices(self.dim, self.p)
        self.m = len(self.kappas)
        self.sib = sibling_half_facets(self.cells)
        self._A = {}

    @property
    def N(self):
        return self.cells.shape[0]

    def A(self, i):
        if i not in self._A:
            self._A[i] = moment_matrix(self.geo, self.stencils[i], i, self.p, self.period)
        return self._A[i]

    def reconstruct_cell(self, ubar, i):
        """h-normalised Taylor coefficients d of cell i (v = d / h^|kappa|) and
        the numerical rank of its scaled system."""
        S = self.stencils[i]
        face = set(self.face_nbrs[i])
        mask = [j in face for j in S]
        uS = np.asarray([ubar[j] for j in S])
        omega = wls_eno_weights(uS, mask, self.geo.h[i], self.eps, self.alpha_c)
        dvec, r, _ = scaled_wls_solve(self.A(i), omega, uS, self.rank_tol)
        return dvec, r

    def derivatives(self, dvec, i):
        """Unscaled derivatives d^kappa u(x_i) from h-normalised coefficients."""
        return np.array([dvec[k] / self.geo.h[i] ** sum(kap) for k, kap in enumerate(self.kappas)])

    def eval_poly(self, dvec, i, x):
        """Reconstruction of cell i at the point x (given near tau_i)."""
        y = (np.asarray(x) - self.geo.centroid[i]) / self.geo.h[i]
        total = 0.0
        for k, kap in enumerate(self.kappas):
            term = dvec[k]
            for c, e in enumerate(kap):
                term *= y[c] ** e / math.factorial(e)
            total += term
        return total


    def basis(self, i, x):
        """The values phi_kappa(y) = prod y_c^kappa_c / kappa_c! at the point x
        (y = (x - x_i) / h_i): eval_poly(d, i, x) = d . basis(i, x)."""
        y = (np.asarray(x) - self.geo.centroid[i]) / self.geo.h[i]
        out = np.empty(len(self.kappas))
        for k, kap in enumerate(self.kappas):
            term = 1.0
            for c, e in enumerate(kap):
                term *= y[c] ** e / math.factorial(e)
            out[k] = term
        return out


# ----------------------------------------------------------------------------
# facet quadrature and the Lax-Friedrichs flux (Sec. 1, Eq. (flux))
# ----------------------------------------------------------------------------

def facet_rule(F):
    """Quadrature points and weights (summing to 1) on a facet with vertices F."""
    d = F.shape[1]
    if d == 1:
        return F.copy(), np.array([1.0])
    if d == 2:
        g = 0.5 / math.sqrt(3.0)
        t = np.array([0.5 - g, 0.5 + g])
        return np.array([F[0] + tt * (F[1] - F[0]) for tt in t]), np.array([0.5, 0.5])
    if d == 3:
        bary = [(2 / 3, 1 / 6, 1 / 6), (1 / 6, 2 / 3, 1 / 6), (1 / 6, 1 / 6, 2 / 3)]
        return np.array([sum(b[k] * F[k] for k in range(3)) for b in bary]), np.full(3, 1.0 / 3.0)
    raise ValueError(d)


def outward_normal(X, f):
    """Unit normal of local facet f (opposite vertex f) pointing out of the simplex X."""
    dp1, d = X.shape
    F = np.delete(X, f, axis=0)
    if d == 1:
        n = np.array([1.0])
    elif d == 2:
        e = F[1] - F[0]
        n = np.array([e[1], -e[0]])
    else:
        n = np.cross(F[1] - F[0], F[2] - F[0])
    n = n / np.linalg.norm(n)
    if np.dot(F.mean(axis=0) - X[f], n) < 0:
        n = -n
    return n


def physical_flux(prob, u):
    """F(u) for the scalar equations as a vector in R^d."""
    d = prob.dim
    if prob.pde == ADVECTION:
        return np.asarray(prob.velocity[:d]) * u
    if prob.pde == BURGERS:
        return np.full(d, 0.5 * u * u)
    raise ValueError(prob.pde)


def normal_speed(prob, u, n):
    if prob.pde == ADVECTION:
        return float(np.linalg.norm(prob.velocity[:prob.dim]))
    if prob.pde == BURGERS:
        return abs(u * float(np.sum(n)))
    raise ValueError(prob.pde)


def lax_friedrichs(prob, um, up, n, alpha):
    """Eq. (flux): 1/2 [ (F(u-) + F(u+)) . n - alpha (u+ - u-) ]."""
    return 0.5 * (np.dot(physical_flux(prob, um) + physical_flux(prob, up), n) - alpha * (up - um))


def facets(prob):
    """Each facet once: (left cell L, its local facet fL, right cell R or -1)."""
    out = []
    for c in range(prob.N):
        for f in range(prob.dim + 1):
            c2, _ = prob.sib[c, f]
            if c2 < 0 or c < c2:
                out.append((c, f, int(c2)))
    return out


def reconstruct_all(prob, ubar):
    out = [prob.reconstruct_cell(ubar, i)[0] for i in range(prob.N)]
    if prob.balanced:
        for i in range(prob.N):
            if out_of_range(prob, ubar, i, out[i]):
                S = balanced_stencil(prob, i, out[i])
                if S is not None:
                    out[i] = reconstruct_on(prob, ubar, i, S)
    return out


# ----------------------------------------------------------------------------
# balanced-stencil re-selection (Sec. 3.2, last paragraph).  Readings: the
# neighbourhood is the stencil S(i); a value is out of range when it leaves
# [min, max] of the stencil averages by more than balance_margin times the
# range of the averages over the mesh (2 %: a smooth extremum exceeds its
# stencil's range by O(h^2), 1.2 % of the range on the 12 x 12 triangle mesh
# with the smooth Burgers data, 0.34 % on 24 x 24, while overshoots at a jump
# are several % of the jump; a margin also keeps averages that equal up to
# rounding (flat regions) from deciding the test);
# the enlarged stencil is the (ceil(ring) + 1)-vertex ring; the new stencil
# keeps the centre and its facet neighbours and fills each side of the plane
# through x_i normal to grad u(x_i) up to half of the old stencil size with
# the side's nearest cells (ties by index; s <= 0 counts as the minus side),
# topping up from the other side when one runs short.
# ----------------------------------------------------------------------------

def cell_facet_points(prob, i):
    X = prob.geo.coords[i]
    out = []
    for f in range(prob.dim + 1):
        pts, _ = facet_rule(np.delete(X, f, axis=0))
        out.extend(pts)
    return out


def out_of_range(prob, ubar, i, dvec):
    uS = np.asarray([ubar[j] for j in prob.stencils[i]])
    lo, hi = float(np.min(uS)), float(np.max(uS))
    tol = prob.balance_margin * (float(np.max(ubar)) - float(np.min(ubar)))
    vals = [prob.eval_poly(dvec, i, x) for x in cell_facet_points(prob, i)]
    return any(v < lo - tol or v > hi + tol for v in vals)


def balanced_stencil(prob, i, dvec):
    """The balanced stencil of cell i from its reconstruction dvec (the
    gradient direction is its first-order coefficients), or None when the
    gradient vanishes."""
    g = np.asarray(dvec[1:1 + prob.dim], dtype=np.float64)
    if not np.any(g != 0.0):
        return None
    n = len(prob.stencils[i])
    face = set(int(j) for j in prob.face_nbrs[i])
    steps = ["vertex"] * (int(math.ceil(prob.ring - 1e-9)) + 1)
    cands = sorted(k_ring(i, steps, prob.nbr) - {i})
    side, dist = {}, {}
    for j in cands:
        dx = min_image(prob.geo.centroid[j] - prob.geo.centroid[i], prob.period)
        side[j] = float(np.dot(dx, g)) > 0.0
        dist[j] = float(np.dot(dx, dx))
    quota = {True: (n - 1 + 1) // 2, False: (n - 1) // 2}
    chosen = set(face)
    for j in face:
        quota[side[j]] -= 1
    pools = {sd: sorted((j for j in cands if side[j] == sd and j not in face), key=lambda j: (dist[j], j))
             for sd in (True, False)}
    for sd in (True, False):
        take = max(0, quota[sd])
        chosen.update(pools[sd][:take])
        pools[sd] = pools[sd][take:]
    rest = sorted(pools[True] + pools[False], key=lambda j: (dist[j], j))
    while len(chosen) < n - 1 and rest:
        chosen.add(rest.pop(0))
    return [i] + sorted(chosen)


def reconstruct_on(prob, ubar, i, S):
    """WLS-ENO reconstruction of cell i on the stencil S (centre first)."""
    A = moment_matrix(prob.geo, S, i, prob.p, prob.period)
    face = set(int(j) for j in prob.face_nbrs[i])
    uS = np.asarray([ubar[j] for j in S])
    omega = wls_eno_weights(uS, [j in face for j in S], prob.geo.h[i], prob.eps, prob.alpha_c)
    dvec, _, _ = scaled_wls_solve(A, omega, uS, prob.rank_tol)
    return dvec


def facet_states(prob, coeffs, L, fL, R):
    """Quadrature points (in L's frame), weights, measure, outward normal of
    L, and the traces u- (from L) and u+ (from R, or u- on a boundary)."""
    X = prob.geo.coords[L]
    F = np.delete(X, fL, axis=0)
    pts, w = facet_rule(F)
    area = facet_measure(F)
    n = outward_normal(X, fL)
    um = np.array([prob.eval_poly(coeffs[L], L, x) for x in pts])
    if R < 0:
        up = um.copy()
    else:
        # the same physical points seen from the nearest copy of tau_R
        shift = min_image(prob.geo.centroid[R] - prob.geo.centroid[L], prob.period) - \
            (prob.geo.centroid[R] - prob.geo.centroid[L])
        up = np.array([prob.eval_poly(coeffs[R], R, x - shift) for x in pts])
    return pts, w, area, n, um, up


def facet_flux(prob, coeffs, L, fL, R):
    """Integral of the LF numerical flux over the facet (outward from L)."""
    pts, w, area, n, um, up = facet_states(prob, coeffs, L, fL, R)
    if prob.pde == ADVECTION:
        alpha = normal_speed(prob, 0.0, n)
    else:
        alpha = max(max(normal_speed(prob, a, n), normal_speed(prob, b, n)) for a, b in zip(um, up))
    return area * sum(w[q] * lax_friedrichs(prob, um[q], up[q], n, alpha) for q in range(len(w)))


def residual(prob, ubar, coeffs=None):
    """L(ubar)_i = -(1/|tau_i|) * sum over facets of the integrated numerical
    flux out of tau_i (Eq. (fvm), divided by |tau_i|)."""
    if prob.pde == EULER:
        return residual_euler_char(prob, ubar) if prob.characteristic else residual_euler(prob, ubar)
    if coeffs is None:
        coeffs = reconstruct_all(prob, ubar)
    flux_out = np.zeros(prob.N)
    for L, fL, R in facets(prob):
        g = facet_flux(prob, coeffs, L, fL, R)
        flux_out[L] += g
        if R >= 0:
            flux_out[R] -= g
    return -flux_out / prob.geo.volume


def max_wave_speed(prob, ubar):
    if prob.pde == ADVECTION:
        return float(np.linalg.norm(prob.velocity[:prob.dim]))
    if prob.pde == BURGERS:
        return math.sqrt(prob.dim) * float(np.max(np.abs(ubar)))
    if prob.pde == EULER:
        rho, vel, p = euler_primitive(np.asarray(ubar), prob.gamma)
        return float(np.max(np.linalg.norm(vel, axis=0) + np.sqrt(prob.gamma * p / rho)))
    raise ValueError(prob.pde)


# ----------------------------------------------------------------------------
# compressible Euler, componentwise WLS-ENO (Sec. 5.2.3 and 5.2.4 use the 2-D
# Euler equations; the reconstruction is applied to each conserved variable)
# ----------------------------------------------------------------------------

POSITIVITY_FLOOR = 1e-12


def euler_primitive(U, gamma):
    """Density, velocity [d][...] and pressure from conserved U = (rho, rho v, E)."""
    rho = U[0]
    vel = U[1:-1] / rho
    p = (gamma - 1.0) * (U[-1] - 0.5 * rho * np.sum(vel * vel, axis=0))
    return rho, vel, p


def euler_normal_flux(U, n, gamma):
    """F(U).n for conserved U (shape [d+2])."""
    rho, vel, p = euler_primitive(np.asarray(U, dtype=np.float64), gamma)
    un = float(np.dot(vel, n))
    out = np.empty(len(U))
    out[0] = rho * un
    out[1:-1] = rho * un * vel + p * np.asarray(n)
    out[-1] = (U[-1] + p) * un
    return out


def euler_wave_speed(U, n, gamma):
    rho, vel, p = euler_primitive(np.asarray(U, dtype=np.float64), gamma)
    return abs(float(np.dot(vel, n))) + math.sqrt(gamma * p / rho)


def euler_coeffs(prob, ubar):
    """Componentwise reconstructions: coeffs[c][i] (each with its own weights)."""
    C = ubar.shape[0]
    return [[prob.reconstruct_cell(ubar[c], i)[0] for i in range(prob.N)] for c in range(C)]


def euler_positive(prob, ubar, coeffs):
    """Reading of the positivity fallback (the paper is silent): a cell whose
    traces give density or pressure <= 1e-12 at any facet quadrature point
    uses its cell averages at all its facets."""
    C = ubar.shape[0]
    ok = np.ones(prob.N, dtype=bool)
    for i in range(prob.N):
        X = prob.geo.coords[i]
        for f in range(prob.dim + 1):
            pts, _ = facet_rule(np.delete(X, f, axis=0))
            for x in pts:
                U = np.array([prob.eval_poly(coeffs[c][i], i, x) for c in range(C)])
                rho, _, p = euler_primitive(U, prob.gamma)
                if not (rho > POSITIVITY_FLOOR and p > POSITIVITY_FLOOR):
                    ok[i] = False
    return ok


def euler_traces(prob, ubar, coeffs, ok, c_cell, pts_in_cell_frame):
    C = ubar.shape[0]
    out = np.empty((len(pts_in_cell_frame), C))
    for q, x in enumerate(pts_in_cell_frame):
        for c in range(C):
            out[q, c] = prob.eval_poly(coeffs[c][c_cell], c_cell, x) if ok[c_cell] else ubar[c, c_cell]
    return out


def residual_euler(prob, ubar):
    """Componentwise WLS-ENO traces, LF flux with alpha = max over the facet's
    points and sides of |u.n| + c (Eq. (flux)), FV residual per component."""
    ubar = np.asarray(ubar, dtype=np.float64)
    C = ubar.shape[0]
    coeffs = euler_coeffs(prob, ubar)
    ok = euler_positive(prob, ubar, coeffs)
    flux_out = np.zeros((C, prob.N))
    for L, fL, R in facets(prob):
        X = prob.geo.coords[L]
        F = np.delete(X, fL, axis=0)
        pts, w = facet_rule(F)
        area = facet_measure(F)
        n = outward_normal(X, fL)
        UL = euler_traces(prob, ubar, coeffs, ok, L, pts)
        if R < 0:
            UR = UL.copy()
        else:
            shift = min_image(prob.geo.centroid[R] - prob.geo.centroid[L], prob.period) - \
                (prob.geo.centroid[R] - prob.geo.centroid[L])
            UR = euler_traces(prob, ubar, coeffs, ok, R, [x - shift for x in pts])
        alpha = max(max(euler_wave_speed(UL[q], n, prob.gamma), euler_wave_speed(UR[q], n, prob.gamma))
                    for q in range(len(w)))
        g = np.zeros(C)
        for q in range(len(w)):
            g += w[q] * 0.5 * (euler_normal_flux(UL[q], n, prob.gamma) + euler_normal_flux(UR[q], n, prob.gamma)
                               - alpha * (UR[q] - UL[q]))
        g *= area
        flux_out[:, L] += g
        if R >= 0:
            flux_out[:, R] -= g
    return -flux_out / prob.geo.volume[None, :]


# ----------------------------------------------------------------------------
# compressible Euler, characteristic-wise WLS-ENO (the characteristic
# decomposition the paper applies to its Euler runs, Sec. 5.1.4 and Sec. 5.2.4,
# in the per-facet form it cites for triangles): for facet f of cell i the
# stencil averages are projected onto the eigenvectors of the Jacobian of
# F(U).n_f at the mean of the two cells' averages, each characteristic field
# is reconstructed with its own WLS-ENO weights, evaluated at the facet's
# points and projected back.
# ----------------------------------------------------------------------------

def euler_char_basis(U, n, gamma):
    """Right eigenvectors R (columns) of d(F(U).n)/dU for 2-D Euler, in the
    order of the eigenvalues u.n - c, u.n (entropy), u.n (shear), u.n + c,
    and L = R^-1; in 1-D the same without the shear wave (u n - c, u n,
    u n + c; the decomposition Sec. 5.1.4 prints for n = 1)."""
    rho, vel, p = euler_primitive(np.asarray(U, dtype=np.float64), gamma)
    if len(n) == 1:
        (u,), (nx,) = vel, n
        c = math.sqrt(gamma * p / rho)
        H = (U[2] + p) / rho
        R = np.array([[1.0, 1.0, 1.0],
                      [u - c * nx, u, u + c * nx],
                      [H - c * u * nx, 0.5 * u * u, H + c * u * nx]])
        return R, np.linalg.inv(R)
    u, v = vel
    nx, ny = n
    c = math.sqrt(gamma * p / rho)
    H = (U[3] + p) / rho
    un = u * nx + v * ny
    ut = -u * ny + v * nx
    R = np.array([[1.0, 1.0, 0.0, 1.0],
                  [u - c * nx, u, -ny, u + c * nx],
                  [v - c * ny, v, nx, v + c * ny],
                  [H - c * un, 0.5 * (u * u + v * v), ut, H + c * un]])
    return R, np.linalg.inv(R)


def euler_char_poly(prob, ubar, i, f):
    """Characteristic reconstruction of cell i for its facet f: (R, the
    dim + 2 fields' coefficient vectors)."""
    j, _ = prob.sib[i, f]
    ustar = 0.5 * (ubar[:, i] + ubar[:, j]) if j >= 0 else ubar[:, i]
    n = outward_normal(prob.geo.coords[i], f)
    R, L = euler_char_basis(ustar, n, prob.gamma)
    S = prob.stencils[i]
    w = {k: L @ ubar[:, k] for k in S}
    return R, [prob.reconstruct_cell({k: w[k][c] for k in S}, i)[0] for c in range(len(ustar))]


def residual_euler_char(prob, ubar):
    """As residual_euler with characteristic-wise traces; the positivity
    fallback is the same reading (a cell with rho or p <= 1e-12 at any of its
    facet points uses its averages at all its facets)."""
    ubar = np.asarray(ubar, dtype=np.float64)
    assert prob.dim in (1, 2)
    C = ubar.shape[0]
    traces = {}
    ok = np.ones(prob.N, dtype=bool)
    for i in range(prob.N):
        X = prob.geo.coords[i]
        for f in range(prob.dim + 1):
            R, coef = euler_char_poly(prob, ubar, i, f)
            pts, _ = facet_rule(np.delete(X, f, axis=0))
            vals = np.array([R @ np.array([prob.eval_poly(coef[c], i, x) for c in range(C)]) for x in pts])
            traces[i, f] = vals
            for U in vals:
                rho, _, pr = euler_primitive(U, prob.gamma)
                if not (rho > POSITIVITY_FLOOR and pr > POSITIVITY_FLOOR):
                    ok[i] = False
    for i in range(prob.N):
        if not ok[i]:
            for f in range(prob.dim + 1):
                traces[i, f] = np.repeat(ubar[:, i][None, :], len(traces[i, f]), axis=0)
    flux_out = np.zeros((C, prob.N))
    for Lc, fL, Rc in facets(prob):
        X = prob.geo.coords[Lc]
        F = np.delete(X, fL, axis=0)
        pts, w = facet_rule(F)
        area = facet_measure(F)
        n = outward_normal(X, fL)
        UL = traces[Lc, fL]
        if Rc < 0:
            UR = UL.copy()
        else:
            # the sibling facet's points in R's frame are the same points; its
            # rule lists them in R's vertex order: match them by position
            fR = int(prob.sib[Lc, fL][1])
            shift = min_image(prob.geo.centroid[Rc] - prob.geo.centroid[Lc], prob.period) - \
                (prob.geo.centroid[Rc] - prob.geo.centroid[Lc])
            ptsR, _ = facet_rule(np.delete(prob.geo.coords[Rc], fR, axis=0))
            order = [int(np.argmin([np.linalg.norm((x - shift) - y) for y in ptsR])) for x in pts]
            UR = traces[Rc, fR][order]
        alpha = max(max(euler_wave_speed(UL[q], n, prob.gamma), euler_wave_speed(UR[q], n, prob.gamma))
                    for q in range(len(w)))
        g = np.zeros(C)
        for q in range(len(w)):
            g += w[q] * 0.5 * (euler_normal_flux(UL[q], n, prob.gamma) + euler_normal_flux(UR[q], n, prob.gamma)
                               - alpha * (UR[q] - UL[q]))
        g *= area
        flux_out[:, Lc] += g
        if Rc >= 0:
            flux_out[:, Rc] -= g
    return -flux_out / prob.geo.volume[None, :]


def cfl_dt(prob, ubar, cfl):
    return cfl * float(np.min(prob.geo.inradius)) / max_wave_speed(prob, ubar)


def rk3_step(L, u, dt):
    """Eq. (3rd-order-Runge-Kutta): the Shu-Osher TVD-RK3 stage sequence."""
    k1 = u + dt * L(u)
    k2 = 0.75 * u + 0.25 * k1 + 0.25 * dt * L(k1)
    return u / 3.0 + 2.0 / 3.0 * k2 + 2.0 / 3.0 * dt * L(k2)


def rk3_run(prob, ubar, n_steps, cfl=None, dt=None):
    """n_steps TVD-RK3 steps; dt from the CFL rule at the start of each step
    unless given.  Returns (ubar, list of dt)."""
    u = np.array(ubar, dtype=np.float64)
    dts = []
    for _ in range(n_steps):
        step = dt if dt is not None else cfl_dt(prob, u, cfl)
        u = rk3_step(lambda x: residual(prob, x), u, step)
        dts.append(step)
    return u, dts


# ----------------------------------------------------------------------------
# reverse mode (the adjoint) of the residual and of one TVD-RK3 step, scalar
# equations.  The paper has no adjoint; this differentiates its scheme as
# written above, step by step in reverse:
#   L_i = -(1/|tau_i|) sum_f g_f (Eq. (fvm)), g_f the facet integral of the
#   LF flux of Eq. (flux) with its per-facet alpha (Burgers: the maximum of
#   |F'(u).n| over the facet's points and both sides, taken at the first
#   maximiser in the order of facet_flux);
#   the traces u(x_q) = d_i . phi_i(x_q) of each cell's polynomial;
#   each cell's weighted least-squares solution (Sec. 3.1.1, rows times
#   omega_j) in its full-rank normal form d = G^-1 A^T W^2 u_S with
#   G = A^T W^2 A, whose differential is G dd = A^T W^2 du_S +
#   A^T d(W^2) (u_S - A d); with lambda = G^-1 dbar this gives
#   u_S-bar = W^2 A lambda and omega_j-bar = 2 omega_j (A lambda)_j r_j;
#   the weights of Sec. 3.1.2, omega_j = 1/beta_j, omega_i = alpha_c/beta_i,
#   beta_j = (u_j - u_i)^2 + eps h^2 and beta_i the minimum over the facet
#   neighbours (at the first minimiser).
# Full-rank cells only (a truncated cell raises), fixed stencils.
# ----------------------------------------------------------------------------

def _lf_partials(prob, um, up, n):
    """dLF/dum, dLF/dup and dLF/dalpha of Eq. (flux) at fixed alpha."""
    if prob.pde == ADVECTION:
        an = float(np.dot(np.asarray(prob.velocity[:prob.dim]), n))
        return lambda alpha: (0.5 * (an + alpha), 0.5 * (an - alpha), -0.5 * (up - um))
    sn = float(np.sum(n))
    return lambda alpha: (0.5 * (um * sn + alpha), 0.5 * (up * sn - alpha), -0.5 * (up - um))


def residual_vjp(prob, ubar, Lbar):
    """(dL/dubar)^T Lbar for the scalar equations (advection, Burgers)."""
    if prob.pde == EULER or prob.balanced:
        raise ValueError("the adjoint covers the scalar equations on fixed stencils")
    ubar = np.asarray(ubar, dtype=np.float64)
    coeffs = []
    for i in range(prob.N):
        d, r = prob.reconstruct_cell(ubar, i)
        if r < prob.m:
            raise ValueError(f"cell {i}: rank {r} < {prob.m}")
        coeffs.append(d)
    # L_i = -flux_out_i / |tau_i|
    fbar = -np.asarray(Lbar, dtype=np.float64) / prob.geo.volume
    dbar = [np.zeros(prob.m) for _ in range(prob.N)]
    for L, fL, R in facets(prob):
        gbar = fbar[L] - (fbar[R] if R >= 0 else 0.0)
        pts, w, area, n, um, up = facet_states(prob, coeffs, L, fL, R)
        if prob.pde == ADVECTION:
            alpha, arg = normal_speed(prob, 0.0, n), None
        else:
            speeds = []
            for a, b in zip(um, up):
                speeds.append(max(normal_speed(prob, a, n), normal_speed(prob, b, n)))
            q_star = int(np.argmax(speeds))
            alpha = speeds[q_star]
            a, b = um[q_star], up[q_star]
            arg = (q_star, "m" if normal_speed(prob, a, n) >= normal_speed(prob, b, n) else "p")
        umbar = np.zeros(len(w))
        upbar = np.zeros(len(w))
        alphabar = 0.0
        for q in range(len(w)):
            dm, dp, da = _lf_partials(prob, um[q], up[q], n)(alpha)
            umbar[q] += gbar * area * w[q] * dm
            upbar[q] += gbar * area * w[q] * dp
            alphabar += gbar * area * w[q] * da
        if arg is not None:  # alpha = |u Sum n| at its first maximiser
            q, side = arg
            u_star = um[q] if side == "m" else up[q]
            dspeed = math.copysign(1.0, u_star * float(np.sum(n))) * float(np.sum(n))
            if side == "m":
                umbar[q] += alphabar * dspeed
            else:
                upbar[q] += alphabar * dspeed
        if R < 0:  # transmissive: u+ = u-
            umbar += upbar
            upbar[:] = 0.0
        for q, x in enumerate(pts):
            dbar[L] += umbar[q] * prob.basis(L, x)
        if R >= 0:
            shift = min_image(prob.geo.centroid[R] - prob.geo.centroid[L], prob.period) - \
                (prob.geo.centroid[R] - prob.geo.centroid[L])
            for q, x in enumerate(pts):
                dbar[R] += upbar[q] * prob.basis(R, x - shift)
    ubar_bar = np.zeros(prob.N)
    for i in range(prob.N):
        S = list(prob.stencils[i])
        face = set(int(j) for j in prob.face_nbrs[i])
        uS = ubar[S]
        A = prob.A(i)
        h = prob.geo.h[i]
        eh2 = prob.eps * h * h
        beta = (uS - uS[0]) ** 2 + eh2
        k_min = min((k for k in range(1, len(S)) if S[k] in face), key=lambda k: (beta[k], k))
        beta[0] = beta[k_min]
        omega = 1.0 / beta
        omega[0] = prob.alpha_c / beta[0]
        W2 = omega * omega
        # lambda = G^-1 dbar with G = (W A)^T (W A) = R^T R (R of the QR of W A)
        Rf = np.linalg.qr(omega[:, None] * A, mode="r")
        lam = scipy.linalg.solve_triangular(Rf, scipy.linalg.solve_triangular(Rf.T, dbar[i], lower=True))
        Alam = A @ lam
        r = uS - A @ coeffs[i]
        uSbar = W2 * Alam
        omegabar = 2.0 * omega * Alam * r
        betabar = -omegabar * omega * omega
        betabar[0] = -omegabar[0] * omega[0] / beta[0]
        betabar[k_min] += betabar[0]  # beta_i = beta of its first minimising facet neighbour
        for k in range(1, len(S)):
            g = 2.0 * (uS[k] - uS[0]) * betabar[k]
            uSbar[k] += g
            uSbar[0] -= g
        np.add.at(ubar_bar, S, uSbar)
    return ubar_bar


def rk3_step_vjp(prob, ubar, dt, gbar_next):
    """(d u^{n+1} / d u^n)^T gbar_next for one fixed-dt step of rk3_step."""
    L = lambda x: residual(prob, x)
    u = np.asarray(ubar, dtype=np.float64)
    k1 = u + dt * L(u)
    k2 = 0.75 * u + 0.25 * k1 + 0.25 * dt * L(k1)
    g3 = np.asarray(gbar_next, dtype=np.float64)
    gu = g3 / 3.0
    g2 = 2.0 / 3.0 * (g3 + dt * residual_vjp(prob, k2, g3))
    gu += 0.75 * g2
    g1 = 0.25 * (g2 + dt * residual_vjp(prob, k1, g2))
    gu += g1 + dt * residual_vjp(prob, u, g1)
    return gu
