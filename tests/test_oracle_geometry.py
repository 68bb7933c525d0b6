"""Pins of the oracle's cell geometry and of the wave speeds in its CFL rule
(Sec. 4.2.1 leaves the time step on unstructured meshes open; the reading
is dt = CFL * min_i r_i / lambda_max with r_i = d|tau_i|/|d tau_i| the
inradius of cell i and lambda_max the largest characteristic speed).

Checked against textbook constructions that share no formula with the
oracle: volumes by Heron's formula and the Cayley-Menger determinant (edge
lengths only), inradii as the distance from the incentre (the vertices
weighted by the opposite facet's measure) to a facet's line or plane, wave
speeds as the largest |d(F.n)/du| (scalar equations) or the spectral radius
of the finite-difference Jacobian of F.n (Euler) over sampled directions."""
import itertools
import math
from types import SimpleNamespace

import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth


def heron(A, B, C):
    a, b, c = np.linalg.norm(B - C), np.linalg.norm(C - A), np.linalg.norm(A - B)
    s = 0.5 * (a + b + c)
    return math.sqrt(max(s * (s - a) * (s - b) * (s - c), 0.0))


def cayley_menger_volume(X):
    D = np.ones((5, 5))
    D[0, 0] = 0.0
    for a in range(4):
        for b in range(4):
            D[a + 1, b + 1] = float(np.sum((X[a] - X[b]) ** 2))
    return math.sqrt(max(np.linalg.det(D) / 288.0, 0.0))


def triangle_inradius(A, B, C):
    """Distance from the incentre to each side (all three returned)."""
    a, b, c = np.linalg.norm(B - C), np.linalg.norm(C - A), np.linalg.norm(A - B)
    I = (a * A + b * B + c * C) / (a + b + c)

    def dist(P, Q):
        e = Q - P
        w = I - P
        return abs(e[0] * w[1] - e[1] * w[0]) / np.linalg.norm(e)
    return dist(B, C), dist(C, A), dist(A, B)


def tet_inradius(X):
    """Distance from the insphere centre to each of the four face planes."""
    areas, normals = [], []
    for k in range(4):
        P = [X[j] for j in range(4) if j != k]
        n = np.cross(P[1] - P[0], P[2] - P[0])
        areas.append(0.5 * np.linalg.norm(n))
        normals.append((P[0], n / np.linalg.norm(n)))
    I = sum(areas[k] * X[k] for k in range(4)) / sum(areas)
    return tuple(abs(float(np.dot(I - P0, n))) for P0, n in normals)


def test_triangle_volumes_and_inradii_are_textbook():
    mesh = synth.tri_mesh(6, seed=2)
    geo = O.geometry(mesh.vertices, mesh.cells, mesh.period)
    for c in range(mesh.cells.shape[0]):
        A, B, C = geo.coords[c]
        assert abs(geo.volume[c] - heron(A, B, C)) <= 1e-13
        r = triangle_inradius(A, B, C)
        assert max(r) - min(r) <= 1e-13
        assert abs(geo.inradius[c] - r[0]) <= 1e-13
        assert np.allclose(geo.centroid[c], (A + B + C) / 3.0, rtol=0, atol=1e-15)
    # the periodic cells tile the unit square
    assert abs(np.sum(geo.volume) - 1.0) <= 1e-12


def test_tetrahedron_volumes_and_inradii_are_textbook():
    mesh = synth.tet_mesh(3, seed=15)
    geo = O.geometry(mesh.vertices, mesh.cells, mesh.period)
    for c in range(mesh.cells.shape[0]):
        X = geo.coords[c]
        assert abs(geo.volume[c] - cayley_menger_volume(X)) <= 1e-12
        r = tet_inradius(X)
        assert max(r) - min(r) <= 1e-13
        assert abs(geo.inradius[c] - r[0]) <= 1e-13
    assert abs(np.sum(geo.volume) - 1.0) <= 1e-12


def test_interval_inradius_is_half_its_length():
    mesh = synth.periodic_line_mesh(16, jitter=0.3, seed=4)
    geo = O.geometry(mesh.vertices, mesh.cells, mesh.period)
    lengths = np.array([abs(x[1, 0] - x[0, 0]) for x in geo.coords])
    assert np.allclose(geo.volume, lengths, rtol=0, atol=1e-15)
    assert np.allclose(geo.inradius, 0.5 * lengths, rtol=0, atol=1e-15)


def directions(dim):
    """Unit vectors: every normalised nonzero integer vector in [-3, 3]^dim."""
    out = []
    for v in itertools.product(range(-3, 4), repeat=dim):
        v = np.array(v, dtype=float)
        if np.any(v):
            out.append(v / np.linalg.norm(v))
    return out


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_burgers_speed_is_the_largest_flux_derivative(dim):
    prob = SimpleNamespace(pde=O.BURGERS, dim=dim, velocity=None)
    rng = np.random.default_rng(dim)
    ubar = rng.uniform(-2.0, 2.0, 50)
    best = 0.0
    for u in ubar:
        for n in directions(dim):
            eps = 1e-5
            deriv = (np.dot(O.physical_flux(prob, u + eps), n) - np.dot(O.physical_flux(prob, u - eps), n)) / (2 * eps)
            assert abs(O.normal_speed(prob, u, n) - abs(deriv)) <= 1e-8
            best = max(best, abs(deriv))
    lam = O.max_wave_speed(prob, ubar)
    assert best <= lam * (1 + 1e-9)
    assert abs(best - lam) <= 1e-8 * lam  # attained at n = (1, .., 1)/sqrt(d)


@pytest.mark.parametrize("dim", [2, 3])
def test_advection_speed_is_the_largest_normal_velocity(dim):
    vel = np.array([1.0, 0.5, 0.25][:dim])
    prob = SimpleNamespace(pde=O.ADVECTION, dim=dim, velocity=vel)
    lam = O.max_wave_speed(prob, np.zeros(3))
    speeds = [abs(float(np.dot(vel, n))) for n in directions(dim)] + [abs(float(np.dot(vel, vel / np.linalg.norm(vel))))]
    assert max(speeds) <= lam * (1 + 1e-12)
    assert abs(max(speeds) - lam) <= 1e-12


def euler_jacobian(U, n, gamma):
    J = np.zeros((len(U), len(U)))
    for k in range(len(U)):
        e = np.zeros(len(U))
        e[k] = 1e-6 * max(1.0, abs(U[k]))
        J[:, k] = (O.euler_normal_flux(U + e, n, gamma) - O.euler_normal_flux(U - e, n, gamma)) / (2 * e[k])
    return J


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_euler_speed_is_the_spectral_radius_of_the_flux_jacobian(dim):
    gamma = 1.4
    rng = np.random.default_rng(10 + dim)
    states = []
    for _ in range(6):
        rho = rng.uniform(0.5, 2.0)
        v = rng.uniform(-1.0, 1.0, dim)
        p = rng.uniform(0.5, 2.0)
        states.append(np.concatenate([[rho], rho * v, [p / (gamma - 1) + 0.5 * rho * v @ v]]))
    for U in states:
        for n in directions(dim)[::3] if dim > 1 else [np.array([1.0]), np.array([-1.0])]:
            rad = float(np.max(np.abs(np.linalg.eigvals(euler_jacobian(U, n, gamma)))))
            assert abs(O.euler_wave_speed(U, n, gamma) - rad) <= 1e-6 * rad
    ubar = np.stack(states, axis=1)
    prob = SimpleNamespace(pde=O.EULER, dim=dim, gamma=gamma, velocity=None)
    lam = O.max_wave_speed(prob, ubar)
    best = 0.0
    for U in states:
        v = U[1:-1] / U[0]
        n = v / np.linalg.norm(v)
        for m in directions(dim) + [n]:
            best = max(best, O.euler_wave_speed(U, m, gamma))
    assert best <= lam * (1 + 1e-12)
    assert abs(best - lam) <= 1e-12 * lam


def test_segment_rule_is_two_point_gauss():
    """Reading R9 in 2-D: exact for degree 3 along an edge (the mean of t^k
    over [0, 1] is 1/(k+1)), not for degree 4."""
    F = np.array([[0.3, -0.2], [1.1, 0.4]])
    pts, w = O.facet_rule(F)
    assert abs(np.sum(w) - 1.0) <= 1e-15
    t = (pts[:, 0] - F[0, 0]) / (F[1, 0] - F[0, 0])
    for k in range(4):
        assert abs(float(np.dot(w, t ** k)) - 1.0 / (k + 1)) <= 1e-15
    assert abs(float(np.dot(w, t ** 4)) - 0.2) > 1e-3


def test_triangle_rule_is_exact_for_degree_two():
    """Reading R9 in 3-D: the mean of l1^a l2^b l3^c over a triangle is
    2 a! b! c! / (a+b+c+2)!; exact for a+b+c <= 2, not for 3."""
    F = np.array([[0.1, 0.0, 0.2], [0.9, 0.3, -0.1], [0.2, 0.8, 0.5]])
    pts, w = O.facet_rule(F)
    T = np.column_stack([F[1] - F[0], F[2] - F[0]])
    lam12 = np.linalg.lstsq(T, (pts - F[0]).T, rcond=None)[0]
    lam = np.vstack([1.0 - lam12.sum(axis=0), lam12])
    for a, b, c in itertools.product(range(4), repeat=3):
        deg = a + b + c
        if deg > 3:
            continue
        exact = 2.0 * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(deg + 2)
        got = float(np.dot(w, lam[0] ** a * lam[1] ** b * lam[2] ** c))
        if deg <= 2:
            assert abs(got - exact) <= 1e-15, (a, b, c)
    assert abs(float(np.dot(w, lam[0] ** 3)) - 2.0 * 6 / math.factorial(5)) > 1e-3


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_outward_normals_close_every_cell(dim):
    """Unit normals, orthogonal to their facet, pointing away from the
    opposite vertex, and sum_f |F_f| n_f = 0 (the divergence theorem for a
    constant field)."""
    mesh = {1: lambda: synth.periodic_line_mesh(8, jitter=0.3, seed=2),
            2: lambda: synth.tri_mesh(5, seed=6), 3: lambda: synth.tet_mesh(3, seed=8)}[dim]()
    geo = O.geometry(mesh.vertices, mesh.cells, mesh.period)
    for X in geo.coords:
        total = np.zeros(dim)
        for f in range(dim + 1):
            n = O.outward_normal(X, f)
            F = np.delete(X, f, axis=0)
            assert abs(np.linalg.norm(n) - 1.0) <= 1e-14
            for e in F[1:] - F[0]:
                assert abs(float(np.dot(n, e))) <= 1e-13
            assert float(np.dot(F[0] - X[f], n)) > 0.0
            total += O.facet_measure(F) * n
        assert np.max(np.abs(total)) <= 1e-13


@pytest.mark.parametrize("make,n_boundary", [
    (lambda: synth.tri_mesh(5, seed=6), 0),
    (lambda: synth.tri_mesh(5, periodic=False, seed=6), 20),
    (lambda: synth.tet_mesh(3, seed=8), 0),
    (lambda: synth.tet_mesh(3, periodic=False, seed=8), 6 * 2 * 9),
    (lambda: synth.periodic_line_mesh(7, jitter=0.2, seed=1), 0),
])
def test_half_facet_siblings_by_brute_force(make, n_boundary):
    """The sibling of half-facet (c, f) (the facet opposite local vertex f)
    is the one other half-facet with the same vertex set, found by comparing
    every pair; boundary facets have none.  The facet list then holds each
    interior facet once and each boundary facet once."""
    mesh = make()
    cells = mesh.cells
    N, dp1 = cells.shape
    keys = {}
    for c in range(N):
        for f in range(dp1):
            keys.setdefault(frozenset(int(v) for k, v in enumerate(cells[c]) if k != f), []).append((c, f))
    assert all(len(v) <= 2 for v in keys.values())
    sib = O.sibling_half_facets(cells)
    boundary = 0
    for group in keys.values():
        if len(group) == 1:
            c, f = group[0]
            assert tuple(sib[c, f]) == (-1, -1)
            boundary += 1
        else:
            (a, fa), (b, fb) = group
            assert tuple(sib[a, fa]) == (b, fb) and tuple(sib[b, fb]) == (a, fa)
    assert boundary == n_boundary
    prob = SimpleNamespace(N=N, dim=dp1 - 1, sib=sib)
    assert len(O.facets(prob)) == (N * dp1 + boundary) // 2


def test_radius_cut_stencils_by_brute_force():
    """Reading R12's 3-D stencil: the 2/3-ring (the cells sharing an edge
    with the centre) plus the cells sharing a vertex with it whose centroid
    lies within 0.95 h_i, found here by comparing vertex sets directly."""
    mesh = synth.tet_mesh(4, seed=5)
    cells = mesh.cells
    geo = O.geometry(mesh.vertices, cells, mesh.period)
    stencils, _ = O.build_stencils(cells, 2.0 / 3.0, 3, radius_cut=0.95, centroid=geo.centroid, h=geo.h,
                                   period=mesh.period)
    sets = [set(int(v) for v in c) for c in cells]
    sizes = []
    for i in range(cells.shape[0]):
        want = {j for j in range(cells.shape[0]) if len(sets[i] & sets[j]) >= 2}
        for j in range(cells.shape[0]):
            if sets[i] & sets[j] and j not in want:
                dx = geo.centroid[j] - geo.centroid[i]
                dx -= np.round(dx / mesh.period) * mesh.period
                if np.linalg.norm(dx) <= 0.95 * geo.h[i]:
                    want.add(j)
        assert stencils[i][0] == i and stencils[i][1:] == sorted(want - {i})
        sizes.append(len(want))
    assert 29 <= min(sizes) and max(sizes) <= 52


def test_short_stencils_grow_by_whole_facet_layers():
    """Reading R13 on a transmissive mesh: a stencil shorter than min_rows is
    the smallest L such that the cells within L facet-adjacency steps of the
    ring have at least min_rows cells (graph distances by scipy's BFS over a
    facet graph built from raw vertex sets)."""
    from scipy.sparse import csr_matrix
    from scipy.sparse.csgraph import shortest_path

    mesh = synth.tri_mesh(7, periodic=False, seed=12)
    cells = mesh.cells
    N = cells.shape[0]
    sets = [set(int(v) for v in c) for c in cells]
    rows, cols = [], []
    for a in range(N):
        for b in range(N):
            if a != b and len(sets[a] & sets[b]) == 2:
                rows.append(a)
                cols.append(b)
    D = shortest_path(csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(N, N)), unweighted=True)
    for min_rows in (9, 15, 22):
        stencils, _ = O.build_stencils(cells, 1.0, 2, min_rows=min_rows)
        plain, _ = O.build_stencils(cells, 1.0, 2)
        grown = 0
        for i in range(N):
            ring = plain[i]
            dist = np.min(D[ring], axis=0)
            L = 0
            while np.sum(dist <= L) < min_rows and np.sum(dist <= L) < np.sum(np.isfinite(dist)):
                L += 1
            want = sorted(set(np.flatnonzero(dist <= L).tolist()) - {i})
            assert stencils[i] == [i] + want, (min_rows, i)
            grown += L > 0
        assert grown > 0


def _rough(mesh, seed):
    return np.random.default_rng(seed).uniform(-1.0, 1.0, mesh.cells.shape[0])


@pytest.mark.parametrize("dim", [2, 3])
def test_reconstruction_is_translation_invariant(dim):
    """Moving a transmissive mesh leaves every h-normalised Taylor
    coefficient about the centroid unchanged (the method sees only relative
    positions).  That includes the cells whose scaled system is rank
    deficient (short stencils in the corners): the pivot rule of reading
    R6 decides the dropped columns by a 1e-6 window, not by rounding."""
    mesh = synth.tri_mesh(8, periodic=False, seed=9) if dim == 2 else synth.tet_mesh(3, periodic=False, seed=9)
    p, ring = (4, 2.0) if dim == 2 else (3, 2.0 / 3.0)
    u = _rough(mesh, 3)
    shift = np.array([0.37, -1.2, 2.5])[:dim]
    a = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, pde=O.BURGERS)
    b = O.Problem(mesh.vertices + shift, mesh.cells, mesh.period, p=p, ring=ring, pde=O.BURGERS)
    deficient = 0
    for i in range(a.N):
        (da, ra), (db, rb) = a.reconstruct_cell(u, i), b.reconstruct_cell(u, i)
        assert ra == rb
        deficient += ra < a.m
        assert np.max(np.abs(da - db)) <= 1e-9 * max(1.0, np.max(np.abs(da))), i
    assert deficient > 0


def test_reflection_flips_the_odd_x_coefficients():
    """x -> -x: the coefficient of (x - x_i)^a (y - y_i)^b changes by (-1)^a,
    and the advection residual with the mirrored velocity is unchanged."""
    mesh = synth.tri_mesh(8, periodic=False, seed=10)
    u = _rough(mesh, 4)
    mirror = mesh.vertices * np.array([-1.0, 1.0])
    a = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=4, ring=2.0, pde=O.ADVECTION,
                  velocity=(1.0, 0.5, 0.0))
    b = O.Problem(mirror, mesh.cells, mesh.period, p=4, ring=2.0, pde=O.ADVECTION, velocity=(-1.0, 0.5, 0.0))
    sign = np.array([(-1.0) ** kap[0] for kap in a.kappas])
    for i in range(a.N):
        da, db = a.reconstruct_cell(u, i)[0], b.reconstruct_cell(u, i)[0]
        assert np.max(np.abs(db - sign * da)) <= 1e-9 * max(1.0, np.max(np.abs(da))), i
    La, Lb = O.residual(a, u), O.residual(b, u)
    assert np.max(np.abs(La - Lb)) <= 1e-9 * np.max(np.abs(La))


def test_burgers_facet_flux_is_consistent_monotone_and_antisymmetric():
    """The facet flux of Eq. (flux) with the per-facet alpha of reading R10
    on constant traces a (from L) and b (from R): F(a, a) = |f| (a^2/2) sum(n);
    non-decreasing in a and non-increasing in b (a monotone flux, as a
    Rusanov flux with alpha >= max |F'(u).n| is); and the same facet seen
    from R gives minus the flux."""
    mesh = synth.tri_mesh(4, seed=2)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0, pde=O.BURGERS)
    rng = np.random.default_rng(12)

    def flux(L, fL, R, a, b):
        coeffs = {L: np.r_[a, np.zeros(prob.m - 1)], R: np.r_[b, np.zeros(prob.m - 1)]}
        return O.facet_flux(prob, coeffs, L, fL, R)

    for L, fL, R in O.facets(prob)[:12]:
        fR = int(prob.sib[L, fL][1])
        X = prob.geo.coords[L]
        F = np.delete(X, fL, axis=0)
        area, n = O.facet_measure(F), O.outward_normal(X, fL)
        for _ in range(20):
            a, b = rng.uniform(-2.0, 2.0, 2)
            assert abs(flux(L, fL, R, a, a) - area * 0.5 * a * a * np.sum(n)) <= 1e-14
            g = flux(L, fL, R, a, b)
            assert flux(L, fL, R, a + 1e-3, b) >= g - 1e-14
            assert flux(L, fL, R, a, b + 1e-3) <= g + 1e-14
            assert abs(flux(R, fR, L, b, a) + g) <= 1e-14
