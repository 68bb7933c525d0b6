"""Pins of the FP64 oracle against things other than itself: the paper's
worked examples (tests/golden, each cited), closed forms, exact integration,
rational brute force, invariants and the accuracy theorem."""
import cmath
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth


def read_golden(golden_dir, name):
    rows = []
    with open(os.path.join(golden_dir, name)) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def frac(s):
    return Fraction(s) if "/" in s else Fraction(s)


# ---------------------------------------------------------------------------
# 1-D worked examples (Sec. 4.2.3, Sec. 4.2.4)
# ---------------------------------------------------------------------------

def uniform_line(ncell=11, dx=1.0):
    return synth.line_mesh(np.arange(ncell + 1) * dx)


def scheme_coefficients(ring, weights=None, dx=1.0):
    """Coefficients of u^-_{i+1/2} in terms of the stencil averages, by
    reconstructing unit vectors (the solve is linear for fixed weights)."""
    mesh = uniform_line(11, dx)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=5, ring=ring)
    i = 5
    S = prob.stencils[i]
    A = prob.A(i)
    w = np.ones(len(S)) if weights is None else weights(prob, S, i)
    xr = prob.geo.centroid[i] + 0.5 * dx
    coef = {}
    for k, j in enumerate(S):
        e = np.zeros(len(S))
        e[k] = 1.0
        dvec, r, _ = O.scaled_wls_solve(A, w, e)
        assert r == 5
        coef[j - i] = prob.eval_poly(dvec, i, xr)
    return coef


def seven_cell_weights(prob, S, i):
    ubar_linear = np.arange(prob.N, dtype=np.float64)  # smooth data, slope 1
    face = set(prob.face_nbrs[i])
    return O.wls_eno_weights(ubar_linear[S], [j in face for j in S], prob.geo.h[i], eps=0.0)


def test_five_cell_scheme(golden_dir):
    coef = scheme_coefficients(ring=2)
    for off, val in read_golden(golden_dir, "five_cell_scheme.txt"):
        assert abs(coef[int(off)] - float(frac(val))) < 1e-13
    assert len(coef) == 5


def test_seven_cell_weights(golden_dir):
    for dx in (1.0, 0.01):
        mesh = uniform_line(11, dx)
        prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=5, ring=3)
        S = prob.stencils[5]
        w = seven_cell_weights(prob, S, 5)
        # ubar_j = j: beta_j = (j - i)^2; express in units of 1/dx^2 where the
        # data has slope 1/dx (rescale ubar by dx)
        ub = np.arange(prob.N) * dx
        face = set(prob.face_nbrs[5])
        w = O.wls_eno_weights(ub[S], [j in face for j in S], 1.0, eps=0.0) * dx * dx
        got = {j - 5: w[k] for k, j in enumerate(S)}
        for off, val in read_golden(golden_dir, "seven_cell_weights.txt"):
            assert abs(got[int(off)] - float(frac(val))) < 1e-12


def test_seven_cell_scheme(golden_dir):
    for dx in (1.0, 0.05):
        coef = scheme_coefficients(ring=3, weights=seven_cell_weights, dx=dx)
        for off, val in read_golden(golden_dir, "seven_cell_scheme.txt"):
            assert abs(coef[int(off)] - float(frac(val))) < 1e-12


def flux_difference(coef):
    """u^-_{i+1/2} - u^-_{i-1/2}: the same stencil shifted by one cell."""
    out = {}
    for off, c in coef.items():
        out[off] = out.get(off, 0.0) + c
        out[off - 1] = out.get(off - 1, 0.0) - c
    return out


@pytest.mark.parametrize("ring,name", [(2, "five_cell_flux_difference.txt"),
                                       (3, "seven_cell_flux_difference.txt")])
def test_flux_differences(golden_dir, ring, name):
    coef = scheme_coefficients(ring, seven_cell_weights if ring == 3 else None)
    fd = flux_difference(coef)
    for off, val in read_golden(golden_dir, name):
        assert abs(fd[int(off)] - float(frac(val))) < 1e-12


def symbol(fd, theta):
    return sum(c * cmath.exp(1j * off * theta) for off, c in fd.items())


def test_five_cell_symbol_real_part():
    fd = flux_difference(scheme_coefficients(2))
    for theta in np.linspace(0, 2 * np.pi, 37):
        z = symbol(fd, theta)
        assert abs(z.real - 16.0 / 15.0 * math.sin(theta / 2) ** 6) < 1e-12


def test_seven_cell_symbol(golden_dir):
    fd = flux_difference(scheme_coefficients(3, seven_cell_weights))
    for k, a, b in read_golden(golden_dir, "seven_cell_symbol.txt"):
        k = int(k)
        ak = fd.get(0, 0.0) if k == 0 else fd.get(k, 0.0) + fd.get(-k, 0.0)
        bk = 0.0 if k == 0 else fd.get(k, 0.0) - fd.get(-k, 0.0)
        assert abs(ak - float(a)) <= 6e-5
        assert abs(bk - float(b)) <= 6e-5


def rk3_gain(z):
    """Amplification of the oracle's TVD-RK3 step on u' = lambda u, z = lambda dt."""
    return complex(O.rk3_step(lambda u: z * u, np.array([1.0 + 0j]), 1.0)[0])


def test_rk3_amplification():
    for z in [0.3, -1.2, 0.5 + 1.0j, -0.7 - 2.1j, 2.0j]:
        g = 1 + z + z * z / 2 + z ** 3 / 6
        assert abs(rk3_gain(z) - g) < 1e-14


def cfl_limit(fd):
    thetas = np.linspace(0, 2 * np.pi, 4001)
    zs = np.array([symbol(fd, t) for t in thetas])

    def stable(sig):
        return all(abs(rk3_gain(-sig * z)) <= 1 + 1e-12 for z in zs)

    lo, hi = 0.1, 3.0
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return lo


def test_cfl_limits(golden_dir):
    ref = {name: float(v) for name, v in read_golden(golden_dir, "cfl_limits.txt")}
    assert abs(cfl_limit(flux_difference(scheme_coefficients(2))) - ref["five_cell"]) <= 0.01
    assert abs(cfl_limit(flux_difference(scheme_coefficients(3, seven_cell_weights)))
               - ref["seven_cell"]) <= 0.01


def test_lf_reduces_to_upwind_1d():
    """With alpha = |a| the LF flux of u_t + a u_x is a * u^- for a > 0 (Sec. 4.2.1)."""
    mesh = uniform_line(11)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1,
                     velocity=(1.0, 0.0, 0.0))
    for um, up in [(0.3, 0.9), (-1.0, 2.0), (5.0, 5.0)]:
        assert abs(O.lax_friedrichs(prob, um, up, np.array([1.0]), 1.0) - um) < 1e-15


# ---------------------------------------------------------------------------
# moments: exact integration (sympy) and the WLS solve: rational brute force
# ---------------------------------------------------------------------------

def test_simplex_moments_vs_sympy():
    sp = pytest.importorskip("sympy")
    x, y, z, s, t, u = sp.symbols("x y z s t u")
    tri = [[Fraction(1, 3), Fraction(-1, 5)], [Fraction(7, 4), Fraction(1, 2)], [Fraction(-1, 2), Fraction(9, 8)]]
    P = [sp.Matrix([sp.Rational(c.numerator, c.denominator) for c in v]) for v in tri]
    # x(s,t) = P0 + s (P1 - P0) + t (P2 - P0), jacobian |det|
    X = P[0] + s * (P[1] - P[0]) + t * (P[2] - P[0])
    jac = abs((P[1] - P[0]).row_join(P[2] - P[0]).det())
    Y = np.array([[float(c) for c in v] for v in tri])
    for kappa in O.multi_indices(2, 5):
        f = X[0] ** kappa[0] * X[1] ** kappa[1] * jac
        exact = sp.integrate(sp.integrate(f, (t, 0, 1 - s)), (s, 0, 1))
        assert abs(O.simplex_monomial_integral(Y, kappa) - float(exact)) < 1e-13 * max(1.0, abs(float(exact)))
    tet = [[0, 0, 0], [Fraction(3, 2), Fraction(1, 4), 0], [Fraction(-1, 3), 1, Fraction(1, 5)],
           [Fraction(1, 2), Fraction(1, 3), Fraction(5, 4)]]
    P = [sp.Matrix([sp.Rational(Fraction(c).numerator, Fraction(c).denominator) for c in v]) for v in tet]
    X = P[0] + s * (P[1] - P[0]) + t * (P[2] - P[0]) + u * (P[3] - P[0])
    jac = abs((P[1] - P[0]).row_join(P[2] - P[0]).row_join(P[3] - P[0]).det())
    Y = np.array([[float(Fraction(c)) for c in v] for v in tet])
    for kappa in O.multi_indices(3, 4):
        f = X[0] ** kappa[0] * X[1] ** kappa[1] * X[2] ** kappa[2] * jac
        exact = sp.integrate(sp.integrate(sp.integrate(f, (u, 0, 1 - s - t)), (t, 0, 1 - s)), (s, 0, 1))
        assert abs(O.simplex_monomial_integral(Y, kappa) - float(exact)) < 1e-13 * max(1.0, abs(float(exact)))


def rational_normal_equations(A, w, b):
    """Solve (A^T W^2 A) v = A^T W^2 b exactly over the rationals."""
    n, m = len(A), len(A[0])
    M = [[sum(A[r][i] * w[r] * w[r] * A[r][j] for r in range(n)) for j in range(m)] for i in range(m)]
    rhs = [sum(A[r][i] * w[r] * w[r] * b[r] for r in range(n)) for i in range(m)]
    for col in range(m):
        piv = next(r for r in range(col, m) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        rhs[col], rhs[piv] = rhs[piv], rhs[col]
        for r in range(m):
            if r != col and M[r][col] != 0:
                f = M[r][col] / M[col][col]
                M[r] = [a - f * c for a, c in zip(M[r], M[col])]
                rhs[r] -= f * rhs[col]
    return [rhs[i] / M[i][i] for i in range(m)]


def test_wls_solve_vs_rational_normal_equations():
    rng = np.random.default_rng(7)
    for n, m in [(7, 3), (9, 6), (13, 6), (15, 10)]:
        A = [[Fraction(int(rng.integers(-9, 10)), int(rng.integers(1, 6))) for _ in range(m)] for _ in range(n)]
        for r in range(n):
            A[r][0] = Fraction(1)
        w = [Fraction(int(rng.integers(1, 20)), int(rng.integers(1, 7))) for _ in range(n)]
        b = [Fraction(int(rng.integers(-30, 31)), int(rng.integers(1, 9))) for _ in range(n)]
        exact = rational_normal_equations(A, w, b)
        v, r, _ = O.scaled_wls_solve(np.array(A, dtype=float), np.array(w, dtype=float),
                                     np.array(b, dtype=float))
        assert r == m
        scale = max(1.0, max(abs(float(e)) for e in exact))
        assert max(abs(v[k] - float(exact[k])) for k in range(m)) < 1e-10 * scale


def test_rank_truncation_drops_dependent_column():
    """A repeated column is rank deficient: r = m - 1 and the basic solution
    reproduces the least-squares fit of the independent columns."""
    rng = np.random.default_rng(3)
    A = rng.normal(size=(9, 4))
    A[:, 3] = 2.0 * A[:, 1]
    w = rng.uniform(0.5, 2.0, size=9)
    b = rng.normal(size=9)
    v, r, _ = O.scaled_wls_solve(A, w, b)
    assert r == 3
    ref, *_ = np.linalg.lstsq(w[:, None] * A[:, :3], w * b, rcond=None)
    fit = A @ v
    assert np.allclose(fit, A[:, :3] @ ref, atol=1e-12)


# ---------------------------------------------------------------------------
# stencils (Sec. 3.2): ring sizes on the regular meshes
# ---------------------------------------------------------------------------

def test_ring_sizes_regular_triangles():
    mesh = synth.tri_mesh(8, jitter=0.0)
    expect = {0.5: 4, 1.0: 13, 1.5: 22, 2.0: 37, 3.0: 73}
    for ring, size in expect.items():
        st, _ = O.build_stencils(mesh.cells, ring, 2)
        assert all(len(s) == size for s in st), ring


def test_ring_sizes_regular_tets():
    mesh = synth.tet_mesh(5, jitter=0.0)
    expect = {1.0 / 3.0: 5, 2.0 / 3.0: 19, 1.0: 71}
    for ring, size in expect.items():
        st, _ = O.build_stencils(mesh.cells, ring, 3)
        assert all(len(s) == size for s in st), ring


def test_one_ring_is_vertex_sharing_brute_force():
    mesh = synth.tri_mesh(6, jitter=0.2, seed=5)
    st, face = O.build_stencils(mesh.cells, 1.0, 2)
    sets = [set(map(int, c)) for c in mesh.cells]
    for i in range(mesh.n_cells):
        brute = sorted(j for j in range(mesh.n_cells) if j != i and sets[i] & sets[j])
        assert st[i] == [i] + brute
        assert face[i] == sorted(j for j in range(mesh.n_cells) if len(sets[i] & sets[j]) == 2)


# ---------------------------------------------------------------------------
# reconstruction: polynomial reproduction and the accuracy theorem (Sec. 4.1)
# ---------------------------------------------------------------------------

def random_poly(d, deg, rng):
    terms = [(k, rng.normal()) for k in O.multi_indices(d, deg + 1)]

    def f(P):
        return sum(c * np.prod([P[:, a] ** e for a, e in enumerate(k)], axis=0) for k, c in terms)

    def deriv(x, kappa):
        tot = 0.0
        for k, c in terms:
            if all(k[a] >= kappa[a] for a in range(d)):
                coef = c
                for a in range(d):
                    coef *= math.factorial(k[a]) / math.factorial(k[a] - kappa[a]) * x[a] ** (k[a] - kappa[a])
                tot += coef
        return tot

    return f, deriv


@pytest.mark.parametrize("dim,p,ring,n", [(2, 3, 1.0, 6), (2, 4, 2.0, 7), (3, 3, 2.0 / 3.0, 3)])
def test_polynomial_reproduction(dim, p, ring, n):
    rng = np.random.default_rng(11 + p)
    mesh = synth.tri_mesh(n, periodic=False, seed=3) if dim == 2 else synth.tet_mesh(n, periodic=False, seed=3)
    m = math.comb(p - 1 + dim, dim)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring,
                     min_rows=math.ceil(1.5 * m))
    f, deriv = random_poly(dim, p - 1, rng)
    ubar = synth.cell_averages(mesh, f)
    for i in range(0, prob.N, max(1, prob.N // 40)):
        dvec, r = prob.reconstruct_cell(ubar, i)
        assert r == prob.m
        got = prob.derivatives(dvec, i)
        ref = np.array([deriv(prob.geo.centroid[i], k) for k in prob.kappas])
        assert np.allclose(got, ref, rtol=1e-8, atol=1e-8 * np.max(np.abs(ref))), i


def test_reconstruction_order_smooth_periodic():
    """Accuracy theorem (Sec. 4.1): degree p-1 WLS gives O(h^p) values; p = 3."""
    errs = []
    hs = []
    for n in (8, 16, 32):
        mesh = synth.tri_mesh(n, jitter=0.2, seed=2)
        prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0)

        def f(P):
            return np.sin(2 * np.pi * P[:, 0]) * np.cos(2 * np.pi * P[:, 1])

        ubar = synth.cell_averages(mesh, f)
        err = 0.0
        for i in range(0, prob.N, max(1, prob.N // 48)):
            dvec, _ = prob.reconstruct_cell(ubar, i)
            for X in prob.geo.coords[i]:
                err = max(err, abs(prob.eval_poly(dvec, i, X) - f(X[None, :])[0]))
        errs.append(err)
        hs.append(1.0 / n)
    orders = [math.log(errs[k] / errs[k + 1]) / math.log(hs[k] / hs[k + 1]) for k in range(2)]
    assert min(orders) > 2.6, orders


@pytest.mark.parametrize("p,ring,min_order", [(3, 2.0, 2.7), (5, 3.0, 4.5)])
def test_reconstruction_order_1d(p, ring, min_order):
    """The 1-D schemes (Sec. 4.2.3, Sec. 4.2.4 build p = 5 on five and seven
    cells): degree p-1 reconstructions of smooth data on jittered periodic
    lines are O(h^p) at the cell ends (Sec. 4.1), here observed >= p - 0.5
    (p = 3 on the 2-ring, p = 5 on the 3-ring)."""
    errs = []
    hs = []
    for n in (16, 32, 64):
        mesh = synth.periodic_line_mesh(n, jitter=0.2, seed=3)
        prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, min_rows=int(2 * ring + 1))

        def f(P):
            return np.sin(2 * np.pi * P[:, 0]) + 0.5 * np.cos(4 * np.pi * P[:, 0])

        ubar = synth.cell_averages(mesh, f, k=8)
        err = 0.0
        for i in range(prob.N):
            dvec, _ = prob.reconstruct_cell(ubar, i)
            for X in prob.geo.coords[i]:
                err = max(err, abs(prob.eval_poly(dvec, i, X) - f(X[None, :])[0]))
        errs.append(err)
        hs.append(1.0 / n)
    orders = [math.log(errs[k] / errs[k + 1]) / math.log(hs[k] / hs[k + 1]) for k in range(2)]
    assert min(orders) >= min_order, orders


# ---------------------------------------------------------------------------
# residual (Eq. (fvm), Eq. (flux)): divergence theorem on exact data
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_advection_residual_is_exact_for_polynomials(dim):
    rng = np.random.default_rng(21)
    if dim == 2:
        mesh = synth.tri_mesh(6, periodic=False, seed=4)
        ring, vel = 1.0, (1.0, -0.6, 0.0)
    else:
        mesh = synth.tet_mesh(3, periodic=False, seed=4)
        ring, vel = 2.0 / 3.0, (1.0, 0.5, -0.25)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=ring,
                     velocity=vel, min_rows=9 if dim == 2 else 15)
    f, deriv = random_poly(dim, 2, rng)

    def div_flux(P):
        g = 0.0
        for a in range(dim):
            kap = [0] * dim
            kap[a] = 1
            g = g + vel[a] * np.array([deriv(x, kap) for x in P])
        return g

    ubar = synth.cell_averages(mesh, f)
    L = O.residual(prob, ubar)
    exact = -synth.cell_averages(mesh, div_flux)
    assert np.max(np.abs(L - exact)) < 1e-9 * np.max(np.abs(exact))


def test_burgers_residual_is_exact_for_linear_data():
    mesh = synth.tri_mesh(6, periodic=False, seed=6)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0, pde=O.BURGERS,
                     min_rows=9)
    a, b, c = 0.4, 1.3, -0.7

    def f(P):
        return a + b * P[:, 0] + c * P[:, 1]

    ubar = synth.cell_averages(mesh, f)
    L = O.residual(prob, ubar)
    exact = -synth.cell_averages(mesh, lambda P: f(P) * (b + c))  # div(u^2/2 (1,1)) = u (u_x + u_y)
    assert np.max(np.abs(L - exact)) < 1e-10 * np.max(np.abs(exact))


def test_periodic_conservation_and_constant_state():
    mesh = synth.tri_mesh(8, seed=9)
    rng = np.random.default_rng(5)
    for pde in (O.ADVECTION, O.BURGERS):
        prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0, pde=pde)
        ubar = rng.uniform(-1.0, 2.0, size=prob.N)
        L = O.residual(prob, ubar)
        vol = prob.geo.volume
        assert abs(np.sum(vol * L)) < 1e-13 * np.sum(vol * np.abs(L))
        Lc = O.residual(prob, np.full(prob.N, 0.75))
        assert np.max(np.abs(Lc)) < 1e-9


# ---------------------------------------------------------------------------
# weights (Sec. 3.1.2): the scalings the text states
# ---------------------------------------------------------------------------

def weights_on_mesh(n, f, i_frac=0.5):
    mesh = synth.tri_mesh(n, jitter=0.2, seed=8)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0)
    ubar = synth.cell_averages(mesh, f)
    out = []
    for i in range(0, prob.N, max(1, prob.N // 16)):
        S = prob.stencils[i]
        face = set(prob.face_nbrs[i])
        w = O.wls_eno_weights(ubar[S], [j in face for j in S], prob.geo.h[i])
        out.append((prob, i, S, face, w, ubar))
    return out


def test_weights_scale_as_inverse_h_squared_on_smooth_data():
    """omega_j = O(1/h^2) and not smaller where u is smooth."""
    f = lambda P: np.sin(2 * np.pi * P[:, 0]) + 0.5 * np.cos(2 * np.pi * P[:, 1])
    ranges = []
    for n in (8, 16, 32, 64):
        vals = [w * prob.geo.h[i] ** 2 for prob, i, S, face, w, _ in weights_on_mesh(n, f)]
        vals = np.concatenate(vals)
        ranges.append((vals.min(), vals.max()))
    # Theta(1/h^2): both ends of the range of omega * h^2 stay put under refinement
    los = [r[0] for r in ranges]
    his = [r[1] for r in ranges]
    assert max(los) / min(los) < 3.0, ranges
    assert max(his) / min(his) < 3.0, ranges
    assert max(his) <= 1.5 / 1e-2 * 1.0000001


def test_weights_are_order_one_across_a_jump():
    """omega_j = O(1) for stencil cells across a discontinuity."""
    f = lambda P: (P[:, 0] > 0.5).astype(float)
    for n in (16, 32, 64):
        mesh = synth.tri_mesh(n, jitter=0.2, seed=8)
        prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0)
        ubar = synth.cell_averages(mesh, f)
        for i in range(prob.N):
            S = prob.stencils[i]
            face = set(prob.face_nbrs[i])
            w = O.wls_eno_weights(ubar[S], [j in face for j in S], prob.geo.h[i])
            for k, j in enumerate(S[1:], start=1):
                if abs(ubar[j] - ubar[i]) > 0.99:
                    assert 0.5 < w[k] <= 1.0 / 0.99 ** 2


def test_centre_weight_dominates_facet_neighbours():
    """The centre cell gets the larger value: alpha times the largest weight of
    the cells that share a facet with it (beta_i is their smallest beta)."""
    rng = np.random.default_rng(4)
    mesh = synth.tri_mesh(8, jitter=0.2, seed=8)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0)
    ubar = rng.normal(size=prob.N)
    for i in range(prob.N):
        S = prob.stencils[i]
        face = set(prob.face_nbrs[i])
        w = O.wls_eno_weights(ubar[S], [j in face for j in S], prob.geo.h[i])
        wf = [w[k] for k, j in enumerate(S) if j in face]
        assert len(wf) == 3
        assert w[0] >= 1.5 * max(wf) * (1 - 1e-15)


# ---------------------------------------------------------------------------
# balanced-stencil re-selection (Sec. 3.2, last paragraph)
# ---------------------------------------------------------------------------

def test_balanced_stencil_selection_invariants():
    """The re-selected stencil keeps the centre (first) and its facet
    neighbours, has at least the old size, and fills both sides of the plane
    normal to the gradient up to their quotas (nearest cells first)."""
    mesh = synth.tri_mesh(12, jitter=0.2, seed=3)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=4, ring=2.0, pde=O.BURGERS)
    rng = np.random.default_rng(8)
    for i in rng.choice(prob.N, 12, replace=False):
        i = int(i)
        a = rng.uniform(0, 2 * np.pi)
        d = np.zeros(prob.m)
        d[1:3] = (np.cos(a), np.sin(a))
        S = O.balanced_stencil(prob, i, d)
        n = len(prob.stencils[i])
        assert S[0] == i and len(S) >= n and len(set(S)) == len(S)
        assert set(prob.face_nbrs[i]) <= set(S)
        g = d[1:3]
        side = {j: float(np.dot(O.min_image(prob.geo.centroid[j] - prob.geo.centroid[i], prob.period), g)) > 0
                for j in S[1:]}
        plus = sum(side.values())
        minus = len(S) - 1 - plus
        face_plus = sum(side[j] for j in prob.face_nbrs[i])
        face_minus = len(prob.face_nbrs[i]) - face_plus
        assert abs(plus - minus) <= 1 + abs(face_plus - face_minus), (plus, minus)


def test_balanced_stencil_selection_invariants_3d():
    """The same invariants on tetrahedra (the paper's motivating case: nearly
    one-sided 3-D neighbourhoods)."""
    mesh = synth.tet_mesh(4, seed=15)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=2.0 / 3.0, pde=O.BURGERS, min_rows=15)
    rng = np.random.default_rng(9)
    for i in rng.choice(prob.N, 10, replace=False):
        i = int(i)
        d = np.zeros(prob.m)
        g = rng.normal(size=3)
        d[1:4] = g
        S = O.balanced_stencil(prob, i, d)
        n = len(prob.stencils[i])
        assert S[0] == i and len(S) == n and len(set(S)) == len(S)
        assert set(prob.face_nbrs[i]) <= set(S)
        side = {j: float(np.dot(O.min_image(prob.geo.centroid[j] - prob.geo.centroid[i], prob.period), g)) > 0
                for j in S[1:]}
        plus = sum(side.values())
        face_plus = sum(side[j] for j in prob.face_nbrs[i])
        face_minus = len(prob.face_nbrs[i]) - face_plus
        assert abs(plus - (len(S) - 1 - plus)) <= 1 + abs(face_plus - face_minus), (plus, len(S))
        # on each side the chosen cells (beyond the facet neighbours) come
        # before every candidate left out, by (squared distance, index)
        steps = ["vertex"] * (int(math.ceil(prob.ring - 1e-9)) + 1)
        cands = O.k_ring(i, steps, prob.nbr) - {i}
        dx = {j: O.min_image(prob.geo.centroid[j] - prob.geo.centroid[i], prob.period) for j in cands}
        key = {j: (float(np.dot(dx[j], dx[j])), j) for j in cands}
        plus_side = {j: float(np.dot(dx[j], g)) > 0 for j in cands}
        face = set(int(j) for j in prob.face_nbrs[i])
        for sd in (True, False):
            mine = [key[j] for j in S[1:] if plus_side[j] == sd and j not in face]
            others = [key[j] for j in cands - set(S) if plus_side[j] == sd]
            if mine and others:
                assert max(mine) < min(others), (i, sd)


def test_balanced_stencil_of_a_symmetric_1d_stencil_is_itself():
    """On a uniform 1-D grid the k-ring is already balanced about the
    centroid: the re-selection returns the same stencil for either sign of
    the gradient."""
    mesh = synth.periodic_line_mesh(20)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=5, ring=2.0)
    for sgn in (1.0, -1.0):
        d = np.zeros(prob.m)
        d[1] = sgn
        assert O.balanced_stencil(prob, 10, d) == prob.stencils[10]


def test_balancing_leaves_smooth_data_alone_and_reduces_overshoot_at_a_jump():
    """Smooth data: no facet value leaves its stencil's range by the margin,
    so the balanced scheme's residual is the plain one.  A jump and random
    data: the balanced reconstructions leave the range at fewer cells."""
    mesh = synth.tri_mesh(12, jitter=0.2, seed=3)
    plain = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=4, ring=2.0, pde=O.BURGERS)
    bal = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=4, ring=2.0, pde=O.BURGERS, balanced=True)
    smooth = synth.burgers_2d_initial(mesh)
    assert np.array_equal(O.residual(plain, smooth), O.residual(bal, smooth))
    jump = synth.cell_averages(mesh, lambda P: (P[:, 0] + 0.4 * P[:, 1] > 0.55).astype(float), k=8)
    before = [O.out_of_range(plain, jump, i, d) for i, d in enumerate(O.reconstruct_all(plain, jump))]
    after = [O.out_of_range(plain, jump, i, d) for i, d in enumerate(O.reconstruct_all(bal, jump))]
    assert sum(before) > 0
    assert sum(after) < sum(before), (sum(before), sum(after))
    # random averages: every local extremum tests the range; balancing keeps
    # most reconstructions inside it (Sec. 3.2: "typically" within range)
    rnd = np.random.default_rng(4).uniform(-1.0, 1.0, plain.N)
    before = sum(O.out_of_range(plain, rnd, i, d) for i, d in enumerate(O.reconstruct_all(plain, rnd)))
    after = sum(O.out_of_range(plain, rnd, i, d) for i, d in enumerate(O.reconstruct_all(bal, rnd)))
    assert before >= 10 and 2 * after <= before, (before, after)


# ---------------------------------------------------------------------------
# moment rows from a cell's own central moments (the binomial shift the
# moments-on-the-fly kernel uses)
# ---------------------------------------------------------------------------

def test_moment_rows_are_binomial_shifts_of_own_central_moments():
    """Row j of cell i's moment matrix (Sec. 3.2, h_i-normalised Taylor
    monomials about x_i) equals sum over alpha <= kappa of cell j's own
    central moments M_j[alpha] (about x_j, absolute units) times
    h_i^-|alpha| d^(kappa-alpha)/(kappa-alpha)!, d = (x_j - x_i)/h_i at the
    minimum image: the binomial theorem; M_j[0] = 1 and the first moments
    vanish about the centroid."""
    rng = np.random.default_rng(12)
    for mesh, p, ring in ((synth.tri_mesh(8, seed=4), 4, 2.0), (synth.tet_mesh(3, seed=5), 3, 2.0 / 3.0),
                          (synth.periodic_line_mesh(12, jitter=0.2, seed=6), 5, 2.0)):
        prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring)
        kap = prob.kappas
        geo = prob.geo
        for i in rng.choice(prob.N, 6, replace=False):
            i = int(i)
            S = prob.stencils[i]
            A = prob.A(i)
            Ys = O.stencil_coords(geo, S, i, prob.period)
            for t, j in enumerate(S):
                cj = Ys[t].mean(axis=0)  # centroid of the image next to tau_i
                own = O.moment_row(Ys[t], cj, 1.0, kap)
                assert abs(own[0] - 1.0) <= 1e-13
                for k, kp in enumerate(kap):
                    if sum(kp) == 1:
                        assert abs(own[k]) <= 1e-13
                d = (cj - geo.centroid[i]) / geo.h[i]
                for k, kp in enumerate(kap):
                    want = 0.0
                    for k2, al in enumerate(kap):
                        if all(a <= b for a, b in zip(al, kp)):
                            term = own[k2] * geo.h[i] ** (-sum(al))
                            for c in range(len(kp)):
                                term *= d[c] ** (kp[c] - al[c]) / math.factorial(kp[c] - al[c])
                            want += term
                    assert abs(A[t, k] - want) <= 1e-11 * max(1.0, abs(want)), (i, j, kp)


# ---------------------------------------------------------------------------
# QR with column pivoting (Sec. 3.3.2) and the pivot rule of reading R6
# ---------------------------------------------------------------------------

def _q_of(vs, n):
    """Q from Q^T e_j, column by column."""
    return np.column_stack([O.apply_qt(vs, e) for e in np.eye(n)]).T


@pytest.mark.parametrize("n,m", [(9, 4), (37, 10), (5, 10), (10, 10)])
def test_qrcp_factors_the_permuted_matrix(n, m):
    """B[:, piv] = Q R with Q orthogonal and R upper triangular, and the
    diagonal of R non-increasing up to the pivot window:
    R_kk^2 >= (1 - 1e-6) R_(k+1)(k+1)^2."""
    rng = np.random.default_rng(n * m)
    B = rng.normal(size=(n, m)) * rng.uniform(0.1, 10.0, size=m)
    R, piv, vs = O.qr_column_pivoting(B)
    assert sorted(piv) == list(range(m))
    Q = _q_of(vs, n)
    k = min(n, m)
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 1e-14
    assert np.max(np.abs(Q[:, :k] @ R - B[:, piv])) <= 1e-13 * np.max(np.abs(B))
    assert np.allclose(R, np.triu(R))
    d = np.abs(np.diag(R))
    assert all(d[j] ** 2 >= (1 - 1e-6) * d[j + 1] ** 2 for j in range(k - 1))


def test_pivot_rule_takes_the_lowest_index_within_the_window():
    """Reading R6: equal norms (every column of the scaled system has norm
    1) pick the lowest index; a squared norm within 1e-6 of the largest
    counts as a tie, one 1e-5 below does not."""
    rng = np.random.default_rng(5)
    B = rng.normal(size=(12, 4))
    B /= np.linalg.norm(B, axis=0)
    assert O.qr_column_pivoting(B)[1][0] == 0
    C = B.copy()
    C[:, 2] *= math.sqrt(1 + 5e-7)   # the largest, but inside the window
    assert O.qr_column_pivoting(C)[1][0] == 0
    C[:, 2] = B[:, 2] * math.sqrt(1 + 1e-5)  # outside the window
    assert O.qr_column_pivoting(C)[1][0] == 2
    # the window is relative to the largest squared norm at every step
    D = np.diag([1.0, 3.0, 2.0, 3.0 * (1 - 4e-7)])
    assert O.qr_column_pivoting(D)[1] == [1, 3, 2, 0]


def test_basic_solution_of_a_short_system():
    """n < m: rank n, and the basic solution is the exact fit on the first
    n pivot columns (zero elsewhere), the definition of Sec. 3.3.2 with E
    restricted to the first r columns."""
    rng = np.random.default_rng(8)
    A = rng.normal(size=(6, 10))
    w = rng.uniform(0.5, 2.0, size=6)
    b = rng.normal(size=6)
    v, r, _ = O.scaled_wls_solve(A, w, b)
    assert r == 6
    s = 1.0 / np.linalg.norm(w[:, None] * A, axis=0)
    _, piv, _ = O.qr_column_pivoting(w[:, None] * A * s)
    keep = piv[:6]
    assert np.all(v[[c for c in range(10) if c not in keep]] == 0.0)
    assert np.allclose(A[:, keep] @ v[keep], b, atol=1e-12)
