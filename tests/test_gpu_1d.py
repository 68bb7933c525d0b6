"""The 1-D path of the library (segments, p = 3 and 5) through the C ABI on
the GPU, against the paper's printed 1-D schemes (Sec. 4.2.3, Sec. 4.2.4;
golden files) and against the oracle."""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL64 = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch.device("cuda:0")


def golden(name):
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    rows = []
    with open(path) as fh:
        for line in fh:
            line = line.split("#", 1)[0].strip()
            if line:
                off, val = line.split()
                rows.append((int(off), float(Fraction(val))))
    return rows


def Context(**kw):
    from paper_1602_02694_gb300.wlseno import Context as C
    return C(0, **kw)


def right_facet_values(ctx, u, n):
    """u^-_{i+1/2} of every cell: local facet 0 (opposite the left vertex)."""
    fv = torch.empty(2 * n, dtype=torch.float64, device=u.device)
    ctx.reconstruct(u, None, fv)
    return fv.cpu().numpy().reshape(n, 2)[:, 0]


def test_five_cell_scheme_on_the_gpu(dev):
    """p = 5 on the 2-ring (five cells, a square system: the weights drop
    out) of a uniform periodic grid: every cell's right facet value is the
    paper's (2 ubar_{i-2} - 13 ubar_{i-1} + 47 ubar_i + 27 ubar_{i+1}
    - 3 ubar_{i+2}) / 60 of random averages."""
    n = 32
    mesh = synth.periodic_line_mesh(n)
    ubar = np.random.default_rng(5).uniform(-1.0, 1.0, n)
    # FP32-bulk: random data make the weights spread widely, kappa(W A S) up
    # to 1.5e5 (median 199; oracle, these cells); one FP64-residual sweep
    # leaves about (kappa 2^-24)^2 = 8e-5 of the O(1) values
    for precision, tol in (("fp64", 1e-13), ("fp32_bulk", 1e-4)):
        ctx = Context(pde="burgers", precision=precision)
        ctx.build_stencils(mesh, order_p=5, ring=2.0, min_rows=5)
        ctx.precompute_moments()
        assert ctx.info()["max_stencil"] == 5
        got = right_facet_values(ctx, torch.tensor(ubar, device=dev), n)
        want = np.zeros(n)
        for off, c in golden("five_cell_scheme.txt"):
            want += c * np.roll(ubar, -off)
        assert np.max(np.abs(got - want)) <= tol, precision
        ctx.close()


def test_seven_cell_scheme_on_the_gpu(dev):
    """p = 5 on the 3-ring (seven cells, weighted least squares): for linear
    data and eps -> 0 the weights are the paper's (1/9, 1/4, 1, 3/2, 1, 1/4,
    1/9); the response of u^-_{i+1/2} to a small change of one average
    (linear data + 1e-7 e_k: the weights move by O(1e-7 / dx)) gives the
    paper's seven-cell coefficients."""
    n, delta = 32, 1e-7
    mesh = synth.periodic_line_mesh(n)
    i = 16
    base = np.arange(n) / n  # linear across cell i's stencil
    ctx = Context(pde="burgers", eps=1e-20)
    ctx.build_stencils(mesh, order_p=5, ring=3.0, min_rows=7)
    ctx.precompute_moments()
    f0 = right_facet_values(ctx, torch.tensor(base, device=dev), n)[i]
    for off, c in golden("seven_cell_scheme.txt"):
        u = base.copy()
        u[i + off] += delta
        f1 = right_facet_values(ctx, torch.tensor(u, device=dev), n)[i]
        assert abs((f1 - f0) / delta - c) <= 2e-5, (off, (f1 - f0) / delta, c)
    ctx.close()


@pytest.mark.parametrize("p,ring", [(5, 3.0), (3, 1.0)])
def test_1d_parity_with_the_oracle(dev, p, ring):
    """Jittered periodic line (48 cells): coefficients, residual and three
    CFL-0.3 Burgers steps against the oracle (FP64), FP32-bulk within 1e-5."""
    n = 48
    mesh = synth.periodic_line_mesh(n, jitter=0.2, seed=7)
    ubar = synth.cell_averages(mesh, lambda P: 0.5 + np.sin(2 * np.pi * P[:, 0]) + (P[:, 0] > 0.6), k=6)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, pde=O.BURGERS)
    m = prob.m
    ref_coef = np.array([prob.reconstruct_cell(ubar, i)[0] for i in range(n)])
    ref_L = O.residual(prob, ubar)
    ref3, _ = O.rk3_run(prob, ubar, 3, cfl=0.3)
    out = {}
    for precision in ("fp64", "fp32_bulk"):
        ctx = Context(pde="burgers", precision=precision)
        # min_rows = the ring's own size (2 ring + 1): no growth, as in the oracle
        ctx.build_stencils(mesh, order_p=p, ring=ring, min_rows=int(2 * ring + 1))
        ctx.precompute_moments()
        ptr, cols = ctx.stencils()
        assert [list(cols[ptr[i]:ptr[i + 1]]) for i in range(n)] == [prob.stencils[i] for i in range(n)]
        u = torch.tensor(ubar, device=dev)
        coef = torch.empty(n * m, dtype=torch.float64, device=dev)
        ctx.reconstruct(u, coef)
        L = torch.empty_like(u)
        ctx.flux_residual(u, L)
        ctx.rk_step(u, cfl=0.3, n_steps=3)
        out[precision] = (coef.cpu().numpy().reshape(n, m), L.cpu().numpy(), u.cpu().numpy())
        ctx.close()
    coef, L, u3 = out["fp64"]
    assert np.max(np.abs(coef - ref_coef)) <= TOL64
    assert np.max(np.abs(L - ref_L)) <= TOL64 * max(1.0, np.max(np.abs(ref_L)))
    assert np.max(np.abs(u3 - ref3)) <= TOL64
    u32 = out["fp32_bulk"][2]
    assert np.sum(np.abs(u32 - ref3)) / np.sum(np.abs(ref3)) <= 1e-5


@pytest.mark.parametrize("p,ring", [(3, 2.0), (5, 3.0)])
def test_1d_euler_shock_tube_parity_with_the_oracle(dev, p, ring):
    """Componentwise 1-D Euler (n_comp = 3) on a jittered transmissive line of
    64 cells with shock-tube data: residual and three CFL-0.3 steps against
    the oracle (FP64 within 1e-10, FP32-bulk within relative L1 1e-5), and
    the same cells falling back to their averages."""
    rng = np.random.default_rng(9)
    n = 64
    nodes = np.linspace(0.0, 1.0, n + 1)
    nodes[1:-1] += rng.uniform(-0.2, 0.2, n - 1) / n
    mesh = synth.line_mesh(nodes)
    ubar = synth.shock_tube_initial(mesh, x0=0.43)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, pde=O.EULER,
                     min_rows=int(2 * ring + 1))
    ref_L = O.residual(prob, ubar)
    ok = O.euler_positive(prob, ubar, O.euler_coeffs(prob, ubar))
    ref3, _ = O.rk3_run(prob, ubar, 3, cfl=0.3)
    out = {}
    for precision in ("fp64", "fp32_bulk"):
        ctx = Context(pde="euler", n_comp=3, precision=precision)
        ctx.build_stencils(mesh, order_p=p, ring=ring, min_rows=int(2 * ring + 1))
        ctx.precompute_moments()
        u = torch.tensor(ubar.ravel(), device=dev)
        L = torch.empty_like(u)
        ctx.flux_residual(u, L)
        fallbacks = ctx.diagnostics()["positivity_fallbacks"]
        ctx.rk_step(u, cfl=0.3, n_steps=3)
        out[precision] = (L.cpu().numpy().reshape(3, n), u.cpu().numpy().reshape(3, n), fallbacks)
        ctx.close()
    L64, u64, fb = out["fp64"]
    assert fb == int(np.sum(~ok))
    assert np.max(np.abs(L64 - ref_L)) <= TOL64 * max(1.0, float(np.max(np.abs(ref_L))))
    assert np.max(np.abs(u64 - ref3)) <= TOL64
    u32 = out["fp32_bulk"][1]
    assert np.sum(np.abs(u32 - ref3)) / np.sum(np.abs(ref3)) <= 1e-5


def test_1d_characteristic_euler_parity_with_the_oracle(dev):
    """Characteristic-wise 1-D Euler (Sec. 5.1.4's decomposition, per facet)
    on the shock tube: residual and three CFL-0.3 steps against the oracle,
    FP64 within 1e-10 and FP32-bulk within relative L1 1e-5."""
    rng = np.random.default_rng(9)
    n = 64
    nodes = np.linspace(0.0, 1.0, n + 1)
    nodes[1:-1] += rng.uniform(-0.2, 0.2, n - 1) / n
    mesh = synth.line_mesh(nodes)
    ubar = synth.shock_tube_initial(mesh, x0=0.43)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=2.0, pde=O.EULER, min_rows=5,
                     characteristic=True)
    ref_L = O.residual(prob, ubar)
    ref3, _ = O.rk3_run(prob, ubar, 3, cfl=0.3)
    out = {}
    for precision in ("fp64", "fp32_bulk"):
        ctx = Context(pde="euler", n_comp=3, precision=precision, characteristic=True)
        ctx.build_stencils(mesh, order_p=3, ring=2.0, min_rows=5)
        ctx.precompute_moments()
        u = torch.tensor(ubar.ravel(), device=dev)
        L = torch.empty_like(u)
        ctx.flux_residual(u, L)
        ctx.rk_step(u, cfl=0.3, n_steps=3)
        out[precision] = (L.cpu().numpy().reshape(3, n), u.cpu().numpy().reshape(3, n))
        ctx.close()
    L64, u64 = out["fp64"]
    assert np.max(np.abs(L64 - ref_L)) <= TOL64 * max(1.0, float(np.max(np.abs(ref_L))))
    assert np.max(np.abs(u64 - ref3)) <= TOL64
    u32 = out["fp32_bulk"][1]
    assert np.sum(np.abs(u32 - ref3)) / np.sum(np.abs(ref3)) <= 1e-5
