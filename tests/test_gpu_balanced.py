"""The balanced-stencil re-selection (Sec. 3.2, last paragraph) through the C
ABI on the GPU against the oracle (Problem(balanced=True)): FP64
coefficients, residuals and RK steps within 1e-10, the number of re-solved
cells exact, FP32-bulk states within relative L1 1e-5; smooth data re-select
nothing and leave the plain scheme's results unchanged."""
import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL64 = 1e-10
MARGIN = 0.02


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch.device("cuda:0")


def Context(**kw):
    from paper_1602_02694_gb300.wlseno import Context as C
    return C(0, **kw)


def jump2(P):
    return (P[:, 0] + 0.4 * P[:, 1] > 0.55).astype(float)


def jump3(P):
    return np.sin(2 * np.pi * P[:, 0]) + (P[:, 0] + 0.3 * P[:, 1] + 0.2 * P[:, 2] > 0.6)


def jump1(P):
    return 0.5 + np.sin(2 * np.pi * P[:, 0]) + (P[:, 0] > 0.6)


# name: (mesh, p, ring, min_rows, data); min_rows as the oracle's (no growth
# beyond it), random data make every local extremum a range violation
CASES = {
    "tri12_p4_jump": (lambda: synth.tri_mesh(12, seed=3), 4, 2.0, 15,
                      lambda m: synth.cell_averages(m, jump2, k=8)),
    "tri12_p4_random": (lambda: synth.tri_mesh(12, seed=3), 4, 2.0, 15,
                        lambda m: np.random.default_rng(4).uniform(-1.0, 1.0, m.cells.shape[0])),
    "tri9_p3_open_random": (lambda: synth.tri_mesh(9, periodic=False, seed=12), 3, 1.0, 9,
                            lambda m: np.random.default_rng(5).uniform(-1.0, 1.0, m.cells.shape[0])),
    "tet4_p3_jump": (lambda: synth.tet_mesh(4, seed=15), 3, 2.0 / 3.0, 15,
                     lambda m: synth.cell_averages(m, jump3, k=4)),
    "line48_p5_jump": (lambda: synth.periodic_line_mesh(48, jitter=0.2, seed=7), 5, 2.0, 5,
                       lambda m: synth.cell_averages(m, jump1, k=6)),
}

_cache = {}


def case(name):
    if name not in _cache:
        make, p, ring, min_rows, data = CASES[name]
        mesh = make()
        prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, pde=O.BURGERS,
                         min_rows=min_rows, balanced=True, balance_margin=MARGIN)
        ubar = data(mesh)
        plain = [prob.reconstruct_cell(ubar, i)[0] for i in range(prob.N)]
        n_bal = sum(1 for i in range(prob.N) if O.out_of_range(prob, ubar, i, plain[i])
                    and O.balanced_stencil(prob, i, plain[i]) is not None)
        _cache[name] = (mesh, prob, ubar, np.array(O.reconstruct_all(prob, ubar)), n_bal)
    return _cache[name]


def make_ctx(mesh, prob, precision="fp64", balanced=True):
    ctx = Context(pde="burgers", precision=precision, balanced=balanced, balance_margin=MARGIN)
    ctx.build_stencils(mesh, order_p=prob.p, ring=prob.ring, min_rows=prob.min_rows)
    ctx.precompute_moments()
    return ctx


@pytest.mark.parametrize("name", list(CASES))
def test_balanced_reconstruction_matches_the_oracle(dev, name):
    mesh, prob, ubar, ref, n_bal = case(name)
    assert n_bal > 0
    ctx = make_ctx(mesh, prob)
    ptr, cols = ctx.stencils()
    assert [list(cols[ptr[i]:ptr[i + 1]]) for i in range(prob.N)] == [list(s) for s in prob.stencils]
    nq = 1 if prob.dim == 1 else prob.dim
    u = torch.tensor(ubar, device=dev)
    coef = torch.empty(prob.N * prob.m, dtype=torch.float64, device=dev)
    fv = torch.empty(prob.N * (prob.dim + 1) * nq, dtype=torch.float64, device=dev)
    # the range test on the facet values, and on the coefficients alone
    for with_fv in (True, False):
        coef.zero_()
        ctx.reconstruct(u, coef, fv if with_fv else None)
        got = coef.cpu().numpy().reshape(prob.N, prob.m)
        assert np.max(np.abs(got - ref)) <= TOL64, with_fv
        assert ctx.diagnostics()["balanced_cells"] == n_bal, with_fv
    ctx.close()


@pytest.mark.parametrize("name", list(CASES))
def test_balanced_residual_matches_the_oracle(dev, name):
    mesh, prob, ubar, ref, n_bal = case(name)
    ref_L = O.residual(prob, ubar, coeffs=list(ref))
    ctx = make_ctx(mesh, prob)
    u = torch.tensor(ubar, device=dev)
    L = torch.empty_like(u)
    ctx.flux_residual(u, L)
    assert np.max(np.abs(L.cpu().numpy() - ref_L)) <= TOL64 * max(1.0, np.max(np.abs(ref_L)))
    assert ctx.diagnostics()["balanced_cells"] == n_bal
    ctx.close()


@pytest.mark.parametrize("name", ["tri12_p4_jump", "line48_p5_jump"])
def test_balanced_rk_steps_match_the_oracle(dev, name):
    """Three CFL-0.3 Burgers steps (the stencils re-selected at every stage),
    FP64 within 1e-10 and FP32-bulk within relative L1 1e-5."""
    mesh, prob, ubar, _, _ = case(name)
    ref3, _ = O.rk3_run(prob, ubar, 3, cfl=0.3)
    for precision in ("fp64", "fp32_bulk"):
        ctx = make_ctx(mesh, prob, precision)
        u = torch.tensor(ubar, device=dev)
        ctx.rk_step(u, cfl=0.3, n_steps=3)
        got = u.cpu().numpy()
        if precision == "fp64":
            assert np.max(np.abs(got - ref3)) <= TOL64
        else:
            assert np.sum(np.abs(got - ref3)) / np.sum(np.abs(ref3)) <= 1e-5
        assert ctx.diagnostics()["launches_by_kind"]["fixup"] > 0
        ctx.close()


def test_balanced_with_rows_formed_on_the_fly(dev):
    """The balanced pass after the FP32-bulk kernel that forms its moment rows
    on the fly: three RK steps within relative L1 1e-5 of the oracle, with
    cells re-selected."""
    mesh, prob, ubar, _, n_bal = case("tri12_p4_jump")
    ref3, _ = O.rk3_run(prob, ubar, 3, cfl=0.3)
    ctx = Context(pde="burgers", precision="fp32_bulk", balanced=True, balance_margin=MARGIN)
    ctx.build_stencils(mesh, order_p=prob.p, ring=prob.ring, min_rows=prob.min_rows, moments_mode=1)
    ctx.precompute_moments()
    u = torch.tensor(ubar, device=dev)
    L = torch.empty_like(u)
    ctx.flux_residual(u, L)
    assert ctx.diagnostics()["balanced_cells"] == n_bal
    ctx.rk_step(u, cfl=0.3, n_steps=3)
    got = u.cpu().numpy()
    assert np.sum(np.abs(got - ref3)) / np.sum(np.abs(ref3)) <= 1e-5
    ctx.close()


def test_smooth_data_reselect_nothing(dev):
    """The smooth Burgers data on the 12 x 12 mesh stay within the margin
    everywhere: no cell is re-solved and the residual is the plain one."""
    mesh = synth.tri_mesh(12, seed=3)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=4, ring=2.0, pde=O.BURGERS, min_rows=15)
    u = torch.tensor(synth.burgers_2d_initial(mesh), device=dev)
    out = []
    for balanced in (False, True):
        ctx = make_ctx(mesh, prob, balanced=balanced)
        L = torch.empty_like(u)
        ctx.flux_residual(u, L)
        out.append(L.cpu().numpy())
        assert ctx.diagnostics()["balanced_cells"] == 0
        ctx.close()
    assert np.array_equal(out[0], out[1])


def test_adjoint_is_refused_for_balanced_stencils(dev):
    from paper_1602_02694_gb300.wlseno import WlsenoError
    mesh, prob, ubar, _, _ = case("tri12_p4_jump")
    ctx = make_ctx(mesh, prob)
    u = torch.tensor(ubar, device=dev)
    g = torch.ones_like(u)
    out = torch.empty_like(u)
    with pytest.raises(WlsenoError):
        ctx.step_adjoint(u, 1e-3, g, out)
    ctx.close()
