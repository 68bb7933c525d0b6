"""Through the C ABI on the GPU:

* the rank rule and basic solution of Sec. 3.3.2 on systems the rule
  truncates: with a rank tolerance of 1e-2 and above, real jittered stencils
  lose columns; every cell goes to the pivoted kernel, whose coefficients
  (dropped ones exactly 0) and count of rank-deficient cells must equal the
  oracle's, cell by cell; and at the default tolerance, weighted stencils
  dominated by cells with collinear centroids lose the columns the line
  cannot determine;
* the error contract of non-finite results: a NaN cell average gives
  WLSENO_ERR_NUMERIC from the call that synchronises, or from the next call
  when the arrays are on the device, and the context works again after the
  report."""
import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL64 = 1e-10
NUMERIC = -6


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch.device("cuda:0")


def Context(**kw):
    from paper_1602_02694_gb300.wlseno import Context as C
    return C(0, **kw)


def oracle_coeffs(prob, ubar):
    d = np.zeros((prob.N, prob.m))
    r = np.zeros(prob.N, dtype=int)
    for i in range(prob.N):
        d[i], r[i] = prob.reconstruct_cell(ubar, i)
    return d, r


@pytest.mark.parametrize("rank_tol,p,ring,shape", [(1e-2, 4, 2.0, (0, 0)), (3e-2, 4, 2.0, (16, 3)),
                                                   (5e-2, 3, 1.0, (0, 0)), (1e-2, 3, 1.0, (8, 2))])
def test_rank_truncation_matches_oracle(dev, rank_tol, p, ring, shape):
    mesh = synth.tri_mesh(10, jitter=0.2, seed=4)
    rng = np.random.default_rng(11)
    cen = mesh.cell_coords.mean(axis=1)
    ubar = 0.5 + np.sin(2 * np.pi * cen[:, 0]) + 0.05 * rng.standard_normal(mesh.n_cells)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, pde=O.BURGERS, rank_tol=rank_tol)
    ref, rank = oracle_coeffs(prob, ubar)
    assert np.sum(rank < prob.m) >= prob.N // 20, "the tolerance must truncate many cells"
    ctx = Context(pde="burgers", rank_tol=rank_tol)
    ctx.build_stencils(mesh, order_p=p, ring=ring, lanes_per_cell=shape[0], rows_per_lane=shape[1])
    ctx.precompute_moments()
    u = torch.tensor(ubar, device=dev)
    coef = torch.empty(prob.N * prob.m, dtype=torch.float64, device=dev)
    ctx.reconstruct(u, coef)
    got = coef.cpu().numpy().reshape(prob.N, prob.m)
    assert ctx.diagnostics()["rank_deficient"] == int(np.sum(rank < prob.m))
    # the oracle's dropped coefficients are exactly zero here too, and no cell
    # keeps more columns than the oracle's rank
    assert np.all(got[ref == 0.0] == 0.0)
    assert np.all(np.sum(got != 0.0, axis=1) <= rank)
    scale = np.maximum(1.0, np.max(np.abs(ref), axis=1))
    assert float(np.max(np.abs(got - ref) / scale[:, None])) <= TOL64
    ctx.close()


def test_collinear_weighted_stencils_drop_columns(dev):
    """On the unjittered "/"-split grid the cells of one kind (lower or upper
    triangles) with the same x + y have collinear centroids, and the exact
    averages of sin(2 pi (x + y)) are equal along those lines.  With a tiny
    eps the weights of Sec. 3.1.2 are 1/(eps h^2) on those cells and about
    1e-13 of that elsewhere, so W A S has only the columns the line
    determines to well above rank_tol = 1e-10 of |R_11|: the rank rule drops
    the others (basic solution, Sec. 3.3.2) in every cell."""
    mesh = synth.tri_mesh(12, jitter=0.0, seed=1)
    ubar = synth.cell_averages(mesh, lambda P: np.sin(2 * np.pi * (P[:, 0] + P[:, 1])), k=6)
    cen = mesh.cell_coords.mean(axis=1)
    key = np.round((cen[:, 0] + cen[:, 1]) * 36).astype(int) % 36
    for k in np.unique(key):
        sel = ubar[key == k]
        assert np.ptp(sel) <= 1e-14, "equal averages along each line"
    eps = 1e-12
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0, pde=O.BURGERS, eps=eps)
    ref, rank = oracle_coeffs(prob, ubar)
    assert np.all(rank < prob.m)
    ctx = Context(pde="burgers", eps=eps)
    ctx.build_stencils(mesh, order_p=3, ring=1.0)
    ctx.precompute_moments()
    coef = torch.empty(prob.N * prob.m, dtype=torch.float64, device=dev)
    ctx.reconstruct(torch.tensor(ubar, device=dev), coef)
    got = coef.cpu().numpy().reshape(prob.N, prob.m)
    assert ctx.diagnostics()["rank_deficient"] == prob.N
    assert np.all(got[ref == 0.0] == 0.0)
    assert np.all(np.sum(got != 0.0, axis=1) <= rank)
    scale = np.maximum(1.0, np.max(np.abs(ref), axis=1))
    assert float(np.max(np.abs(got - ref) / scale[:, None])) <= TOL64
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_nan_average_reports_numeric(dev, precision):
    from paper_1602_02694_gb300.wlseno import WlsenoError
    mesh = synth.tri_mesh(8, jitter=0.2, seed=1)
    ubar = synth.burgers_2d_initial(mesh)
    bad = ubar.copy()
    bad[17] = np.nan
    ctx = Context(pde="burgers", precision=precision)
    ctx.build_stencils(mesh, order_p=3, ring=1.0)
    ctx.precompute_moments()
    # host arrays: the call synchronises and reports its own result
    res = np.zeros(mesh.n_cells)
    with pytest.raises(WlsenoError) as ei:
        ctx.flux_residual(bad, res)
    assert ei.value.status == NUMERIC
    ctx.flux_residual(ubar, res)  # reported once: the context works again
    assert np.all(np.isfinite(res))
    # device arrays: the call returns at once; the next call reports it
    ud = torch.tensor(bad, device=dev)
    rd = torch.empty_like(ud)
    ctx.flux_residual(ud, rd)
    torch.cuda.synchronize()
    assert ctx.diagnostics()["nonfinite"] > 0
    with pytest.raises(WlsenoError) as ei:
        ctx.rk_step(torch.tensor(ubar, device=dev), cfl=0.3)
    assert ei.value.status == NUMERIC
    good = torch.tensor(ubar, device=dev)
    ctx.rk_step(good, cfl=0.3)
    torch.cuda.synchronize()
    assert bool(torch.all(torch.isfinite(good)))
    # a NaN state inside rk_step: reported by the synchronising dt read
    ub = torch.tensor(bad, device=dev)
    with pytest.raises(WlsenoError) as ei:
        ctx.rk_step(ub, dt=1e-4, want_dt=True)
    assert ei.value.status == NUMERIC
    ctx.close()
