"""The FP32-bulk reconstruction with its moment rows formed on the fly
(moments_mode = 1: the offset of each stencil cell and its own central
moments, binomially shifted) against the oracle and against the stored-row
kernel: without refinement both carry the FP32 rounding of the same problem,
with every cell refined both reach the FP64 solution, and three RK steps stay
within relative L1 1e-5 of the oracle."""
import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch.device("cuda:0")


def Context(**kw):
    from paper_1602_02694_gb300.wlseno import Context as C
    return C(0, **kw)


# name: (mesh, p, ring, min_rows)
CASES = {
    "tri9_p3_ring1": (lambda: synth.tri_mesh(9, seed=11), 3, 1.0, 9),
    "tri10_p4_ring2": (lambda: synth.tri_mesh(10, seed=13), 4, 2.0, 15),
    "tri7_p3_open": (lambda: synth.tri_mesh(7, periodic=False, seed=12), 3, 1.0, 9),
    "tet4_p3": (lambda: synth.tet_mesh(4, seed=15), 3, 2.0 / 3.0, 15),
    "line48_p5": (lambda: synth.periodic_line_mesh(48, jitter=0.2, seed=7), 5, 2.0, 5),
}


def field(mesh):
    if mesh.dim == 1:
        return synth.cell_averages(mesh, lambda P: 0.5 + np.sin(2 * np.pi * P[:, 0]) + (P[:, 0] > 0.6), k=6)
    if mesh.dim == 2:
        return synth.cell_averages(mesh, lambda P: np.sin(2 * np.pi * P[:, 0]) * np.cos(2 * np.pi * P[:, 1])
                                   + (P[:, 0] + 0.3 * P[:, 1] > 0.55))
    return synth.cell_averages(mesh, lambda P: np.sin(2 * np.pi * (P[:, 0] + P[:, 2])) + (P[:, 1] > 0.5))


_cache = {}


def case(name):
    if name not in _cache:
        make, p, ring, min_rows = CASES[name]
        mesh = make()
        prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, pde=O.BURGERS,
                         min_rows=min_rows)
        ubar = field(mesh)
        ref = np.array([prob.reconstruct_cell(ubar, i)[0] for i in range(prob.N)])
        _cache[name] = (mesh, prob, ubar, ref)
    return _cache[name]


def coeffs(dev, mesh, prob, ubar, mode, kflag):
    ctx = Context(pde="burgers", precision="fp32_bulk", kappa_flag=kflag)
    ctx.build_stencils(mesh, order_p=prob.p, ring=prob.ring, min_rows=prob.min_rows, moments_mode=mode)
    assert ctx.info()["moments_mode"] == mode
    ctx.precompute_moments()
    c = torch.empty(prob.N * prob.m, dtype=torch.float64, device=dev)
    ctx.reconstruct(torch.tensor(ubar, device=dev), c)
    ctx.close()
    return c.cpu().numpy().reshape(prob.N, prob.m)


@pytest.mark.parametrize("name", list(CASES))
def test_on_the_fly_rows_match_stored_rows(dev, name):
    mesh, prob, ubar, ref = case(name)
    scale = max(1.0, float(np.max(np.abs(ref))))
    # no refinement: both are FP32 solves of the same problem (rows rounded
    # differently), each within the FP32 reach of the FP64 solution
    err = {mode: float(np.max(np.abs(coeffs(dev, mesh, prob, ubar, mode, 1e30) - ref))) / scale
           for mode in (0, 1)}
    assert err[0] <= 1e-2 and err[1] <= 2.0 * err[0] + 1e-6, err
    # every cell refined with the FP64 residual (preconditioned by the FP32
    # factor of each mode's rows): one sweep leaves about (kappa eps)^2, where
    # eps is a few FP32 ulps for the shifted rows (their binomial sums round
    # a few times) against half an ulp for the stored ones
    fine = {mode: float(np.max(np.abs(coeffs(dev, mesh, prob, ubar, mode, 1e-30) - ref))) / scale
            for mode in (0, 1)}
    assert fine[0] <= 1e-5 and fine[1] <= max(10.0 * fine[0], 1e-6), fine


@pytest.mark.parametrize("name", ["tri10_p4_ring2", "tet4_p3", "line48_p5"])
def test_on_the_fly_rk_steps_match_the_oracle(dev, name):
    mesh, prob, ubar, _ = case(name)
    ref3, _ = O.rk3_run(prob, ubar, 3, cfl=0.3)
    ctx = Context(pde="burgers", precision="fp32_bulk")
    ctx.build_stencils(mesh, order_p=prob.p, ring=prob.ring, min_rows=prob.min_rows, moments_mode=1)
    ctx.precompute_moments()
    u = torch.tensor(ubar, device=dev)
    ctx.rk_step(u, cfl=0.3, n_steps=3)
    got = u.cpu().numpy()
    assert np.sum(np.abs(got - ref3)) / np.sum(np.abs(ref3)) <= 1e-5
    ctx.close()


def test_autotune_tries_both_moments_modes(dev):
    mesh, prob, ubar, _ = case("tri10_p4_ring2")
    ctx = Context(pde="burgers", precision="fp32_bulk")
    ctx.build_stencils(mesh, order_p=prob.p, ring=prob.ring, min_rows=prob.min_rows)
    ctx.precompute_moments()
    u = torch.tensor(ubar, device=dev)
    ctx.autotune(u, reps=2)
    info = ctx.info()
    assert info["moments_mode"] in (0, 1)
    if info["moments_mode"] == 1:
        assert (info["lanes_per_cell"], info["rows_per_lane"]) == (1, 0)
    v = u.clone()
    ctx.rk_step(v, cfl=0.3, n_steps=2)  # the captured step uses the chosen variant
    assert bool(torch.isfinite(v).all())
    ctx.close()


def test_moments_mode_is_rejected_where_it_does_not_apply(dev):
    from paper_1602_02694_gb300.wlseno import WlsenoError
    mesh, prob, _, _ = case("tri9_p3_ring1")
    for precision, shape in (("fp64", (1, 0)), ("fp32_bulk", (8, 2))):
        ctx = Context(pde="burgers", precision=precision)
        with pytest.raises(WlsenoError):
            ctx.build_stencils(mesh, order_p=3, ring=1.0, min_rows=9, lanes_per_cell=shape[0],
                               rows_per_lane=shape[1], moments_mode=1)
        ctx.close()
