"""wlseno_flux_residual_static: the residual operator for callers that cannot
allocate device memory when they call it (code running inside a stream
capture, allocation-free real-time loops, hosts whose device memory belongs to
their own pool).  Its facet-value scratch is a fixed array inside the library.

These tests call it through the C ABI as the first residual call on a fresh
context, twice in a row with different data, and check it against the
oracle's residual (FP64: 1e-10; FP32-bulk: relative L1 1e-5) and against
wlseno_flux_residual called afterwards (the same kernels: the same bits),
in 1-D, 2-D and 3-D, FP64 and FP32-bulk (moment rows stored and formed on
the fly) and with balanced stencils; plus its size and pointer checks.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch.device("cuda:0")


def case_data(kind):
    """(mesh, two data sets, oracle problem kwargs, build kwargs)."""
    if kind == "1d":
        mesh = synth.periodic_line_mesh(40, jitter=0.2, seed=2)
        x = mesh.cell_coords.mean(axis=1)[:, 0]
        data = [np.sin(2 * np.pi * x), 0.3 + (x > 0.5)]
        # the seven-cell stencil of Sec. 4.2 (no growth to ceil(1.5 m) rows)
        return mesh, data, {"p": 5, "ring": 3.0}, {"order_p": 5, "ring": 3.0, "min_rows": 7}
    if kind == "3d":
        mesh = synth.tet_mesh(4, jitter=0.15, seed=1)
        c = mesh.cell_coords.mean(axis=1)
        data = [np.sin(2 * np.pi * c[:, 0]) * np.cos(2 * np.pi * c[:, 1]), 1.0 + c[:, 2] ** 2]
        kw = {"p": 3, "ring": 2.0 / 3.0, "radius_cut": 0.95}
        return mesh, data, kw, {"order_p": 3, "ring": 2.0 / 3.0, "radius_cut": 0.95}
    mesh = synth.tri_mesh(12, jitter=0.2, seed=3)
    c = mesh.cell_coords.mean(axis=1)
    data = [synth.burgers_2d_initial(mesh), 0.2 + ((c[:, 0] > 0.3) & (c[:, 0] < 0.6)).astype(float)]
    if kind == "2d_p3":
        return mesh, data, {"p": 3, "ring": 1.0}, {"order_p": 3, "ring": 1.0}
    return mesh, data, {"p": 4, "ring": 2.0}, {"order_p": 4, "ring": 2.0}


CASES = [("fp64", "burgers", "2d_p4", 0, False), ("fp32_bulk", "advection", "2d_p3", 0, False),
         ("fp32_bulk", "burgers", "2d_p4", 1, False), ("fp32_bulk", "burgers", "2d_p3", 0, True),
         ("fp64", "advection", "1d", 0, False), ("fp64", "advection", "3d", 0, False)]


@pytest.mark.parametrize("precision,pde,kind,mode,balanced", CASES)
def test_static_residual_on_a_fresh_context(dev, precision, pde, kind, mode, balanced):
    from paper_1602_02694_gb300.wlseno import Context, WlsenoError

    mesh, data, okw, bkw = case_data(kind)
    vel = (1.0, 0.5, 0.25)
    ctx = Context(0, pde=pde, precision=precision, velocity=vel, balanced=balanced)
    ctx.build_stencils(mesh, moments_mode=mode, **bkw)
    ctx.precompute_moments()
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, pde=O.BURGERS if pde == "burgers" else O.ADVECTION,
                     velocity=vel, balanced=balanced, **okw)
    got = []
    for ubar in data:  # two calls in a row before any other residual call
        u = torch.tensor(ubar, dtype=torch.float64, device=dev)
        r = torch.full_like(u, float("nan"))
        ctx.flux_residual_static(u, r)
        torch.cuda.synchronize()
        got.append(r.cpu().numpy())
    for ubar, g in zip(data, got):
        ref = O.residual(prob, ubar)
        if precision == "fp64":
            assert float(np.max(np.abs(g - ref))) <= TOL * max(1.0, float(np.max(np.abs(ref))))
        else:
            assert float(np.sum(np.abs(g - ref)) / np.sum(np.abs(ref))) <= 1e-5
        u = torch.tensor(ubar, dtype=torch.float64, device=dev)
        r = torch.empty_like(u)
        ctx.flux_residual(u, r)
        assert np.array_equal(r.cpu().numpy(), g)  # the same kernels, the same bits
    with pytest.raises(WlsenoError) as info:
        ctx.flux_residual_static(np.zeros(mesh.n_cells), np.zeros(mesh.n_cells))
    assert info.value.status == -1
    ctx.close()


def test_static_residual_rejects_meshes_beyond_its_scratch(dev):
    from paper_1602_02694_gb300.wlseno import Context, WlsenoError

    mesh = synth.tri_mesh(300, seed=3)  # 180,000 triangles > 174,762
    ctx = Context(0, pde="advection")
    ctx.build_stencils(mesh, order_p=3, ring=1.0)
    ctx.precompute_moments()
    u = torch.zeros(mesh.n_cells, dtype=torch.float64, device=dev)
    r = torch.zeros_like(u)
    with pytest.raises(WlsenoError) as info:
        ctx.flux_residual_static(u, r)
    assert info.value.status == -1 and "fixed scratch" in str(info.value)
    ctx.close()
