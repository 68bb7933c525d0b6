"""wlseno_flux_residual_static: the residual operator for callers that cannot
allocate device memory when they call it (code running inside a stream
capture, allocation-free real-time loops, hosts whose device memory belongs to
their own pool).  Its facet-value scratch is a fixed array inside the library;
these tests check it against wlseno_flux_residual through the C ABI, on two
calls in a row with different data, and its size and pointer checks.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch.device("cuda:0")


def test_static_residual_matches_flux_residual(dev):
    from paper_1602_02694_gb300 import synth
    from paper_1602_02694_gb300.wlseno import Context, WlsenoError

    mesh = synth.tri_mesh(64, seed=3)  # 8,192 cells
    data = [synth.burgers_2d_initial(mesh), synth.advection_2d_initial(mesh)]
    for precision, pde, p, ring, mode in (("fp64", "burgers", 4, 2.0, 0), ("fp32_bulk", "advection", 3, 1.0, 0),
                                          ("fp32_bulk", "burgers", 4, 2.0, 1)):
        ctx = Context(0, pde=pde, precision=precision)
        ctx.build_stencils(mesh, order_p=p, ring=ring, moments_mode=mode)
        ctx.precompute_moments()
        for ubar in data:  # two calls in a row; the second sees other data
            u = torch.tensor(ubar, dtype=torch.float64, device=dev)
            ref = torch.empty_like(u)
            ctx.flux_residual(u, ref)
            got = torch.full_like(u, float("nan"))
            ctx.flux_residual_static(u, got)
            torch.cuda.synchronize()
            scale = max(1.0, float(torch.max(torch.abs(ref))))
            err = float(torch.max(torch.abs(got - ref)))
            assert err <= TOL * scale, (precision, err)
        with pytest.raises(WlsenoError) as info:
            ctx.flux_residual_static(np.zeros(mesh.n_cells), np.zeros(mesh.n_cells))
        assert info.value.status == -1
        ctx.close()


def test_static_residual_rejects_meshes_beyond_its_scratch(dev):
    from paper_1602_02694_gb300 import synth
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
