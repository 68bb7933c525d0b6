"""Cell reordering through the C ABI on the GPU: a randomly shuffled copy of
a jittered periodic mesh, renumbered by the library along the Hilbert curve
(opts.reorder = 1, perm_out = new -> old), gives the oracle's residuals and
reconstructions of the shuffled mesh after un-permuting (FP64, 1e-10), and
the same FP32-bulk RK steps to FP32 rounding."""
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


def shuffled(n, seed):
    mesh = synth.tri_mesh(n, jitter=0.2, seed=1)
    u = synth.burgers_2d_initial(mesh)
    order = np.random.default_rng(seed).permutation(mesh.n_cells)
    return synth.Mesh(mesh.vertices, mesh.cells[order], mesh.period, mesh.cell_coords[order], n=0), u[order]


def test_reordered_mesh_matches_oracle(dev):
    mesh, u = shuffled(16, 3)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=4, ring=2.0, pde=O.BURGERS)
    ref = O.residual(prob, u)
    ctx = Context(pde="burgers")
    ctx.build_stencils(mesh, order_p=4, ring=2.0, reorder=1)
    perm = ctx.perm
    assert sorted(perm.tolist()) == list(range(mesh.n_cells)) and not np.array_equal(perm, np.arange(len(perm)))
    ctx.precompute_moments()
    ud = torch.tensor(u[perm], device=dev)
    L = torch.empty_like(ud)
    ctx.flux_residual(ud, L)
    got = L.cpu().numpy()
    scale = max(1.0, float(np.max(np.abs(ref))))
    assert float(np.max(np.abs(got - ref[perm]))) <= 1e-10 * scale
    coef = torch.empty(mesh.n_cells * 10, dtype=torch.float64, device=dev)
    ctx.reconstruct(ud, coef)
    coef = coef.cpu().numpy().reshape(-1, 10)
    for k in range(0, mesh.n_cells, 37):
        d, _ = prob.reconstruct_cell(u, int(perm[k]))
        assert np.max(np.abs(coef[k] - d)) <= 1e-10
    # the library's stencils are the oracle's, renumbered
    ptr, cols = ctx.stencils()
    for k in range(0, mesh.n_cells, 29):
        assert sorted(perm[cols[ptr[k]:ptr[k + 1]]].tolist()) == sorted(prob.stencils[int(perm[k])])
    ctx.close()


def test_reordered_rk_steps_fp32_bulk(dev):
    mesh, u = shuffled(48, 5)
    out = {}
    for reorder in (0, 1):
        ctx = Context(pde="burgers", precision="fp32_bulk")
        ctx.build_stencils(mesh, order_p=4, ring=2.0, reorder=reorder)
        perm = ctx.perm
        ctx.precompute_moments()
        ud = torch.tensor(u[perm], device=dev)
        ctx.rk_step(ud, dt=5e-5, n_steps=3)
        back = np.empty(mesh.n_cells)
        back[perm] = ud.cpu().numpy()
        out[reorder] = back
        ctx.close()
    a, b = out[0], out[1]
    assert np.sum(np.abs(a - b)) / np.sum(np.abs(b)) <= 1e-6
