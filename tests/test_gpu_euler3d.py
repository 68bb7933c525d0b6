"""Componentwise 3-D Euler (n_comp = 5) through the C ABI against the oracle:
a periodic tetrahedral mesh with a dense high-pressure ball in a light
stream (a 3-D Riemann-type state with smooth velocities), residual and two
CFL-0.3 steps in FP64 within 1e-10, FP32-bulk within relative L1 1e-5, and
the same cells falling back to their averages."""
import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL64 = 1e-10
GAMMA = 1.4


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch.device("cuda:0")


def primitive(P):
    inside = (np.sum((P - 0.5) ** 2, axis=1) < 0.3 ** 2).astype(float)
    rho = 0.125 + 0.875 * inside
    p = 0.1 + 0.9 * inside
    u = 0.3 * np.sin(2 * np.pi * P[:, 1])
    v = 0.2 * np.cos(2 * np.pi * P[:, 2])
    w = 0.1 * np.sin(2 * np.pi * P[:, 0])
    return rho, u, v, w, p


def conserved(k):
    def f(P):
        rho, u, v, w, p = primitive(P)
        return [rho, rho * u, rho * v, rho * w, p / (GAMMA - 1.0) + 0.5 * rho * (u * u + v * v + w * w)][k]
    return f


def test_3d_euler_parity_with_the_oracle(dev):
    from paper_1602_02694_gb300.wlseno import Context

    mesh = synth.tet_mesh(3, seed=15)
    N = mesh.n_cells
    ubar = np.stack([synth.cell_averages(mesh, conserved(k), k=4) for k in range(5)])
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=2.0 / 3.0, pde=O.EULER, min_rows=15)
    ref_L = O.residual(prob, ubar)
    ok = O.euler_positive(prob, ubar, O.euler_coeffs(prob, ubar))
    ref2, _ = O.rk3_run(prob, ubar, 2, cfl=0.3)
    out = {}
    for precision in ("fp64", "fp32_bulk"):
        ctx = Context(0, pde="euler", n_comp=5, gamma=GAMMA, precision=precision)
        ctx.build_stencils(mesh, order_p=3, ring=2.0 / 3.0, min_rows=15)
        ptr, cols = ctx.stencils()
        assert [list(cols[ptr[i]:ptr[i + 1]]) for i in range(N)] == [list(s) for s in prob.stencils]
        ctx.precompute_moments()
        u = torch.tensor(ubar.ravel(), device=dev)
        L = torch.empty_like(u)
        ctx.flux_residual(u, L)
        fallbacks = ctx.diagnostics()["positivity_fallbacks"]
        ctx.rk_step(u, cfl=0.3, n_steps=2)
        out[precision] = (L.cpu().numpy().reshape(5, N), u.cpu().numpy().reshape(5, N), fallbacks)
        ctx.close()
    L64, u64, fb = out["fp64"]
    assert fb == int(np.sum(~ok))
    assert np.max(np.abs(L64 - ref_L)) <= TOL64 * max(1.0, float(np.max(np.abs(ref_L))))
    assert np.max(np.abs(u64 - ref2)) <= TOL64
    u32 = out["fp32_bulk"][1]
    assert np.sum(np.abs(u32 - ref2)) / np.sum(np.abs(ref2)) <= 1e-5
