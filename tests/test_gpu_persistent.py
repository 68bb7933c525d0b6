"""The persistent step (one cooperative kernel per TVD-RK3 step whose
resident blocks walk all cells of all meshes through every phase, with
bounded grid barriers), through the C ABI on the GPU:

* the same bits as the kernel-per-phase step, FP64 and FP32-bulk (moment
  rows stored or formed on the fly), CFL, fixed and per-mesh time steps,
  one mesh and a batch of meshes of uneven sizes;
* the oracle's 100 steps of the 2-D advection workload;
* a barrier poll limit too small to wait for the other blocks: the step
  gives up in every block (no hang, no trap), the call that synchronises
  or the next call returns WLSENO_ERR_TIMEOUT, and with the default limit
  the context gives the right bits again."""
import math

import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TIMEOUT = -7


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch.device("cuda:0")


def Context(**kw):
    from paper_1602_02694_gb300.wlseno import Context as C
    return C(0, **kw)


def run(meshes, u0, pde, precision, persistent, steps, p=3, ring=1.0, moments_mode=0, **step):
    ctx = Context(pde=pde, precision=precision, velocity=(1.0, 1.0, 0.0))
    ctx.build_stencils(meshes, order_p=p, ring=ring, moments_mode=moments_mode, persistent=persistent)
    ctx.precompute_moments()
    if step.get("dt", 0.0) < 0.0:
        inr = ctx.geometry()["inradius"]
        dts, off = [], 0
        for m in (meshes if isinstance(meshes, list) else [meshes]):
            dts.append(0.3 * float(np.min(inr[off:off + m.n_cells])) / (math.sqrt(2.0) * float(np.max(np.abs(u0)))))
            off += m.n_cells
        ctx.set_mesh_dt(dts)
    u = torch.tensor(u0, device="cuda")
    ctx.rk_step(u, n_steps=steps, **step)
    torch.cuda.synchronize()
    d = ctx.diagnostics()
    ctx.close()
    return u, d


CASES = [
    ("advection", "fp64", 3, 1.0, 0, {"cfl": 0.4}),
    ("burgers", "fp64", 4, 2.0, 0, {"cfl": 0.3}),
    ("burgers", "fp32_bulk", 4, 2.0, 0, {"cfl": 0.3}),
    ("burgers", "fp32_bulk", 4, 2.0, 1, {"cfl": 0.3}),
    ("burgers", "fp32_bulk", 3, 1.0, 1, {"dt": 2e-4}),
    ("advection", "fp32_bulk", 3, 1.0, 0, {"cfl": 0.4}),
]


@pytest.mark.parametrize("pde,precision,p,ring,mode,step", CASES)
def test_persistent_equals_phase_kernels(dev, pde, precision, p, ring, mode, step):
    mesh = synth.tri_mesh(24, jitter=0.2, seed=1)
    u0 = synth.burgers_2d_initial(mesh) if pde == "burgers" else synth.advection_2d_initial(mesh)
    a, da = run(mesh, u0, pde, precision, 0, 5, p, ring, mode, **step)
    b, db = run(mesh, u0, pde, precision, 1, 5, p, ring, mode, **step)
    assert torch.equal(a, b)
    assert da["launches_by_kind"]["step"] == 0 and db["launches_by_kind"]["step"] == 5
    assert db["launches_by_kind"]["reconstruct"] == 0 and db["nonfinite"] == 0


@pytest.mark.parametrize("precision", ["fp64", "fp32_bulk"])
def test_persistent_batch_of_uneven_meshes(dev, precision):
    meshes = [synth.tri_mesh(n, jitter=0.2, seed=40 + n) for n in (8, 20, 13, 32)]
    u0 = np.concatenate([synth.smooth_random_initial(m, seed=50 + k) for k, m in enumerate(meshes)])
    a, _ = run(meshes, u0, "burgers", precision, 0, 4, dt=-1.0)
    b, _ = run(meshes, u0, "burgers", precision, 1, 4, dt=-1.0)
    assert torch.equal(a, b)
    a, _ = run(meshes, u0, "burgers", precision, 0, 4, cfl=0.3)
    b, _ = run(meshes, u0, "burgers", precision, 1, 4, cfl=0.3)
    assert torch.equal(a, b)


def test_persistent_matches_oracle_advection_workload(dev):
    mesh = synth.tri_mesh(32, jitter=0.2, seed=1)
    ubar = synth.advection_2d_initial(mesh)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0, velocity=(1.0, 1.0, 0.0))
    ref, _ = O.rk3_run(prob, ubar, 100, cfl=0.4)
    u, d = run(mesh, ubar, "advection", "fp64", 1, 100, cfl=0.4)
    assert float(np.max(np.abs(u.cpu().numpy() - ref))) <= 1e-10


def test_barrier_wait_limit_gives_timeout_and_recovers(dev):
    from paper_1602_02694_gb300.wlseno import WlsenoError
    mesh = synth.tri_mesh(128, jitter=0.2, seed=1)  # 32,768 cells: 256 blocks
    u0 = synth.burgers_2d_initial(mesh)
    want, _ = run(mesh, u0, "burgers", "fp32_bulk", 0, 2, cfl=0.3)
    ctx = Context(pde="burgers", precision="fp32_bulk")
    ctx.build_stencils(mesh, order_p=3, ring=1.0, persistent=1)
    ctx.precompute_moments()
    ctx.set_wait_limit(1)
    u = torch.tensor(u0, device="cuda")
    with pytest.raises(WlsenoError) as ei:  # the dt read synchronises
        ctx.rk_step(u, cfl=0.3, n_steps=1, want_dt=True)
    assert ei.value.status == TIMEOUT
    u = torch.tensor(u0, device="cuda")
    ctx.rk_step(u, cfl=0.3, n_steps=1)  # asynchronous: reported by the next call
    torch.cuda.synchronize()
    with pytest.raises(WlsenoError) as ei:
        ctx.rk_step(u, cfl=0.3, n_steps=1)
    assert ei.value.status == TIMEOUT
    ctx.set_wait_limit(0)
    u = torch.tensor(u0, device="cuda")
    ctx.rk_step(u, cfl=0.3, n_steps=2)
    torch.cuda.synchronize()
    assert torch.equal(u, want)
    ctx.close()
