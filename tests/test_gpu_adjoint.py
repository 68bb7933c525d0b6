"""The hand-written adjoint of the TVD-RK3 step (wlseno_step_adjoint and the
torch.autograd rollout): element by element against the oracle's own reverse
mode (one step, and a batched three-step rollout), the full gradient against central differences of the FP64 oracle's
forward step, random directions against central differences of the GPU
forward (step 1e-6, FP64), and stage checkpointing against storing every
state."""
import math

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


@pytest.mark.parametrize("pde", ["burgers", "advection"])
def test_step_adjoint_matches_oracle_finite_differences(dev, pde):
    """Full gradient of J = sum w_i ubar_i(t + dt)^2 after one step: GPU
    adjoint vs central differences (h = 1e-6) of the oracle's RK3 step."""
    mesh = synth.tri_mesh(6, seed=21)
    if pde == "burgers":
        ubar = synth.burgers_2d_initial(mesh)
    else:
        ubar = synth.cell_averages(mesh, lambda P: np.sin(2 * np.pi * P[:, 0]) + 0.5 * np.cos(2 * np.pi * P[:, 1]))
    w = synth.loss_weights(mesh.n_cells, 3)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0,
                     pde=O.BURGERS if pde == "burgers" else O.ADVECTION, velocity=(1.0, 1.0, 0.0))
    dt = 0.3 * float(np.min(prob.geo.inradius)) / 2.5

    def J_oracle(u):
        u1 = O.rk3_step(lambda x: O.residual(prob, x), u, dt)
        return float(np.sum(w * u1 * u1))

    h = 1e-6
    g_fd = np.zeros(prob.N)
    for i in range(prob.N):
        e = np.zeros(prob.N)
        e[i] = h
        g_fd[i] = (J_oracle(ubar + e) - J_oracle(ubar - e)) / (2 * h)

    ctx = Context(pde=pde, velocity=(1.0, 1.0, 0.0))
    ctx.build_stencils(mesh, order_p=3, ring=1.0)
    ctx.precompute_moments()
    u0 = torch.tensor(ubar, device=dev)
    u1 = u0.clone()
    ctx.rk_step(u1, dt=dt, n_steps=1)
    gnext = 2.0 * torch.tensor(w, device=dev) * u1
    g = torch.empty_like(u0)
    ctx.step_adjoint(u0, dt, gnext, g)
    err = float(np.max(np.abs(g.cpu().numpy() - g_fd)))
    assert err <= 1e-4 * float(np.max(np.abs(g_fd))), err
    assert err <= 1e-7 * max(1.0, float(np.max(np.abs(g_fd)))), err
    ctx.close()


def batch_problem(dev):
    """Three periodic Burgers problems of different sizes in one context, each
    stepping at its own dt (CFL 0.3 from its initial data)."""
    meshes = [synth.tri_mesh(n, seed=30 + n) for n in (8, 12, 16)]
    u0 = np.concatenate([synth.smooth_random_initial(m, seed=40 + k) for k, m in enumerate(meshes)])
    ctx = Context(pde="burgers")
    ctx.build_stencils(meshes, order_p=3, ring=1.0)
    ctx.precompute_moments()
    inr = ctx.geometry()["inradius"]
    dts, off = [], 0
    for m in meshes:
        sl = slice(off, off + m.n_cells)
        dts.append(0.3 * float(np.min(inr[sl])) / (math.sqrt(2.0) * float(np.max(np.abs(u0[sl])))))
        off += m.n_cells
    ctx.set_mesh_dt(dts)
    return ctx, torch.tensor(u0, device=dev)


def test_rollout_gradient_random_directions(dev):
    """Batched problems, 3 steps with checkpoints every 2 steps: <g, v> against
    central differences of the GPU forward on 16 random unit directions."""
    from paper_1602_02694_gb300.autograd import rollout
    ctx, u0 = batch_problem(dev)
    N = u0.numel()
    w = torch.tensor(synth.loss_weights(N, 3), device=dev)
    steps = 3

    def J(u):
        v = u.clone()
        ctx.rk_step(v, dt=-1.0, n_steps=steps)
        return float(torch.sum(w * v * v))

    x = u0.clone().requires_grad_(True)
    uT = rollout(ctx, x, steps, -1.0, checkpoint_every=2)
    torch.sum(w * uT * uT).backward()
    g = x.grad.detach()
    gnorm = float(torch.linalg.norm(g))
    dirs = synth.random_unit_directions(N, 16, 4)
    h = 1e-6
    for d in dirs:
        v = torch.tensor(d, device=dev)
        fd = (J(u0 + h * v) - J(u0 - h * v)) / (2 * h)
        ad = float(torch.dot(g, v))
        assert abs(fd - ad) <= 1e-4 * gnorm, (fd, ad, gnorm)
    ctx.close()


def test_checkpoint_spacing_does_not_change_the_gradient(dev):
    from paper_1602_02694_gb300.autograd import rollout
    ctx, u0 = batch_problem(dev)
    w = torch.tensor(synth.loss_weights(u0.numel(), 5), device=dev)
    grads = []
    for every in (1, 2, 5):
        x = u0.clone().requires_grad_(True)
        uT = rollout(ctx, x, 5, -1.0, checkpoint_every=every)
        torch.sum(w * uT * uT).backward()
        grads.append(x.grad.detach().clone())
    for gk in grads[1:]:
        assert torch.equal(gk, grads[0])
    ctx.close()


def test_adjoint_refuses_fp32_bulk_contexts(dev):
    """The adjoint is the derivative of the FP64 step: an FP32-bulk context
    gets INVALID_ARG with a message instead of a VJP of another step."""
    from paper_1602_02694_gb300.wlseno import WlsenoError
    mesh = synth.tri_mesh(6, seed=21)
    u = torch.tensor(synth.burgers_2d_initial(mesh), device=dev)
    ctx = Context(pde="burgers", precision="fp32_bulk")
    ctx.build_stencils(mesh, order_p=3, ring=1.0)
    ctx.precompute_moments()
    with pytest.raises(WlsenoError) as ei:
        ctx.step_adjoint(u, 1e-3, torch.ones_like(u), torch.empty_like(u))
    assert ei.value.status == -1 and "FP64" in str(ei.value)
    ctx.close()


@pytest.mark.parametrize("pde", ["burgers", "advection"])
def test_step_adjoint_matches_oracle_reverse_mode(dev, pde):
    """The GPU adjoint of one fixed-dt TVD-RK3 step against the oracle's own
    reverse mode (rk3_step_vjp, pinned against central differences of its
    forward step in tests/test_oracle_adjoint.py), element by element, on
    periodic and transmissive triangle meshes and a periodic tetrahedral one:
    FP64 to 1e-10 of the gradient's largest entry."""
    cases = [(synth.tri_mesh(6, seed=21), {"ring": 1.0}),
             (synth.tri_mesh(8, jitter=0.2, seed=23, periodic=False), {"ring": 1.0, "min_rows": 9}),
             (synth.tet_mesh(3, jitter=0.15, seed=1), {"ring": 2.0 / 3.0, "radius_cut": 0.95})]
    for mesh, kw in cases:
        c = mesh.cell_coords.mean(axis=1)
        if pde == "burgers":
            ubar = 0.5 + np.sin(2 * np.pi * (c[:, 0] + c[:, 1]))
        else:
            ubar = np.sin(2 * np.pi * c[:, 0]) + 0.5 * np.cos(2 * np.pi * c[:, 1])
        prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3,
                         pde=O.BURGERS if pde == "burgers" else O.ADVECTION, velocity=(1.0, 1.0, 0.0), **kw)
        dt = 0.3 * float(np.min(prob.geo.inradius)) / 2.5
        w = synth.loss_weights(mesh.n_cells, 3)
        u1 = O.rk3_step(lambda x: O.residual(prob, x), ubar, dt)
        gnext = 2.0 * w * u1
        ref = O.rk3_step_vjp(prob, ubar, dt, gnext)
        ctx = Context(pde=pde, velocity=(1.0, 1.0, 0.0))
        ctx.build_stencils(mesh, order_p=3, **kw)
        ctx.precompute_moments()
        g = torch.empty(mesh.n_cells, dtype=torch.float64, device=dev)
        ctx.step_adjoint(torch.tensor(ubar, device=dev), dt, torch.tensor(gnext, device=dev), g)
        err = float(np.max(np.abs(g.cpu().numpy() - ref)))
        assert err <= 1e-10 * max(1.0, float(np.max(np.abs(ref)))), (pde, mesh.n_cells, err)
        ctx.close()


def test_batched_rollout_gradient_matches_oracle_reverse_mode(dev):
    """Three periodic Burgers problems of different sizes in one context, each
    at its own dt, 3 steps with a checkpoint every 2: the autograd gradient of
    sum w_i ubar_i(T)^2 against the oracle's reverse mode run problem by
    problem (3 forward steps, then rk3_step_vjp backwards), element by
    element to 1e-10 of the gradient's largest entry."""
    from paper_1602_02694_gb300.autograd import rollout
    ctx, u0 = batch_problem(dev)
    N = u0.numel()
    w = synth.loss_weights(N, 3)
    steps = 3
    x = u0.clone().requires_grad_(True)
    uT = rollout(ctx, x, steps, -1.0, checkpoint_every=2)
    torch.sum(torch.tensor(w, device=dev) * uT * uT).backward()
    g = x.grad.detach().cpu().numpy()
    meshes = [synth.tri_mesh(n, seed=30 + n) for n in (8, 12, 16)]
    inr = ctx.geometry()["inradius"]
    ctx.close()
    ref = np.empty(N)
    u_all = u0.cpu().numpy()
    off = 0
    for m in meshes:
        sl = slice(off, off + m.n_cells)
        dt = 0.3 * float(np.min(inr[sl])) / (math.sqrt(2.0) * float(np.max(np.abs(u_all[sl]))))
        prob = O.Problem(m.vertices, m.cells, m.period, p=3, ring=1.0, pde=O.BURGERS)
        states = [u_all[sl]]
        for _ in range(steps):
            states.append(O.rk3_step(lambda y: O.residual(prob, y), states[-1], dt))
        gb = 2.0 * w[sl] * states[-1]
        for k in range(steps - 1, -1, -1):
            gb = O.rk3_step_vjp(prob, states[k], dt, gb)
        ref[sl] = gb
        off += m.n_cells
    err = float(np.max(np.abs(g - ref)))
    assert err <= 1e-10 * max(1.0, float(np.max(np.abs(ref)))), err
