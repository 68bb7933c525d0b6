"""Pins of the oracle's reverse mode (residual_vjp, rk3_step_vjp) against
what the mathematics fixes: for every direction v, <Lbar, J v> equals the
central difference (L(u + h v) - L(u - h v)) / 2h of the oracle's own
residual (h = 1e-6; the truncation and rounding of the difference stay
below 1e-7 of the value here), for linear advection and Burgers, periodic
and transmissive 2-D meshes, a 1-D line and a 3-D tetrahedral mesh, and the
same for one TVD-RK3 step.  Burgers data with jumps put the per-facet LF
alpha's maximiser and the centre weight's minimising facet neighbour on
every kind of cell.  Mistakes planted in the reverse mode (the weights held
fixed, the alpha term dropped, the centre weight's minimiser ignored, the
transmissive trace not folded back) each fail these checks."""
import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth

H = 1e-6
TOL = 1e-7


def _cases():
    tri = synth.tri_mesh(6, jitter=0.2, seed=21)
    tri_open = synth.tri_mesh(6, jitter=0.2, seed=22, periodic=False)
    line = synth.periodic_line_mesh(24, jitter=0.2, seed=2)
    tet = synth.tet_mesh(3, jitter=0.15, seed=1)
    out = []
    for mesh, kw, name in ((tri, {"p": 3, "ring": 1.0}, "tri"),
                           (tri_open, {"p": 3, "ring": 1.0, "min_rows": 9}, "tri_open"),
                           (line, {"p": 3, "ring": 2.0}, "line"),
                           (tet, {"p": 3, "ring": 2.0 / 3.0, "radius_cut": 0.95}, "tet")):
        for pde in (O.ADVECTION, O.BURGERS):
            out.append((mesh, kw, pde, f"{name}-{'burgers' if pde == O.BURGERS else 'advection'}"))
    return out


def _data(mesh, seed):
    c = mesh.cell_coords.mean(axis=1)
    rng = np.random.default_rng(seed)
    smooth = 0.5 + np.sin(2 * np.pi * c[:, 0]) * np.cos(2 * np.pi * c[:, -1])
    return smooth + 0.3 * (c[:, 0] > 0.5) + 0.05 * rng.normal(size=len(c))


@pytest.mark.parametrize("mesh,kw,pde,name", _cases(), ids=[c[3] for c in _cases()])
def test_residual_vjp_matches_central_differences(mesh, kw, pde, name):
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, pde=pde, velocity=(1.0, 0.5, 0.25), **kw)
    u = _data(mesh, 3)
    rng = np.random.default_rng(4)
    for _ in range(2):
        Lbar = rng.normal(size=prob.N)
        v = rng.normal(size=prob.N)
        got = float(O.residual_vjp(prob, u, Lbar) @ v)
        fd = float(Lbar @ (O.residual(prob, u + H * v) - O.residual(prob, u - H * v)) / (2 * H))
        assert abs(got - fd) <= TOL * max(1.0, abs(fd)), (name, got, fd)


@pytest.mark.parametrize("pde", [O.ADVECTION, O.BURGERS])
def test_rk3_step_vjp_matches_central_differences(pde):
    mesh = synth.tri_mesh(6, jitter=0.2, seed=21)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0, pde=pde, velocity=(1.0, 1.0, 0.0))
    u = _data(mesh, 5)
    dt = 0.3 * float(np.min(prob.geo.inradius)) / 2.5
    rng = np.random.default_rng(6)
    g = rng.normal(size=prob.N)
    v = rng.normal(size=prob.N)
    step = lambda x: O.rk3_step(lambda y: O.residual(prob, y), x, dt)
    got = float(O.rk3_step_vjp(prob, u, dt, g) @ v)
    fd = float(g @ (step(u + H * v) - step(u - H * v)) / (2 * H))
    assert abs(got - fd) <= TOL * max(1.0, abs(fd)), (got, fd)


def test_reverse_mode_refuses_truncated_cells():
    mesh = synth.tri_mesh(6, jitter=0.2, seed=21)
    prob = O.Problem(mesh.vertices, mesh.cells, mesh.period, p=3, ring=1.0, pde=O.BURGERS, rank_tol=0.5)
    with pytest.raises(ValueError):
        O.residual_vjp(prob, _data(mesh, 3), np.ones(prob.N))
