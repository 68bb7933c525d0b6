"""The Python binding refuses arrays shorter than the built context needs
before it passes their pointers to the library (which cannot see their
length): per-cell arrays [n_comp][n_cells], coefficients [n_comp][n_cells][m],
facet values [n_comp][n_cells][dim+1][quad_per_facet], per-mesh steps
[n_meshes].  Runs without a GPU: the library is replaced by a stub that
accepts every call."""
import numpy as np
import pytest

from paper_1602_02694_gb300 import wlseno as W


class StubLib:
    def __getattr__(self, name):
        return lambda *args: 0


def context(n_comp, n_cells, m, dim, nq, n_meshes=1):
    ctx = W.Context.__new__(W.Context)
    ctx.lib = StubLib()
    ctx.h = None  # close() and __del__ then do nothing
    ctx._info = {"n_comp": n_comp, "n_cells": n_cells, "m": m, "dim": dim, "quad_per_facet": nq,
                 "n_meshes": n_meshes}
    return ctx


@pytest.mark.parametrize("C,N,m,dim,nq", [(1, 10, 6, 2, 2), (4, 7, 6, 2, 2), (3, 9, 3, 1, 1), (5, 4, 10, 3, 3)])
def test_exact_sizes_pass_and_short_arrays_are_refused(C, N, m, dim, nq):
    ctx = context(C, N, m, dim, nq, n_meshes=2)
    u = np.zeros(C * N)
    coef = np.zeros(C * N * m)
    fv = np.zeros(C * N * (dim + 1) * nq)
    ctx.reconstruct(u, coef, fv)
    ctx.reconstruct(u, None, fv)
    ctx.flux_residual(u, np.zeros(C * N))
    ctx.flux_residual_static(u, np.zeros(C * N))
    ctx.rk_step(u, cfl=0.3)
    ctx.step_adjoint(u, 1e-3, np.zeros(C * N), np.zeros(C * N))
    ctx.set_mesh_dt([1e-3, 2e-3])
    short = np.zeros(C * N - 1)
    calls = [lambda: ctx.reconstruct(short),
             lambda: ctx.reconstruct(u, coef[:-1]),
             lambda: ctx.reconstruct(u, None, fv[:-1]),
             lambda: ctx.flux_residual(u, short),
             lambda: ctx.flux_residual_static(short, np.zeros(C * N)),
             lambda: ctx.rk_step(short, cfl=0.3),
             lambda: ctx.autotune(short),
             lambda: ctx.step_adjoint(u, 1e-3, short, np.zeros(C * N)),
             lambda: ctx.step_adjoint(u, 1e-3, np.zeros(C * N), short),
             lambda: ctx.set_mesh_dt([1e-3])]
    for call in calls:
        with pytest.raises(ValueError):
            call()


def test_longer_arrays_and_unbuilt_contexts_are_left_to_the_library():
    ctx = context(1, 10, 6, 2, 2)
    ctx.flux_residual(np.zeros(12), np.zeros(11))
    ctx._info = None
    ctx.flux_residual(np.zeros(1), np.zeros(1))  # the library reports the missing build
    with pytest.raises(TypeError):
        ctx.flux_residual([0.0] * 10, np.zeros(10))


def test_torch_tensors_are_measured_by_numel():
    torch = pytest.importorskip("torch")
    ctx = context(4, 7, 6, 2, 2)
    u = torch.zeros(28, dtype=torch.float64)
    ctx.flux_residual(u, torch.zeros(28, dtype=torch.float64))
    with pytest.raises(ValueError):
        ctx.flux_residual(u, torch.zeros(27, dtype=torch.float64))
    with pytest.raises(ValueError):
        ctx.reconstruct(u, torch.zeros(4 * 7 * 6 - 1, dtype=torch.float64))
