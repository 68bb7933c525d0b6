"""The linear stability of the scheme itself, on the oracle alone (no GPU):
with the weights of Sec. 3.1.2 frozen at a smooth state (0.5 + sin 2 pi
(x + y), the Burgers workload's data), the WLS-ENO reconstruction is a
linear map and the residual of linear advection a linear operator whose
spectrum decides how a perturbation of that state grows.

* Quadratic reconstruction (p = 3) on the 1-ring: no eigenvalue has a
  positive real part (the largest is the zero of conservation).
* The 1-D scheme of Sec. 4.2 (p = 5 on seven cells) with the same weights:
  stable likewise.
* Cubic reconstruction (p = 4) on the 2-ring with eps = 1e-2: eigenvalues
  with real parts of many c/h -- grid-scale modes that grow without
  oscillating.  With eps = 1e8 (weights near uniform) the largest real part
  drops by more than an order of magnitude.  The frozen weights already
  show it, so the growth is not the weights' dependence on the solution; it
  is why FP32-bulk and FP64 runs of the Burgers workload part after a few
  tens of steps (both amplify their rounding at the same rate)."""
import math

import numpy as np
import pytest

from oracle import wlseno_oracle as O
from paper_1602_02694_gb300 import synth


class FrozenWeights(O.Problem):
    """The oracle's reconstruction with the weights taken from a fixed state."""
    u_frozen = None

    def reconstruct_cell(self, ubar, i):
        S = self.stencils[i]
        face = set(self.face_nbrs[i])
        mask = [j in face for j in S]
        uS = np.asarray([ubar[j] for j in S])
        uF = np.asarray([self.u_frozen[j] for j in S])
        omega = O.wls_eno_weights(uF, mask, self.geo.h[i], self.eps, self.alpha_c)
        return O.scaled_wls_solve(self.A(i), omega, uS, self.rank_tol)[:2]


def spectrum(mesh, u0, p, ring, eps, velocity):
    prob = FrozenWeights(mesh.vertices, mesh.cells, mesh.period, p=p, ring=ring, pde=O.ADVECTION,
                         eps=eps, velocity=velocity)
    prob.u_frozen = u0
    N = len(u0)
    J = np.empty((N, N))
    for k in range(N):  # the operator is linear: its columns are the residuals of unit vectors
        e = np.zeros(N)
        e[k] = 1.0
        J[:, k] = O.residual(prob, e)
    return np.linalg.eigvals(J)


def smooth(mesh, dim):
    if dim == 1:
        return synth.cell_averages(mesh, lambda P: 0.5 + np.sin(2 * np.pi * P[:, 0]), k=6)
    return synth.cell_averages(mesh, lambda P: 0.5 + np.sin(2 * np.pi * (P[:, 0] + P[:, 1])), k=4)


def test_quadratic_1ring_is_stable():
    mesh = synth.tri_mesh(8, jitter=0.2, seed=1)
    lam = spectrum(mesh, smooth(mesh, 2), 3, 1.0, 1e-2, (1.0, 1.0, 0.0))
    assert lam.real.max() <= 1e-8 * np.abs(lam).max()


def test_one_dimensional_scheme_is_stable():
    mesh = synth.periodic_line_mesh(48, jitter=0.2, seed=1)
    lam = spectrum(mesh, smooth(mesh, 1), 5, 3.0, 1e-2, (1.0, 0.0, 0.0))
    assert lam.real.max() <= 1e-8 * np.abs(lam).max()


@pytest.mark.parametrize("eps,low,high", [(1e-2, 5.0, None), (1e8, None, 1.0)])
def test_cubic_2ring_grows_at_the_grid_scale(eps, low, high):
    n = 8
    mesh = synth.tri_mesh(n, jitter=0.2, seed=1)
    lam = spectrum(mesh, smooth(mesh, 2), 4, 2.0, eps, (1.0, 1.0, 0.0))
    rate = lam.real.max() * (1.0 / n) / math.sqrt(2.0)  # in units of c/h
    if low is not None:
        assert rate > low, rate   # observed 14.4
    if high is not None:
        assert rate < high, rate  # observed 0.42
