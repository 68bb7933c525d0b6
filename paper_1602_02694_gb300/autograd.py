"""torch.autograd wrapper of the hand-written adjoint of wlseno_rk_step.

`rollout(ctx, u0, n_steps, dt, checkpoint_every)` advances u0 by n_steps
fixed-dt TVD-RK3 steps through the C ABI and, on backward, returns the
gradient with respect to u0 from wlseno_step_adjoint.  Stage checkpointing:
the forward pass keeps every `checkpoint_every`-th state; the backward pass
recomputes the states of each segment from its checkpoint (the adjoint
itself recomputes the two inner stages of every step) and walks the segment
in reverse, so memory is O(n_steps / k + k) states instead of O(n_steps).
Argument marshalling only: every step and adjoint runs in the library.
"""
from __future__ import annotations

import torch


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(fctx, u0, wctx, dt, n_steps, every):
        u = u0.detach().clone().contiguous()
        ckpts = {0: u.clone()}
        for s in range(n_steps):
            wctx.rk_step(u, dt=dt, n_steps=1)
            if (s + 1) % every == 0 and s + 1 < n_steps:
                ckpts[s + 1] = u.clone()
        fctx.wctx, fctx.dt, fctx.n, fctx.every, fctx.ckpts = wctx, dt, n_steps, every, ckpts
        return u

    @staticmethod
    def backward(fctx, gout):
        wctx, dt, n, every, ckpts = fctx.wctx, fctx.dt, fctx.n, fctx.every, fctx.ckpts
        g = gout.detach().clone().contiguous()
        gnext = torch.empty_like(g)
        starts = sorted(ckpts)
        for a in reversed(starts):
            b = min(a + every, n)
            states = [ckpts[a].clone()]
            for _ in range(a, b - 1):
                nxt = states[-1].clone()
                wctx.rk_step(nxt, dt=dt, n_steps=1)
                states.append(nxt)
            for s in range(b - 1, a - 1, -1):
                gnext.copy_(g)
                wctx.step_adjoint(states[s - a], dt, gnext, g)
        return g, None, None, None, None


def rollout(wctx, u0: torch.Tensor, n_steps: int, dt: float, checkpoint_every: int = 1) -> torch.Tensor:
    """Differentiable n_steps x TVD-RK3 (dt > 0 fixed, or dt < 0 for the
    per-mesh steps set with Context.set_mesh_dt)."""
    if n_steps < 1 or checkpoint_every < 1:
        raise ValueError("n_steps and checkpoint_every must be >= 1")
    if dt == 0:
        raise ValueError("the adjoint needs a fixed dt")
    return _Rollout.apply(u0, wctx, float(dt), int(n_steps), int(checkpoint_every))
