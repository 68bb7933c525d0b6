"""Host-side failure modes on a GPU context, with no GPU fault: calls made in
the wrong order return WLSENO_ERR_STATE, and a context whose device
allocations are capped by WLSENO_DEVICE_BYTES_LIMIT fails its set-up with
WLSENO_ERR_OOM and a message, can be destroyed, and leaves the next context
(without the cap) working."""
import numpy as np
import pytest

from paper_1602_02694_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    return torch.device("cuda:0")


def test_calls_out_of_order_return_state(dev):
    from paper_1602_02694_gb300.wlseno import Context, WlsenoError
    mesh = synth.tri_mesh(6, seed=1)
    u = torch.tensor(synth.burgers_2d_initial(mesh), device=dev)
    ctx = Context(0, pde="burgers")
    with pytest.raises(WlsenoError) as info:
        ctx.rk_step(u, cfl=0.3, n_steps=1)
    assert info.value.status == -8
    ctx.build_stencils(mesh, order_p=3, ring=1.0)
    with pytest.raises(WlsenoError) as info:
        ctx.flux_residual(u, torch.empty_like(u))
    assert info.value.status == -8
    ctx.precompute_moments()
    r = torch.empty_like(u)
    ctx.flux_residual(u, r)
    assert bool(torch.all(torch.isfinite(r)))
    ctx.close()


def test_device_bytes_limit_gives_oom(dev, monkeypatch):
    from paper_1602_02694_gb300.wlseno import Context, WlsenoError
    mesh = synth.tri_mesh(12, seed=1)
    monkeypatch.setenv("WLSENO_DEVICE_BYTES_LIMIT", "65536")
    ctx = Context(0, pde="burgers")
    with pytest.raises(WlsenoError) as info:
        ctx.build_stencils(mesh, order_p=3, ring=1.0)
        ctx.precompute_moments()
    assert info.value.status == -5
    assert "WLSENO_DEVICE_BYTES_LIMIT" in str(info.value)
    ctx.close()
    monkeypatch.delenv("WLSENO_DEVICE_BYTES_LIMIT")
    ctx = Context(0, pde="burgers")
    ctx.build_stencils(mesh, order_p=3, ring=1.0)
    ctx.precompute_moments()
    u = torch.tensor(synth.burgers_2d_initial(mesh), device=dev)
    r = torch.empty_like(u)
    ctx.flux_residual(u, r)
    assert bool(torch.all(torch.isfinite(r)))
    ctx.close()
