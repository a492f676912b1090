"""fire_step_noalloc, the entry point for callers that cannot allocate device
memory (graph capture, pooled or framework-owned memory, allocator-free time
loops), called through the C ABI: on the same state and inputs it must give
what fire_step gives, on two calls in a row.  The buffers here are allocated
by the test; the entry point itself allocates nothing."""
import numpy as np
import pytest

from paper_1102_1343_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_step_matches_fire_step(prec):
    import torch

    from paper_1102_1343_gb300 import build
    build.build()
    import paper_1102_1343_gb300 as pkg

    torch.cuda.set_device(0)
    w = synth.random_landscape(14, 11, seed=31, ignition="center", steps=12)
    m = pkg.FireModel.from_workload(w, precision=prec)
    u, v = m.wind(w.u, w.v)
    for _ in range(8):  # a fire that burns
        m.step(u, v, w.dt)
    psi, tign, frac, t = m.state()
    dt_ = m.dtype
    dev = m.device
    fuel = torch.as_tensor(w.fuel).to(dev).contiguous()
    zx = torch.as_tensor(w.dzdx).to(dev, dt_).contiguous()
    zy = torch.as_tensor(w.dzdy).to(dev, dt_).contiguous()
    grid = pkg.make_grid(w.nxa, w.nya, w.srx, w.sry, w.dx_atm, w.dy_atm,
                         pkg.FIRE_FP64 if prec == "fp64" else pkg.FIRE_FP32, w.band, w.eps)
    psi_b = torch.empty_like(psi)
    frac_b = torch.empty_like(frac)
    hs = torch.zeros((w.nya, w.nxa), dtype=torch.float64, device=dev)
    hl = torch.zeros_like(hs)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    tol = 1e-10 if prec == "fp64" else 1e-6
    for call in range(2):
        pkg.fire_step_noalloc(grid, w.classes, psi, psi_b, frac, frac_b, tign, fuel, None, zx, zy,
                              u, v, t, w.dt, hs, hl, status)
        ref_hs, ref_hl = m.step(u, v, w.dt)
        p_ref, t_ref, f_ref, t_next = m.state()
        torch.cuda.synchronize()
        scale = max(1.0, float(p_ref.abs().max()))
        assert float((psi_b - p_ref).abs().max()) <= tol * scale
        assert float((frac_b - f_ref).abs().max()) <= tol
        fin = torch.isfinite(t_ref)
        assert torch.equal(fin, torch.isfinite(tign))
        assert float((tign[fin] - t_ref[fin]).abs().max()) <= tol * max(1.0, t_next)
        hmax = max(1.0, float(ref_hs.abs().max()))
        assert float((hs - ref_hs).abs().max()) <= tol * hmax
        assert float((hl - ref_hl).abs().max()) <= tol * max(1.0, float(ref_hl.abs().max()))
        assert int(status.item()) == 0 and m.status() == pkg.FIRE_OK
        psi, psi_b = psi_b, psi
        frac, frac_b = frac_b, frac
        t = t_next
    m.close()


def test_noalloc_rejects_too_many_classes():
    from paper_1102_1343_gb300 import build
    build.build()
    import paper_1102_1343_gb300 as pkg
    grid = pkg.make_grid(4, 4, 10, 10, 60.0, 60.0)
    classes = [synth.nominal_class()] * (pkg.FIRE_MAX_CLASSES + 1)
    with pytest.raises(pkg.FireError) as e:
        pkg.fire_step_noalloc(grid, classes, 1, 2, 3, 4, 5, 6, None, 7, 8, 9, 10, 0.0, 0.5)
    assert e.value.code == pkg.FIRE_ERR_ARG
