"""fire_step_noalloc, the entry point for callers that cannot allocate device
memory (pooled or framework-owned memory, allocator-free time loops), called
through the C ABI: on the same state and inputs it must give what fire_step
gives, on two calls in a row.  The buffers here are allocated by the test; the
entry point itself allocates nothing.  Both launch families are covered: a
small mesh (one-cell 2-D tiles) and a mesh large enough for strips (warp
strips in FP32, marching strips in FP64, the defaults of realistic meshes)."""
import numpy as np
import pytest

from paper_1102_1343_gb300 import synth

pytestmark = pytest.mark.gpu

# (atmospheric cells x, y, expected default kernel per precision)
CASES = {"tiles": (14, 11, {"fp64": 0, "fp32": 0}),
         "strips": (200, 16, {"fp64": 1, "fp32": 2})}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_step_matches_fire_step(prec, case):
    import torch

    from paper_1102_1343_gb300 import build
    build.build()
    import paper_1102_1343_gb300 as pkg

    torch.cuda.set_device(0)
    nxa, nya, want = CASES[case]
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    assert pkg.fire_default_kernel(prec, nxa, nya, 10, 10, n_sm)[0] == want[prec]
    w = synth.random_landscape(nxa, nya, seed=31, ignition="center", steps=12)
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
        torch.cuda.synchronize()
        free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
        pkg.fire_step_noalloc(grid, w.classes, psi, psi_b, frac, frac_b, tign, fuel, None, zx, zy,
                              u, v, t, w.dt, hs, hl, status)
        torch.cuda.synchronize()
        if call == 1:  # the first call may load the library's code onto the device
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        ref_hs, ref_hl = m.step(u, v, w.dt)
        p_ref, t_ref, f_ref, t_next = m.state()
        torch.cuda.synchronize()
        scale = max(1.0, float(p_ref.abs().max()))
        assert float((psi_b - p_ref).abs().max()) <= tol * scale
        assert float((frac_b - f_ref).abs().max()) <= tol
        fin = torch.isfinite(t_ref)
        assert torch.equal(fin, torch.isfinite(tign))
        assert float((tign[fin] - t_ref[fin]).abs().max()) <= tol * max(1.0, t_next)
        assert float(frac_b.min()) < 1.0  # the fire burns in the compared state
        hmax = max(1.0, float(ref_hs.abs().max()))
        assert float((hs - ref_hs).abs().max()) <= tol * hmax
        assert float((hl - ref_hl).abs().max()) <= tol * max(1.0, float(ref_hl.abs().max()))
        assert int(status.item()) == 0 and m.status() == pkg.FIRE_OK
        psi, psi_b = psi_b, psi
        frac, frac_b = frac_b, frac
        t = t_next
    # without a status buffer the step is the same (faults are then not seen)
    psi_c = torch.empty_like(psi)
    frac_c = torch.empty_like(frac)
    tign_c = tign.clone()
    pkg.fire_step_noalloc(grid, w.classes, psi, psi_c, frac, frac_c, tign_c, fuel, None, zx, zy,
                          u, v, t, w.dt, None, None, None)
    pkg.fire_step_noalloc(grid, w.classes, psi, psi_b, frac, frac_b, tign, fuel, None, zx, zy,
                          u, v, t, w.dt, None, None, status)
    torch.cuda.synchronize()
    assert torch.equal(psi_c, psi_b) and torch.equal(frac_c, frac_b)
    assert torch.equal(tign_c, tign)
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


def test_noalloc_binding_checks_tensors():
    """Tensors of the wrong dtype or size are refused by the binding before
    the call (no kernel runs)."""
    import torch

    import paper_1102_1343_gb300 as pkg
    torch.cuda.set_device(0)
    grid = pkg.make_grid(4, 4, 10, 10, 60.0, 60.0, pkg.FIRE_FP64)
    n = 40 * 40
    d = dict(device="cuda")
    f64 = lambda k=n: torch.zeros(k, dtype=torch.float64, **d)  # noqa: E731
    args = [f64(), f64(), f64(), f64(), f64(), torch.zeros(n, dtype=torch.uint8, **d), None,
            f64(), f64(), f64(4 * 5), f64(5 * 4), 0.0, 0.5]
    bad = list(args)
    bad[4] = torch.zeros(n, dtype=torch.float32, **d)  # tign must be double
    with pytest.raises(pkg.FireError) as e:
        pkg.fire_step_noalloc(grid, [synth.nominal_class()], *bad)
    assert e.value.code == pkg.FIRE_ERR_ARG and "tign" in str(e.value)
    bad = list(args)
    bad[1] = f64(n - 1)  # short psi_out
    with pytest.raises(pkg.FireError) as e:
        pkg.fire_step_noalloc(grid, [synth.nominal_class()], *bad)
    assert e.value.code == pkg.FIRE_ERR_ARG and "psi_out" in str(e.value)
