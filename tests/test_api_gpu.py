"""Entry points of the C ABI that the other GPU tests use only in passing:
the accessors (fire_mesh_size, fire_time, fire_last_cuda_error, the kernel
timing), inputs changed between steps (fire_set_spread_mult,
fire_set_fuel_classes, fire_set_moisture, each against the oracle restarted
from the same state with the new inputs), and the ensemble's strip shape
(fire_ensemble_set_kernel)."""
import numpy as np
import pytest

import oracle
from gpu_helpers import compare_fp64, rel_inf, state_np
from paper_1102_1343_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    from paper_1102_1343_gb300 import build
    build.build()
    import paper_1102_1343_gb300 as p
    p.load_library()
    assert torch.cuda.is_available()
    return p


def test_accessors_and_kernel_timing(pkg):
    w = synth.random_landscape(23, 17, seed=31, ignition="line", steps=12)
    m = pkg.FireModel.from_workload(w, precision="fp64")
    assert pkg.fire_mesh_size(m.ctx) == (w.nx, w.ny)
    assert pkg.fire_time(m.ctx) == 0.0
    u, v = m.wind(w.u, w.v)
    pkg.fire_enable_timing(m.ctx, True)
    for _ in range(5):
        m.step(u, v, w.dt)
    ms, n = pkg.fire_kernel_time_ms(m.ctx)
    assert n == 5 and ms > 0.0
    pkg.fire_enable_timing(m.ctx, False)
    m.run(7, u, v, w.dt)
    assert pkg.fire_time(m.ctx) == m.time == 12 * w.dt  # dt = 0.5: every sum exact
    assert m.status() == pkg.FIRE_OK
    assert isinstance(pkg.fire_last_cuda_error(), str)
    m.close()


def restart(w, orc, classes, mult, moisture):
    """The oracle with new inputs, continuing from orc's state (the
    instantaneous ignitions are in that state already)."""
    o = oracle.OracleFire(w.nxa, w.nya, (w.srx, w.sry), w.dx_atm, classes, w.fuel, w.dzdx,
                          w.dzdy, [], moisture=moisture, mult=mult, eps=w.eps, band=w.band,
                          dy_atm=w.dy_atm)
    o.set_state(orc.psi, orc.tign, orc.frac, orc.t)
    return o


def test_inputs_changed_between_steps(pkg):
    """FP64: 15 steps, then a new multiplier and new fuel classes (moisture
    +0.03, one class's load doubled), 15 steps, then a per-node moisture
    field, 10 steps, then the multiplier removed, 10 steps; after each
    segment the state and every step's heat equal the oracle's within
    1e-10."""
    w = synth.random_landscape(23, 17, seed=32, ignition="points", n_points=4,
                               edge_margin=300.0, ignition_radius=40.0, steps=50)
    m = pkg.FireModel.from_workload(w, precision="fp64")
    orc = oracle.OracleFire.from_workload(w)
    u, v = m.wind(w.u, w.v)
    rng = np.random.default_rng(33)
    classes = [dict(c, fuelmc_g=c["fuelmc_g"] + 0.03) for c in w.classes]
    classes[int(np.bincount(w.fuel.ravel()).argmax())]["fgi"] *= 2.0
    mult = rng.uniform(0.5, 1.5, (w.ny, w.nx))
    moist = np.clip(np.array([c["fuelmc_g"] for c in classes])[w.fuel]
                    + rng.uniform(-0.02, 0.02, (w.ny, w.nx)), 0.01, None)
    segments = [(15, None), (15, ("mult+classes", classes, mult, None)),
                (10, ("moisture", classes, mult, moist)), (10, ("no mult", classes, None, moist))]
    for n, change in segments:
        if change:
            what, cl, mu, mo = change
            if what == "mult+classes":
                m.set_mult(mu)
                m.set_classes(cl)
            elif what == "moisture":
                m.set_moisture(mo)
            else:
                m.set_mult(None)
            orc = restart(w, orc, cl, mu, mo)
        worst = 0.0
        for _ in range(n):
            hs, hl = m.step(u, v, w.dt)
            hs_o, hl_o, _ = orc.step(w.u, w.v, w.dt)
            worst = max(worst, rel_inf(hs.cpu().numpy(), hs_o), rel_inf(hl.cpu().numpy(), hl_o))
        ok, e = compare_fp64(state_np(m), orc)
        assert ok, (change and change[0], e)
        assert worst <= 1e-10, change and change[0]
    assert np.isfinite(orc.tign).sum() > 100
    m.close()


def test_ensemble_strip_shape(pkg):
    """fire_ensemble_set_kernel: the strips rounded to whole atmospheric
    cells and even widths per member; members still equal single runs at
    the member's resulting shape."""
    import torch
    ws = [synth.random_landscape(12, 9, seed=51, ignition="center", steps=10),
          synth.random_landscape(17, 13, sr=5, seed=54, ignition="center", steps=10)]
    members, keep, winds = [], [], []
    for w in ws:
        fuel = torch.as_tensor(w.fuel).cuda()
        zx = torch.as_tensor(w.dzdx).to("cuda", torch.float32).contiguous()
        zy = torch.as_tensor(w.dzdy).to("cuda", torch.float32).contiguous()
        keep += [fuel, zx, zy]
        members.append(dict(grid=pkg.make_grid(w.nxa, w.nya, w.srx, w.sry, w.dx_atm, w.dy_atm,
                                               pkg.FIRE_FP32, w.band, w.eps),
                            classes=w.classes, fuel_class_dev=fuel, dzdx_dev=zx, dzdy_dev=zy,
                            ignitions=w.ignitions))
        winds.append((torch.as_tensor(w.u).to("cuda", torch.float32).contiguous(),
                      torch.as_tensor(w.v).to("cuda", torch.float32).contiguous()))
    ens = pkg.fire_ensemble_create(members)
    pkg.fire_ensemble_set_kernel(ens, 25, 33)
    grid, items = pkg.fire_ensemble_get_kernel(ens)
    assert grid > 0 and items > 0
    shapes = [pkg.fire_get_kernel(pkg.fire_ensemble_member(ens, k)) for k in range(len(ws))]
    for (var, kx, ky), w in zip(shapes, ws):
        assert var == pkg.FIRE_KERNEL_WARP
        assert (kx * w.srx) % 2 == 0 and kx * w.srx <= 60 and ky >= 1
    hs = [torch.zeros((w.nya, w.nxa), dtype=torch.float64, device="cuda") for w in ws]
    hl = [torch.zeros_like(h) for h in hs]
    pkg.fire_ensemble_step(ens, 10, ws[0].dt, [a for a, _ in winds], [b for _, b in winds], hs, hl)
    for k, w in enumerate(ws):
        single = pkg.FireModel.from_workload(w, precision="fp32")
        pkg.fire_set_kernel(single.ctx, *shapes[k])
        for _ in range(10):
            hs1, hl1 = single.step(*winds[k], w.dt)
        a = state_np(single)
        ctx = pkg.fire_ensemble_member(ens, k)
        psi = torch.empty((w.ny, w.nx), dtype=torch.float32, device="cuda")
        tign = torch.empty((w.ny, w.nx), dtype=torch.float64, device="cuda")
        frac = torch.empty_like(psi)
        pkg.fire_get_state(ctx, psi, tign, frac)
        torch.cuda.synchronize()
        assert np.array_equal(a[0], psi.double().cpu().numpy())
        assert np.array_equal(a[1], tign.cpu().numpy())
        assert np.array_equal(a[2], frac.double().cpu().numpy())
        assert np.array_equal(hs1.cpu().numpy(), hs[k].cpu().numpy())
        single.close()
    pkg.fire_ensemble_destroy(ens)
