"""Autotuners of the step kernel (fire_autotune) and of the ensemble's strip
shape (fire_ensemble_autotune): the state is untouched, the chosen shape is
valid, and results with it still match the oracle / single runs."""
import numpy as np
import pytest

import oracle
from gpu_helpers import compare_fp64, state_np
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


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotune_keeps_state_and_parity(pkg, prec):
    w = synth.random_landscape(23, 17, seed=21, ignition="line", steps=40)
    m = pkg.FireModel.from_workload(w, precision=prec)
    u, v = m.wind(w.u, w.v)
    m.run(5, u, v, w.dt)
    before = state_np(m)
    variant, kx, ky = m.autotune(u, v, w.dt, probe_steps=2)
    after = state_np(m)
    for a, b in zip(before[:3], after[:3]):
        assert np.array_equal(a, b)
    assert before[3] == after[3]
    assert pkg.fire_get_kernel(m.ctx) == (variant, kx, ky)
    allowed = {pkg.FIRE_KERNEL_TILE, pkg.FIRE_KERNEL_MARCH}
    if prec == "fp32":
        allowed.add(pkg.FIRE_KERNEL_WARP)
    assert variant in allowed
    assert 1 <= kx <= w.nxa and 1 <= ky <= w.nya
    m.run(30, u, v, w.dt)
    if prec == "fp64":
        orc = oracle.OracleFire.from_workload(w)
        for _ in range(35):
            orc.step(w.u, w.v, w.dt)
        ok, e = compare_fp64(state_np(m), orc)
        assert ok, e
    m.close()


def test_ensemble_autotune(pkg):
    import torch
    ws = [synth.random_landscape(12, 9, seed=51, ignition="center", steps=30),
          synth.random_landscape(23, 17, seed=52, ignition="line", steps=30),
          synth.random_landscape(8, 8, seed=53, ignition="center", steps=30)]
    keep, members, us, vs = [], [], [], []
    for w in ws:
        fuel = torch.as_tensor(w.fuel).cuda().contiguous()
        zx = torch.as_tensor(w.dzdx).to("cuda", torch.float32).contiguous()
        zy = torch.as_tensor(w.dzdy).to("cuda", torch.float32).contiguous()
        keep += [fuel, zx, zy]
        members.append(dict(grid=pkg.make_grid(w.nxa, w.nya, w.srx, w.sry, w.dx_atm, w.dy_atm,
                                               pkg.FIRE_FP32, w.band, w.eps),
                            classes=w.classes, fuel_class_dev=fuel, dzdx_dev=zx, dzdy_dev=zy,
                            ignitions=w.ignitions))
        us.append(torch.as_tensor(w.u).to("cuda", torch.float32).contiguous())
        vs.append(torch.as_tensor(w.v).to("cuda", torch.float32).contiguous())
    ens = pkg.fire_ensemble_create(members)
    pkg.fire_ensemble_step(ens, 4, ws[0].dt, us, vs)

    def member_states():
        out = []
        for k, w in enumerate(ws):
            ctx = pkg.fire_ensemble_member(ens, k)
            psi = torch.empty((w.ny, w.nx), dtype=torch.float32, device="cuda")
            tign = torch.empty((w.ny, w.nx), dtype=torch.float64, device="cuda")
            frac = torch.empty_like(psi)
            t = pkg.fire_get_state(ctx, psi, tign, frac)
            torch.cuda.synchronize()
            out.append((psi.cpu().numpy(), tign.cpu().numpy(), frac.cpu().numpy(), t))
        return out

    before = member_states()
    cols, rows = pkg.fire_ensemble_autotune(ens, 2, ws[0].dt, us, vs)
    after = member_states()
    for a, b in zip(before, after):
        for x, y in zip(a[:3], b[:3]):
            assert np.array_equal(x, y)
        assert a[3] == b[3]
    assert 20 <= cols <= 240 and 20 <= rows <= 320
    pkg.fire_ensemble_step(ens, 10, ws[0].dt, us, vs)
    code, per = pkg.fire_ensemble_status(ens, len(ws))
    assert code == pkg.FIRE_OK, per
    # each member equals the same member run alone with the tuned shape
    final = member_states()
    for k, w in enumerate(ws):
        single = pkg.FireModel.from_workload(w, precision="fp32")
        pkg.fire_set_kernel(single.ctx, *pkg.fire_get_kernel(pkg.fire_ensemble_member(ens, k)))
        for _ in range(14):
            single.step(us[k], vs[k], w.dt)
        s = state_np(single)
        for x, y in zip(s[:3], final[k][:3]):
            assert np.array_equal(x, y)
        single.close()
    pkg.fire_ensemble_destroy(ens)


def _ctas(variant, kx, ky, nx, ny, srx, sry):
    W, L = kx * srx, ky * sry
    if variant == 2:  # warp strips, 4 per CTA
        return -(-(-(-nx // W)) // 4) * -(-ny // L)
    return -(-nx // W) * -(-ny // L)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_default_shape_follows_mesh_size(pkg, prec):
    """fire_init's default: tiles of one atmospheric cell on a mesh too small
    for strips, strips on larger ones, as tall as the waves of CTAs allow."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tiny = synth.plain_circle()
    m = pkg.FireModel.from_workload(tiny, precision=prec)
    assert pkg.fire_get_kernel(m.ctx) == (pkg.FIRE_KERNEL_TILE, 1, 1)
    m.close()
    w = synth.random_landscape(200, 200, seed=3, ignition="line", steps=1)
    m = pkg.FireModel.from_workload(w, precision=prec)
    variant, kx, ky = pkg.fire_get_kernel(m.ctx)
    m.close()
    if prec == "fp32":
        assert (variant, kx) == (pkg.FIRE_KERNEL_WARP, 6)
        slots, waves2, ky_max = 3 * sms, 7, 16
    else:
        assert (variant, kx) == (pkg.FIRE_KERNEL_MARCH, 24)
        slots, waves2, ky_max = 2 * sms, 5, 6
    n = _ctas(variant, kx, ky, w.nx, w.ny, 10, 10)
    # the tallest strips with enough waves (or one atmospheric cell high)
    assert ky == 1 or 2 * n >= waves2 * slots
    if ky < ky_max:
        assert 2 * _ctas(variant, kx, ky + 1, w.nx, w.ny, 10, 10) < waves2 * slots
