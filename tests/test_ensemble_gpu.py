"""Batched ensemble (one persistent launch per call, members of different
sizes): each member equals the same member run alone through fire_step, the
members agree with the FP64 oracle, replayed launches equal one long launch,
and the bounded grid barrier reports FIRE_ERR_TIMEOUT instead of hanging when a
CTA never arrives."""
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


def member_workloads():
    ws = [synth.random_landscape(12, 9, seed=51, ignition="center", steps=30),
          synth.random_landscape(23, 17, seed=52, ignition="line", steps=30),
          synth.random_landscape(8, 8, seed=53, ignition="center", steps=30),
          synth.random_landscape(17, 26, sr=5, seed=54, ignition="points", n_points=3,
                                 edge_margin=200.0, steps=30)]
    # the third member also has a growing segment ignition (its window forces
    # the step-by-step path for the first steps)
    ws[2].ignitions = ws[2].ignitions + [synth.line_ignition(150.0, 150.0, 220.0, 180.0,
                                                             radius=6.0, t_start=0.5,
                                                             speed=2.0)]
    return ws


def add_node_moisture(ws, members=(0, 1)):
    """Per-node fuel moisture on some members (class moisture + a smooth
    +-0.04 field); the others keep their class moisture, and the ensemble
    then gives every member per-node coefficients."""
    from scipy.ndimage import gaussian_filter
    for k in members:
        w = ws[k]
        rng = np.random.default_rng(60 + k)
        f = gaussian_filter(rng.standard_normal((w.ny, w.nx)), 6.0, mode="reflect")
        f *= 0.04 / max(np.abs(f).max(), 1e-12)
        w.moisture = np.maximum(0.01, np.array([c["fuelmc_g"] for c in w.classes])[w.fuel] + f)
    return ws


def make_ensemble(pkg, ws, prec):
    import torch
    P = pkg.FIRE_FP64 if prec == "fp64" else pkg.FIRE_FP32
    dt_ = torch.float64 if prec == "fp64" else torch.float32
    keep, members, winds = [], [], []
    for w in ws:
        fuel = torch.as_tensor(w.fuel).cuda().contiguous()
        zx = torch.as_tensor(w.dzdx).to("cuda", dt_).contiguous()
        zy = torch.as_tensor(w.dzdy).to("cuda", dt_).contiguous()
        mo = (None if w.moisture is None
              else torch.as_tensor(w.moisture).to("cuda", dt_).contiguous())
        keep += [fuel, zx, zy, mo]
        members.append(dict(grid=pkg.make_grid(w.nxa, w.nya, w.srx, w.sry, w.dx_atm, w.dy_atm, P,
                                               w.band, w.eps),
                            classes=w.classes, fuel_class_dev=fuel, dzdx_dev=zx, dzdy_dev=zy,
                            moisture_dev=mo, ignitions=w.ignitions))
        winds.append((torch.as_tensor(w.u).to("cuda", dt_).contiguous(),
                      torch.as_tensor(w.v).to("cuda", dt_).contiguous()))
    ens = pkg.fire_ensemble_create(members)
    torch.cuda.synchronize()
    return ens, winds


def member_state(pkg, ens, m, w, prec):
    import torch
    ctx = pkg.fire_ensemble_member(ens, m)
    dt_ = torch.float64 if prec == "fp64" else torch.float32
    psi = torch.empty((w.ny, w.nx), dtype=dt_, device="cuda")
    tign = torch.empty((w.ny, w.nx), dtype=torch.float64, device="cuda")
    frac = torch.empty_like(psi)
    t = pkg.fire_get_state(ctx, psi, tign, frac)
    torch.cuda.synchronize()
    return psi.double().cpu().numpy(), tign.cpu().numpy(), frac.double().cpu().numpy(), t


@pytest.mark.parametrize("moisture", [False, True])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_members_equal_single_runs(pkg, prec, moisture):
    import torch
    ws = member_workloads()
    if moisture:
        ws = add_node_moisture(ws)
    ens, winds = make_ensemble(pkg, ws, prec)
    hs = [torch.zeros((w.nya, w.nxa), dtype=torch.float64, device="cuda") for w in ws]
    hl = [torch.zeros_like(h) for h in hs]
    us = [u for u, _ in winds]
    vs = [v for _, v in winds]
    pkg.fire_ensemble_step(ens, 20, ws[0].dt, us, vs, hs, hl)
    pkg.fire_ensemble_step(ens, 7, ws[0].dt, us, vs, hs, hl)
    code, per = pkg.fire_ensemble_status(ens, len(ws))
    assert code == pkg.FIRE_OK, per
    for m, w in enumerate(ws):
        single = pkg.FireModel.from_workload(w, precision=prec)
        v_, kx, ky = pkg.fire_get_kernel(pkg.fire_ensemble_member(ens, m))
        pkg.fire_set_kernel(single.ctx, v_, kx, ky)
        u, v = winds[m]
        for _ in range(27):
            hs1, hl1 = single.step(u, v, w.dt)
        a = state_np(single)
        b = member_state(pkg, ens, m, w, prec)
        for k in range(3):
            assert np.array_equal(a[k], b[k]), (m, k)
        assert a[3] == b[3]
        assert np.array_equal(hs1.cpu().numpy(), hs[m].cpu().numpy())
        assert np.array_equal(hl1.cpu().numpy(), hl[m].cpu().numpy())
        single.close()
    pkg.fire_ensemble_destroy(ens)


def test_full_ensemble_members_equal_single_runs(pkg):
    """The benchmark's ensemble: 64 members of fire meshes 390^2..2050^2
    (96.8 M nodes), FP32, 60 steps in one call with the autotuned strips.
    The smallest, the largest and two middle members equal the same members
    run alone with the same strip shape bit for bit (psi, t_i, F and both
    heat grids), so the single-run parity and FP32 tolerances carry over to
    every member size of that workload."""
    import torch
    sizes = synth.ensemble_sizes(64)
    ws = [synth.ensemble_member(k, s, steps=60) for k, s in enumerate(sizes)]
    ens, winds = make_ensemble(pkg, ws, "fp32")
    us = [u for u, _ in winds]
    vs = [v for _, v in winds]
    dt = ws[0].dt
    pkg.fire_ensemble_autotune(ens, 3, dt, us, vs)
    hs = [torch.zeros((w.nya, w.nxa), dtype=torch.float64, device="cuda") for w in ws]
    hl = [torch.zeros_like(h) for h in hs]
    pkg.fire_ensemble_step(ens, 60, dt, us, vs, hs, hl)
    code, per = pkg.fire_ensemble_status(ens, len(ws))
    assert code == pkg.FIRE_OK, per
    order = sorted(range(len(ws)), key=lambda k: ws[k].nx * ws[k].ny)
    for m in (order[0], order[len(order) // 3], order[2 * len(order) // 3], order[-1]):
        w = ws[m]
        single = pkg.FireModel.from_workload(w, precision="fp32")
        v_, kx, ky = pkg.fire_get_kernel(pkg.fire_ensemble_member(ens, m))
        pkg.fire_set_kernel(single.ctx, v_, kx, ky)
        u, v = winds[m]
        for _ in range(60):
            hs1, hl1 = single.step(u, v, w.dt)
        a = state_np(single)
        b = member_state(pkg, ens, m, w, "fp32")
        assert np.isfinite(a[1]).sum() > 0, m
        for k in range(3):
            assert np.array_equal(a[k], b[k]), (m, w.nx, k)
        assert a[3] == b[3]
        assert np.array_equal(hs1.cpu().numpy(), hs[m].cpu().numpy())
        assert np.array_equal(hl1.cpu().numpy(), hl[m].cpu().numpy())
        single.close()
    pkg.fire_ensemble_destroy(ens)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_max_members_equal_single_runs(pkg, prec):
    """FIRE_MAX_MEMBERS (1024) small members of 1x1 to 6x5 atmospheric cells
    at refinement 10 or 5 (odd mesh widths among them) in one ensemble, 12
    steps in two calls: the first, middle and last members, the smallest
    and largest, and random others equal the same members run alone bit for
    bit.  One member more is refused."""
    import torch
    rng = np.random.default_rng(17)
    ws = []
    for k in range(pkg.FIRE_MAX_MEMBERS):
        nxa, nya = int(rng.integers(1, 7)), int(rng.integers(1, 6))
        sr = 10 if k % 3 else 5
        ws.append(synth.random_landscape(nxa, nya, sr=sr, seed=1000 + k, ignition="center",
                                         steps=12))
    ens, winds = make_ensemble(pkg, ws, prec)
    hs = [torch.zeros((w.nya, w.nxa), dtype=torch.float64, device="cuda") for w in ws]
    hl = [torch.zeros_like(h) for h in hs]
    us = [u for u, _ in winds]
    vs = [v for _, v in winds]
    pkg.fire_ensemble_step(ens, 7, ws[0].dt, us, vs, hs, hl)
    pkg.fire_ensemble_step(ens, 5, ws[0].dt, us, vs, hs, hl)
    code, per = pkg.fire_ensemble_status(ens, len(ws))
    assert code in (pkg.FIRE_OK, pkg.FIRE_ERR_BOUNDARY), per
    size = [w.nx * w.ny for w in ws]
    check = {0, 1, 511, 1022, 1023, int(np.argmin(size)), int(np.argmax(size))}
    check |= {int(k) for k in rng.choice(len(ws), 9, replace=False)}
    for m in sorted(check):
        w = ws[m]
        single = pkg.FireModel.from_workload(w, precision=prec)
        v_, kx, ky = pkg.fire_get_kernel(pkg.fire_ensemble_member(ens, m))
        pkg.fire_set_kernel(single.ctx, v_, kx, ky)
        u, v = winds[m]
        for _ in range(12):
            hs1, hl1 = single.step(u, v, w.dt)
        a = state_np(single)
        b = member_state(pkg, ens, m, w, prec)
        for k in range(3):
            assert np.array_equal(a[k], b[k]), (m, k)
        assert a[3] == b[3]
        assert np.array_equal(hs1.cpu().numpy(), hs[m].cpu().numpy()), m
        assert np.array_equal(hl1.cpu().numpy(), hl[m].cpu().numpy()), m
        assert single.status() == per[m], m
        single.close()
    pkg.fire_ensemble_destroy(ens)
    with pytest.raises(pkg.FireError):
        make_ensemble(pkg, ws + ws[:1], prec)


@pytest.mark.parametrize("moisture", [False, True])
def test_members_match_oracle_fp64(pkg, moisture):
    ws = member_workloads()
    if moisture:
        ws = add_node_moisture(ws)
    ens, winds = make_ensemble(pkg, ws, "fp64")
    pkg.fire_ensemble_step(ens, 24, ws[0].dt, [u for u, _ in winds], [v for _, v in winds])
    for m, w in enumerate(ws):
        orc = oracle.OracleFire.from_workload(w)
        for _ in range(24):
            orc.step(w.u, w.v, w.dt)
        ok, e = compare_fp64(member_state(pkg, ens, m, w, "fp64"), orc)
        assert ok, (m, e)
    pkg.fire_ensemble_destroy(ens)


def test_replayed_launches_equal_one_launch(pkg):
    ws = member_workloads()[:2]
    a, wa = make_ensemble(pkg, ws, "fp32")
    b, wb = make_ensemble(pkg, ws, "fp32")
    for _ in range(3):
        pkg.fire_ensemble_step(a, 8, ws[0].dt, [u for u, _ in wa], [v for _, v in wa])
    pkg.fire_ensemble_step(b, 24, ws[0].dt, [u for u, _ in wb], [v for _, v in wb])
    for m, w in enumerate(ws):
        sa, sb = member_state(pkg, a, m, w, "fp32"), member_state(pkg, b, m, w, "fp32")
        for k in range(3):
            assert np.array_equal(sa[k], sb[k])
        assert sa[3] == sb[3]
    pkg.fire_ensemble_destroy(a)
    pkg.fire_ensemble_destroy(b)


def test_barrier_wait_times_out_without_hanging(pkg):
    """A CTA that never arrives at the barrier (test hook) makes the others'
    bounded waits give up: FIRE_ERR_TIMEOUT, and the ensemble stays usable."""
    ws = member_workloads()[:2]
    ens, winds = make_ensemble(pkg, ws, "fp32")
    grid, items = pkg.fire_ensemble_get_kernel(ens)
    assert grid >= 2
    us, vs = [u for u, _ in winds], [v for _, v in winds]
    pkg.fire_ensemble_set_barrier_test(ens, 0, 20000)  # ~2 ms of polling
    pkg.fire_ensemble_step(ens, 3, ws[0].dt, us, vs)
    code, _ = pkg.fire_ensemble_status(ens, len(ws))
    assert code == pkg.FIRE_ERR_TIMEOUT
    pkg.fire_ensemble_clear_status(ens)
    pkg.fire_ensemble_set_barrier_test(ens, -1, 20000000)
    pkg.fire_ensemble_step(ens, 3, ws[0].dt, us, vs)
    code, _ = pkg.fire_ensemble_status(ens, len(ws))
    assert code == pkg.FIRE_OK
    pkg.fire_ensemble_destroy(ens)
