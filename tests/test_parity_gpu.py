"""GPU parity of the CUDA fire step against the FP64 oracle, through the C ABI.

FP64 path: every result within 1e-10 norm-wise relative error of the oracle.
FP32 path: ignition time within 0.1 s (nodes ignited in both), burnt area
within 0.5 %, integrated heat within 1e-4 relative (multi-step runs); one-step
results from a shared state within bounds derived from FP32 rounding.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from gpu_helpers import (as_path_precision, check_step_on_cell, compare_fp64, crop_step,
                         node_moisture, rel_inf, state_np)
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


def run_pair(pkg, w, prec, steps=None, tile=None, check_every=None, heat_tol=1e-10, scheme=0):
    """Run the CUDA path and the oracle side by side; returns both and the
    worst per-step heat error and the integrated heats."""
    import torch
    steps = w.steps if steps is None else steps
    wp = as_path_precision(w, prec)
    orc = oracle.OracleFire.from_workload(wp, scheme=scheme)
    m = pkg.FireModel.from_workload(w, precision=prec)
    if scheme:
        pkg.fire_set_fraction_scheme(m.ctx, scheme)
    if tile:
        pkg.fire_set_kernel(m.ctx, *tile)
    u, v = m.wind(w.u, w.v)
    worst = 0.0
    Qg = Qo = 0.0
    area = w.dx_atm * w.dy_atm
    for n in range(steps):
        hs, hl = m.step(u, v, w.dt)
        hs_o, hl_o, _ = orc.step(wp.u, wp.v, w.dt)
        hs_g = hs.cpu().numpy()
        hl_g = hl.cpu().numpy()
        worst = max(worst, rel_inf(hs_g, hs_o), rel_inf(hl_g, hl_o))
        Qg += hs_g.sum() * w.dt * area
        Qo += hs_o.sum() * w.dt * area
    torch.cuda.synchronize()
    return m, orc, worst, Qg, Qo


# ---------------------------------------------------------------------------
# FP64: 1e-10
# ---------------------------------------------------------------------------

def test_fp64_plain_circle(pkg):
    """100x100 FP64 circle, constant wind 3 m/s, 120 steps of 0.5 s."""
    w = synth.plain_circle()
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64")
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10
    assert Qo > 0 and abs(Qg - Qo) <= 1e-10 * Qo
    assert m.status() == pkg.FIRE_OK


@pytest.mark.parametrize("tile", [None, (1, 1, 1), (1, 7, 3), (1, 12, 17), (0, 1, 1), (0, 3, 2),
                                  (0, 5, 3), (2, 1, 1), (2, 2, 3), (2, 6, 5), (2, 4, 17)])
def test_fp64_landscape_ragged_tiles(pkg, tile):
    """Hills, 13 fuels, smooth wind, line ignition on 230x170 nodes: several
    strips (marching and warp kernels) or tiles (2-D tile kernel), with a
    ragged last row and column."""
    w = synth.random_landscape(23, 17, seed=21, ignition="line", steps=120)
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10
    assert Qo > 0


@pytest.mark.parametrize("mesh", [(1, 1, 10, "center"), (12, 1, 10, "center"),
                                  (1, 9, 10, "center"), (6, 4, 2, "center"), (8, 6, 10, "none")])
@pytest.mark.parametrize("tile", [None, (0, 1, 1), (1, 1, 1), (2, 1, 1)])
def test_fp64_degenerate_meshes(pkg, mesh, tile):
    """Edge cases of the mesh: one atmospheric cell, one atmospheric row (the
    wind interpolation's single-row case), one column, refinement 2, and a
    fire with no ignition at all (psi stays psi_far, no heat); each kernel
    with strips or tiles one atmospheric cell wide, against the oracle; the
    fire reaching the boundary ring sets the same status on both sides."""
    nxa, nya, sr, ign = mesh
    w = synth.random_landscape(nxa, nya, sr=sr, seed=41, ignition=ign, steps=30)
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10
    boundary = bool(orc.status & oracle.STATUS_BOUNDARY)
    assert (m.status() == pkg.FIRE_ERR_BOUNDARY) == boundary
    if ign == "none":
        assert Qo == 0.0 and Qg == 0.0 and not np.isfinite(orc.tign).any()


@pytest.mark.parametrize("tile", [None, (1, 2, 3), (0, 4, 4), (2, 12, 3), (2, 4, 7)])
def test_fp64_odd_mesh_width(pkg, tile):
    """Refinement 5 on 23x17 atmos cells: an odd fire-mesh width (115), so the
    marching kernel takes its unpaired (scalar) loads and stores."""
    w = synth.random_landscape(23, 17, sr=5, seed=22, ignition="points", n_points=4,
                               edge_margin=150.0, steps=80)
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10


@pytest.mark.parametrize("tile", [None, (2, 5, 3)])
def test_fp64_anisotropic_multiplier_and_segments(pkg, tile):
    """Refinement 4 x 6 with unequal atmos spacing, a per-node spread
    multiplier, a growing segment ignition and a delayed instantaneous one."""
    w = synth.random_landscape(31, 19, sr=5, seed=33, ignition="center", steps=90)
    nx, ny = 31 * 4, 19 * 6
    zx, zy = synth.hills_gradient(np.random.default_rng(3), nx, ny, 10.0, 9.0)
    w = dataclasses.replace(w, srx=4, sry=6, dx_atm=40.0, dy_atm=54.0,
                            fuel=synth.voronoi_fuel(np.random.default_rng(1), nx, ny, 10.0),
                            dzdx=zx, dzdy=zy)
    rng = np.random.default_rng(2)
    w.mult = rng.uniform(0.5, 1.5, (ny, nx))
    w.ignitions = [synth.line_ignition(200.0, 300.0, 330.0, 420.0, radius=12.0, t_start=1.0,
                                       speed=0.8),
                   synth.point_ignition(600.0, 250.0, radius=9.0, t_start=7.25),
                   synth.point_ignition(300.0, 700.0, radius=15.0)]
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10


def max_tables_case(seed=91, steps=40):
    """The limits of the tables: FIRE_MAX_CLASSES (64) fuel classes, every
    one of them on the map, and FIRE_MAX_IGNITIONS (256) ignitions on 400x300
    nodes: 160 instantaneous points, 48 delayed ones, 32 growing points and
    16 growing line segments, many windows open at once."""
    w = synth.random_landscape(40, 30, seed=seed, ignition="none", steps=steps)
    rng = np.random.default_rng(seed)
    classes = synth.random_classes(rng, n=64, chaparral_index=63)
    fuel = synth.voronoi_fuel(rng, w.nx, w.ny, w.dx, n_classes=64, n_sites=3000)
    Lx, Ly = w.nx * w.dx, w.ny * w.dy

    def xy():
        return float(rng.uniform(100.0, Lx - 100.0)), float(rng.uniform(100.0, Ly - 100.0))

    ign = [synth.point_ignition(*xy(), radius=float(rng.uniform(5.0, 15.0)))
           for _ in range(160)]
    ign += [synth.point_ignition(*xy(), radius=float(rng.uniform(5.0, 15.0)),
                                 t_start=float(rng.uniform(0.5, 15.0))) for _ in range(48)]
    ign += [synth.point_ignition(*xy(), radius=float(rng.uniform(5.0, 15.0)),
                                 t_start=float(rng.uniform(0.0, 10.0)),
                                 speed=float(rng.uniform(0.5, 2.0))) for _ in range(32)]
    for _ in range(16):
        ax, ay = xy()
        ign.append(synth.line_ignition(ax, ay, ax + float(rng.uniform(-60.0, 60.0)),
                                       ay + float(rng.uniform(30.0, 60.0)), radius=8.0,
                                       t_start=float(rng.uniform(0.0, 10.0)), speed=1.0))
    return dataclasses.replace(w, classes=classes, fuel=fuel, ignitions=ign)


@pytest.mark.parametrize("tile", [None, (0, 2, 2), (1, 6, 2), (2, 4, 2)])
def test_fp64_max_classes_and_ignitions(pkg, tile):
    """64 fuel classes and 256 ignitions (the tables' limits) through every
    FP64 kernel, against the oracle at 1e-10."""
    w = max_tables_case()
    assert len(w.classes) == pkg.FIRE_MAX_CLASSES and len(w.ignitions) == pkg.FIRE_MAX_IGNITIONS
    assert len(np.unique(w.fuel)) == 64
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10
    assert Qo > 0 and np.isfinite(orc.tign).sum() > 2000


@pytest.mark.parametrize("tile", [None, (4, 4, 2), (3, 8, 2)])
def test_fp32_max_classes_and_ignitions(pkg, tile):
    """The same case through the FP32 warp kernels (two-column, dense and
    four-column, each with its 64-class table in shared memory), against the
    oracle within the FP32 bounds."""
    w = max_tables_case()
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp32", tile=tile)
    if tile is None:
        assert pkg.fire_get_kernel(m.ctx)[0] in (pkg.FIRE_KERNEL_WARP, pkg.FIRE_KERNEL_TILE)
    psi, tign, frac, _ = state_np(m)
    both = np.isfinite(tign) & np.isfinite(orc.tign)
    assert both.sum() > 2000
    assert np.abs(tign[both] - orc.tign[both]).max() <= 0.1
    A, Ao = (psi <= 0).sum(), (orc.psi <= 0).sum()
    B, Bo = (1 - frac).sum(), (1 - orc.frac).sum()
    assert abs(A - Ao) / Ao <= 0.005 and abs(B - Bo) / Bo <= 0.005
    assert abs(Qg - Qo) / Qo <= 1e-4


def ignition_edge_case(steps=40):
    """Zero wind on hills and 13 fuels, 300x250 nodes, with the edge cases of
    the ignition forms: a point of radius 0 on a node, a zero-length segment,
    a segment partly and one wholly outside the domain, a growing point whose
    window opens exactly at a step start (t = 4 dt), one that opens after the
    run, two overlapping fires lit at different times, and a fire in the
    boundary band (the boundary status on both sides)."""
    w = synth.random_landscape(30, 25, seed=71, ignition="none", steps=steps)
    u, v = synth.constant_wind(w.nxa, w.nya, 0.0, 0.0)
    dx, dt = w.dx, w.dt
    node = lambda i, j: ((i + 0.5) * dx, (j + 0.5) * dx)
    ign = [synth.point_ignition(*node(40, 40), radius=0.0),
           synth.line_ignition(*node(120, 60), *node(120, 60), radius=12.0),
           synth.line_ignition(-80.0, 500.0, 60.0, 520.0, radius=9.0),
           synth.line_ignition(-500.0, -500.0, -300.0, -450.0, radius=20.0),
           synth.point_ignition(*node(200, 150), radius=15.0, t_start=4 * dt, speed=1.5),
           synth.point_ignition(*node(60, 200), radius=15.0, t_start=(steps + 5) * dt,
                                speed=1.0),
           synth.point_ignition(*node(220, 60), radius=18.0),
           synth.point_ignition(*node(225, 64), radius=10.0, t_start=3.0),
           synth.point_ignition(*node(2, 120), radius=8.0)]
    return dataclasses.replace(w, u=u, v=v, ignitions=ign)


@pytest.mark.parametrize("tile", [None, (0, 3, 2), (1, 6, 3), (2, 4, 5)])
def test_fp64_ignition_edge_cases(pkg, tile):
    w = ignition_edge_case()
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10
    tign = orc.tign
    assert np.isfinite(tign[40, 40]) and tign[40, 40] == 0.0  # radius 0 on a node
    assert tign[60, 120] == 0.0 and tign[64, 225] == 3.0  # zero-length segment, overlap
    assert not np.isfinite(tign[200, 60])  # the window after the run never opened
    assert np.isfinite(tign[80:90, 0:12]).any()  # the part of a segment inside the domain
    assert np.isfinite(tign[150, 200]) and tign[150, 200] == 4 * w.dt  # opened at 4 dt
    assert m.status() == pkg.FIRE_ERR_BOUNDARY and orc.status & oracle.STATUS_BOUNDARY


def largest_shape(pkg, ctx, variant, ky_cap):
    """The largest accepted (kx, ky): the widest kx, and the tallest ky at it
    up to ky_cap (strips taller than the mesh change nothing); a shape one
    step wider, or taller below the cap, is refused."""
    def ok(a, b):
        try:
            pkg.fire_set_kernel(ctx, variant, a, b)
            return True
        except pkg.FireError:
            return False
    kx = 1
    while ok(kx + 1, 1):
        kx += 1
    ky = 1
    while ky < ky_cap and ok(kx, ky + 1):
        ky += 1
    assert ok(kx, ky) and not ok(kx + 1, 1)
    assert ky == ky_cap or not ok(kx, ky + 1)
    return kx, ky


@pytest.mark.parametrize("prec,variant", [("fp64", "warp"), ("fp64", "march"), ("fp64", "tile"),
                                          ("fp32", "warp4"), ("fp32", "dense")])
def test_largest_strip_and_tile_shapes(pkg, prec, variant):
    """Each kernel at the largest strip or tile shape fire_set_kernel accepts
    on 500x600 nodes (warp strips of 60 x 510 rows, marching strips of 240
    columns as tall as the mesh, the 2-D tiles and the FP32 four-column and
    dense strips as large as their shared memory or row limit allows, strips
    no taller than the mesh): FP64 against the oracle at
    1e-10, FP32 bit for bit equal to the two-column warp kernel at the same
    shape (the four-column kernel at its own widest strips against the
    two-column kernel's widest)."""
    w = synth.random_landscape(50, 60, seed=72, ignition="points", n_points=5,
                               edge_margin=300.0, steps=30)
    V = {"warp": pkg.FIRE_KERNEL_WARP, "march": pkg.FIRE_KERNEL_MARCH,
         "tile": pkg.FIRE_KERNEL_TILE, "warp4": pkg.FIRE_KERNEL_WARP4,
         "dense": pkg.FIRE_KERNEL_WARP_DENSE}[variant]
    probe = pkg.FireModel.from_workload(w, precision=prec)
    kx, ky = largest_shape(pkg, probe.ctx, V, w.nya)
    probe.close()
    if variant in ("warp", "dense"):
        assert (kx, ky) == (6, 51)  # 60 columns, 510 rows (at most 512)
    if variant == "march":
        assert kx == 24  # 240 columns (at most 248)
    if prec == "fp64":
        m, orc, heat_err, Qg, Qo = run_pair(pkg, w, prec, tile=(V, kx, ky))
        ok, e = compare_fp64(state_np(m), orc)
        assert ok, e
        assert heat_err <= 1e-10
        assert m.status() == pkg.FIRE_OK
        return
    import torch
    runs = []
    for var, shape in ((V, (kx, ky)), (pkg.FIRE_KERNEL_WARP, (6, min(ky, 51)))):
        m = pkg.FireModel.from_workload(w, precision=prec)
        pkg.fire_set_kernel(m.ctx, var, *shape)
        u, v = m.wind(w.u, w.v)
        for _ in range(w.steps):
            hs, hl = m.step(u, v, w.dt)
        torch.cuda.synchronize()
        runs.append(state_np(m)[:3] + (hs.cpu().numpy(), hl.cpu().numpy()))
        assert m.status() == pkg.FIRE_OK
        m.close()
    assert np.isfinite(runs[0][1]).sum() > 20
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def drip_torch_case(seed=61, steps=120):
    """Two drip torches (Sect. "Ignition"): one crossing at 3.2 m/s for 20 s,
    its line burning out to 15 m at 2 m/s, one starting at 10.25 s."""
    w = synth.random_landscape(23, 17, seed=seed, ignition="none", steps=steps)
    w.ignitions = [synth.drip_torch(300.0, 400.0, 3.0, 1.0, t_start=1.0, t_end=21.0,
                                    radius=15.0, speed=2.0),
                   synth.drip_torch(900.0, 300.0, -2.0, 2.5, t_start=10.25, t_end=25.0,
                                    radius=9.0, speed=4.0)]
    return w


@pytest.mark.parametrize("tile", [None, (1, 6, 2), (0, 2, 2), (2, 6, 4)])
def test_fp64_drip_torch(pkg, tile):
    """Drip-torch ignition in every kernel against the oracle at 1e-10 (psi,
    F, the ignition times including those the torches set, every step's
    heat)."""
    w = drip_torch_case()
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10
    assert np.isfinite(orc.tign).sum() > 100 and Qo > 0


@pytest.mark.parametrize("case,tile", [("line", None), ("line", (0, 2, 2)), ("points", (0, 3, 1))])
def test_fp64_linear_fraction_scheme(pkg, case, tile):
    """The fuel-fraction scheme exact for linear psi and t_i (the tile
    kernel) against the oracle's, at 1e-10 on psi, F, t_i and the heat."""
    w = synth.random_landscape(23, 17, seed=21, ignition=case, n_points=4, edge_margin=200.0,
                               steps=120)
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile, scheme=1)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10
    assert Qo > 0 and pkg.fire_get_kernel(m.ctx)[0] == pkg.FIRE_KERNEL_TILE
    # other kernels are refused while the scheme is set, and so is the adjoint
    with pytest.raises(pkg.FireError):
        pkg.fire_set_kernel(m.ctx, pkg.FIRE_KERNEL_MARCH, 2, 2)
    u, v = m.wind(w.u, w.v)
    with pytest.raises(pkg.FireError) as ex:
        m.adjoint(u, v, w.dt, 5, np.full((w.ny, w.nx), np.nan), grads=False)
    assert ex.value.code == pkg.FIRE_ERR_STATE
    pkg.fire_set_fraction_scheme(m.ctx, pkg.FIRE_FRACTION_SUBCELL)
    pkg.fire_set_kernel(m.ctx, pkg.FIRE_KERNEL_MARCH, 2, 2)
    m.close()


def test_fp32_linear_fraction_scheme(pkg):
    w = synth.random_landscape(32, 26, seed=44, ignition="line", steps=300)
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp32", scheme=1)
    psi, tign, frac, _ = state_np(m)
    both = np.isfinite(tign) & np.isfinite(orc.tign)
    assert both.sum() > 100
    dti = np.abs(tign[both] - orc.tign[both]).max()
    B, Bo = (1 - frac).sum(), (1 - orc.frac).sum()
    assert dti <= 0.1
    assert abs((psi <= 0).sum() - (orc.psi <= 0).sum()) / (orc.psi <= 0).sum() <= 0.005
    assert abs(B - Bo) / Bo <= 0.005
    assert abs(Qg - Qo) / Qo <= 1e-4
    m.close()


@pytest.mark.parametrize("tile", [None, (2, 6, 4)])
def test_fp64_chaparral(pkg, tile):
    """The chaparral rate of eq. (chapparal) (6 m/s in a wind above 4.6 m/s)
    with a time step inside the scheme's stability limit (c = S dt/dx = 0.2)."""
    w = synth.random_landscape(20, 16, seed=77, ignition="center", steps=100, dt=0.2)
    w.classes = synth.random_classes(np.random.default_rng(78), chaparral_index=3)
    jj, ii = np.nonzero(w.fuel[40:-40, 40:-40] == 3)
    k = len(jj) // 2
    w.ignitions = [synth.point_ignition((ii[k] + 40.5) * w.dx, (jj[k] + 40.5) * w.dy, 10.0)]
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10


@pytest.mark.parametrize("tile", [None, (1, 12, 3), (0, 3, 2), (2, 6, 5)])
def test_fp64_node_moisture(pkg, tile):
    """A per-node fuel moisture (class moisture + a smooth +-0.05 field): the
    coefficients R0, c, d and the heat factors of each node from Table 2 at
    that node's moisture, in every kernel, against the oracle's per-node
    coefficients (orc_node_coefficients with the moisture field)."""
    w = node_moisture(synth.random_landscape(23, 17, seed=21, ignition="line", steps=120))
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10
    assert Qo > 0 and abs(Qg - Qo) <= 1e-10 * Qo


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_class_valued_node_moisture_changes_no_bit(pkg, prec):
    """A per-node moisture equal to every node's class moisture gives the same
    coefficients, so the per-node kernels give the same bits as the class
    table; fire_set_moisture(None) returns to the class table."""
    import torch
    w = synth.random_landscape(24, 10, seed=31, ignition="points", n_points=6, edge_margin=150.0,
                               steps=120)
    if prec == "fp32":
        # the FP32 path stores the moisture in float: class values that a
        # float holds exactly give exactly the class coefficients
        w.classes = [dict(c, fuelmc_g=float(np.float32(c["fuelmc_g"]))) for c in w.classes]
    a = pkg.FireModel.from_workload(w, precision=prec)
    w.moisture = np.array([c["fuelmc_g"] for c in w.classes])[w.fuel]
    b = pkg.FireModel.from_workload(w, precision=prec)
    c = pkg.FireModel.from_workload(w, precision=prec)
    c.set_moisture(None)
    u, v = a.wind(w.u, w.v)
    for _ in range(w.steps):
        hs_a, hl_a = a.step(u, v, w.dt)
        hs_b, hl_b = b.step(u, v, w.dt)
        hs_c, _ = c.step(u, v, w.dt)
    torch.cuda.synchronize()
    sa, sb, sc = state_np(a), state_np(b), state_np(c)
    assert np.isfinite(sa[1]).sum() > 50
    for k in range(3):
        assert np.array_equal(sa[k], sb[k]) and np.array_equal(sa[k], sc[k])
    assert np.array_equal(hs_a.cpu().numpy(), hs_b.cpu().numpy())
    assert np.array_equal(hl_a.cpu().numpy(), hl_b.cpu().numpy())
    assert np.array_equal(hs_a.cpu().numpy(), hs_c.cpu().numpy())
    for x in (a, b, c):
        x.close()


# ---------------------------------------------------------------------------
# FP32: ignition time 0.1 s, burnt area 0.5 %, integrated heat 1e-4
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("case,tile", [("line", None), ("points", None), ("line", (0, 8, 4)),
                                       ("line", (2, 6, 20)), ("points", (2, 6, 20)),
                                       ("line-moisture", None), ("points-moisture", (1, 12, 4)),
                                       ("drip", None), ("line", (3, 12, 8)),
                                       ("points", (3, 12, 20)), ("points-moisture", (3, 6, 4)),
                                       ("drip", (3, 12, 5))])
def test_fp32_against_fp64_oracle(pkg, case, tile):
    if case == "drip":
        w = drip_torch_case(steps=300)
    else:
        w = synth.random_landscape(32, 26, seed=44, ignition=case.split("-")[0], n_points=6,
                                   edge_margin=300.0, steps=300)
    if case.endswith("moisture"):
        w = node_moisture(w)
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp32", tile=tile)
    psi, tign, frac, _ = state_np(m)
    both = np.isfinite(tign) & np.isfinite(orc.tign)
    assert both.sum() > 100
    dti = np.abs(tign[both] - orc.tign[both]).max()
    A, Ao = (psi <= 0).sum(), (orc.psi <= 0).sum()
    B, Bo = (1 - frac).sum(), (1 - orc.frac).sum()
    errs = dict(tign_max_s=dti, area=abs(A - Ao) / Ao, burned=abs(B - Bo) / Bo,
                heat=abs(Qg - Qo) / Qo)
    print("fp32 errors vs fp64 oracle:", errs)
    assert dti <= 0.1, errs
    assert errs["area"] <= 0.005 and errs["burned"] <= 0.005, errs
    assert errs["heat"] <= 1e-4, errs


# ---------------------------------------------------------------------------
# faults, equivalences of the entry points
# ---------------------------------------------------------------------------

def test_boundary_and_nonfinite_status(pkg):
    w = synth.plain_circle(steps=2)
    w.ignitions = [synth.point_ignition(3.0, 300.0, radius=8.0)]
    m = pkg.FireModel.from_workload(w, precision="fp32")
    u, v = m.wind(w.u, w.v)
    m.step(u, v, w.dt)
    assert m.status() == pkg.FIRE_ERR_BOUNDARY
    pkg.fire_clear_status(m.ctx)
    assert m.status() == pkg.FIRE_OK
    w2 = synth.plain_circle(steps=1)
    m2 = pkg.FireModel.from_workload(w2, precision="fp64")
    uu = w2.u.copy()
    uu[3, 4] = np.nan
    u2, v2 = m2.wind(uu, w2.v)
    m2.step(u2, v2, w2.dt)
    assert m2.status() == pkg.FIRE_ERR_NONFINITE


@pytest.mark.parametrize("prec,pinned", [("fp32", False), ("fp64", False), ("fp32", True),
                                          ("fp64", True)])
def test_run_graph_and_host_path_equal_steps(pkg, prec, pinned):
    """fire_run (graph replay) and fire_step_host give the same bits as a
    sequence of fire_step calls; with page-locked heat buffers the kernel
    writes them directly, with pageable ones through a copy."""
    import torch
    w = synth.random_landscape(12, 9, seed=5, ignition="center", steps=15)
    a = pkg.FireModel.from_workload(w, precision=prec)
    b = pkg.FireModel.from_workload(w, precision=prec)
    c = pkg.FireModel.from_workload(w, precision=prec)
    u, v = a.wind(w.u, w.v)
    for _ in range(w.steps):
        hs_a, hl_a = a.step(u, v, w.dt)
    hs_b, hl_b = b.run(w.steps, u, v, w.dt)
    dt_np = np.float64 if prec == "fp64" else np.float32
    uh = np.ascontiguousarray(w.u, dt_np)
    vh = np.ascontiguousarray(w.v, dt_np)
    if pinned:
        hs_c = torch.zeros((w.nya, w.nxa), dtype=torch.float64).pin_memory().numpy()
        hl_c = torch.zeros((w.nya, w.nxa), dtype=torch.float64).pin_memory().numpy()
    else:
        hs_c = np.zeros((w.nya, w.nxa))
        hl_c = np.zeros((w.nya, w.nxa))
    for _ in range(w.steps):
        pkg.fire_step_host(c.ctx, uh, vh, w.dt, hs_c, hl_c)
    torch.cuda.synchronize()
    sa, sb, sc = state_np(a), state_np(b), state_np(c)
    for x, y in ((sa, sb), (sa, sc)):
        for k in range(3):
            assert np.array_equal(x[k], y[k])
        assert x[3] == y[3]
    assert np.array_equal(hs_a.cpu().numpy(), hs_b.cpu().numpy())
    assert np.any(hs_c != 0.0) and np.any(hl_c != 0.0)
    assert np.array_equal(hs_a.cpu().numpy(), hs_c)
    assert np.array_equal(hl_a.cpu().numpy(), hl_c)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_run_follows_changed_arguments(pkg, prec):
    """fire_run in several calls that change what its captured graph holds:
    a new wind buffer, the same buffer with new contents, a new dt, no heat
    outputs and then others, and a growing ignition window that opens between
    them.  The state and the last heat grids equal a plain fire_step loop's
    bit for bit."""
    import torch
    w = synth.random_landscape(30, 20, seed=6, ignition="center", steps=1)
    # a window from t = 6 to 9 s on node (199, 116): the steps in it run one
    # by one, the ones after it replay the graph again
    w.ignitions = w.ignitions + [synth.point_ignition(1197.0, 699.0, radius=3.0, t_start=6.0,
                                                      speed=1.0)]
    a = pkg.FireModel.from_workload(w, precision=prec)
    b = pkg.FireModel.from_workload(w, precision=prec)
    u1, v1 = a.wind(w.u, w.v)
    u2, v2 = a.wind(w.u * 1.3, w.v * 0.7)
    u3, v3 = u1.clone(), v1.clone()
    hs = torch.zeros_like(a.heat_s)
    hl = torch.zeros_like(a.heat_l)
    plan = [(9, u1, v1, 0.5, (a.heat_s, a.heat_l)), (10, u2, v2, 0.5, (None, None)),
            (6, u3, v3, 0.5, (hs, hl)), (8, u3, v3, 0.25, (hs, hl))]
    for n, u, v, dt, (h1, h2) in plan:
        if u is u3 and dt == 0.25:
            u3.mul_(0.9)  # new contents of the buffer the graph holds
        for _ in range(n):
            pkg.fire_step(a.ctx, u, v, dt, a.heat_s, a.heat_l)
        pkg.fire_run(b.ctx, n, dt, u, v, h1, h2)
    torch.cuda.synchronize()
    sa, sb = state_np(a), state_np(b)
    for k in range(3):
        assert np.array_equal(sa[k], sb[k]), k
    assert sa[3] == sb[3] == 25 * 0.5 + 8 * 0.25
    assert np.array_equal(a.heat_s.cpu().numpy(), hs.cpu().numpy())
    assert np.array_equal(a.heat_l.cpu().numpy(), hl.cpu().numpy())
    assert sa[1][116, 199] == 6.0  # the second fire
    a.close()
    b.close()


def test_checkpoint_resume(pkg):
    """get_state / set_state: a resumed run continues with the same bits."""
    import torch
    w = synth.random_landscape(12, 9, seed=6, ignition="center", steps=10)
    a = pkg.FireModel.from_workload(w, precision="fp32")
    u, v = a.wind(w.u, w.v)
    for _ in range(5):
        a.step(u, v, w.dt)
    ck = a.state()
    ck = tuple(x.clone() if hasattr(x, "clone") else x for x in ck)
    for _ in range(5):
        a.step(u, v, w.dt)
    b = pkg.FireModel.from_workload(w, precision="fp32")
    b.set_state(*ck)
    for _ in range(5):
        b.step(u, v, w.dt)
    torch.cuda.synchronize()
    sa, sb = state_np(a), state_np(b)
    for k in range(3):
        assert np.array_equal(sa[k], sb[k])
    assert sa[3] == sb[3]


# ---------------------------------------------------------------------------
# full-size meshes: one step from the GPU's own state, sampled atmos cells
# recomputed by the oracle on crops
# ---------------------------------------------------------------------------

def _sample_cells(w, rng, n_random, near):
    cells = set()
    for g in w.ignitions:
        I = int(g["ax"] / w.dx_atm)
        J = int(g["ay"] / w.dy_atm)
        for dI in (-1, 0, 1):
            for dJ in (-1, 0, 1):
                cells.add((I + dI, J + dJ))
        if len(cells) >= near:
            break
    while len(cells) < near + n_random:
        cells.add((int(rng.integers(1, w.nxa - 1)), int(rng.integers(1, w.nya - 1))))
    return [(I, J) for I, J in cells if 1 <= I < w.nxa - 1 and 1 <= J < w.nya - 1]


@pytest.mark.parametrize("name,prec,warm,tile", [("line2000", "fp64", 60, None),
                                                 ("line2000", "fp32", 200, None),
                                                 ("points8200", "fp32", 200, None),
                                                 ("points8200", "fp32", 200, (2, 6, 20)),
                                                 ("line2000", "fp64", 60, (2, 6, 20)),
                                                 ("burning8200", "fp32", 20, None)])
def test_full_size_sampled_cells(pkg, name, prec, warm, tile):
    """The 2000x2000 line-fire mesh (FP64 and FP32), the 8200x8200 50-point
    mesh (FP32) in the tile shape the benchmark uses, and the same mesh 42 %
    burnt (the benchmark's burning leg, on the dense warp kernel that the
    adaptive choice takes there): after `warm` steps, one more GPU step is
    compared on sampled atmospheric cells (around the ignitions and at
    random) with the oracle run on 3x3-cell crops from the same state."""
    import torch
    w = {"line2000": synth.line_fire_2000, "points8200": synth.points_fire_8200,
         "burning8200": synth.burning_fire_8200}[name]()
    wp = as_path_precision(w, prec)
    m = pkg.FireModel.from_workload(w, precision=prec)
    if tile:
        pkg.fire_set_kernel(m.ctx, *tile)
    u, v = m.wind(w.u, w.v)
    m.run(warm, u, v, w.dt)
    if name == "burning8200":
        assert pkg.fire_get_kernel(m.ctx)[0] == pkg.FIRE_KERNEL_WARP_DENSE
    psi0, tign0, frac0, t0 = state_np(m)
    hs, hl = m.step(u, v, w.dt)
    torch.cuda.synchronize()
    psi1, tign1, frac1, _ = state_np(m)
    hs = hs.cpu().numpy()
    hl = hl.cpu().numpy()
    assert m.status() == pkg.FIRE_OK
    rng = np.random.default_rng(9)
    cells = _sample_cells(w, rng, n_random=24, near=36)
    Hs_max = max(oracle.fuel_coefficients(c)[7] for c in w.classes)
    Hq_max = max(oracle.fuel_coefficients(c)[8] for c in w.classes)
    burning_cells = 0
    for I, J in cells:
        sub, hs_o, hl_o, (cy, cx), (ys, xs) = crop_step(wp, psi0, tign0, frac0, t0, I, J, w.dt)
        burning_cells += check_step_on_cell(
            prec, sub, cy, cx, psi0[ys, xs], t0, psi1[ys, xs][cy, cx],
            tign1[ys, xs][cy, cx], frac1[ys, xs][cy, cx], hs[J, I], hl[J, I], hs_o, hl_o,
            Hs_max, Hq_max, w.dt)
    assert burning_cells >= 4


@pytest.mark.parametrize("mesh", [(32, 26, 10), (23, 17, 10), (23, 17, 5), (13, 40, 10)])
def test_warp4_equals_two_column_warp_kernel(pkg, mesh):
    """The four-column warp kernel and the dense two-column one (t_i read a
    row ahead, packed fuel fractions) compute every node with the same
    operations as the two-column one: the same bits for psi, t_i, F and both
    heat grids (meshes whose width is a multiple of 4 (float4 rows), even
    (float2 pairs) and odd (scalars); strips of 12 and of 6 atmospheric
    cells), with multipliers and a per-node moisture on one mesh."""
    import torch
    nxa, nya, sr = mesh
    w = synth.random_landscape(nxa, nya, sr=sr, seed=46, ignition="points", n_points=5,
                               edge_margin=150.0, steps=150, ignition_radius=25.0)
    if nxa == 13:
        w = node_moisture(w)
        w.mult = np.random.default_rng(5).uniform(0.7, 1.3, (w.ny, w.nx))
    a = pkg.FireModel.from_workload(w, precision="fp32")
    b = pkg.FireModel.from_workload(w, precision="fp32")
    c = pkg.FireModel.from_workload(w, precision="fp32")
    d = pkg.FireModel.from_workload(w, precision="fp32")
    ky = max(1, 30 // sr)
    pkg.fire_set_kernel(a.ctx, pkg.FIRE_KERNEL_WARP, 60 // sr, ky)
    pkg.fire_set_kernel(b.ctx, pkg.FIRE_KERNEL_WARP4, 120 // sr, ky)
    pkg.fire_set_kernel(c.ctx, pkg.FIRE_KERNEL_WARP4, 60 // sr, 2 * ky)
    pkg.fire_set_kernel(d.ctx, pkg.FIRE_KERNEL_WARP_DENSE, 60 // sr, ky)
    u, v = a.wind(w.u, w.v)
    for _ in range(w.steps):
        ha = a.step(u, v, w.dt)
        hb = b.step(u, v, w.dt)
        hc = c.step(u, v, w.dt)
        hd = d.step(u, v, w.dt)
    torch.cuda.synchronize()
    sa, sb, sc, sd = state_np(a), state_np(b), state_np(c), state_np(d)
    assert np.isfinite(sa[1]).sum() > 30
    for k in range(3):
        assert np.array_equal(sa[k], sb[k]) and np.array_equal(sa[k], sc[k]), k
        assert np.array_equal(sa[k], sd[k]), k
    for x, y in ((ha, hb), (ha, hc), (ha, hd)):
        assert np.array_equal(x[0].cpu().numpy(), y[0].cpu().numpy())
        assert np.array_equal(x[1].cpu().numpy(), y[1].cpu().numpy())
    assert a.status() == b.status() == c.status() == d.status() == pkg.FIRE_OK
    m64 = pkg.FireModel.from_workload(w, precision="fp64")
    for variant in (pkg.FIRE_KERNEL_WARP4, pkg.FIRE_KERNEL_WARP_DENSE):
        with pytest.raises(pkg.FireError):
            pkg.fire_set_kernel(m64.ctx, variant, 60 // sr, ky)
    for x in (a, b, c, d, m64):
        x.close()


def test_fp32_warp_kernels_equal_on_anisotropic_refinement(pkg):
    """Refinement 4 x 6 with unequal atmospheric spacing (40 x 54 m): the
    two-column, four-column and dense warp kernels give the same bits."""
    import torch
    w = synth.random_landscape(31, 19, sr=5, seed=34, ignition="none", steps=80)
    nx, ny = 31 * 4, 19 * 6
    zx, zy = synth.hills_gradient(np.random.default_rng(4), nx, ny, 10.0, 9.0)
    w = dataclasses.replace(w, srx=4, sry=6, dx_atm=40.0, dy_atm=54.0,
                            fuel=synth.voronoi_fuel(np.random.default_rng(2), nx, ny, 10.0),
                            dzdx=zx, dzdy=zy,
                            ignitions=[synth.point_ignition(420.0, 500.0, radius=30.0),
                                       synth.line_ignition(150.0, 200.0, 260.0, 330.0,
                                                           radius=12.0)])
    runs = []
    for var, kx, ky in ((pkg.FIRE_KERNEL_WARP, 15, 5), (pkg.FIRE_KERNEL_WARP4, 30, 5),
                        (pkg.FIRE_KERNEL_WARP_DENSE, 15, 3)):
        m = pkg.FireModel.from_workload(w, precision="fp32")
        pkg.fire_set_kernel(m.ctx, var, kx, ky)
        u, v = m.wind(w.u, w.v)
        for _ in range(w.steps):
            hs, hl = m.step(u, v, w.dt)
        torch.cuda.synchronize()
        runs.append(state_np(m)[:3] + (hs.cpu().numpy(), hl.cpu().numpy()))
        assert m.status() == pkg.FIRE_OK
        m.close()
    assert np.isfinite(runs[0][1]).sum() > 50
    for r in runs[1:]:
        for a, b in zip(runs[0], r):
            assert np.array_equal(a, b)


@pytest.mark.parametrize("tile", [None, (0, 2, 2), (1, 6, 3), (2, 4, 5)])
def test_fp64_fully_burning_mesh(pkg, tile):
    """One ignition larger than the domain: every node burns from t = 0, so
    every cell runs the quadrature in every step and the fire sits in the
    boundary band (the boundary status on both sides)."""
    w = synth.random_landscape(20, 15, seed=73, ignition="none", steps=40)
    w = dataclasses.replace(w, ignitions=[synth.point_ignition(600.0, 450.0, radius=5000.0)])
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10 and Qo > 0
    assert (orc.tign == 0.0).all() and (orc.frac < 1.0).all()
    assert m.status() == pkg.FIRE_ERR_BOUNDARY and orc.status & oracle.STATUS_BOUNDARY


@pytest.mark.parametrize("tile", [None, (0, 3, 2), (2, 4, 5)])
def test_fp64_fuel_at_and_above_extinction_moisture(pkg, tile):
    """Classes whose fuel moisture equals, or exceeds, the moisture of
    extinction (the reaction intensity's moisture damping is 0 there) beside
    ordinary ones, against the oracle at 1e-10."""
    w = synth.random_landscape(23, 17, seed=74, ignition="points", n_points=5,
                               edge_margin=200.0, ignition_radius=30.0, steps=60)
    classes = [dict(c) for c in w.classes]
    for k in (0, 3, 5):
        classes[k]["fuelmc_g"] = classes[k]["fuelmce"]
    for k in (1, 7):
        classes[k]["fuelmc_g"] = classes[k]["fuelmce"] + 0.05
    w = dataclasses.replace(w, classes=classes)
    assert any(np.isin(w.fuel, [0, 1, 3, 5, 7]).ravel())
    m, orc, heat_err, Qg, Qo = run_pair(pkg, w, "fp64", tile=tile)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert heat_err <= 1e-10


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_multiplier_of_ones_changes_no_bit(pkg, prec):
    """A spread multiplier of ones (loaded and multiplied per node) gives the
    same bits as no multiplier: m = 1 multiplies exactly."""
    w = synth.random_landscape(24, 10, seed=31, ignition="points", n_points=6, edge_margin=150.0,
                               steps=200)
    a = pkg.FireModel.from_workload(w, precision=prec)
    w.mult = np.ones((w.ny, w.nx))
    b = pkg.FireModel.from_workload(w, precision=prec)
    for m in (a, b):
        pkg.fire_set_kernel(m.ctx, pkg.FIRE_KERNEL_WARP, 6, 3)
    u, v = a.wind(w.u, w.v)
    for _ in range(w.steps):
        hs_a, hl_a = a.step(u, v, w.dt)
        hs_b, hl_b = b.step(u, v, w.dt)
    sa, sb = state_np(a), state_np(b)
    assert np.isfinite(sa[1]).sum() > 50
    for k in range(3):
        assert np.array_equal(sa[k], sb[k])
    assert np.array_equal(hs_a.cpu().numpy(), hs_b.cpu().numpy())
    assert np.array_equal(hl_a.cpu().numpy(), hl_b.cpu().numpy())
    a.close()
    b.close()
