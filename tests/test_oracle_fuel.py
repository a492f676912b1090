"""Pins of the oracle's fuel fraction (Sect. 3.3), heat fluxes (Sect. 2.3,
Sect. 5 items 5-6), ignition (Sect. 3.4) and boundary handling: the exactness
cases the paper claims, brute-force integrals, the exact total heat, and
arrival times of ignition segments."""
import math

import numpy as np
import pytest

from paper_1102_1343_gb300 import synth

H = 6.0  # fire cell size for the single-cell tests


def nodes3(f):
    """3x3 node values of f(x, y) at offsets -H, 0, H around the cell centre."""
    o = np.array([-H, 0.0, H])
    return np.array([[f(x, y) for x in o] for y in o])


def test_no_fire_leaves_all_fuel(orc):
    """Exact when no part of the cell is on fire: F = 1."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        p = rng.uniform(0.0, 5.0, (3, 3))
        p[rng.integers(0, 3), rng.integers(0, 3)] = 0.0
        assert orc.cell_fuel_fraction(p, np.full((3, 3), np.inf), 100.0, 30.0) == 1.0


def test_fully_burning_cell_uniform_ignition(orc):
    """Whole cell on fire with one ignition time: F = exp(-(t - t_i)/T_f),
    eq. (fuel)."""
    for ti, t, Tf in [(0.0, 10.0, 60.0), (3.5, 4.0, 7.0), (100.0, 160.0, 8.0)]:
        p = -np.abs(np.random.default_rng(int(t)).uniform(0.1, 3.0, (3, 3)))
        F = orc.cell_fuel_fraction(p, np.full((3, 3), ti), t, Tf)
        assert F == pytest.approx(math.exp(-(t - ti) / Tf), rel=1e-15)


def _burnout_fraction(orc, f):
    """F for a fast-burning fuel with ignition long ago: 1 - burnt area."""
    p = nodes3(f)
    ti = np.where(p < 0, -1e6, np.inf)
    return orc.cell_fuel_fraction(p, ti, 0.0, 1e-6)


@pytest.mark.parametrize("x0", [-2.9, -1.5, -0.2, 0.0, 0.7, 2.2, 2.99])
def test_axis_aligned_front_area_exact(orc, x0):
    """eq. (approx-area) is exact when psi is linear and the fireline is
    aligned with a coordinate direction: F = 1 - (x0 + H/2)/H."""
    want = 1.0 - (x0 + H / 2) / H
    assert _burnout_fraction(orc, lambda x, y: x - x0) == pytest.approx(want, abs=1e-14)
    assert _burnout_fraction(orc, lambda x, y: y - x0) == pytest.approx(want, abs=1e-14)
    assert _burnout_fraction(orc, lambda x, y: x0 - x) == pytest.approx(1 - want, abs=1e-14)


def test_diagonal_front_area_exact(orc):
    """eq. (approx-area) is exact when the fireline crosses subcells along
    their diagonals: x + y = 0 burns half the cell, x + y = H/2 burns 7/8."""
    assert _burnout_fraction(orc, lambda x, y: x + y) == pytest.approx(0.5, abs=1e-15)
    assert _burnout_fraction(orc, lambda x, y: x + y - H / 2) == pytest.approx(0.125, abs=1e-15)


def _true_fraction(fpsi, fti, t, Tf, n=400):
    """Brute-force integral of eq. (fuel_left) over the cell [-H/2, H/2]^2
    with a midpoint rule of n x n points."""
    c = (np.arange(n) + 0.5) / n * H - H / 2
    X, Y = np.meshgrid(c, c)
    p = fpsi(X, Y)
    ti = fti(X, Y)
    burn = np.where(p <= 0, 1.0 - np.exp(-(t - ti) / Tf), 0.0)
    return 1.0 - burn.mean()


def test_brute_force_fully_burning_linear_ignition_time(orc):
    """Fully burning cell with t_i linear in space: the quadrature averages
    t - t_i exactly on each subcell, so its error is the Jensen gap
    |mean e^-g - e^-mean g| <= Var(g)/2 per subcell (g = (t - t_i)/T_f >= 0),
    Var of a linear function over a square of side s: (a^2 + b^2) s^2 / 12."""
    rng = np.random.default_rng(5)
    for _ in range(20):
        a, b = rng.uniform(-2, 2, 2)
        t, Tf = 50.0, float(rng.uniform(5, 60))
        t0 = 30.0
        fpsi = lambda x, y: -10.0 + 0 * x
        fti = lambda x, y: t0 + a * x + b * y
        F = orc.cell_fuel_fraction(nodes3(fpsi), nodes3(fti), t, Tf)
        Ft = _true_fraction(fpsi, fti, t, Tf)
        bound = 0.5 * (a * a + b * b) * (H / 2) ** 2 / 12 / Tf ** 2
        assert abs(F - Ft) <= bound + 1e-6, (F, Ft, bound)


def test_brute_force_general_fronts_error_reported(orc):
    """Straight fronts of any direction through the cell with linear ignition
    times: the paper gives no error bound (Sect. 7); the quadrature is exact
    in the limit cases and stays within 0.1 of the true fraction here."""
    rng = np.random.default_rng(6)
    worst = 0.0
    for _ in range(30):
        th = rng.uniform(0, 2 * np.pi)
        c0 = rng.uniform(-2, 2)
        S = 0.1
        t, Tf = 100.0, float(rng.uniform(10, 100))
        fpsi = lambda x, y: np.cos(th) * x + np.sin(th) * y - c0
        fti = lambda x, y: t + (np.cos(th) * x + np.sin(th) * y - c0) / S
        F = orc.cell_fuel_fraction(nodes3(fpsi), nodes3(fti), t, Tf)
        worst = max(worst, abs(F - _true_fraction(fpsi, fti, t, Tf)))
    assert worst < 0.1


def _small_run(orc, steps=60, seed=11, nxa=9, nya=7):
    w = synth.random_landscape(nxa, nya, sr=10, seed=seed, steps=steps, ignition="center")
    o = orc.OracleFire.from_workload(w)
    return w, o


def test_heat_telescopes_to_fuel_burned(orc):
    """Total heat released equals fuel burned x heat content, regardless of
    the quadrature (Sect. 3.3): sum_n sum_cells phi_h dt area =
    sum_nodes (1 - F_end) H_s dx dy, and the same for the latent flux."""
    w, o = _small_run(orc, steps=80)
    tot_s = tot_l = 0.0
    for _ in range(w.steps):
        hs, hl, st = o.step(w.u, w.v, w.dt)
        tot_s += hs.sum() * w.dt * w.dx_atm * w.dy_atm
        tot_l += hl.sum() * w.dt * w.dx_atm * w.dy_atm
    assert st == 0
    co = orc.node_coefficients(w.classes, w.fuel)
    want_s = ((1 - o.frac) * co[..., 7]).sum() * w.dx * w.dy
    want_l = ((1 - o.frac) * co[..., 8]).sum() * w.dx * w.dy
    assert want_s > 0
    assert tot_s == pytest.approx(want_s, rel=1e-10)
    assert tot_l == pytest.approx(want_l, rel=1e-10)
    assert np.all(o.frac <= 1.0) and np.all(o.frac >= 0.0)


def test_heat_ratio_single_fuel(orc):
    w = synth.plain_circle(steps=20)
    o = orc.OracleFire.from_workload(w)
    c = w.classes[0]
    for _ in range(w.steps):
        hs, hl, st = o.step(w.u, w.v, w.dt)
    m = hs != 0
    assert m.any()
    ratio = (c["fuelmc_g"] + 0.56) * 2.5e6 / c["cmbcnst"]
    assert np.allclose(hl[m] / hs[m], ratio, rtol=1e-13)


def test_instantaneous_ignition_is_distance_function(orc):
    """psi = min(psi_far, dist - r_g), t_i = t_g inside (Sect. 3.4)."""
    w = synth.plain_circle()
    o = orc.OracleFire.from_workload(w)
    x = (np.arange(w.nx)[None, :] + 0.5) * w.dx
    y = (np.arange(w.ny)[:, None] + 0.5) * w.dy
    g = w.ignitions[0]
    d = np.hypot(x - g["ax"], y - g["ay"])
    assert np.allclose(o.psi, np.minimum(o.psi_far, d - 10.0), rtol=0, atol=1e-13)
    assert np.array_equal(np.isfinite(o.tign), d <= 10.0)
    assert np.all(o.tign[d <= 10.0] == 0.0)
    assert np.all(o.frac == 1.0)


def test_segment_ignition_arrival_times(orc):
    """A growing ignition on a segment (eqs. ignition-lfn, ignition-min) in a
    fuel that does not spread by itself: after the window t_g..t_g + r_g/S_g
    psi = dist - r_g and newly ignited nodes carry the arrival time
    t_g + dist/S_g."""
    nxa, sr, dxa = 6, 10, 10.0
    nx = nxa * sr
    dx = dxa / sr
    cls = [synth.nominal_class(fgi=0.0)]
    z = np.zeros((nx, nx))
    seg = synth.line_ignition(20.0, 25.0, 38.0, 31.0, radius=3.0, t_start=1.0, speed=0.5)
    o = orc.OracleFire(nxa, nxa, sr, dxa, cls, np.zeros((nx, nx), np.uint8), z, z, [seg])
    u, v = synth.constant_wind(nxa, nxa)
    assert np.all(np.isinf(o.tign))
    for _ in range(20):
        o.step(u, v, 0.5)
    x = (np.arange(nx)[None, :] + 0.5) * dx
    y = (np.arange(nx)[:, None] + 0.5) * dx
    ax, ay, bx, by = 20.0, 25.0, 38.0, 31.0
    s = np.clip(((x - ax) * (bx - ax) + (y - ay) * (by - ay)) / ((bx - ax) ** 2 + (by - ay) ** 2),
                0, 1)
    d = np.hypot(x - ax - s * (bx - ax), y - ay - s * (by - ay))
    assert np.allclose(o.psi, np.minimum(o.psi_far, d - 3.0), atol=1e-12)
    lit = d <= 3.0
    assert np.array_equal(np.isfinite(o.tign), lit)
    assert np.allclose(o.tign[lit], 1.0 + d[lit] / 0.5, rtol=1e-14)


def test_boundary_termination_flag(orc):
    """Fire near the boundary is reported (Sect. 3.1, last paragraph)."""
    w = synth.plain_circle(steps=1)
    o = orc.OracleFire.from_workload(w)
    assert o.step(w.u, w.v, w.dt)[2] == 0
    w2 = synth.plain_circle(steps=1)
    w2.ignitions = [synth.point_ignition(3.0, 300.0, radius=8.0)]
    o2 = orc.OracleFire.from_workload(w2)
    assert o2.step(w2.u, w2.v, w2.dt)[2] & orc.STATUS_BOUNDARY


def test_nonfinite_wind_flagged(orc):
    w = synth.plain_circle(steps=1)
    o = orc.OracleFire.from_workload(w)
    u = w.u.copy()
    u[5, 5] = np.nan
    assert o.step(u, w.v, w.dt)[2] & orc.STATUS_NONFINITE
