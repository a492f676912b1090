"""Pins of the oracle's second fuel-fraction scheme, the one the Discussion
describes as "always second order": exact when the level-set function and
the time from ignition are linear in space.

The reference integrals are computed here independently of the oracle: for a
linear front the burnt part of the cell at each x is an interval of y, on
which the integrand 1 - exp(-(t - t_i)/T_f) integrates in closed form, and
the remaining 1-D integral is done by adaptive quadrature; fully burning
cells are integrated in 40-digit arithmetic (mpmath)."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle

NODES = np.array([-1.0, 0.0, 1.0])  # node offsets in cell widths


def exact_linear(a, b, c, lam, Tf):
    """Fuel fraction of the unit cell [-1/2, 1/2]^2 for psi = a x + b y + c
    and t - t_i = -lam psi where psi <= 0 (so 1 - exp(lam psi / Tf) burns)."""
    k = lam / Tf

    def inner(x):
        # burnt y in [-1/2, 1/2] with a x + b y + c <= 0
        lo, hi = -0.5, 0.5
        if b > 0:
            hi = min(hi, -(a * x + c) / b)
        elif b < 0:
            lo = max(lo, -(a * x + c) / b)
        elif a * x + c > 0:
            return 0.0
        if hi <= lo:
            return 0.0
        if k == 0.0:
            return 0.0
        if b == 0.0:
            return (hi - lo) * (1.0 - math.exp(k * (a * x + c)))
        e1 = math.exp(k * (a * x + b * hi + c))
        e0 = math.exp(k * (a * x + b * lo + c))
        return (hi - lo) - (e1 - e0) / (k * b)

    brk = []
    if b != 0.0:
        for yb in (-0.5, 0.5):
            if a != 0.0:
                xb = -(b * yb + c) / a
                if -0.5 < xb < 0.5:
                    brk.append(xb)
    val, err = integrate.quad(inner, -0.5, 0.5, points=brk or None, epsabs=1e-15,
                              epsrel=1e-13, limit=200)
    return 1.0 - val


def stencil(a, b, c, lam, t=100.0):
    """3x3 node values of psi and of the ignition times (infinite where psi
    >= 0) for psi = a x + b y + c and t_i = t + lam psi at burnt nodes."""
    X, Y = np.meshgrid(NODES, NODES)
    p = a * X + b * Y + c
    ti = np.where(p < 0.0, t + lam * p, np.inf)
    return p, ti


@pytest.mark.parametrize("seed", range(12))
def test_exact_for_linear_psi_and_ignition_time(orc, seed):
    """Fronts crossing the cell in any direction (and cells fully burning or
    not burning at all), any slope of the ignition time: the scheme equals
    the exact integral; the subcell scheme of Sect. 3.3 generally does not."""
    rng = np.random.default_rng(seed)
    a, b = rng.uniform(-3.0, 3.0, 2)
    c = rng.uniform(-1.0, 1.0)
    lam = rng.uniform(0.5, 40.0)
    Tf = rng.uniform(5.0, 100.0)
    t = 100.0
    p, ti = stencil(a, b, c, lam, t)
    want = exact_linear(a, b, c, lam, Tf)
    got = orc.cell_fuel_fraction_linear(p, ti, t, Tf)
    assert got == pytest.approx(want, abs=2e-13)


def test_subcell_scheme_is_not_exact_where_the_new_one_is(orc):
    a, b, c, lam, Tf, t = 1.3, 0.7, 0.1, 30.0, 8.0, 100.0
    p, ti = stencil(a, b, c, lam, t)
    want = exact_linear(a, b, c, lam, Tf)
    assert orc.cell_fuel_fraction_linear(p, ti, t, Tf) == pytest.approx(want, abs=1e-13)
    assert abs(orc.cell_fuel_fraction(p, ti, t, Tf) - want) > 1e-3


def test_special_cases(orc):
    """No node burning: F = 1 exactly; a cell burning with one ignition time
    everywhere: F = exp(-(t - t_i)/T_f) (eq. fuel); a front that has just
    arrived (t_i = t at every burnt node): nothing burned yet."""
    t, Tf = 50.0, 20.0
    p = np.full((3, 3), 2.0)
    assert orc.cell_fuel_fraction_linear(p, np.full((3, 3), np.inf), t, Tf) == 1.0
    p = -np.full((3, 3), 3.0)
    ti = np.full((3, 3), 41.0)
    assert orc.cell_fuel_fraction_linear(p, ti, t, Tf) == pytest.approx(math.exp(-9.0 / 20.0),
                                                                         rel=1e-14)
    p, _ = stencil(0.8, -0.4, 0.05, 1.0)
    assert orc.cell_fuel_fraction_linear(p, np.where(p < 0, t, np.inf), t, Tf) == 1.0


@pytest.mark.parametrize("grad", [(1e-9, 2e-9), (0.3, -0.2), (0.9, 0.95), (4.0, -7.0),
                                  (30.0, 29.999), (-80.0, 5.0)])
def test_fully_burning_cells_against_40_digit_integrals(orc, grad):
    """Every node burning with t - t_i linear: the integral of exp over each
    triangle goes through the second divided difference of exp, evaluated
    by a series (spread < 1) or by differences (spread >= 1); gradients from
    nearly flat to steep and nearly equal vertex values."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    gx, gy = grad
    d0 = 100.0
    X, Y = np.meshgrid(NODES, NODES)
    D = d0 + gx * X + gy * Y          # t - t_i at the nodes (all > 0)
    t, Tf = 500.0, 37.0
    p = -np.ones((3, 3))              # all burning
    got = orc.cell_fuel_fraction_linear(p, t - D, t, Tf)
    f = lambda x, y: 1 - mp.exp(-(d0 + gx * x + gy * y) / Tf)  # noqa: E731
    want = 1 - mp.quad(f, [-0.5, 0.5], [-0.5, 0.5])
    assert got == pytest.approx(float(want), rel=1e-13, abs=1e-15)


def test_planar_front_steps_give_the_exact_fraction(orc):
    """Through whole fire steps: a planar front moving at a uniform speed
    (eq. F-disc keeps psi linear and t_i is linear behind it) gives every
    interior cell the exact fuel fraction with the scheme; the subcell
    scheme departs from it near the front."""
    from paper_1102_1343_gb300 import synth
    R = 0.25
    cls = [synth.nominal_class(fgi=0.3, weight=25.0, weight_is_tf=1.0)]
    nxa, nya, sr = 8, 3, 10
    dx = 6.0
    nx, ny = nxa * sr, nya * sr
    co = oracle.fuel_coefficients(cls[0])
    # an S0-only spread rate: chaparral-like coefficients scaled to R
    coef = np.zeros((ny, nx, 9))
    coef[..., 0] = R
    coef[..., 2] = 1.0
    coef[..., 5] = 30.0
    coef[..., 6] = co[6]
    coef[..., 7] = co[7]
    coef[..., 8] = co[8]
    fuel = np.zeros((ny, nx), np.uint8)
    z = np.zeros((ny, nx))
    for scheme in (1, 0):
        o = oracle.OracleFire(nxa, nya, sr, 60.0, cls, fuel, z, z, [], eps=0.4, band=0,
                              scheme=scheme)
        o.coef = np.ascontiguousarray(coef)
        xs = (np.arange(nx) + 0.5) * dx
        x0 = 150.0
        psi = np.broadcast_to(xs - x0, (ny, nx)).copy()
        tign = np.where(psi <= 0.0, 0.0 + psi / R, np.inf)
        tign = np.where(np.isfinite(tign), np.minimum(tign, 0.0), tign)
        o.set_state(psi, tign, np.ones((ny, nx)), 0.0)
        u = np.zeros((nya, nxa + 1))
        v = np.zeros((nya + 1, nxa))
        for _ in range(40):
            o.step(u, v, 0.5)
        t = o.t
        # exact: psi = x - x0 - R t, t_i = (x - x0)/R
        front = x0 + R * t
        rows = slice(3, ny - 3)
        errs = []
        for i in range(5, nx - 5):
            xc = xs[i]
            c = (xc - front) / dx
            lam = dx / R  # t - t_i = -psi / R in seconds, psi in cell widths
            want = exact_linear(1.0, 0.0, c, lam, co[6])
            errs.append(np.abs(o.frac[rows, i] - want).max())
        if scheme == 1:
            assert max(errs) <= 1e-12, max(errs)
        else:
            assert max(errs) > 1e-4
