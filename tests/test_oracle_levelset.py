"""Pins of the oracle's level-set core (Sect. 3.1) and wind interpolation
(Sect. 5): textbook upwinding, extrapolation properties, exact results of the
discretisation on planar and quadratic level-set functions, a planar front and
a circle advanced with known speed."""
import math

import numpy as np
import pytest

from paper_1102_1343_gb300 import synth


def test_godunov_matches_textbook_hamiltonian(orc):
    """eq. (Godunov) selects the one-sided difference whose square is the
    Godunov Hamiltonian for outward motion (S > 0):
    grad_x^2 = max(max(D-, 0)^2, min(D+, 0)^2)  (Osher & Fedkiw, p. 58)."""
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.standard_normal(4000), [0.0, -0.0, 1.0, -1.0, 2.5, -2.5]])
    pairs = [(a, b) for a, b in rng.choice(vals, size=(6000, 2))]
    pairs += [(a, -a) for a in vals[:200]] + [(a, a) for a in vals[:200]]
    for dm, dp in pairs:
        g = orc.godunov(dm, dp)
        assert g in (dm, dp, 0.0)
        a, b = max(dm, 0.0), min(dp, 0.0)
        assert g * g == max(a * a, b * b)
    # the printed case order decides ties: D- when |D-| = |D+| in the last case
    assert orc.godunov(2.0, -2.0) == 2.0


def test_extrapolation_properties(orc):
    """Boundary extrapolation (Sect. 3.1): a level-set function increasing
    outward is continued linearly; the ghost never falls below either value
    it is extrapolated from; corners continue bilinear fields."""
    nx, ny = 7, 5
    x = np.arange(nx)[None, :] * 1.0
    y = np.arange(ny)[:, None] * 1.0
    # V-shaped in x, V-shaped in y: increasing outward at every edge
    psi = np.abs(x - 3.0) * 2.0 + np.abs(y - 2.0) * 3.0 + 1.0
    e = orc.extend(psi)
    assert np.array_equal(e[1:-1, 0], psi[:, 0] + (psi[:, 0] - psi[:, 1]))
    assert np.array_equal(e[1:-1, -1], psi[:, -1] + (psi[:, -1] - psi[:, -2]))
    assert np.array_equal(e[0, 1:-1], psi[0] + (psi[0] - psi[1]))
    # corners continue the field: |x-3|*2 + |y-2|*3 + 1 at (-1,-1) = 8 + 9 + 1
    assert e[0, 0] == 18.0 and e[-1, -1] == 18.0
    rng = np.random.default_rng(1)
    for _ in range(50):
        a = rng.standard_normal((ny, nx))
        e = orc.extend(a)
        assert np.all(e[1:-1, 0] >= np.maximum(a[:, 0], a[:, 1]))
        assert np.all(e[1:-1, 0] >= 2 * a[:, 0] - a[:, 1] - 1e-15)
        assert np.all(e[0, 1:-1] >= np.maximum(a[0], a[1]))
        assert np.all(e[-1, 1:-1] >= np.maximum(a[-1], a[-2]))
        assert np.array_equal(e[1:-1, 1:-1], a)


def test_wind_interpolation_reproduces_affine_fields(orc):
    """Bilinear interpolation from the staggered grid is exact for affine
    wind fields where the node lies inside the grid of wind points, and uses
    the edge value outside it."""
    nxa, nya, sr = 6, 4, 5
    al, be, ga = 1.5, 0.25, -0.75
    # u at (I, J+1/2), v at (I+1/2, J) in atmos cell units
    I = np.arange(nxa + 1)[None, :]
    J = np.arange(nya)[:, None] + 0.5
    u = al + be * I + ga * J
    I2 = np.arange(nxa)[None, :] + 0.5
    J2 = np.arange(nya + 1)[:, None] * 1.0
    v = -al + 2 * be * I2 - ga * J2
    un, vn = orc.wind_at_nodes(nxa, nya, sr, sr, u, v)
    xa = (np.arange(nxa * sr)[None, :] + 0.5) / sr
    ya = (np.arange(nya * sr)[:, None] + 0.5) / sr
    u_want = al + be * xa + ga * np.clip(ya, 0.5, nya - 0.5)
    v_want = -al + 2 * be * np.clip(xa, 0.5, nxa - 0.5) - ga * ya
    assert np.allclose(un, u_want, rtol=0, atol=1e-13)
    assert np.allclose(vn, v_want, rtol=0, atol=1e-13)


def _const_rate_setup(orc, ny, nx, **cls_over):
    cls = synth.nominal_class(**cls_over)
    co = orc.fuel_coefficients(cls)
    z = np.zeros((ny, nx))
    return co, co[1], z  # zero wind and flat terrain: S = R0


def test_rhs_planar_and_quadratic(orc):
    """eq. (F-disc) on fields where the discretisation is exact:
    planar psi = a x + b y: F = -S sqrt(a^2 + b^2) at interior nodes;
    quadratic psi = x^2: upwind gradient 2x - dx, scaled Laplacian 2 dx, so
    F = -S (2x - dx) + eps S 2 dx."""
    ny, nx, dx, dy, eps = 9, 12, 2.0, 3.0, 0.4
    co, S, z = _const_rate_setup(orc, ny, nx)
    x = (np.arange(nx)[None, :] + 0.5) * dx + 0 * np.arange(ny)[:, None]
    y = (np.arange(ny)[:, None] + 0.5) * dy + 0 * np.arange(nx)[None, :]
    for a, b in [(1.0, 0.0), (-0.6, 0.8), (0.3, -2.0), (-1.0, -1.0)]:
        psi = a * x + b * y + 7.0
        F = orc.rhs(psi, dx, dy, eps, co, z, z, z, z)
        assert np.allclose(F[1:-1, 1:-1], -S * math.hypot(a, b), rtol=1e-13)
    psi = x ** 2
    F = orc.rhs(psi, dx, dy, eps, co, z, z, z, z)
    want = -S * (2 * x - dx) + eps * S * 2 * dx
    assert np.allclose(F[1:-1, 1:-1], want[1:-1, 1:-1], rtol=1e-13)


def test_rhs_uses_normal_wind_and_slope(orc):
    """The spread rate uses U = wind . n and tan(phi) = grad z . n with n from
    central differences (Sect. 2.2 and after eq. Godunov)."""
    ny, nx, dx = 8, 8, 1.0
    cls = synth.nominal_class()
    co = orc.fuel_coefficients(cls)
    x = (np.arange(nx)[None, :] + 0.5) * dx + 0 * np.arange(ny)[:, None]
    y = (np.arange(ny)[:, None] + 0.5) * dx + 0 * np.arange(nx)[None, :]
    c, s = 0.6, 0.8
    psi = c * x + s * y
    un = np.full((ny, nx), 4.0)
    vn = np.full((ny, nx), -1.0)
    zx = np.full((ny, nx), 0.2)
    zy = np.full((ny, nx), 0.1)
    F = orc.rhs(psi, dx, dx, 0.4, co, un, vn, zx, zy)
    S = orc.spread_rate(co, 4.0 * c - 1.0 * s, 0.2 * c + 0.1 * s)
    assert np.allclose(F[1:-1, 1:-1], -S, rtol=1e-13)
    m = np.full((ny, nx), 1.7)
    F2 = orc.rhs(psi, dx, dx, 0.4, co, un, vn, zx, zy, mult=m)
    assert np.allclose(F2, 1.7 * F, rtol=1e-15)


def _uniform_run(orc, nxa, nya, sr, dx_atm, psi0, steps, dt, eps, U=0.0, V=0.0):
    nx, ny = nxa * sr, nya * sr
    cls = [synth.nominal_class(fgi=0.5)]
    u, v = synth.constant_wind(nxa, nya, U, V)
    z = np.zeros((ny, nx))
    o = orc.OracleFire(nxa, nya, sr, dx_atm, cls, np.zeros((ny, nx), np.uint8), z, z, [],
                       eps=eps)
    o.set_state(psi0, np.full((ny, nx), np.inf), np.ones((ny, nx)), 0.0)
    return o, u, v


def test_planar_front_exact(orc):
    """Planar front with uniform spread rate: psi = x - x0 keeps slope 1, the
    scheme gives psi^{n+1} = psi^n - S dt exactly away from the boundary and
    eq. (set-ignition-time) gives t_i = (x - x0)/S exactly."""
    nxa, nya, sr, dxa = 16, 2, 10, 10.0
    nx, ny = nxa * sr, nya * sr
    dx = dxa / sr
    x = (np.arange(nx)[None, :] + 0.5) * dx + np.zeros((ny, 1))
    x0 = 120.3
    o, u, v = _uniform_run(orc, nxa, nya, sr, dxa, x - x0, 0, 0.5, 0.4, U=2.0)
    S = orc.rothermel_rate(synth.nominal_class(fgi=0.5), 2.0, 0.0)
    steps, dt = 40, 0.5
    for n in range(steps):
        o.step(u, v, dt)
    # only the left edge (psi decreasing outward) disturbs the field, by at
    # most two nodes per step (one per Heun stage)
    lo, hi = 2 * steps + 2, nx - 2
    want = x - x0 - steps * S * dt
    assert np.allclose(o.psi[:, lo:hi], want[:, lo:hi], rtol=0, atol=1e-12)
    crossed = np.isfinite(o.tign[:, lo:hi])
    assert crossed.sum() >= ny
    ti_want = (x[:, lo:hi] - x0) / S
    assert np.allclose(o.tign[:, lo:hi][crossed], ti_want[crossed], rtol=1e-11)


def _radius_along_axes(psi, dx, c):
    """Zero crossing of psi along the +-x, +-y rays through the centre c,
    by linear interpolation between nodes (c lies between nodes)."""
    ny, nx = psi.shape
    ic = int(c / dx - 0.5)  # node just below the centre
    out = []
    rows = (psi[ic] + psi[ic + 1]) / 2  # mean of the two rows straddling y = c
    cols = (psi[:, ic] + psi[:, ic + 1]) / 2
    for line in (rows, cols):
        xs = (np.arange(len(line)) + 0.5) * dx - c
        for sgn in (1, -1):
            d = sgn * xs
            order = np.argsort(d)
            d, p = d[order], line[order]
            k = np.where((d > 0) & (p > 0))[0][0]
            d0, d1, p0, p1 = d[k - 1], d[k], p[k - 1], p[k]
            out.append(d0 + (0 - p0) * (d1 - d0) / (p1 - p0))
    return np.array(out)


@pytest.mark.parametrize("eps", [0.0, 0.4])
def test_circle_growth(orc, eps):
    """Circle under constant S (zero wind and slope): with eps = 0 the radius
    grows as r0 + S t; with the viscosity the scaled Laplacian of a distance
    function is about dx/r, so dr/dt = S (1 - eps dx / r).  First-order
    upwinding gives O(dx) front errors: the radius must agree within dx/20
    without viscosity and within dx/4 with it (the ODE drops O(dx^2/r^2))."""
    nxa, sr, dxa = 12, 10, 10.0
    nx = nxa * sr
    dx = dxa / sr
    c = nx * dx / 2
    x = (np.arange(nx)[None, :] + 0.5) * dx
    y = (np.arange(nx)[:, None] + 0.5) * dx
    r0 = 15.0
    psi0 = np.hypot(x - c, y - c) - r0
    o, u, v = _uniform_run(orc, nxa, nxa, sr, dxa, psi0, 0, 0.0, eps)
    S = orc.rothermel_rate(synth.nominal_class(fgi=0.5), 0.0, 0.0)
    dt = 0.25 * dx / S / 4
    steps = int(round(25.0 / S / dt))  # grow by about 25 m
    for n in range(steps):
        o.step(u, v, dt)
    T = steps * dt
    # ODE dr/dt = S (1 - eps dx / r), integrated with small RK4 steps
    r, h = r0, T / 4000
    f = lambda r: S * (1 - eps * dx / r)
    for _ in range(4000):
        k1 = f(r); k2 = f(r + h / 2 * k1); k3 = f(r + h / 2 * k2); k4 = f(r + h * k3)
        r += h / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    rad = _radius_along_axes(o.psi, dx, c)
    tol = dx / 20 if eps == 0.0 else dx / 4
    assert np.all(np.abs(rad - r) < tol), (rad, r)
    if eps == 0.0:
        assert r == pytest.approx(r0 + S * T, rel=1e-12)


@pytest.mark.parametrize("c_target", [0.1, 0.3, 0.5])
def test_checkerboard_amplification_linear_theory(orc, c_target):
    """Linear stability of eqs. (Heun), (F-disc), (Godunov) on a planar front
    psi = x with constant S, perturbed by a checkerboard d (-1)^(i+j):
    central differences do not see the checkerboard (n stays (1,0)), the
    upwind x-difference adds 2 d s/dx, the scaled Laplacian -4 d s (1/dx+1/dy)
    and the y-terms are second order, so one Euler stage multiplies the
    checkerboard by 1 + z with z = -S dt (2/dx + 4 eps (1/dx + 1/dy)), and a
    Heun step by 1 + z + z^2/2 (above 1 in magnitude when z < -2)."""
    nxa, sr, dxa, eps = 6, 8, 8.0, 0.4
    nx = nxa * sr
    dx = dxa / sr
    cls = synth.nominal_class(fgi=0.5)
    S = orc.rothermel_rate(cls, 0.0, 0.0)
    dt = c_target * dx / S
    x = (np.arange(nx)[None, :] + 0.5) * dx + np.zeros((nx, 1))
    s = (-1.0) ** (np.arange(nx)[None, :] + np.arange(nx)[:, None])
    d = 1e-7 * dx
    o, u, v = _uniform_run(orc, nxa, nxa, sr, dxa, x + 1000.0 + d * s, 0, dt, eps)
    o.step(u, v, dt)
    core = (slice(6, -6), slice(6, -6))
    pert = (o.psi - (x + 1000.0 - S * dt))[core] / (d * s[core])
    z = -S * dt * (2 / dx + 4 * eps * (1 / dx + 1 / dx))
    assert np.allclose(pert, 1 + z + z * z / 2, rtol=1e-5, atol=1e-5)


def test_synthetic_landscapes_within_stability_limit(orc):
    """The random landscapes used as workloads keep the explicit scheme stable:
    with the fastest class at the largest wind of the field and the largest
    slope, the worst linear factor z = -c (2 sqrt 2 + 8 eps) (c = S dt/dx,
    diagonal front) stays inside Heun's interval [-2, 0] with margin."""
    for seed, nxa in [(synth.BASE_SEED, 200), (21, 23), (44, 32), (33, 31)]:
        w = synth.random_landscape(nxa, nxa, seed=seed, steps=1)
        umax = float(np.hypot(np.abs(w.u).max(), np.abs(w.v).max()))
        smax = max(orc.rothermel_rate(c, umax, 0.4) for c in w.classes)
        c = smax * w.dt / w.dx
        z = -c * (2 * np.sqrt(2) + 8 * w.eps)
        assert z > -1.5, (seed, smax, z)


def test_step_is_well_conditioned_at_symmetric_points(orc):
    """Rounding-level perturbations of psi (1e-13 relative) stay at that level
    over 60 steps, also where a line ignition lies on a node column and the
    central gradient at the nodes on the line is pure rounding noise: there
    the normal is taken as zero instead of being picked by the noise."""
    w = synth.random_landscape(23, 17, seed=21, ignition="line", steps=60)
    a = orc.OracleFire.from_workload(w)
    b = orc.OracleFire.from_workload(w)
    rng = np.random.default_rng(4)
    b.psi *= 1.0 + 1e-13 * rng.standard_normal(b.psi.shape)
    for _ in range(w.steps):
        a.step(w.u, w.v, w.dt)
        b.step(w.u, w.v, w.dt)
    scale = np.abs(a.psi).max()
    assert np.abs(a.psi - b.psi).max() <= 1e-10 * scale
    assert np.abs(a.frac - b.frac).max() <= 1e-10
