"""Pins of the oracle's reference adjoint of the arrival-time misfit
J = 1/2 sum over nodes ignited in both runs of (t_i - t_obs)^2 (the data
assimilation use of Sect. 7 that motivates the level-set formulation):

- d(coefficients)/d(M_f) against central differences of the Table 2 chain;
- a planar front under uniform spread rate, where the discrete scheme moves
  the front exactly at S, so t_i = t0 + (x - x0)/(m S) and the derivative of J
  along a uniform change of the multiplier, the moisture or the wind has a
  closed form (the sum of the per-node / per-face gradient);
- central finite differences along random directions on a random landscape
  (wind, slope, patchy fuel), away from switch points (the set of ignited nodes
  is the same in the perturbed runs);
- a zero misfit gives a zero gradient;
- the dot-product test of one linearised step, <J v, w> = <v, J^T w>, for
  directions of the state, the multiplier and the moisture.
"""
import numpy as np
import pytest

import oracle
from paper_1102_1343_gb300 import synth


def test_coefficient_moisture_derivative_matches_fd(orc):
    rng = np.random.default_rng(5)
    classes = synth.random_classes(rng) + [synth.nominal_class()]
    for c in classes:
        Mf = c["fuelmc_g"]
        d = orc.fuel_coefficients_dMf(c)
        h = 1e-6
        fd = (orc.fuel_coefficients(c, Mf + h) - orc.fuel_coefficients(c, Mf - h)) / (2 * h)
        scale = np.maximum(np.abs(fd), 1e-12)
        assert np.all(np.abs(d - fd) <= 1e-6 * scale + 1e-14), (c, d, fd)
        # b, e, T_f and S0 do not depend on the moisture
        assert d[2] == 0.0 and d[5] == 0.0 and d[6] == 0.0 and d[0] == 0.0
    chap = synth.nominal_class(chaparral=1.0)
    d = orc.fuel_coefficients_dMf(chap)
    assert np.all(d[:7] == 0.0)


def planar_case(U0):
    """Planar front x = x0 moving in +x on a flat, uniform-fuel mesh of 1 m
    cells; uniform wind (U0, 0)."""
    nxa, nya, sr = 12, 2, 10
    dx_atm = 10.0
    cls = [synth.nominal_class()]
    nx, ny = nxa * sr, nya * sr
    fuel = np.zeros((ny, nx), np.uint8)
    z = np.zeros((ny, nx))
    co = oracle.fuel_coefficients(cls[0])
    S = oracle.spread_rate(co, U0, 0.0)
    dt = 0.25 / S  # z = -S dt (2/dx + 4 eps 2/dx) = -1.3: stable
    fire = oracle.OracleFire(nxa, nya, sr, dx_atm, cls, fuel, z, z.copy(), ignitions=[],
                             mult=np.ones((ny, nx)))
    x = (np.arange(nx) + 0.5) * 1.0
    x0 = 70.3
    psi = np.broadcast_to(x - x0, (ny, nx)).copy()
    tign = np.where(psi <= 0, 0.0, np.inf)
    fire.set_state(psi, tign, np.ones((ny, nx)), 0.0)
    u = np.full((nya, nxa + 1), U0)
    v = np.zeros((nya + 1, nxa))
    return fire, cls, co, S, dt, u, v, x, x0


@pytest.mark.parametrize("U0", [0.0, 3.0])
def test_planar_front_uniform_directions_closed_form(orc, U0):
    fire, cls, co, S, dt, u, v, x, x0 = planar_case(U0)
    nsteps = 24
    ny, nx = fire.ny, fire.nx
    # observations from a slower front: residuals of both signs along x
    tobs = np.broadcast_to((x - x0) / (0.9 * S) - 2.0 * dt, (ny, nx)).copy()
    J, gm, gM, gu, gv = fire.adjoint(u, v, dt, nsteps, tobs)
    ti = fire.tign
    ign = np.isfinite(ti) & (fire.psi <= 0) & (np.broadcast_to(x, (ny, nx)) > x0)
    assert ign.sum() >= 5 * ny  # several columns crossed
    # the scheme moves the planar front exactly at S
    expect_t = np.broadcast_to((x - x0) / S, (ny, nx))
    assert np.max(np.abs(ti[ign] - expect_t[ign])) < 1e-9
    r = np.where(ign, ti - tobs, 0.0)
    dti_dS = -(np.broadcast_to(x, (ny, nx)) - x0) / S ** 2  # dt_i/dS at each crossed node
    # uniform multiplier: dS/dm = S
    want_m = np.sum(r * dti_dS * S)
    assert abs(gm.sum() - want_m) <= 1e-8 * abs(want_m)
    # uniform moisture: dS/dM_f = dR0 + dc U^b (+ dd tan^2 = 0), by central
    # differences of the coefficient chain
    h = 1e-6
    Mf = cls[0]["fuelmc_g"]
    cp = orc.fuel_coefficients(cls[0], Mf + h)
    cm = orc.fuel_coefficients(cls[0], Mf - h)
    dS = (orc.spread_rate(cp, U0, 0.0) - orc.spread_rate(cm, U0, 0.0)) / (2 * h)
    want_M = np.sum(r * dti_dS * dS)
    assert abs(gM.sum() - want_M) <= 1e-6 * abs(want_M)
    # uniform wind u (every face): dS/dU; v is perpendicular to the normal
    if U0 > 0:
        dSdU = (orc.spread_rate(co, U0 + 1e-5, 0.0) - orc.spread_rate(co, U0 - 1e-5, 0.0)) / 2e-5
        want_u = np.sum(r * dti_dS * dSdU)
        assert abs(gu.sum() - want_u) <= 1e-6 * abs(want_u)
    else:
        # max{0, U} has a kink at 0: one-sided (frozen) derivative 0
        assert gu.sum() == 0.0
    assert np.max(np.abs(gv)) <= 1e-12 * np.max(np.abs(gu) + 1.0)
    # J itself
    assert abs(J - 0.5 * np.sum(np.where(np.isfinite(ti), (ti - tobs) ** 2, 0.0))) <= 1e-12 * J


def landscape(seed=7, nxa=8, nya=8, sr=5, dx_atm=10.0, dy_atm=None):
    """Small random landscape (2 m cells; dy_atm != dx_atm gives anisotropic
    cells) with a centred ignition; with the multiplier 3 used below the
    front crosses several cells in 60 steps of 0.25 s."""
    w = synth.random_landscape(nxa, nya, sr=sr, dx_atm=dx_atm, seed=seed, ignition="center",
                               steps=60, dt=0.25)
    if dy_atm is not None:
        w.dy_atm = dy_atm
    # no chaparral class (its rate does not depend on the moisture, fine, but
    # its 6 m/s cap needs a smaller step)
    for c in w.classes:
        c["chaparral"] = 0.0
    return w


def run_J(w, mult, moist, u, v, nsteps, tobs):
    f = oracle.OracleFire.from_workload(w, mult=mult, moisture=moist)
    for _ in range(nsteps):
        f.step(u, v, w.dt)
    ok = np.isfinite(f.tign) & np.isfinite(tobs)
    return 0.5 * np.sum((f.tign[ok] - tobs[ok]) ** 2), np.isfinite(f.tign)


@pytest.mark.parametrize("dy_atm", [None, 14.0])
def test_gradient_matches_central_differences(orc, dy_atm):
    w = landscape(dy_atm=dy_atm)
    nsteps = 60
    ny, nx = w.ny, w.nx
    rng = np.random.default_rng(11)
    mult = 3.0 * (1.0 + 0.05 * rng.standard_normal((ny, nx)))
    moist = np.array([w.classes[c]["fuelmc_g"] for c in w.fuel.ravel()]).reshape(ny, nx)
    # truth: stronger fire, drier fuel, stronger wind
    truth_mult = mult * 1.2
    f = oracle.OracleFire.from_workload(w, mult=truth_mult, moisture=moist - 0.02)
    for _ in range(nsteps):
        f.step(w.u * 1.1, w.v * 1.1, w.dt)
    tobs = np.where(np.isfinite(f.tign), f.tign, np.nan)

    base = oracle.OracleFire.from_workload(w, mult=mult, moisture=moist)
    J, gm, gM, gu, gv = base.adjoint(w.u, w.v, w.dt, nsteps, tobs)
    J0, ign0 = run_J(w, mult, moist, w.u, w.v, nsteps, tobs)
    assert abs(J - J0) <= 1e-12 * J0
    assert J > 0 and np.count_nonzero(np.isfinite(tobs) & ign0) > 20

    checked, worst = 0, 0.0
    for q in range(8):
        dm = rng.standard_normal((ny, nx))
        dM = rng.standard_normal((ny, nx))
        du = rng.standard_normal(w.u.shape)
        dv = rng.standard_normal(w.v.shape)
        for which in ("m", "M", "u", "v"):
            h = 1e-6
            args_p = [mult, moist, w.u, w.v]
            args_m = [mult, moist, w.u, w.v]
            k = "mMuv".index(which)
            d = (dm, dM * 0.01, du, dv)[k]
            args_p[k] = args_p[k] + h * d
            args_m[k] = args_m[k] - h * d
            Jp, ip = run_J(w, *args_p, nsteps, tobs)
            Jm, im = run_J(w, *args_m, nsteps, tobs)
            if not (np.array_equal(ip, ign0) and np.array_equal(im, ign0)):
                continue  # a node entered or left the ignited set: switch point
            fd = (Jp - Jm) / (2 * h)
            g = (gm, gM, gu, gv)[k]
            ad = float(np.sum(g * d))
            assert abs(fd - ad) <= 1e-6 * max(abs(fd), 1e-3 * J), (which, q, fd, ad)
            worst = max(worst, abs(fd - ad) / max(abs(fd), 1e-3 * J))
            checked += 1
    print("checked", checked, "worst rel", worst)
    assert checked >= 28


def test_zero_misfit_zero_gradient(orc):
    w = landscape(seed=8)
    nsteps = 20
    w.mult = np.full((w.ny, w.nx), 3.0)
    f = oracle.OracleFire.from_workload(w)
    for _ in range(nsteps):
        f.step(w.u, w.v, w.dt)
    tobs = np.where(np.isfinite(f.tign), f.tign, np.nan)
    g = oracle.OracleFire.from_workload(w)
    J, gm, gM, gu, gv = g.adjoint(w.u, w.v, w.dt, nsteps, tobs)
    assert J == 0.0
    for a in (gm, gM, gu, gv):
        assert np.all(a == 0.0)
    # the adjoint call advanced the state exactly like the plain steps
    assert np.array_equal(g.psi, f.psi) and np.array_equal(g.tign, f.tign)
    assert np.array_equal(g.frac, f.frac) and g.t == f.t


@pytest.mark.parametrize("dy_atm", [None, 14.0])
def test_step_vjp_dot_product(orc, dy_atm):
    """Dot-product test of the linearised level-set step: <J v, w> from
    central differences of the forward step equals <v, J^T w> from the
    reverse step (orc_step_vjp), for random directions v of the state psi,
    the multiplier and the moisture and a random cotangent w.  Directions
    whose +-h steps straddle a switch point (a Godunov selection, a clamp,
    a zeroed central difference) show up as central differences that
    change when h is halved; those are skipped."""
    w = landscape(dy_atm=dy_atm)
    ny, nx = w.ny, w.nx
    rng = np.random.default_rng(23)
    mult = 3.0 * (1.0 + 0.05 * rng.standard_normal((ny, nx)))
    moist = np.array([w.classes[c]["fuelmc_g"] for c in w.fuel.ravel()]).reshape(ny, nx)
    f = oracle.OracleFire.from_workload(w, mult=mult, moisture=moist)
    for _ in range(30):
        f.step(w.u, w.v, w.dt)
    psi0, tign0, frac0, t0 = f.psi.copy(), f.tign.copy(), f.frac.copy(), f.t

    def step_psi(psi, m, M):
        g = oracle.OracleFire(w.nxa, w.nya, w.srx, w.dx_atm, w.classes, w.fuel, w.dzdx, w.dzdy,
                              [], moisture=M, mult=m, dy_atm=w.dy_atm)
        g.set_state(psi, tign0, frac0, t0)
        g.step(w.u, w.v, w.dt)
        return g.psi

    cot = rng.standard_normal((ny, nx))
    lam, gm, gM, _, _ = f.step_vjp(w.u, w.v, w.dt, cot)
    assert np.abs(lam).max() > 0 and np.abs(gm).max() > 0 and np.abs(gM).max() > 0
    checked, worst = 0, 0.0
    for q in range(6):
        for which in ("psi", "m", "M"):
            d = rng.standard_normal((ny, nx)) * (0.01 if which == "M" else 1.0)
            fd = []
            for h in (1e-6, 5e-7):
                args_p = [psi0, mult, moist]
                args_m = [psi0, mult, moist]
                k = ("psi", "m", "M").index(which)
                args_p[k] = args_p[k] + h * d
                args_m[k] = args_m[k] - h * d
                fd.append(float(np.sum((step_psi(*args_p) - step_psi(*args_m)) * cot)) / (2 * h))
            if abs(fd[0] - fd[1]) > 1e-6 * max(abs(fd[0]), 1e-12):
                continue  # a switch point within the step
            ad = float(np.sum(d * (lam, gm, gM)[("psi", "m", "M").index(which)]))
            err = abs(fd[0] - ad) / max(abs(fd[0]), 1e-12)
            # central differences agree to ~1e-6 here (truncation); an
            # error of the transposition would be of order one
            assert err <= 1e-5, (which, q, fd, ad)
            worst = max(worst, err)
            checked += 1
    print("checked", checked, "worst rel", worst)
    assert checked >= 12


# ---------------------------------------------------------------------------
# heat misfit: Q = sensible heat released per unit area of each atmospheric
# cell over the run, J = 1/2 sum (Q - q_obs)^2
# ---------------------------------------------------------------------------

def released_heat(w, mult, moist, u, v, nsteps):
    """Q per atmospheric cell as the time integral of the step's sensible
    heat flux output (eqs. sensible-heat-flux, average)."""
    f = oracle.OracleFire.from_workload(w, mult=mult, moisture=moist)
    Q = np.zeros((w.nya, w.nxa))
    for _ in range(nsteps):
        hs, _, _ = f.step(u, v, w.dt)
        Q += hs * w.dt
    return Q


def heat_case(seed=7, dy_atm=None, corner=False):
    """The small landscape; corner=True ignites at the domain corner instead,
    so that the quadrature's ghost nodes (x, y and corner) carry ignition
    times."""
    w = landscape(seed=seed, dy_atm=dy_atm)
    if corner:
        w.ignitions = [synth.point_ignition(1.0, 1.0, radius=7.0)]
    rng = np.random.default_rng(seed + 40)
    mult = 3.0 * (1.0 + 0.05 * rng.standard_normal((w.ny, w.nx)))
    moist = np.array([w.classes[c]["fuelmc_g"] for c in w.fuel.ravel()]).reshape(w.ny, w.nx)
    return w, mult, moist


def test_heat_objective_is_the_integrated_heat_flux(orc):
    """J with observations Q_flux + delta equals 1/2 sum delta^2: the Q of the
    objective (from the fuel fractions at the start and the end) is the time
    integral of the step's heat flux output (the sum telescopes)."""
    w, mult, moist = heat_case()
    nsteps = 40
    Q = released_heat(w, mult, moist, w.u, w.v, nsteps)
    assert Q.max() > 0
    rng = np.random.default_rng(1)
    delta = rng.standard_normal(Q.shape) * Q.max()
    f = oracle.OracleFire.from_workload(w, mult=mult, moisture=moist)
    J, *_ = f.adjoint_heat(w.u, w.v, w.dt, nsteps, Q + delta)
    assert abs(J - 0.5 * np.sum(delta ** 2)) <= 1e-9 * J
    # unobserved cells do not count
    qobs = Q + delta
    qobs[0, :] = np.nan
    g = oracle.OracleFire.from_workload(w, mult=mult, moisture=moist)
    J2, *_ = g.adjoint_heat(w.u, w.v, w.dt, nsteps, qobs)
    assert abs(J2 - 0.5 * np.sum(delta[1:] ** 2)) <= 1e-9 * J2


def test_heat_misfit_zero_gives_zero_gradient(orc):
    w, mult, moist = heat_case(seed=8)
    nsteps = 30
    Q = released_heat(w, mult, moist, w.u, w.v, nsteps)
    f = oracle.OracleFire.from_workload(w, mult=mult, moisture=moist)
    J, gm, gM, gu, gv = f.adjoint_heat(w.u, w.v, w.dt, nsteps, Q)
    g = oracle.OracleFire.from_workload(w, mult=mult, moisture=moist)
    J1, gm1, gM1, gu1, gv1 = g.adjoint_heat(w.u, w.v, w.dt, nsteps, Q * 0.9)
    assert J <= 1e-24 * max(J1, 1.0)
    for a, b in ((gm, gm1), (gM, gM1), (gu, gu1), (gv, gv1)):
        assert np.abs(a).max() <= 1e-9 * np.abs(b).max()


@pytest.mark.parametrize("dy_atm,corner", [(None, False), (14.0, False), (None, True)])
def test_heat_gradient_matches_central_differences(orc, dy_atm, corner):
    """Central differences of J_heat along random directions of the
    multiplier, the moisture and the wind; directions whose +-h runs cross a
    switch point (ignited set, quadrature branches) show up as differences
    that change when h is halved, and are skipped."""
    w, mult, moist = heat_case(dy_atm=dy_atm, corner=corner)
    nsteps = 50
    # observations: a truth run with a stronger fire, drier fuel, more wind
    qobs = released_heat(w, mult * 1.2, moist - 0.02, w.u * 1.1, w.v * 1.1, nsteps)
    base = oracle.OracleFire.from_workload(w, mult=mult, moisture=moist)
    J, gm, gM, gu, gv = base.adjoint_heat(w.u, w.v, w.dt, nsteps, qobs)
    assert J > 0

    def J_at(m, M, u, v):
        f = oracle.OracleFire.from_workload(w, mult=m, moisture=M)
        Jv, *_ = f.adjoint_heat(u, v, w.dt, nsteps, qobs)
        return Jv

    rng = np.random.default_rng(17)
    checked, worst = 0, 0.0
    for q in range(8):
        dirs = {"m": rng.standard_normal((w.ny, w.nx)),
                "M": rng.standard_normal((w.ny, w.nx)) * 0.01,
                "u": rng.standard_normal(w.u.shape),
                "v": rng.standard_normal(w.v.shape)}
        for name, d in dirs.items():
            k = "mMuv".index(name)
            fd = []
            for h in (1e-6, 5e-7):
                ap = [mult, moist, w.u, w.v]
                am = [mult, moist, w.u, w.v]
                ap[k] = ap[k] + h * d
                am[k] = am[k] - h * d
                fd.append((J_at(*ap) - J_at(*am)) / (2 * h))
            if abs(fd[0] - fd[1]) > 1e-6 * max(abs(fd[0]), 1e-3 * J):
                continue
            ad = float(np.sum((gm, gM, gu, gv)[k] * d))
            err = abs(fd[0] - ad) / max(abs(fd[0]), 1e-3 * J)
            assert err <= 1e-5, (name, q, fd, ad)
            worst = max(worst, err)
            checked += 1
    print("checked", checked, "worst rel", worst)
    assert checked >= 20


@pytest.mark.parametrize("shape", [(6, 5), (2, 2), (9, 3)])
def test_extend_vjp_dot_product(orc, shape):
    """The transpose of the ghost extension (x ghosts, then y ghosts over the
    extended rows, corners included) used by the heat adjoint:
    <extend(a + h v) - extend(a - h v), D> / 2h = <v, extend^T D>.  The
    extension is piecewise linear, so away from its kinks (fields without
    ties in the ghosts' max) the two agree to rounding; fields of each branch
    type are tried."""
    ny, nx = shape
    rng = np.random.default_rng(nx * 10 + ny)
    for field in ("random", "linear", "bowl"):
        y, x = np.mgrid[0:ny, 0:nx]
        a = {"random": rng.standard_normal((ny, nx)),
             "linear": 0.7 * x - 0.3 * y + 0.1,          # 2 p0 - p1 branch
             # off-centre, so that no ghost sits on a tie of its max
             "bowl": (x - nx / 2.0 - 0.37) ** 2 + (y - ny / 2.0 - 0.21) ** 2}[field]
        for _ in range(4):
            v = rng.standard_normal((ny, nx))
            D = rng.standard_normal((ny + 2, nx + 2))
            h = 1e-7
            ep, em = oracle.extend(a + h * v), oracle.extend(a - h * v)
            lhs = float(np.sum((ep - em) * D)) / (2 * h)
            rhs = float(np.sum(v * oracle.extend_vjp(a, D)))
            assert abs(lhs - rhs) <= 1e-6 * max(1.0, abs(rhs)), (field, lhs, rhs)
