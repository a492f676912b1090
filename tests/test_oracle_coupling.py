"""Pins of the oracle's coupling steps (Sect. "Coupling of the fire and the
atmospheric models"): the wind at z_f = 6.1 m by vertical log-linear
interpolation with u(z_0) = 0, and the insertion of the fire's heat fluxes
into the tendencies of mu theta and mu q_m with an exp(-z/z_ext) profile."""
import json
import math
import os

import numpy as np
import pytest

from paper_1102_1343_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
ZF = GOLD["midflame_height_m"]["z_f"]


def columns(seed=3, shape=(7, 9), nz=12):
    rng = np.random.default_rng(seed)
    return synth.atmos_columns(rng, shape, nz=nz)


def test_log_profile_is_reproduced_exactly(orc):
    """u = c ln(z/z0) is linear in ln z, so its log-linear interpolant is the
    profile itself at any height between z0 and the top level."""
    zw, z, z0, _ = columns()
    c = np.random.default_rng(4).uniform(-2.0, 2.0, z0.shape)
    u = c * np.log(z / z0)
    for zf in (ZF, 0.7, 33.0, float(z.min()) * 1.01, 1500.0):
        got = orc.wind_at_height(u, z, z0, zf)
        want = np.where(zf > z0, c * np.log(zf / z0), 0.0)
        inside = zf <= z[-1]
        assert np.allclose(got[inside], want[inside], rtol=1e-13, atol=1e-13)


def test_below_roughness_and_at_levels(orc):
    """0 at and below z0; the level's own value at a level height; the top
    value above the highest level."""
    zw, z, z0, u = columns(seed=5)
    assert np.all(orc.wind_at_height(u, z, z0, 1e-4) == 0.0)
    one = orc.wind_at_height(u, z, np.full_like(z0, ZF), ZF)
    assert np.all(one == 0.0)
    p = (2, 3)
    for k in (0, 3, len(z) - 1):
        got = orc.wind_at_height(u[:, p[0]:p[0] + 1, p[1]:p[1] + 1],
                                 z[:, p[0]:p[0] + 1, p[1]:p[1] + 1],
                                 z0[p[0]:p[0] + 1, p[1]:p[1] + 1], float(z[k][p]))
        assert got[0, 0] == pytest.approx(u[k][p], rel=1e-14, abs=1e-14)
    top = orc.wind_at_height(u, z, z0, 10.0 * float(z.max()))
    assert np.array_equal(top, u[-1])


def test_piecewise_linear_in_log_height(orc):
    """Between two levels the interpolant is a + b ln z through their values
    (below the first level: through (ln z0, 0) and the first level)."""
    z = np.array([10.0, 25.0, 70.0])[:, None]
    u = np.array([4.0, 6.5, 7.0])[:, None]
    z0 = np.array([0.1])
    for zf, (za, ua, zb, ub) in ((6.1, (0.1, 0.0, 10.0, 4.0)), (17.0, (10.0, 4.0, 25.0, 6.5)),
                                 (40.0, (25.0, 6.5, 70.0, 7.0))):
        want = ua + (ub - ua) * (math.log(zf) - math.log(za)) / (math.log(zb) - math.log(za))
        assert orc.wind_at_height(u, z, z0, zf)[0] == pytest.approx(want, rel=1e-14)


def test_levels_below_roughness_are_skipped(orc):
    """A level at or below z0 is not a point of the interpolant (u = 0 up to
    z0): the value at z_f comes from (ln z0, 0) and the next level above."""
    z = np.array([0.3, 12.0, 40.0])[:, None]
    u = np.array([9.0, 5.0, 8.0])[:, None]
    z0 = np.array([0.5])
    want = 5.0 * (math.log(ZF) - math.log(0.5)) / (math.log(12.0) - math.log(0.5))
    assert orc.wind_at_height(u, z, z0, ZF)[0] == pytest.approx(want, rel=1e-14)


def heat_inputs(seed=7, shape=(6, 8), nz=15, top=3000.0):
    rng = np.random.default_rng(seed)
    zw, z, z0, _ = synth.atmos_columns(rng, shape, nz=nz, top=top)
    rho, mu = synth.air_columns(rng, shape, zw)
    hs = rng.uniform(0.0, 5e4, shape)
    hl = rng.uniform(0.0, 2e4, shape)
    return hs, hl, zw, rho, mu


@pytest.mark.parametrize("zext", [50.0, 200.0, 5000.0])
def test_inserted_heat_integrates_to_the_surface_flux(orc, zext):
    """The column integral of sigma rho (source/mu) dz is the fire's flux
    times 1 - exp(-z_top/z_ext) (the part of the decaying flux absorbed
    below the model top): the sum over layers telescopes."""
    hs, hl, zw, rho, mu = heat_inputs()
    cp, L = 1004.0, 2.5e6
    rth, rqv = orc.heat_insertion(hs, hl, zw, rho, mu, zext, cp, L)
    dz = zw[1:] - zw[:-1]
    absorbed = 1.0 - np.exp(-zw[-1] / zext)
    assert np.allclose((cp * rho * rth / mu * dz).sum(0), hs * absorbed, rtol=1e-12)
    assert np.allclose((L * rho * rqv / mu * dz).sum(0), hl * absorbed, rtol=1e-12)
    assert np.all(rth >= 0) and np.all(rqv >= 0)


def test_thin_layers_approach_the_exponential_profile(orc):
    """With layers much thinner than z_ext the layer source is the flux
    convergence phi/z_ext exp(-z/z_ext) at the layer centre to second order
    in dz/z_ext."""
    shape = (3, 4)
    nz, zext = 400, 100.0
    zw = np.broadcast_to(np.linspace(0.0, 400.0, nz + 1)[:, None, None], (nz + 1,) + shape).copy()
    rho = np.ones((nz,) + shape)
    mu = np.ones(shape)
    hs = np.full(shape, 1004.0)
    hl = np.zeros(shape)
    rth, _ = orc.heat_insertion(hs, hl, zw, rho, mu, zext, 1004.0, 2.5e6)
    zc = 0.5 * (zw[1:] + zw[:-1])
    want = np.exp(-zc / zext) / zext
    err = np.abs(rth - want) / want
    assert err.max() <= (1.0 / zext) ** 2 * 1.0 ** 2  # (dz/z_ext)^2 / 24 with dz = 1 m


def test_sources_add_to_the_tendencies(orc):
    hs, hl, zw, rho, mu = heat_inputs(seed=9)
    base = np.random.default_rng(1).standard_normal(rho.shape)
    a, b = orc.heat_insertion(hs, hl, zw, rho, mu, 150.0)
    a2, b2 = orc.heat_insertion(hs, hl, zw, rho, mu, 150.0, rth=base, rqv=2 * base)
    assert np.allclose(a2, a + base, rtol=1e-15, atol=1e-15)
    assert np.allclose(b2, b + 2 * base, rtol=1e-15, atol=1e-15)
    z1, z2 = orc.heat_insertion(0 * hs, 0 * hl, zw, rho, mu, 150.0)
    assert np.all(z1 == 0.0) and np.all(z2 == 0.0)
