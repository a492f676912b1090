"""Pins of the oracle's fire physics (Sect. 2, Tables 1-2) against what the
paper prints and against properties of the Rothermel model."""
import json
import math
import os

import numpy as np
import pytest

from paper_1102_1343_gb300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def classes():
    rng = np.random.default_rng(7)
    return synth.random_classes(rng, n=13, chaparral_index=12)[:12] + [synth.nominal_class()]


def test_chaparral_closed_form(orc):
    """eq. (chapparal): S = min{6, max{0.03333, 1.2974 U}} for the chaparral
    class, both through the coefficient form and the direct rule."""
    g = GOLD["chaparral"]
    cls = synth.nominal_class(chaparral=1.0)
    co = orc.fuel_coefficients(cls)
    for U in np.concatenate([np.linspace(-10, 10, 401), [0.0, 0.03333 / 1.2974, 6 / 1.2974]]):
        want = min(g["upper_m_per_s"], max(g["lower_m_per_s"], g["slope_per_wind"] * U))
        assert orc.spread_rate(co, U, 0.3) == pytest.approx(want, rel=1e-14, abs=1e-15)
        assert orc.rothermel_rate(cls, U, 0.3) == pytest.approx(want, rel=1e-14, abs=1e-15)


@pytest.mark.parametrize("k", range(13))
def test_coefficient_form_equals_direct_chain(orc, k):
    """eq. (spread-WRF-Fire) with the stored coefficients reproduces
    S = R0 (1 + phi_W + phi_S) of eq. (spread) evaluated directly through
    Table 2 in English units (wind converted inside the chain, limits of the
    caption of Table 2 applied to the raw inputs)."""
    cls = classes()[k]
    co = orc.fuel_coefficients(cls)
    for U in [-3.0, 0.0, 1e-3, 0.5, 2.0, 7.5, 29.9, 30.0, 45.0]:
        for tp in [-0.5, 0.0, 0.05, 0.2, 0.7]:
            a = orc.spread_rate(co, U, tp)
            b = orc.rothermel_rate(cls, U, tp)
            assert a == pytest.approx(b, rel=1e-12, abs=1e-300)


def test_rothermel_invariants(orc):
    """Properties of the Rothermel model with the CAWFE limits:
    S(U<=0, tan<=0) = R0 > 0; S increases with U on [0, 30] and with the slope;
    constant for U >= 30 m/s; decreases with moisture; zero at or above the
    moisture of extinction."""
    lim = GOLD["wind_limits"]["wind_max_m_per_s"]
    for cls in classes():
        co = orc.fuel_coefficients(cls)
        R0 = co[1]
        assert R0 > 0
        assert orc.spread_rate(co, -2.0, -0.3) == R0
        assert orc.spread_rate(co, 0.0, 0.0) == R0
        Us = np.linspace(0.0, lim, 31)
        S = [orc.spread_rate(co, U, 0.0) for U in Us]
        assert all(np.diff(S) > 0)
        assert orc.spread_rate(co, lim + 5, 0.0) == pytest.approx(S[-1], rel=1e-15)
        T = [orc.spread_rate(co, 0.0, t) for t in np.linspace(0, 1, 11)]
        assert all(np.diff(T) > 0)
        Ms = np.linspace(0.01, cls["fuelmce"] * 0.99, 12)
        R = [orc.fuel_coefficients(cls, Mf=m)[1] for m in Ms]
        assert all(np.diff(R) < 0)
        assert orc.fuel_coefficients(cls, Mf=cls["fuelmce"])[1] == 0.0
        assert orc.rothermel_rate(cls, 5.0, 0.2, Mf=cls["fuelmce"] * 1.5) == 0.0


def test_no_fuel_does_not_spread(orc):
    cls = synth.nominal_class(fgi=0.0)
    co = orc.fuel_coefficients(cls)
    assert orc.spread_rate(co, 10.0, 0.5) == 0.0
    assert co[7] == 0.0 and co[8] == 0.0


def test_burn_time_from_weight(orc):
    """Sect. 'Fuel burned and heat released': w = 1000 leaves 0.6 of the fuel
    after 600 s, and T_f is approximately w/0.8514 (4 printed digits)."""
    g = GOLD["burn_time"]
    Tf = orc.fuel_coefficients(synth.nominal_class(weight=g["w_reference"]))[6]
    assert math.exp(-600.0 / Tf) == pytest.approx(g["remaining_after_600s"], rel=1e-14)
    for w in [7.0, 50.0, 180.0, 1000.0]:
        Tf = orc.fuel_coefficients(synth.nominal_class(weight=w))[6]
        assert w / Tf == pytest.approx(g["w_over_Tf_printed"], abs=0.5e-4)
    assert orc.fuel_coefficients(synth.nominal_class(weight=60.0, weight_is_tf=1.0))[6] == 60.0


def test_heat_factor_ratio(orc):
    """eqs. (sensible-heat-flux), (latent-heat-flux): the latent/sensible
    ratio is (M_f + 0.56) L / h, independent of the load."""
    g = GOLD["latent_heat"]
    for cls in classes():
        co = orc.fuel_coefficients(cls)
        want = (cls["fuelmc_g"] + g["water_ratio"]) * g["L_J_per_kg"] / cls["cmbcnst"]
        assert co[8] / co[7] == pytest.approx(want, rel=1e-14)
        # sensible factor: heat content of the dry part of the load
        assert co[7] == pytest.approx(cls["fgi"] * cls["cmbcnst"] / (1 + cls["fuelmc_g"]),
                                      rel=1e-14)


def test_spread_rate_magnitude_plausible(orc):
    """Grass-like nominal class: no-wind rate of a few cm/s and a head rate of
    order 0.1 m/s in a 3 m/s wind (order of magnitude of BEHAVE grass fires).
    A sanity check of the unit conversions, not a pin of the value."""
    cls = synth.nominal_class(fgi=0.5, fuelmc_g=0.08)
    R0 = orc.rothermel_rate(cls, 0.0, 0.0)
    assert 0.005 < R0 < 0.1
    S3 = orc.rothermel_rate(cls, 3.0, 0.0)
    assert 0.05 < S3 < 1.0
