"""Pins of the oracle's Rothermel chain (Table 2 of the paper), step by step.

The oracle evaluates Table 2 in English units (BTU-lb-ft-min), as the
table's caption prescribes.  These tests pin it without reusing its code:

* the chain restated here in SI units, every constant taken from the paper's
  printed Table 2 (``golden/rothermel_table2.json``) and converted by its
  dimension with the exact unit definitions, so that a wrong constant, a wrong
  unit or a conversion in the wrong direction in the oracle shows up;
* exact properties of the model that hold whatever the constants: the
  optimum packing ratio maximises the reaction velocity, the moisture
  damping is 1 for dry fuel and vanishes at the moisture of extinction, the
  heat balance of Eq. (52);
* a round trip of a class given in English units through the oracle's
  metric input;
* planted mistakes: copies of the oracle source, each with one plausible
  slip (a swapped constant, a flipped sign, a unit), must fail at least one
  of the pins above.
"""
import ctypes as C
import json
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1102_1343_gb300 import synth

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "rothermel_table2.json")))
U_ = G["units"]
FT = U_["m_per_ft"]          # m per ft
LB = U_["kg_per_lb"]         # kg per lb
BTU = U_["J_per_BTU"]        # J per BTU
MIN = U_["s_per_min"]        # s per min


def classes():
    rng = np.random.default_rng(11)
    out = [synth.nominal_class(), synth.nominal_class(fgi=1.2, fueldepthm=0.9, fuelmc_g=0.15,
                                                        fuelmce=0.3, savr=1500 / FT)]
    out += synth.random_classes(rng, n=8, chaparral_index=None)
    return out


# ---------------------------------------------------------------------------
# the chain in SI units (sigma in 1/m, loads in kg/m^2, ...), constants of the
# printed table converted by their dimensions
# ---------------------------------------------------------------------------
def si_chain(cls, Mf=None):
    Mf = cls["fuelmc_g"] if Mf is None else Mf
    s = cls["savr"]                         # 1/m; the table's sigma (1/ft) is FT * s
    k = FT
    w0 = cls["fgi"] / (1.0 + Mf)            # kg/m^2
    rho_b = w0 / cls["fueldepthm"]          # kg/m^3
    beta = rho_b / cls["fueldens"]
    nb = G["not_printed"]
    beta_op = nb["beta_op_a"] * k ** nb["beta_op_p"] * s ** nb["beta_op_p"]
    a = G["A"]
    A = 1.0 / (a["a"] * k ** a["p"] * s ** a["p"] - a["b"])
    gm = G["Gmax"]
    s15 = (k * s) ** gm["p"]
    Gmax = s15 / (gm["d0"] + gm["d1"] * s15) / MIN        # 1/s
    r = beta / beta_op
    Gamma = Gmax * r ** A * math.exp(A * (1.0 - r))
    wn = w0 / (1.0 + cls["st"])
    m = G["etaM"]
    rm = Mf / cls["fuelmce"]
    etaM = m["c0"] + m["c1"] * rm + m["c2"] * rm ** 2 + m["c3"] * rm ** 3
    etaM = min(1.0, max(0.0, etaM)) if rm < 1.0 else 0.0
    etaS = G["etaS"]["k"] * cls["se"] ** G["etaS"]["p"]
    IR = Gamma * wn * cls["cmbcnst"] * etaM * etaS        # W/m^2
    x = G["xi"]
    xi = (math.exp((x["a"] + x["b"] * (k * s) ** x["p"]) * (beta + x["beta_shift"]))
          / (x["d0"] + x["d1"] * k * s))
    eps = math.exp(-(G["eps"]["c_per_ft"] / k) / s)      # 138 per ft = 138/0.3048 per m
    q = G["Qig"]
    Qig = (q["c0"] + q["c1"] * Mf) * BTU / LB             # J/kg
    R0 = IR * xi / (rho_b * eps * Qig)                    # m/s
    c = G["C"]
    Cw = c["a"] * math.exp(-c["b"] * (k * s) ** c["p"])
    B = nb["B_a"] * (k * s) ** nb["B_p"]
    e = G["E"]
    E = e["a"] * math.exp(-e["b"] * k * s)
    return dict(w0=w0, rho_b=rho_b, beta=beta, beta_op=beta_op, A=A, Gmax=Gmax, Gamma=Gamma,
                wn=wn, etaM=etaM, etaS=etaS, IR=IR, xi=xi, eps=eps, Qig=Qig, R0=R0, C=Cw, B=B,
                E=E)


def si_rate(cls, U, tanphi, Mf=None):
    """S = R0 (1 + phi_W + phi_S) (eq. spread) with the limits of the caption."""
    p = si_chain(cls, Mf)
    lim = G["limits"]["wind_max_m_per_s"]
    Ul = min(max(U, 0.0), lim)
    tp = max(tanphi, 0.0)
    Ua = cls["windrf"] * Ul * MIN / FT                    # ft/min
    phiW = p["C"] * Ua ** p["B"] * (p["beta"] / p["beta_op"]) ** (-p["E"])
    phiS = G["phiS"]["a"] * p["beta"] ** G["phiS"]["p"] * tp * tp
    return p["R0"] * (1.0 + phiW + phiS)


# the oracle's intermediates converted to SI with the exact unit definitions
def oracle_si(cls, Mf=None, library=None):
    o = oracle.rothermel_intermediates(cls, Mf, library=library)
    return dict(w0=o["w0"] * LB / FT ** 2, rho_b=o["rho_b"] * LB / FT ** 3, beta=o["beta"],
                beta_op=o["beta_op"], A=o["A"], Gmax=o["Gmax"] / MIN, Gamma=o["Gamma"] / MIN,
                wn=o["wn"] * LB / FT ** 2, etaM=o["etaM"], etaS=o["etaS"],
                IR=o["IR"] * BTU / (FT ** 2 * MIN), xi=o["xi"], eps=o["eps"],
                Qig=o["Qig"] * BTU / LB, R0=o["R0_ftmin"] * FT / MIN, C=o["C"], B=o["B"],
                E=o["E"])


def _coefficients(cls, library=None, Mf=None):
    if library is None:
        return oracle.fuel_coefficients(cls, Mf)
    v = oracle.fuel_vector(cls)
    out = np.zeros(9)
    library.orc_fuel_coefficients(v.ctypes.data_as(C.POINTER(C.c_double)),
                                  -1.0 if Mf is None else float(Mf),
                                  out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def _spread(co, U, tp):
    """eq. (spread-WRF-Fire) from a coefficient vector (S0 R0 b c d e ...)."""
    Ue = min(max(U, 0.0), co[5])
    return max(co[0], co[1] + co[3] * Ue ** co[2] + co[4] * max(tp, 0.0) ** 2)


# ---------------------------------------------------------------------------
# pins (each takes an oracle build, so that the planted mistakes can run them)
# ---------------------------------------------------------------------------
def check_si_chain(library=None):
    for cls in classes():
        for Mf in (None, 0.0, 0.5 * cls["fuelmce"]):
            want, got = si_chain(cls, Mf), oracle_si(cls, Mf, library)
            for key, w in want.items():
                assert got[key] == pytest.approx(w, rel=1e-12, abs=1e-300), key


def check_si_rate(library=None):
    for cls in classes():
        co = _coefficients(cls, library)
        for U in (0.0, 0.3, 2.0, 9.0, 29.0, 40.0):
            for tp in (0.0, 0.1, 0.45):
                assert _spread(co, U, tp) == pytest.approx(si_rate(cls, U, tp), rel=1e-12)


def check_english_round_trip(library=None):
    """A class defined in English units, converted to the oracle's metric
    input here (English -> SI, the opposite direction of the oracle's own
    conversion), comes back with the English values."""
    eng = dict(sigma=2750.0, wl=0.092, depth=1.4, rho_p=32.0, h=8000.0)
    cls = synth.nominal_class(savr=eng["sigma"] / FT, fgi=eng["wl"] * LB / FT ** 2,
                              fueldepthm=eng["depth"] * FT, fueldens=eng["rho_p"] * LB / FT ** 3,
                              cmbcnst=eng["h"] * BTU / LB)
    o = oracle.rothermel_intermediates(cls, library=library)
    for key, w in eng.items():
        assert o[key] == pytest.approx(w, rel=1e-13), key


def check_optimum_packing_ratio(library=None):
    """Eq. (36): Gamma = Gamma_max exactly at beta = beta_op and below it at
    every other packing ratio (beta_op is the optimum); the depth sets beta."""
    for cls in classes()[:5]:
        o = oracle.rothermel_intermediates(cls, library=library)
        w0 = o["wl"] / (1.0 + cls["fuelmc_g"])
        depth_op_ft = w0 / (o["rho_p"] * o["beta_op"])       # beta = beta_op
        at = oracle.rothermel_intermediates(dict(cls, fueldepthm=depth_op_ft * FT),
                                            library=library)
        assert at["beta"] == pytest.approx(at["beta_op"], rel=1e-13)
        assert at["Gamma"] == pytest.approx(at["Gmax"], rel=1e-12)
        for f in (0.2, 0.5, 0.8, 0.95, 1.05, 1.5, 3.0, 10.0):
            off = oracle.rothermel_intermediates(dict(cls, fueldepthm=depth_op_ft * FT * f),
                                                 library=library)
            assert off["Gamma"] < at["Gamma"] * (1.0 - 1e-6), f
        # the maximum over a fine scan of depths sits at beta/beta_op = 1
        fs = np.exp(np.linspace(-1.0, 1.0, 201))
        g = [oracle.rothermel_intermediates(dict(cls, fueldepthm=depth_op_ft * FT * f),
                                            library=library)["Gamma"] for f in fs]
        assert abs(math.log(fs[int(np.argmax(g))])) <= 0.011


def check_moisture_damping(library=None):
    """Eq. (29): eta_M = 1 for dry fuel, and it falls continuously to 0 at the
    moisture of extinction (the coefficients sum to zero), so R0 -> 0."""
    for cls in classes()[:5]:
        Mx = cls["fuelmce"]
        assert oracle.rothermel_intermediates(cls, 0.0, library=library)["etaM"] == 1.0
        for d in (1e-4, 1e-6):
            near = oracle.rothermel_intermediates(cls, Mx * (1.0 - d), library=library)
            assert 0.0 <= near["etaM"] <= 3.0 * d, d
        e = [oracle.rothermel_intermediates(cls, m, library=library)["etaM"]
             for m in np.linspace(0.0, Mx * 0.999, 50)]
        assert all(np.diff(e) < 0)


def check_mineral_damping(library=None):
    """Eq. (30) at the usual effective mineral content S_E = 0.010:
    0.174 * 0.01^-0.19 = 0.174 * 10^0.38 (about 0.42)."""
    o = oracle.rothermel_intermediates(synth.nominal_class(se=0.010), library=library)
    assert o["etaS"] == pytest.approx(0.174 * 10.0 ** 0.38, rel=1e-14)
    assert 0.41 < o["etaS"] < 0.42


def check_heat_balance(library=None):
    """Eq. (52): R0 rho_b eps Q_ig = I_R xi and I_R = Gamma w_n h eta_M eta_S;
    w_0 = w_l/(1+M_f), w_n = w_0/(1+S_T), rho_b = w_0/delta, beta = rho_b/rho_P."""
    for cls in classes():
        o = oracle.rothermel_intermediates(cls, library=library)
        assert o["R0_ftmin"] * o["rho_b"] * o["eps"] * o["Qig"] == pytest.approx(
            o["IR"] * o["xi"], rel=1e-13)
        assert o["IR"] == pytest.approx(o["Gamma"] * o["wn"] * o["h"] * o["etaM"] * o["etaS"],
                                        rel=1e-13)
        assert o["w0"] == pytest.approx(o["wl"] / (1 + cls["fuelmc_g"]), rel=1e-14)
        assert o["wn"] == pytest.approx(o["w0"] / (1 + cls["st"]), rel=1e-14)
        assert o["rho_b"] == pytest.approx(o["w0"] / o["depth"], rel=1e-14)
        assert o["beta"] == pytest.approx(o["rho_b"] / o["rho_p"], rel=1e-14)


def check_wind_factor_unit_speed(library=None):
    """Eq. (47) at a midflame wind of exactly 1 ft/min: phi_W = C
    (beta/beta_op)^(-E) whatever B is; at 2 ft/min it is 2^B times that.  The
    6.1 m wind giving U_a = 1 ft/min is U = (0.3048/60)/a m/s."""
    for cls in classes()[:5]:
        o = oracle.rothermel_intermediates(cls, library=library)
        co = _coefficients(cls, library)
        U1 = FT / MIN / cls["windrf"]
        phi1 = (_spread(co, U1, 0.0) - co[1]) / co[1]
        phi2 = (_spread(co, 2 * U1, 0.0) - co[1]) / co[1]
        assert phi1 == pytest.approx(o["C"] * (o["beta"] / o["beta_op"]) ** (-o["E"]), rel=1e-11)
        assert phi2 / phi1 == pytest.approx(2.0 ** o["B"], rel=1e-11)
        # R0 of the coefficient form in m/s is the chain's ft/min value converted
        assert co[1] == pytest.approx(o["R0_ftmin"] * FT / MIN, rel=1e-14)


PINS = [check_si_chain, check_si_rate, check_english_round_trip, check_optimum_packing_ratio,
        check_moisture_damping, check_mineral_damping, check_heat_balance,
        check_wind_factor_unit_speed]


@pytest.mark.parametrize("pin", PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin()


# ---------------------------------------------------------------------------
# planted mistakes: each must fail at least one pin
# ---------------------------------------------------------------------------
MUTANTS = {
    "xi constants swapped": ("exp((0.792 + 0.681 * sqrt(sigma))",
                             "exp((0.681 + 0.792 * sqrt(sigma))"),
    "xi denominator typo": ("192.0 + 0.2595 * sigma", "192.0 + 0.2559 * sigma"),
    "A exponent sign": ("pow(ratio, A) * exp(A * (1.0 - ratio))",
                        "pow(ratio, -A) * exp(-A * (1.0 - ratio))"),
    "A constant typo": ("4.77 * pow(sigma, 0.1) - 7.27", "4.77 * pow(sigma, 0.1) - 7.72"),
    "eta_M coefficient typo": ("5.11 * rm * rm", "5.21 * rm * rm"),
    "eps with sigma in 1/m": ("exp(-138.0 / sigma)", "exp(-138.0 / fc[FC_SAVR])"),
    "Gamma_max as printed": ("495.0 + 0.0594 * s15", "495.0 + 0.594 * s15"),
    "beta_op exponent typo": ("pow(sigma, -0.8189)", "pow(sigma, -0.8198)"),
    "Q_ig as printed": ("250.0 + 1116.0 * Mf", "250.0 * beta + 1116.0 * Mf"),
    "eta_S exponent typo": ("0.174 * pow(SE, -0.19)", "0.174 * pow(SE, -0.91)"),
    "w_n minerals": ("w0 / (1.0 + ST)", "w0 * (1.0 - ST)"),
    "depth conversion inverted": ("fc[FC_DEPTH] / M_PER_FT", "fc[FC_DEPTH] * M_PER_FT"),
    "C constant typo": ("7.47 * exp(-0.133", "7.47 * exp(-0.331"),
    "E constant typo": ("0.715 * exp(-3.59e-4", "0.715 * exp(-3.95e-4"),
    "B exponent typo": ("0.02526 * pow(sigma, 0.54)", "0.02526 * pow(sigma, 0.45)"),
    "slope exponent typo": ("R0 * 5.275 * pow(p.beta, -0.3)", "R0 * 5.275 * pow(p.beta, -0.03)"),
    "wind conversion inverted": ("pow(fc[FC_WINDRF] * (60.0 / M_PER_FT), p.B)",
                                 "pow(fc[FC_WINDRF] * (M_PER_FT / 60.0), p.B)"),
    "R0 not converted to m/s": ("double R0 = p.R0_ftmin * (M_PER_FT / 60.0);",
                                "double R0 = p.R0_ftmin * (60.0 / M_PER_FT);"),
}


def _build_mutant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "wrffire_oracle.c")).read()
    # the first occurrence is the chain of rothermel_parts (the adjoint's
    # dual-number copy of the chain comes later in the file)
    start = src.index("rothermel_parts(const double *fc, double Mf)")
    at = src.find(old, start)
    assert at >= 0, f"{name}: the planted text is not in the oracle's chain"
    d = tmp_path / name.replace(" ", "_").replace("/", "_")
    d.mkdir()
    c = d / "mutant.c"
    c.write_text(src[:at] + new + src[at + len(old):])
    so = d / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", str(c),
                    "-o", str(so), "-lm"], check=True)
    L = C.CDLL(str(so))
    D = C.POINTER(C.c_double)
    L.orc_rothermel_intermediates.restype = None
    L.orc_rothermel_intermediates.argtypes = [D, C.c_double, D]
    L.orc_fuel_coefficients.restype = None
    L.orc_fuel_coefficients.argtypes = [D, C.c_double, D]
    return L


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc to build the mutants")
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(tmp_path, orc, name):
    old, new = MUTANTS[name]
    L = _build_mutant(tmp_path, name, old, new)
    failed = []
    for pin in PINS:
        try:
            pin(L)
        except AssertionError:
            failed.append(pin.__name__)
    assert failed, f"planted mistake '{name}' passed every pin"
