"""Plain FP64 CPU oracle of the WRF-Fire fire step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use this package; the product library never
imports it, and it never imports the product library.  The arithmetic lives in
``wrffire_oracle.c`` (plain C, -O2 -ffp-contract=off); this module only
marshals numpy arrays.

Inputs come in the neutral form produced by ``paper_1102_1343_gb300.synth``
(fuel classes as dicts of Table 1 identifiers, ignitions as dicts), which holds
no arithmetic of the method.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wrffire_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
# a library built from a modified copy of the source, loaded instead of the
# build (the planted-mistake tests run the pins against such copies)
_LIB_OVERRIDE = os.environ.get("WRFFIRE_ORACLE_LIBRARY")
_lock = threading.Lock()
_lib = None

# order of the 13 doubles of one fuel class (Table 1), as in wrffire_oracle.c
FUEL_FIELDS = ("windrf", "weight", "weight_is_tf", "fgi", "fueldepthm", "savr",
               "fuelmce", "fueldens", "st", "se", "cmbcnst", "fuelmc_g", "chaparral")
# order of the 9 coefficients (eq. spread-WRF-Fire + T_f + heat factors)
COEF_FIELDS = ("S0", "R0", "b", "c", "d", "e", "Tf", "Hs", "Hq")
IGN_FIELDS = ("ax", "ay", "bx", "by", "t_start", "radius", "speed", "vx", "vy", "t_end")
STATUS_BOUNDARY = 1
STATUS_NONFINITE = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", _SRC, "-o", tmp, "-lm"]
    # with OpenMP where the compiler has it (the per-node loops over rows;
    # results do not depend on the thread count), else single-threaded
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Grid(C.Structure):
    _fields_ = [("nxa", C.c_int), ("nya", C.c_int), ("srx", C.c_int), ("sry", C.c_int),
                ("dx_atm", C.c_double), ("dy_atm", C.c_double), ("eps", C.c_double),
                ("band", C.c_int), ("scheme", C.c_int)]


_D = C.POINTER(C.c_double)
_U8 = C.POINTER(C.c_ubyte)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(_LIB_OVERRIDE or build())
            L.orc_rothermel_rate.restype = C.c_double
            L.orc_rothermel_rate.argtypes = [_D, C.c_double, C.c_double, C.c_double]
            L.orc_rothermel_intermediates.restype = None
            L.orc_rothermel_intermediates.argtypes = [_D, C.c_double, _D]
            L.orc_fuel_coefficients.restype = None
            L.orc_fuel_coefficients.argtypes = [_D, C.c_double, _D]
            L.orc_spread_rate.restype = C.c_double
            L.orc_spread_rate.argtypes = [_D, C.c_double, C.c_double]
            L.orc_node_coefficients.restype = None
            L.orc_node_coefficients.argtypes = [_D, C.c_int, _U8, _D, C.c_long, _D]
            L.orc_godunov.restype = C.c_double
            L.orc_godunov.argtypes = [C.c_double, C.c_double]
            L.orc_extend.restype = None
            L.orc_extend.argtypes = [C.c_int, C.c_int, _D, _D]
            L.orc_wind_at_nodes.restype = None
            L.orc_wind_at_nodes.argtypes = [C.c_int] * 4 + [_D, _D, _D, _D]
            L.orc_rhs.restype = None
            L.orc_rhs.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                  _D, _D, _D, _D, _D, _D, _D, _D]
            L.orc_cell_fuel_fraction.restype = C.c_double
            L.orc_cell_fuel_fraction.argtypes = [_D, _D, C.c_double, C.c_double]
            L.orc_cell_fuel_fraction_linear.restype = C.c_double
            L.orc_cell_fuel_fraction_linear.argtypes = [_D, _D, C.c_double, C.c_double]
            L.orc_ignite.restype = None
            L.orc_ignite.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, _D, C.c_int,
                                     _U8, C.c_double, _D, _D]
            L.orc_init_state.restype = None
            L.orc_init_state.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                         _D, C.c_int, _U8, _D, _D, _D]
            L.orc_step.restype = C.c_int
            L.orc_step.argtypes = [C.POINTER(_Grid), _D, _D, _D, _D, _D, _D, _D, C.c_int, _U8,
                                   C.c_double, C.c_double, _D, _D, _D, _D, _D]
            L.orc_fuel_coefficients_dMf.restype = None
            L.orc_fuel_coefficients_dMf.argtypes = [_D, C.c_double, _D]
            L.orc_node_coefficients_dMf.restype = None
            L.orc_node_coefficients_dMf.argtypes = [_D, C.c_int, _U8, _D, C.c_long, _D]
            L.orc_adjoint.restype = C.c_double
            L.orc_adjoint.argtypes = ([C.POINTER(_Grid)] + [_D] * 7 + [C.c_double, C.c_double,
                                      C.c_int] + [_D] * 8)
            L.orc_adjoint_heat.restype = C.c_double
            L.orc_adjoint_heat.argtypes = ([C.POINTER(_Grid)] + [_D] * 7 + [C.c_double, C.c_double,
                                           C.c_int] + [_D] * 8)
            L.orc_extend_vjp.restype = None
            L.orc_extend_vjp.argtypes = [C.c_int, C.c_int, _D, _D, _D]
            L.orc_step_vjp.restype = None
            L.orc_step_vjp.argtypes = ([C.POINTER(_Grid)] + [_D] * 7 + [C.c_double] + [_D] * 7)
            L.orc_wind_at_height.restype = None
            L.orc_wind_at_height.argtypes = [C.c_int, C.c_long, _D, _D, _D, C.c_double, _D]
            L.orc_heat_insertion.restype = None
            L.orc_heat_insertion.argtypes = ([C.c_int, C.c_long] + [_D] * 5
                                             + [C.c_double] * 3 + [_D, _D])
            L.orc_set_threads.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            L.orc_set_threads(1)  # one thread unless asked (set_threads)
            _lib = L
    return _lib


def set_threads(n: int) -> int:
    """Threads of the oracle's per-node loops (OpenMP builds); returns the
    count in effect, 1 where the oracle was built without OpenMP.  The
    results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def fuel_vector(cls: dict) -> np.ndarray:
    """One fuel class (dict of Table 1 identifiers) as the oracle's 13 doubles."""
    return np.array([float(cls.get(k, 0.0)) for k in FUEL_FIELDS], dtype=np.float64)


def fuel_table(classes) -> np.ndarray:
    return np.ascontiguousarray(np.stack([fuel_vector(c) for c in classes]))


def ignition_table(ignitions) -> np.ndarray:
    if not ignitions:
        return np.zeros((1, len(IGN_FIELDS)), dtype=np.float64)
    return np.ascontiguousarray(
        np.array([[float(g.get(k, 0.0)) for k in IGN_FIELDS] for g in ignitions],
                 dtype=np.float64))


def rothermel_rate(cls: dict, U: float, tanphi: float, Mf: float | None = None) -> float:
    v = fuel_vector(cls)
    return lib().orc_rothermel_rate(_dp(v), -1.0 if Mf is None else float(Mf), float(U),
                                    float(tanphi))


# names of the values orc_rothermel_intermediates returns (English units)
ROTHERMEL_FIELDS = ("sigma", "wl", "depth", "rho_p", "h", "w0", "rho_b", "beta", "beta_op", "A",
                    "Gmax", "Gamma", "wn", "etaM", "etaS", "IR", "xi", "eps", "Qig", "R0_ftmin",
                    "B", "C", "E", "nofuel")


def rothermel_intermediates(cls: dict, Mf: float | None = None, library=None) -> dict:
    """Every intermediate of the oracle's Table 2 chain for one class (dict
    keyed by ROTHERMEL_FIELDS, English units).  ``library`` selects another
    build of the oracle source (the mutation tests)."""
    v = fuel_vector(cls)
    out = np.zeros(len(ROTHERMEL_FIELDS))
    (library or lib()).orc_rothermel_intermediates(_dp(v), -1.0 if Mf is None else float(Mf),
                                                   _dp(out))
    return dict(zip(ROTHERMEL_FIELDS, out.tolist()))


def fuel_coefficients(cls: dict, Mf: float | None = None) -> np.ndarray:
    v = fuel_vector(cls)
    out = np.zeros(9)
    lib().orc_fuel_coefficients(_dp(v), -1.0 if Mf is None else float(Mf), _dp(out))
    return out


def spread_rate(coef, U: float, tanphi: float) -> float:
    co = _f64(coef)
    return lib().orc_spread_rate(_dp(co), float(U), float(tanphi))


def node_coefficients(classes, fuel, moisture=None) -> np.ndarray:
    tab = fuel_table(classes)
    fuel = np.ascontiguousarray(fuel, dtype=np.uint8)
    mo = _f64(moisture)
    out = np.zeros(fuel.shape + (9,))
    lib().orc_node_coefficients(_dp(tab), len(classes), fuel.ctypes.data_as(_U8), _dp(mo),
                                fuel.size, _dp(out))
    return out


def fuel_coefficients_dMf(cls: dict, Mf: float | None = None) -> np.ndarray:
    """d(coefficients)/d(M_f) of one class (dual-number evaluation of Table 2)."""
    v = fuel_vector(cls)
    out = np.zeros(9)
    lib().orc_fuel_coefficients_dMf(_dp(v), -1.0 if Mf is None else float(Mf), _dp(out))
    return out


def node_coefficients_dMf(classes, fuel, moisture=None) -> np.ndarray:
    tab = fuel_table(classes)
    fuel = np.ascontiguousarray(fuel, dtype=np.uint8)
    mo = _f64(moisture)
    out = np.zeros(fuel.shape + (9,))
    lib().orc_node_coefficients_dMf(_dp(tab), len(classes), fuel.ctypes.data_as(_U8), _dp(mo),
                                    fuel.size, _dp(out))
    return out


def godunov(dm: float, dp: float) -> float:
    return lib().orc_godunov(float(dm), float(dp))


def extend(a) -> np.ndarray:
    a = _f64(a)
    ny, nx = a.shape
    ext = np.zeros((ny + 2, nx + 2))
    lib().orc_extend(nx, ny, _dp(a), _dp(ext))
    return ext


def extend_vjp(a, D) -> np.ndarray:
    """(d extend(a) / d a)^T D for D of the extended shape (ny+2, nx+2)."""
    a = _f64(a)
    ny, nx = a.shape
    D = _f64(D)
    assert D.shape == (ny + 2, nx + 2)
    out = np.zeros_like(a)
    lib().orc_extend_vjp(nx, ny, _dp(a), _dp(D), _dp(out))
    return out


def wind_at_nodes(nxa, nya, srx, sry, u, v):
    u, v = _f64(u), _f64(v)
    assert u.shape == (nya, nxa + 1) and v.shape == (nya + 1, nxa)
    un = np.zeros((nya * sry, nxa * srx))
    vn = np.zeros_like(un)
    lib().orc_wind_at_nodes(nxa, nya, srx, sry, _dp(u), _dp(v), _dp(un), _dp(vn))
    return un, vn


def rhs(psi, dx, dy, eps, coef, un, vn, dzdx, dzdy, mult=None) -> np.ndarray:
    """Right-hand side of eq. (F-disc) for every node (ghosts extrapolated)."""
    psi = _f64(psi)
    ny, nx = psi.shape
    ext = extend(psi)
    co = _f64(coef)
    if co.ndim == 1:
        co = np.ascontiguousarray(np.broadcast_to(co, (ny, nx, 9)))
    un, vn, dzdx, dzdy, mult = map(_f64, (un, vn, dzdx, dzdy, mult))
    F = np.zeros_like(psi)
    lib().orc_rhs(nx, ny, float(dx), float(dy), float(eps), _dp(ext), _dp(co), _dp(mult),
                  _dp(un), _dp(vn), _dp(dzdx), _dp(dzdy), _dp(F))
    return F


def cell_fuel_fraction(psi3, tign3, t: float, Tf: float) -> float:
    """Fuel fraction of the cell at the centre of a 3x3 node neighbourhood.

    tign3 holds node ignition times; eq. (ti-comp) is applied here (t where
    psi >= 0), as in the step."""
    p = _f64(psi3).reshape(3, 3)
    ti = _f64(tign3).reshape(3, 3)
    th = np.ascontiguousarray(np.where(p < 0.0, ti, t))
    p = np.ascontiguousarray(p)
    return lib().orc_cell_fuel_fraction(_dp(p), _dp(th), float(t), float(Tf))


def wind_at_height(u3d, z3d, z0, zf):
    """Vertical log-linear interpolation of a wind component to height zf
    (Sect. "Coupling"): u3d, z3d [nz][...] (levels first), z0 [...];
    returns [...]."""
    u3d, z3d, z0 = _f64(u3d), _f64(z3d), _f64(z0)
    nz = u3d.shape[0]
    assert z3d.shape == u3d.shape and z0.shape == u3d.shape[1:]
    out = np.zeros(u3d.shape[1:])
    lib().orc_wind_at_height(nz, z0.size, _dp(u3d), _dp(z3d), _dp(z0), float(zf), _dp(out))
    return out


def heat_insertion(hs, hl, zw, rho, mu, zext, cp=1004.0, L=2.5e6, rth=None, rqv=None):
    """Sources added to the tendencies of mu theta and mu q_m (Sect.
    "Coupling", the heat insertion): hs, hl, mu [...], zw [nz+1][...], rho
    [nz][...]; returns (rth, rqv) [nz][...] (added to the given arrays)."""
    hs, hl, zw, rho, mu = map(_f64, (hs, hl, zw, rho, mu))
    nz = rho.shape[0]
    rth = np.zeros(rho.shape) if rth is None else _f64(rth).copy()
    rqv = np.zeros(rho.shape) if rqv is None else _f64(rqv).copy()
    lib().orc_heat_insertion(nz, hs.size, _dp(hs), _dp(hl), _dp(zw), _dp(rho), _dp(mu),
                             float(zext), float(cp), float(L), _dp(rth), _dp(rqv))
    return rth, rqv


def cell_fuel_fraction_linear(psi3, tign3, t: float, Tf: float) -> float:
    """Fuel fraction of the cell at the centre of a 3x3 node neighbourhood by
    the scheme exact for linear psi and t_i (tign3: node ignition times;
    eq. (ti-comp) applied here as in cell_fuel_fraction)."""
    p = _f64(psi3).reshape(3, 3)
    ti = _f64(tign3).reshape(3, 3)
    th = np.ascontiguousarray(np.where(p < 0.0, ti, t))
    p = np.ascontiguousarray(p)
    return lib().orc_cell_fuel_fraction_linear(_dp(p), _dp(th), float(t), float(Tf))


def default_psi_far(nx, ny, dx, dy) -> float:
    """Reading of "const > 0" for the initial level-set function: the domain diagonal."""
    return float(np.hypot(nx * dx, ny * dy))


class OracleFire:
    """The oracle's fire model: state + the six-item step, FP64."""

    def __init__(self, nxa, nya, sr, dx_atm, classes, fuel, dzdx, dzdy, ignitions=(),
                 moisture=None, mult=None, eps=0.4, band=1, psi_far=None, dy_atm=None,
                 scheme=0):
        srx, sry = (sr, sr) if np.isscalar(sr) else sr
        dy_atm = dx_atm if dy_atm is None else dy_atm
        self.g = _Grid(nxa, nya, srx, sry, float(dx_atm), float(dy_atm), float(eps), int(band),
                       int(scheme))
        self.nx, self.ny = nxa * srx, nya * sry
        self.dx, self.dy = dx_atm / srx, dy_atm / sry
        fuel = np.ascontiguousarray(fuel, dtype=np.uint8)
        assert fuel.shape == (self.ny, self.nx)
        self.coef = node_coefficients(classes, fuel, moisture)
        self.classes, self.fuel, self.moisture = list(classes), fuel, _f64(moisture)
        self.mult = _f64(mult)
        self.dzdx, self.dzdy = _f64(dzdx), _f64(dzdy)
        self.ign = ignition_table(list(ignitions))
        self.n_ign = len(list(ignitions))
        self.applied = np.zeros(max(1, self.n_ign), dtype=np.uint8)
        self.psi_far = (default_psi_far(self.nx, self.ny, self.dx, self.dy)
                        if psi_far is None else float(psi_far))
        self.psi = np.zeros((self.ny, self.nx))
        self.tign = np.zeros_like(self.psi)
        self.frac = np.zeros_like(self.psi)
        lib().orc_init_state(self.nx, self.ny, self.dx, self.dy, self.psi_far, _dp(self.ign),
                             self.n_ign, self.applied.ctypes.data_as(_U8), _dp(self.psi),
                             _dp(self.tign), _dp(self.frac))
        self.t = 0.0
        self.status = 0

    @classmethod
    def from_workload(cls, w, **kw):
        args = dict(nxa=w.nxa, nya=w.nya, sr=(w.srx, w.sry), dx_atm=w.dx_atm, dy_atm=w.dy_atm,
                    classes=w.classes, fuel=w.fuel, dzdx=w.dzdx, dzdy=w.dzdy,
                    ignitions=w.ignitions, moisture=w.moisture, mult=w.mult, eps=w.eps,
                    band=w.band)
        args.update(kw)
        return cls(**args)

    def step(self, u, v, dt):
        u, v = _f64(u), _f64(v)
        g = self.g
        assert u.shape == (g.nya, g.nxa + 1) and v.shape == (g.nya + 1, g.nxa)
        hs = np.zeros((g.nya, g.nxa))
        hl = np.zeros_like(hs)
        st = lib().orc_step(C.byref(g), _dp(self.coef), _dp(self.mult), _dp(self.dzdx),
                            _dp(self.dzdy), _dp(u), _dp(v), _dp(self.ign), self.n_ign,
                            self.applied.ctypes.data_as(_U8), self.t, float(dt),
                            _dp(self.psi), _dp(self.tign), _dp(self.frac), _dp(hs), _dp(hl))
        self.t = self.t + float(dt)
        self.status |= st
        return hs, hl, st

    def adjoint(self, u, v, dt, nsteps, tobs):
        """Reference adjoint: advance nsteps (no ignition may become active),
        return J = 1/2 sum over nodes ignited in both of (t_i - tobs)^2 and
        dJ/d(multiplier) [ny][nx], dJ/d(M_f) per node [ny][nx], dJ/du
        [nya][nxa+1], dJ/dv [nya+1][nxa].  tobs is NaN/inf where unobserved."""
        u, v = _f64(u), _f64(v)
        g = self.g
        tobs = _f64(tobs)
        assert tobs.shape == (self.ny, self.nx)
        dco = node_coefficients_dMf(self.classes, self.fuel, self.moisture)
        gm = np.zeros((self.ny, self.nx))
        gM = np.zeros_like(gm)
        gu = np.zeros((g.nya, g.nxa + 1))
        gv = np.zeros((g.nya + 1, g.nxa))
        J = lib().orc_adjoint(C.byref(g), _dp(self.coef), _dp(dco), _dp(self.mult),
                              _dp(self.dzdx), _dp(self.dzdy), _dp(u), _dp(v), self.t,
                              float(dt), int(nsteps), _dp(self.psi), _dp(self.tign),
                              _dp(self.frac), _dp(tobs), _dp(gm), _dp(gM), _dp(gu), _dp(gv))
        for _ in range(int(nsteps)):
            self.t = self.t + float(dt)
        return J, gm, gM, gu, gv

    def adjoint_heat(self, u, v, dt, nsteps, qobs):
        """Reference adjoint of the heat misfit: advance nsteps (no ignition
        may become active), return J = 1/2 sum over atmospheric cells with a
        finite observation of (Q - qobs)^2, Q the sensible heat released per
        unit area over the run [nya][nxa], and the gradients as adjoint()."""
        u, v = _f64(u), _f64(v)
        g = self.g
        qobs = _f64(qobs)
        assert qobs.shape == (g.nya, g.nxa)
        dco = node_coefficients_dMf(self.classes, self.fuel, self.moisture)
        gm = np.zeros((self.ny, self.nx))
        gM = np.zeros_like(gm)
        gu = np.zeros((g.nya, g.nxa + 1))
        gv = np.zeros((g.nya + 1, g.nxa))
        J = lib().orc_adjoint_heat(C.byref(g), _dp(self.coef), _dp(dco), _dp(self.mult),
                                   _dp(self.dzdx), _dp(self.dzdy), _dp(u), _dp(v), self.t,
                                   float(dt), int(nsteps), _dp(self.psi), _dp(self.tign),
                                   _dp(self.frac), _dp(qobs), _dp(gm), _dp(gM), _dp(gu), _dp(gv))
        for _ in range(int(nsteps)):
            self.t = self.t + float(dt)
        return J, gm, gM, gu, gv

    def step_vjp(self, u, v, dt, w):
        """For one level-set step from the current state with the wind u, v:
        lam = (d psi^{n+1} / d psi^n)^T w and the parameter terms
        w^T d psi^{n+1} / dp for the per-node multiplier, the per-node
        moisture and the node wind (un, vn), each [ny][nx].  The state is
        not advanced."""
        u, v, w = _f64(u), _f64(v), _f64(w)
        assert w.shape == (self.ny, self.nx)
        dco = node_coefficients_dMf(self.classes, self.fuel, self.moisture)
        lam = np.zeros((self.ny, self.nx))
        gm, gM, gun, gvn = (np.zeros_like(lam) for _ in range(4))
        lib().orc_step_vjp(C.byref(self.g), _dp(self.coef), _dp(dco), _dp(self.mult),
                           _dp(self.dzdx), _dp(self.dzdy), _dp(u), _dp(v), float(dt),
                           _dp(self.psi), _dp(w), _dp(lam), _dp(gm), _dp(gM), _dp(gun),
                           _dp(gvn))
        return lam, gm, gM, gun, gvn

    def set_state(self, psi, tign, frac, t):
        self.psi = _f64(psi).copy()
        self.tign = _f64(tign).copy()
        self.frac = _f64(frac).copy()
        self.t = float(t)
