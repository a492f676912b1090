"""GB300 (sm_103a) fire-model step of WRF-Fire: thin Python binding.

The binding mirrors the C ABI of ``include/wrffire.h`` name for name
(``fire_init``, ``fire_step``, ``fire_step_host``, ``fire_run``,
``fire_get_state``, ``fire_set_state``, ``fire_status``, ...).  It only marshals
arguments: torch CUDA tensors are passed as device pointers, numpy arrays as
host pointers, and every step of the fire model runs in the CUDA library
``libwrffire_gb300.so``.  There is no CPU fallback: if the library is missing
the import of the native handle raises.

``FireModel`` wraps one context with torch-allocated inputs and outputs.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# the library this module loads; WRFFIRE_LIBRARY names another build of it
# (the bounds-checked one of build.build(checked=True), for tests)
LIB_PATH = os.environ.get("WRFFIRE_LIBRARY") or os.path.join(_HERE, "libwrffire_gb300.so")

FIRE_FP64 = 0
FIRE_FP32 = 1
FIRE_OK = 0
FIRE_ERR_ARG = -1
FIRE_ERR_CUDA = -2
FIRE_ERR_OOM = -3
FIRE_ERR_BOUNDARY = -4
FIRE_ERR_NONFINITE = -5
FIRE_ERR_TIMEOUT = -6
FIRE_ERR_STATE = -7
FIRE_ERR_BOUNDS = -8
FIRE_KERNEL_TILE = 0
FIRE_KERNEL_MARCH = 1
FIRE_KERNEL_WARP = 2
FIRE_KERNEL_WARP4 = 3
FIRE_KERNEL_WARP_DENSE = 4
FIRE_MAX_CLASSES = 64
FIRE_MAX_IGNITIONS = 256
FIRE_MAX_MEMBERS = 1024

# every entry point the header declares (checked by the ABI test)
ABI_SYMBOLS = ("fire_init", "fire_step", "fire_step_host", "fire_run", "fire_get_state",
               "fire_set_state", "fire_status", "fire_clear_status", "fire_mesh_size",
               "fire_time", "fire_set_kernel", "fire_get_kernel", "fire_enable_timing",
               "fire_kernel_time_ms", "fire_strerror", "fire_last_cuda_error", "fire_destroy",
               "fire_step_noalloc",
               "fire_ensemble_create", "fire_ensemble_step", "fire_ensemble_member",
               "fire_ensemble_status", "fire_ensemble_clear_status", "fire_ensemble_set_kernel",
               "fire_ensemble_get_kernel", "fire_ensemble_set_barrier_test",
               "fire_ensemble_destroy", "fire_set_spread_mult", "fire_set_fuel_classes",
               "fire_adjoint", "fire_autotune", "fire_ensemble_autotune",
               "fire_default_kernel", "fire_adjoint_heat", "fire_set_moisture",
               "fire_wind_at_height", "fire_heat_insertion", "fire_set_fraction_scheme",
               "fire_bounds_checked", "fire_bounds_selftest", "fire_set_adaptive",
               "fire_adaptive_info")
FIRE_FRACTION_SUBCELL = 0
FIRE_FRACTION_LINEAR = 1


class FireError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        msg = f"{what}: {fire_strerror(code)} ({code})" if what else f"{fire_strerror(code)} ({code})"
        if code in (FIRE_ERR_CUDA, FIRE_ERR_OOM):
            msg += f" [{fire_last_cuda_error()}]"
        super().__init__(msg)


class fire_grid_desc(C.Structure):
    _fields_ = [("nx_atm", C.c_int), ("ny_atm", C.c_int), ("sr_x", C.c_int), ("sr_y", C.c_int),
                ("dx_atm", C.c_double), ("dy_atm", C.c_double), ("precision", C.c_int),
                ("boundary_band", C.c_int), ("eps_visc", C.c_double), ("psi_far", C.c_double)]


class fire_fuel_class(C.Structure):
    _fields_ = [("windrf", C.c_double), ("weight", C.c_double), ("weight_is_tf", C.c_int),
                ("chaparral", C.c_int), ("fgi", C.c_double), ("fueldepthm", C.c_double),
                ("savr", C.c_double), ("fuelmce", C.c_double), ("fueldens", C.c_double),
                ("st", C.c_double), ("se", C.c_double), ("cmbcnst", C.c_double),
                ("fuelmc_g", C.c_double)]


class fire_ignition(C.Structure):
    _fields_ = [("ax", C.c_double), ("ay", C.c_double), ("bx", C.c_double), ("by", C.c_double),
                ("t_start", C.c_double), ("radius", C.c_double), ("speed", C.c_double),
                ("vx", C.c_double), ("vy", C.c_double), ("t_end", C.c_double)]


_P = C.c_void_p


class fire_member_desc(C.Structure):
    _fields_ = [("grid", fire_grid_desc), ("classes", C.POINTER(fire_fuel_class)),
                ("n_classes", C.c_int), ("fuel_class_dev", _P), ("moisture_dev", _P),
                ("spread_mult_dev", _P),
                ("dzdx_dev", _P), ("dzdy_dev", _P), ("ignitions", C.POINTER(fire_ignition)),
                ("n_ign", C.c_int)]


_lib = None


def load_library(path: str | None = None):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -m paper_1102_1343_gb300.build` (needs nvcc)")
    L = C.CDLL(path)
    L.fire_init.argtypes = [C.POINTER(_P), C.POINTER(fire_grid_desc), C.POINTER(fire_fuel_class),
                            C.c_int, _P, _P, _P, _P, _P, C.POINTER(fire_ignition), C.c_int, _P]
    L.fire_step.argtypes = [_P, _P, _P, C.c_double, _P, _P]
    L.fire_step_host.argtypes = [_P, _P, _P, C.c_double, _P, _P]
    L.fire_run.argtypes = [_P, C.c_int, C.c_double, _P, _P, _P, _P]
    L.fire_get_state.argtypes = [_P, _P, _P, _P, C.POINTER(C.c_double)]
    L.fire_set_state.argtypes = [_P, _P, _P, _P, C.c_double]
    L.fire_status.argtypes = [_P]
    L.fire_clear_status.argtypes = [_P]
    L.fire_mesh_size.argtypes = [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.fire_time.argtypes = [_P]
    L.fire_time.restype = C.c_double
    L.fire_set_kernel.argtypes = [_P, C.c_int, C.c_int, C.c_int]
    L.fire_set_adaptive.argtypes = [_P, C.c_int]
    L.fire_adaptive_info.argtypes = [_P, C.POINTER(C.c_int), C.POINTER(C.c_longlong),
                                     C.POINTER(C.c_double)]
    L.fire_get_kernel.argtypes = [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.fire_enable_timing.argtypes = [_P, C.c_int]
    L.fire_kernel_time_ms.argtypes = [_P, C.POINTER(C.c_double), C.POINTER(C.c_long)]
    L.fire_strerror.argtypes = [C.c_int]
    L.fire_strerror.restype = C.c_char_p
    L.fire_bounds_checked.argtypes = []
    L.fire_bounds_selftest.argtypes = [C.POINTER(C.c_int)]
    L.fire_last_cuda_error.argtypes = []
    L.fire_last_cuda_error.restype = C.c_char_p
    L.fire_destroy.argtypes = [_P]
    L.fire_destroy.restype = None
    L.fire_step_noalloc.argtypes = ([C.POINTER(fire_grid_desc), C.POINTER(fire_fuel_class), C.c_int]
                                    + [_P] * 11 + [C.c_double, C.c_double] + [_P] * 4)
    L.fire_step_noalloc.restype = C.c_int
    L.fire_ensemble_create.argtypes = [C.POINTER(_P), C.c_int, C.POINTER(fire_member_desc), _P]
    L.fire_ensemble_step.argtypes = [_P, C.c_int, C.c_double, C.POINTER(_P), C.POINTER(_P),
                                     C.POINTER(_P), C.POINTER(_P)]
    L.fire_ensemble_member.argtypes = [_P, C.c_int, C.POINTER(_P)]
    L.fire_ensemble_status.argtypes = [_P, C.POINTER(C.c_int)]
    L.fire_ensemble_clear_status.argtypes = [_P]
    L.fire_ensemble_set_kernel.argtypes = [_P, C.c_int, C.c_int]
    L.fire_ensemble_get_kernel.argtypes = [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.fire_ensemble_set_barrier_test.argtypes = [_P, C.c_int, C.c_longlong]
    L.fire_ensemble_destroy.argtypes = [_P]
    L.fire_ensemble_destroy.restype = None
    L.fire_set_spread_mult.argtypes = [_P, _P]
    L.fire_set_spread_mult.restype = C.c_int
    L.fire_set_fuel_classes.argtypes = [_P, C.POINTER(fire_fuel_class), C.c_int]
    L.fire_set_fuel_classes.restype = C.c_int
    L.fire_set_moisture.argtypes = [_P, _P]
    L.fire_set_moisture.restype = C.c_int
    L.fire_set_fraction_scheme.argtypes = [_P, C.c_int]
    L.fire_set_fraction_scheme.restype = C.c_int
    L.fire_wind_at_height.argtypes = [C.c_int, C.c_int, C.c_longlong, _P, _P, _P, C.c_double,
                                      _P, _P]
    L.fire_wind_at_height.restype = C.c_int
    L.fire_heat_insertion.argtypes = ([C.c_int, C.c_longlong] + [_P] * 5
                                      + [C.c_double] * 3 + [_P, _P, _P])
    L.fire_heat_insertion.restype = C.c_int
    L.fire_adjoint.argtypes = [_P, C.c_int, C.c_double, _P, _P, _P, C.c_int,
                               C.POINTER(C.c_double), _P, _P, _P, _P]
    L.fire_adjoint.restype = C.c_int
    L.fire_adjoint_heat.argtypes = L.fire_adjoint.argtypes
    L.fire_adjoint_heat.restype = C.c_int
    L.fire_autotune.argtypes = [_P, _P, _P, C.c_double, C.c_int, C.POINTER(C.c_int),
                                C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.fire_autotune.restype = C.c_int
    L.fire_ensemble_autotune.argtypes = [_P, C.c_int, C.c_double, C.POINTER(_P), C.POINTER(_P),
                                         C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.fire_ensemble_autotune.restype = C.c_int
    L.fire_default_kernel.argtypes = [C.c_int] * 6 + [C.POINTER(C.c_int)] * 3
    L.fire_default_kernel.restype = C.c_int
    for name in ("fire_ensemble_create", "fire_ensemble_step", "fire_ensemble_member",
                 "fire_ensemble_status", "fire_ensemble_clear_status", "fire_ensemble_set_kernel",
                 "fire_ensemble_get_kernel", "fire_ensemble_set_barrier_test"):
        getattr(L, name).restype = C.c_int
    for name in ABI_SYMBOLS:
        f = getattr(L, name)
        if f.restype is C.c_int or name in ("fire_init", "fire_step", "fire_step_host",
                                             "fire_run", "fire_get_state", "fire_set_state",
                                             "fire_status", "fire_clear_status",
                                             "fire_mesh_size", "fire_set_kernel", "fire_get_kernel",
                                             "fire_enable_timing", "fire_kernel_time_ms"):
            f.restype = C.c_int
    _lib = L
    return L


def _ptr(x):
    """Device pointer of a torch tensor, host pointer of a numpy array, or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous (row-major)")
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if isinstance(x, int):
        return x
    raise TypeError(f"cannot pass {type(x)} as a buffer")


def _check(code, what):
    if code != FIRE_OK:
        raise FireError(code, what)
    return code


# ---------------------------------------------------------------------------
# the C ABI, name for name
# ---------------------------------------------------------------------------

def fire_strerror(code: int) -> str:
    return load_library().fire_strerror(int(code)).decode()


def fire_bounds_checked() -> bool:
    """Whether the loaded library is the bounds-checked build."""
    return bool(load_library().fire_bounds_checked())


def fire_bounds_selftest():
    """The index check of a bounds-checked build on the indices -1, 0, 9, 10
    of a 10-element buffer: whether each was flagged (1 0 0 1 expected)."""
    f = (C.c_int * 4)()
    _check(load_library().fire_bounds_selftest(f), "fire_bounds_selftest")
    return list(f)


def fire_last_cuda_error() -> str:
    return load_library().fire_last_cuda_error().decode()


def make_grid(nx_atm, ny_atm, sr_x, sr_y, dx_atm, dy_atm, precision=FIRE_FP32, boundary_band=1,
              eps_visc=0.4, psi_far=0.0) -> fire_grid_desc:
    return fire_grid_desc(int(nx_atm), int(ny_atm), int(sr_x), int(sr_y), float(dx_atm),
                          float(dy_atm), int(precision), int(boundary_band), float(eps_visc),
                          float(psi_far))


def make_classes(classes) -> C.Array:
    arr = (fire_fuel_class * len(classes))()
    for k, c in enumerate(classes):
        for name, typ in fire_fuel_class._fields_:
            val = c.get(name, 0)
            setattr(arr[k], name, int(val) if typ is C.c_int else float(val))
    return arr


def make_ignitions(ignitions) -> C.Array:
    arr = (fire_ignition * max(1, len(ignitions)))()
    for k, g in enumerate(ignitions):
        for name, _ in fire_ignition._fields_:
            # the drip-torch fields (vx, vy, t_end) are optional: 0 otherwise
            setattr(arr[k], name, float(g[name] if name in ("ax", "ay", "bx", "by", "t_start",
                                                            "radius", "speed")
                                        else g.get(name, 0.0)))
    return arr


def fire_init(grid: fire_grid_desc, classes, fuel_class_dev, moisture_dev, spread_mult_dev,
              dzdx_dev, dzdy_dev, ignitions, cuda_stream=None) -> int:
    """Returns the context handle (an int); raises FireError on failure."""
    L = load_library()
    cls = make_classes(classes)
    ign = make_ignitions(list(ignitions))
    out = _P()
    code = L.fire_init(C.byref(out), C.byref(grid), cls, len(classes), _ptr(fuel_class_dev),
                       _ptr(moisture_dev), _ptr(spread_mult_dev), _ptr(dzdx_dev),
                       _ptr(dzdy_dev), ign, len(list(ignitions)), _ptr(cuda_stream) or None)
    _check(code, "fire_init")
    return out.value


def fire_step(ctx, wind_u_dev, wind_v_dev, dt, heat_sens_dev=None, heat_lat_dev=None) -> int:
    return _check(load_library().fire_step(ctx, _ptr(wind_u_dev), _ptr(wind_v_dev), float(dt),
                                           _ptr(heat_sens_dev), _ptr(heat_lat_dev)), "fire_step")


def fire_step_host(ctx, wind_u_host, wind_v_host, dt, heat_sens_host=None,
                   heat_lat_host=None) -> int:
    return _check(load_library().fire_step_host(ctx, _ptr(wind_u_host), _ptr(wind_v_host),
                                                float(dt), _ptr(heat_sens_host),
                                                _ptr(heat_lat_host)), "fire_step_host")


def fire_run(ctx, nsteps, dt, wind_u_dev, wind_v_dev, heat_sens_dev=None,
             heat_lat_dev=None) -> int:
    return _check(load_library().fire_run(ctx, int(nsteps), float(dt), _ptr(wind_u_dev),
                                          _ptr(wind_v_dev), _ptr(heat_sens_dev),
                                          _ptr(heat_lat_dev)), "fire_run")


def fire_get_state(ctx, psi_dev=None, tign_dev=None, frac_dev=None) -> float:
    t = C.c_double()
    _check(load_library().fire_get_state(ctx, _ptr(psi_dev), _ptr(tign_dev), _ptr(frac_dev),
                                         C.byref(t)), "fire_get_state")
    return t.value


def fire_set_state(ctx, psi_dev, tign_dev, frac_dev, t) -> int:
    return _check(load_library().fire_set_state(ctx, _ptr(psi_dev), _ptr(tign_dev),
                                                _ptr(frac_dev), float(t)), "fire_set_state")


def fire_status(ctx) -> int:
    """Synchronises; returns FIRE_OK or a device fault code (not raised)."""
    return load_library().fire_status(ctx)


def fire_clear_status(ctx) -> int:
    return _check(load_library().fire_clear_status(ctx), "fire_clear_status")


def fire_mesh_size(ctx):
    nx, ny = C.c_int(), C.c_int()
    _check(load_library().fire_mesh_size(ctx, C.byref(nx), C.byref(ny)), "fire_mesh_size")
    return nx.value, ny.value


def fire_time(ctx) -> float:
    return load_library().fire_time(ctx)


def fire_set_kernel(ctx, variant, kx, ky) -> int:
    return _check(load_library().fire_set_kernel(ctx, int(variant), int(kx), int(ky)),
                  "fire_set_kernel")


def fire_default_kernel(precision, nx_atm, ny_atm, sr_x, sr_y, n_sm):
    """(variant, kx, ky) that fire_init takes by default on a device with
    n_sm SMs (host computation, no device needed)."""
    v, kx, ky = C.c_int(), C.c_int(), C.c_int()
    prec = {"fp32": FIRE_FP32, "fp64": FIRE_FP64}.get(precision, precision)
    _check(load_library().fire_default_kernel(int(prec), int(nx_atm), int(ny_atm), int(sr_x),
                                              int(sr_y), int(n_sm), C.byref(v), C.byref(kx),
                                              C.byref(ky)), "fire_default_kernel")
    return v.value, kx.value, ky.value


def fire_set_adaptive(ctx, on=True) -> int:
    return _check(load_library().fire_set_adaptive(ctx, int(bool(on))), "fire_set_adaptive")


def fire_adaptive_info(ctx):
    """(on, count launches so far, last burnt fraction or -1)."""
    on, n, f = C.c_int(), C.c_longlong(), C.c_double()
    _check(load_library().fire_adaptive_info(ctx, C.byref(on), C.byref(n), C.byref(f)),
           "fire_adaptive_info")
    return bool(on.value), n.value, f.value


def fire_get_kernel(ctx):
    v, kx, ky = C.c_int(), C.c_int(), C.c_int()
    _check(load_library().fire_get_kernel(ctx, C.byref(v), C.byref(kx), C.byref(ky)),
           "fire_get_kernel")
    return v.value, kx.value, ky.value


def fire_enable_timing(ctx, on=True) -> int:
    return _check(load_library().fire_enable_timing(ctx, int(bool(on))), "fire_enable_timing")


def fire_kernel_time_ms(ctx):
    ms, n = C.c_double(), C.c_long()
    _check(load_library().fire_kernel_time_ms(ctx, C.byref(ms), C.byref(n)),
           "fire_kernel_time_ms")
    return ms.value, n.value


def _check_noalloc_tensors(items):
    """Each (name, tensor, dtype name, elements) with a torch tensor: on the
    current CUDA device, contiguous, of that dtype and element count."""
    dev = None
    for name, x, dtype, n in items:
        if x is None or not hasattr(x, "data_ptr"):
            continue
        import torch
        if not x.is_cuda:
            raise FireError(FIRE_ERR_ARG, f"fire_step_noalloc: {name} is not a CUDA tensor")
        if dev is None:
            dev = torch.cuda.current_device()
        if x.device.index != dev:
            raise FireError(FIRE_ERR_ARG,
                            f"fire_step_noalloc: {name} is on cuda:{x.device.index}, "
                            f"the current device is cuda:{dev}")
        if not x.is_contiguous():
            raise FireError(FIRE_ERR_ARG, f"fire_step_noalloc: {name} is not contiguous")
        if x.dtype != getattr(torch, dtype):
            raise FireError(FIRE_ERR_ARG,
                            f"fire_step_noalloc: {name} is {x.dtype}, expected torch.{dtype}")
        if (x.numel() != n) if name != "status" else (x.numel() < n):
            raise FireError(FIRE_ERR_ARG,
                            f"fire_step_noalloc: {name} has {x.numel()} elements, expected {n}")


def fire_step_noalloc(grid: fire_grid_desc, classes, psi_in_dev, psi_out_dev, frac_in_dev,
                      frac_out_dev, tign_dev, fuel_class_dev, spread_mult_dev, dzdx_dev,
                      dzdy_dev, wind_u_dev, wind_v_dev, t, dt, heat_sens_dev=None,
                      heat_lat_dev=None, status_dev=None, cuda_stream=None) -> int:
    """One fire step on caller-owned buffers without any allocation (see the
    header): the state is passed in and out, nothing is kept between calls.
    Torch tensors are checked before the call (device, layout, dtype and
    size; FireError FIRE_ERR_ARG on a mismatch), so that a wrong buffer never
    reaches the kernels; raw integer pointers are passed through as given."""
    nx, ny = grid.nx_atm * grid.sr_x, grid.ny_atm * grid.sr_y
    nxa, nya = grid.nx_atm, grid.ny_atm
    path = "float64" if grid.precision == FIRE_FP64 else "float32"
    _check_noalloc_tensors(
        [("psi_in", psi_in_dev, path, nx * ny), ("psi_out", psi_out_dev, path, nx * ny),
         ("frac_in", frac_in_dev, path, nx * ny), ("frac_out", frac_out_dev, path, nx * ny),
         ("tign", tign_dev, "float64", nx * ny), ("fuel_class", fuel_class_dev, "uint8", nx * ny),
         ("spread_mult", spread_mult_dev, path, nx * ny), ("dzdx", dzdx_dev, path, nx * ny),
         ("dzdy", dzdy_dev, path, nx * ny), ("wind_u", wind_u_dev, path, nya * (nxa + 1)),
         ("wind_v", wind_v_dev, path, (nya + 1) * nxa),
         ("heat_sens", heat_sens_dev, "float64", nya * nxa),
         ("heat_lat", heat_lat_dev, "float64", nya * nxa), ("status", status_dev, "int32", 1)])
    L = load_library()
    cls = make_classes(classes)
    code = L.fire_step_noalloc(C.byref(grid), cls, len(classes), _ptr(psi_in_dev),
                               _ptr(psi_out_dev), _ptr(frac_in_dev), _ptr(frac_out_dev),
                               _ptr(tign_dev), _ptr(fuel_class_dev), _ptr(spread_mult_dev),
                               _ptr(dzdx_dev), _ptr(dzdy_dev), _ptr(wind_u_dev), _ptr(wind_v_dev),
                               float(t), float(dt), _ptr(heat_sens_dev), _ptr(heat_lat_dev),
                               _ptr(status_dev), _ptr(cuda_stream) or None)
    return _check(code, "fire_step_noalloc")


def _ptr_array(items):
    arr = (_P * len(items))()
    for k, x in enumerate(items):
        arr[k] = _ptr(x)
    return arr


def fire_ensemble_create(members, cuda_stream=None) -> int:
    """members: list of dicts with the fire_init arguments (grid, classes,
    fuel_class_dev, moisture_dev, spread_mult_dev, dzdx_dev, dzdy_dev,
    ignitions; moisture_dev and spread_mult_dev optional)."""
    L = load_library()
    descs = (fire_member_desc * len(members))()
    keep = []
    for k, m in enumerate(members):
        cls = make_classes(m["classes"])
        ign = make_ignitions(list(m.get("ignitions", ())))
        keep += [cls, ign]
        descs[k].grid = m["grid"]
        descs[k].classes = C.cast(cls, C.POINTER(fire_fuel_class))
        descs[k].n_classes = len(m["classes"])
        descs[k].fuel_class_dev = _ptr(m["fuel_class_dev"])
        descs[k].moisture_dev = _ptr(m.get("moisture_dev"))
        descs[k].spread_mult_dev = _ptr(m.get("spread_mult_dev"))
        descs[k].dzdx_dev = _ptr(m["dzdx_dev"])
        descs[k].dzdy_dev = _ptr(m["dzdy_dev"])
        descs[k].ignitions = C.cast(ign, C.POINTER(fire_ignition))
        descs[k].n_ign = len(list(m.get("ignitions", ())))
    out = _P()
    _check(L.fire_ensemble_create(C.byref(out), len(members), descs, _ptr(cuda_stream) or None),
           "fire_ensemble_create")
    return out.value


def fire_ensemble_step(ens, nsteps, dt, wind_u_dev, wind_v_dev, heat_sens_dev=None,
                       heat_lat_dev=None) -> int:
    L = load_library()
    hs = _ptr_array(heat_sens_dev) if heat_sens_dev is not None else None
    hl = _ptr_array(heat_lat_dev) if heat_lat_dev is not None else None
    return _check(L.fire_ensemble_step(ens, int(nsteps), float(dt), _ptr_array(wind_u_dev),
                                       _ptr_array(wind_v_dev), hs, hl), "fire_ensemble_step")


def fire_ensemble_member(ens, member) -> int:
    out = _P()
    _check(load_library().fire_ensemble_member(ens, int(member), C.byref(out)),
           "fire_ensemble_member")
    return out.value


def fire_ensemble_status(ens, n_members=None):
    """Synchronises; returns (code, per-member codes or None)."""
    if n_members:
        arr = (C.c_int * n_members)()
        code = load_library().fire_ensemble_status(ens, arr)
        return code, list(arr)
    return load_library().fire_ensemble_status(ens, None), None


def fire_ensemble_clear_status(ens) -> int:
    return _check(load_library().fire_ensemble_clear_status(ens), "fire_ensemble_clear_status")


def fire_ensemble_set_kernel(ens, strip_columns, strip_rows) -> int:
    return _check(load_library().fire_ensemble_set_kernel(ens, int(strip_columns),
                                                          int(strip_rows)),
                  "fire_ensemble_set_kernel")


def fire_ensemble_get_kernel(ens):
    g, n = C.c_int(), C.c_int()
    _check(load_library().fire_ensemble_get_kernel(ens, C.byref(g), C.byref(n)),
           "fire_ensemble_get_kernel")
    return g.value, n.value


def fire_ensemble_set_barrier_test(ens, skip_block, spin_limit) -> int:
    return _check(load_library().fire_ensemble_set_barrier_test(ens, int(skip_block),
                                                                int(spin_limit)),
                  "fire_ensemble_set_barrier_test")


def fire_ensemble_destroy(ens) -> None:
    if ens:
        load_library().fire_ensemble_destroy(ens)


def fire_set_spread_mult(ctx, mult_dev) -> int:
    return _check(load_library().fire_set_spread_mult(ctx, _ptr(mult_dev)),
                  "fire_set_spread_mult")


def fire_set_moisture(ctx, moisture_dev) -> int:
    return _check(load_library().fire_set_moisture(ctx, _ptr(moisture_dev)), "fire_set_moisture")


def fire_set_fraction_scheme(ctx, scheme) -> int:
    return _check(load_library().fire_set_fraction_scheme(ctx, int(scheme)),
                  "fire_set_fraction_scheme")


def fire_wind_at_height(u3d, z3d, z0, z_f, out=None, cuda_stream=None):
    """The wind component at height z_f by vertical log-linear interpolation
    (fire_wind_at_height): u3d, z3d [nz][...] and z0 [...] CUDA tensors of one
    precision (float32 or float64); returns `out` (allocated like z0 if None)."""
    import torch
    nz = u3d.shape[0]
    if z3d.shape != u3d.shape or z0.shape != u3d.shape[1:]:
        raise FireError(FIRE_ERR_ARG, "fire_wind_at_height: shapes")
    if out is None:
        out = torch.empty_like(z0)
    for x in (u3d, z3d, z0, out):
        if not (x.is_cuda and x.is_contiguous() and x.dtype == z0.dtype):
            raise FireError(FIRE_ERR_ARG, "fire_wind_at_height: tensors must be contiguous "
                                          "CUDA tensors of one dtype")
    prec = FIRE_FP64 if z0.dtype == torch.float64 else FIRE_FP32
    _check(load_library().fire_wind_at_height(prec, nz, z0.numel(), _ptr(u3d), _ptr(z3d),
                                              _ptr(z0), float(z_f), _ptr(out),
                                              _ptr(cuda_stream) or None), "fire_wind_at_height")
    return out


def fire_heat_insertion(heat_sens, heat_lat, zw, rho, mu, z_ext, rth, rqv, cp=1004.0,
                        latent=2.5e6, cuda_stream=None) -> int:
    """Add the fire's heat sources to the tendencies rth, rqv [nz][...]
    (fire_heat_insertion); all float64 CUDA tensors, zw [nz+1][...], rho
    [nz][...], the fluxes and mu [...]; rth or rqv may be None."""
    nz = rho.shape[0]
    ncols = mu.numel()
    for name, x, n in (("heat_sens", heat_sens, ncols), ("heat_lat", heat_lat, ncols),
                       ("zw", zw, (nz + 1) * ncols), ("rho", rho, nz * ncols), ("mu", mu, ncols),
                       ("rth", rth, nz * ncols), ("rqv", rqv, nz * ncols)):
        if x is None:
            continue
        import torch
        if not (x.is_cuda and x.is_contiguous() and x.dtype == torch.float64 and x.numel() == n):
            raise FireError(FIRE_ERR_ARG, f"fire_heat_insertion: {name}")
    return _check(load_library().fire_heat_insertion(
        nz, ncols, _ptr(heat_sens), _ptr(heat_lat), _ptr(zw), _ptr(rho), _ptr(mu), float(z_ext),
        float(cp), float(latent), _ptr(rth), _ptr(rqv), _ptr(cuda_stream) or None),
        "fire_heat_insertion")


def fire_set_fuel_classes(ctx, classes) -> int:
    cls = make_classes(classes)
    return _check(load_library().fire_set_fuel_classes(ctx, cls, len(classes)),
                  "fire_set_fuel_classes")


def fire_adjoint(ctx, nsteps, dt, wind_u_dev, wind_v_dev, t_obs_dev, ckpt_every=20,
                 g_mult_dev=None, g_moist_dev=None, g_u_dev=None, g_v_dev=None) -> float:
    """Runs the misfit and its adjoint; returns J (gradients written in place)."""
    J = C.c_double()
    _check(load_library().fire_adjoint(ctx, int(nsteps), float(dt), _ptr(wind_u_dev),
                                       _ptr(wind_v_dev), _ptr(t_obs_dev), int(ckpt_every),
                                       C.byref(J), _ptr(g_mult_dev), _ptr(g_moist_dev),
                                       _ptr(g_u_dev), _ptr(g_v_dev)), "fire_adjoint")
    return J.value


def fire_adjoint_heat(ctx, nsteps, dt, wind_u_dev, wind_v_dev, q_obs_dev, ckpt_every=20,
                      g_mult_dev=None, g_moist_dev=None, g_u_dev=None, g_v_dev=None) -> float:
    """The heat misfit and its adjoint; returns J (gradients written in place)."""
    J = C.c_double()
    _check(load_library().fire_adjoint_heat(ctx, int(nsteps), float(dt), _ptr(wind_u_dev),
                                            _ptr(wind_v_dev), _ptr(q_obs_dev), int(ckpt_every),
                                            C.byref(J), _ptr(g_mult_dev), _ptr(g_moist_dev),
                                            _ptr(g_u_dev), _ptr(g_v_dev)), "fire_adjoint_heat")
    return J.value


def fire_autotune(ctx, wind_u_dev, wind_v_dev, dt, probe_steps=3):
    """Times candidate step-kernel shapes, keeps the fastest; returns
    (variant, kx, ky)."""
    a, b, c = C.c_int(), C.c_int(), C.c_int()
    _check(load_library().fire_autotune(ctx, _ptr(wind_u_dev), _ptr(wind_v_dev), float(dt),
                                        int(probe_steps), C.byref(a), C.byref(b), C.byref(c)),
           "fire_autotune")
    return a.value, b.value, c.value


def fire_ensemble_autotune(ens, probe_steps, dt, wind_u_dev, wind_v_dev):
    """Times candidate strip shapes of the persistent launch, keeps the
    fastest; returns (strip_columns, strip_rows)."""
    a, b = C.c_int(), C.c_int()
    _check(load_library().fire_ensemble_autotune(ens, int(probe_steps), float(dt),
                                                 _ptr_array(wind_u_dev), _ptr_array(wind_v_dev),
                                                 C.byref(a), C.byref(b)),
           "fire_ensemble_autotune")
    return a.value, b.value


def fire_destroy(ctx) -> None:
    if ctx:
        load_library().fire_destroy(ctx)


# ---------------------------------------------------------------------------
# convenience wrapper (torch for memory and streams only)
# ---------------------------------------------------------------------------

class FireModel:
    """One fire-model context on the current CUDA device.

    Inputs are copied to the device once; ``step`` takes the wind (torch CUDA
    tensors of the context precision, or anything torch can convert) and
    returns the averaged sensible and latent heat flux densities as float64
    CUDA tensors."""

    def __init__(self, nxa, nya, sr, dx_atm, classes, fuel, dzdx, dzdy, ignitions=(),
                 precision="fp32", mult=None, eps=0.4, band=1, psi_far=0.0, dy_atm=None,
                 stream=None, device=None, moisture=None):
        import torch
        self.torch = torch
        srx, sry = (sr, sr) if np.isscalar(sr) else sr
        dy_atm = dx_atm if dy_atm is None else dy_atm
        self.precision = FIRE_FP64 if precision in ("fp64", FIRE_FP64, "f64") else FIRE_FP32
        self.dtype = torch.float64 if self.precision == FIRE_FP64 else torch.float32
        self.device = torch.device(device or "cuda")
        self.nxa, self.nya, self.srx, self.sry = nxa, nya, srx, sry
        self.nx, self.ny = nxa * srx, nya * sry
        self.stream = stream or torch.cuda.current_stream(self.device)
        dev = self.device

        def t(a, dtype):
            return torch.as_tensor(np.ascontiguousarray(a)).to(dev, dtype).contiguous()

        fuel_d = t(fuel, torch.uint8)
        zx, zy = t(dzdx, self.dtype), t(dzdy, self.dtype)
        m = None if mult is None else t(mult, self.dtype)
        mo = None if moisture is None else t(moisture, self.dtype)
        grid = make_grid(nxa, nya, srx, sry, dx_atm, dy_atm, self.precision, band, eps, psi_far)
        torch.cuda.synchronize(dev)
        self.ctx = fire_init(grid, classes, fuel_d, mo, m, zx, zy, list(ignitions),
                             self.stream.cuda_stream)
        self.classes = [dict(c) for c in classes]
        self.fuel_dev = fuel_d
        self.heat_s = torch.zeros((nya, nxa), dtype=torch.float64, device=dev)
        self.heat_l = torch.zeros_like(self.heat_s)

    @classmethod
    def from_workload(cls, w, precision="fp32", **kw):
        return cls(w.nxa, w.nya, (w.srx, w.sry), w.dx_atm, w.classes, w.fuel, w.dzdx, w.dzdy,
                   w.ignitions, precision=precision, mult=w.mult, eps=w.eps, band=w.band,
                   dy_atm=w.dy_atm, moisture=w.moisture, **kw)

    def wind(self, u, v):
        torch = self.torch
        return (torch.as_tensor(np.ascontiguousarray(u)).to(self.device, self.dtype).contiguous(),
                torch.as_tensor(np.ascontiguousarray(v)).to(self.device, self.dtype).contiguous())

    def step(self, u, v, dt):
        fire_step(self.ctx, u, v, dt, self.heat_s, self.heat_l)
        return self.heat_s, self.heat_l

    def run(self, nsteps, u, v, dt):
        fire_run(self.ctx, nsteps, dt, u, v, self.heat_s, self.heat_l)
        return self.heat_s, self.heat_l

    def state(self):
        torch = self.torch
        psi = torch.empty((self.ny, self.nx), dtype=self.dtype, device=self.device)
        tign = torch.empty((self.ny, self.nx), dtype=torch.float64, device=self.device)
        frac = torch.empty_like(psi)
        t = fire_get_state(self.ctx, psi, tign, frac)
        return psi, tign, frac, t

    def set_state(self, psi, tign, frac, t):
        fire_set_state(self.ctx, psi.contiguous(), tign.contiguous(), frac.contiguous(), t)

    def status(self):
        return fire_status(self.ctx)

    def autotune(self, u, v, dt, probe_steps=3):
        return fire_autotune(self.ctx, u, v, dt, probe_steps)

    def set_mult(self, mult):
        """Per-node spread multiplier (None: 1)."""
        m = None if mult is None else self.torch.as_tensor(mult).to(self.device, self.dtype).contiguous()
        fire_set_spread_mult(self.ctx, m)

    def set_moisture(self, moisture):
        """Per-node fuel moisture [ny][nx] (None: the class moisture)."""
        mo = (None if moisture is None
              else self.torch.as_tensor(moisture).to(self.device, self.dtype).contiguous())
        fire_set_moisture(self.ctx, mo)

    def set_classes(self, classes):
        self.classes = [dict(c) for c in classes]
        fire_set_fuel_classes(self.ctx, self.classes)

    def adjoint(self, u, v, dt, nsteps, tobs, ckpt_every=20, grads=True):
        """J = 1/2 sum (t_i - t_obs)^2 after nsteps steps and (if grads) its
        gradients dJ/dm, dJ/dM_f per node and dJ/du, dJ/dv (float64 CUDA
        tensors).  Advances the model like run()."""
        torch = self.torch
        tobs = torch.as_tensor(tobs).to(self.device, torch.float64).contiguous()
        if not grads:
            return fire_adjoint(self.ctx, nsteps, dt, u, v, tobs, ckpt_every), None, None, None, None
        f64 = dict(dtype=torch.float64, device=self.device)
        gm = torch.empty((self.ny, self.nx), **f64)
        gM = torch.empty_like(gm)
        gu = torch.empty((self.nya, self.nxa + 1), **f64)
        gv = torch.empty((self.nya + 1, self.nxa), **f64)
        J = fire_adjoint(self.ctx, nsteps, dt, u, v, tobs, ckpt_every, gm, gM, gu, gv)
        return J, gm, gM, gu, gv

    def adjoint_heat(self, u, v, dt, nsteps, qobs, ckpt_every=20, grads=True):
        """J = 1/2 sum over atmospheric cells of (Q - q_obs)^2, Q the sensible
        heat released per unit area over the nsteps steps, and (if grads) its
        gradients as adjoint().  Advances the model like run()."""
        torch = self.torch
        qobs = torch.as_tensor(qobs).to(self.device, torch.float64).contiguous()
        if not grads:
            return (fire_adjoint_heat(self.ctx, nsteps, dt, u, v, qobs, ckpt_every), None, None,
                    None, None)
        f64 = dict(dtype=torch.float64, device=self.device)
        gm = torch.empty((self.ny, self.nx), **f64)
        gM = torch.empty_like(gm)
        gu = torch.empty((self.nya, self.nxa + 1), **f64)
        gv = torch.empty((self.nya + 1, self.nxa), **f64)
        J = fire_adjoint_heat(self.ctx, nsteps, dt, u, v, qobs, ckpt_every, gm, gM, gu, gv)
        return J, gm, gM, gu, gv

    @property
    def time(self):
        return fire_time(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            fire_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fire_adjoint_function(objective="arrival"):
    import torch

    heat = objective == "heat"

    class _Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, model, state0, mult, moisture, u, v, obs, dt, nsteps, ckpt_every):
            psi0, tign0, frac0, t0 = state0
            model.set_state(psi0, tign0, frac0, t0)
            model.set_mult(mult.detach())
            model.set_moisture(moisture.detach())
            ud = u.detach().to(model.device, model.dtype).contiguous()
            vd = v.detach().to(model.device, model.dtype).contiguous()
            run = model.adjoint_heat if heat else model.adjoint
            J, gm, gM, gu, gv = run(ud, vd, dt, nsteps, obs, ckpt_every)
            ctx.save_for_backward(gm, gM, gu, gv)
            ctx.dtypes = (mult.dtype, moisture.dtype, u.dtype, v.dtype)
            ctx.devices = (mult.device, moisture.device, u.device, v.device)
            return torch.tensor(J, dtype=torch.float64, device=model.device)

        @staticmethod
        def backward(ctx, gJ):
            gm, gM, gu, gv = ctx.saved_tensors
            out = [(gJ * g).to(d, dt_) for g, dt_, d in zip((gm, gM, gu, gv), ctx.dtypes,
                                                             ctx.devices)]
            return (None, None, out[0], out[1], out[2], out[3], None, None, None, None)

    if heat:
        class FireHeatAdjointFn(_Fn):
            """J(m, M_f, u, v) = 1/2 sum over atmospheric cells with a finite
            observation of (Q - q_obs)^2, Q the sensible heat released per
            unit area over nsteps steps from the given initial state, as a
            differentiable torch function of the per-node spread multiplier
            m [ny][nx], the per-node fuel moisture M_f [ny][nx] and the
            staggered wind u [nya][nxa+1], v [nya+1][nxa].  The forward call
            sets m and M_f on the model, runs fire_adjoint_heat and keeps
            the gradients; backward scales them.

            apply(model, state0, mult, moisture, u, v, q_obs, dt, nsteps,
            ckpt_every) with q_obs [nya][nxa] and state0 as for
            FireAdjointFn."""

        return FireHeatAdjointFn

    class FireAdjointFn(_Fn):
        """J(m, M_f, u, v) = 1/2 sum over nodes ignited in both of
        (t_i - t_obs)^2 after nsteps steps from the given initial state, as a
        differentiable torch function of the per-node spread multiplier m
        [ny][nx], the per-node fuel moisture M_f [ny][nx] and the staggered
        wind u [nya][nxa+1], v [nya+1][nxa].  The forward call sets m and M_f
        on the model (fire_set_spread_mult, fire_set_moisture), runs
        fire_adjoint (forward sweep, checkpoints and the reverse sweep in the
        CUDA library) and keeps the gradients, all per node as the library
        returns them; backward scales them.

        apply(model, state0, mult, moisture, u, v, t_obs, dt, nsteps, ckpt_every)
        with state0 = (psi, tign, frac, t) as returned by FireModel.state()."""

    return FireAdjointFn


def __getattr__(name):
    if name in ("FireAdjointFn", "FireHeatAdjointFn"):
        fn = _fire_adjoint_function("heat" if name == "FireHeatAdjointFn" else "arrival")
        globals()[name] = fn
        return fn
    raise AttributeError(name)
