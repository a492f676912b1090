"""The C-ABI library loads on a machine without a GPU and exports every entry
point include/wrffire.h declares; argument validation answers without touching
the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "wrffire.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fire_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1102_1343_gb300 import build
    build.build()
    import paper_1102_1343_gb300 as pkg
    return pkg.load_library()


def test_header_declares_the_abi():
    syms = declared_symbols()
    for s in ("fire_init", "fire_step", "fire_step_host", "fire_run", "fire_status",
              "fire_get_state", "fire_set_state", "fire_destroy", "fire_strerror"):
        assert s in syms


def header_constants():
    """FIRE_* names with their values: #define lines and enumerators."""
    src = open(os.path.join(ROOT, "include", "wrffire.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {k: int(v) for k, v in re.findall(r"#define\s+(FIRE_[A-Z_0-9]+)\s+(-?\d+)", src)}
    for body in re.findall(r"enum\s+\w+\s*\{(.*?)\}", src, flags=re.S):
        out.update({k: int(v) for k, v in re.findall(r"(FIRE_[A-Z_0-9]+)\s*=\s*(-?\d+)", body)})
    return out


def test_binding_constants_match_the_header():
    import paper_1102_1343_gb300 as pkg
    consts = header_constants()
    assert {"FIRE_OK", "FIRE_ERR_BOUNDS", "FIRE_KERNEL_WARP_DENSE", "FIRE_MAX_MEMBERS"} <= set(consts)
    for k, v in consts.items():
        assert getattr(pkg, k) == v, k


def test_library_exports_every_declared_symbol(lib):
    import paper_1102_1343_gb300 as pkg
    for s in declared_symbols():
        assert hasattr(lib, s), s
    assert set(pkg.ABI_SYMBOLS) <= set(declared_symbols())


def test_strerror_and_argument_checks_without_gpu(lib):
    import paper_1102_1343_gb300 as pkg
    assert pkg.fire_strerror(pkg.FIRE_ERR_BOUNDARY).startswith("fire reached")
    out = C.c_void_p()
    assert lib.fire_init(C.byref(out), None, None, 0, None, None, None, None, None, None, 0,
                         None) == pkg.FIRE_ERR_ARG
    assert out.value is None
    g = pkg.make_grid(10, 10, 10, 10, 60.0, 60.0)
    cls = pkg.make_classes([{"fgi": 0.5, "weight": 7.0, "savr": 1e4, "fueldepthm": 0.3,
                             "fueldens": 500.0, "fuelmce": 0.3, "se": 0.01}])
    # no fuel class: rejected before any device call
    assert lib.fire_init(C.byref(out), C.byref(g), cls, 0, 1, 1, None, 1, 1, None, 0,
                         None) == pkg.FIRE_ERR_ARG
    assert lib.fire_set_moisture(None, None) == pkg.FIRE_ERR_ARG
    bad = pkg.make_grid(1, 1, 1, 1, 60.0, 60.0)  # a 1x1 fire mesh cannot be extrapolated
    assert lib.fire_init(C.byref(out), C.byref(bad), cls, 1, 1, None, None, 1, 1, None, 0,
                         None) == pkg.FIRE_ERR_ARG
    assert lib.fire_step(None, None, None, 0.5, None, None) == pkg.FIRE_ERR_ARG
    assert lib.fire_status(None) == pkg.FIRE_ERR_ARG


def test_null_context_is_rejected_by_every_entry_point(lib):
    """Each call returns a status and never aborts: a null context (or null
    required pointers) gives FIRE_ERR_ARG before any device work, so this
    runs without a GPU."""
    import paper_1102_1343_gb300 as pkg
    J = C.c_double()
    i1, i2, i3 = C.c_int(), C.c_int(), C.c_int()
    E = pkg.FIRE_ERR_ARG
    assert lib.fire_run(None, 3, 0.5, None, None, None, None) == E
    assert lib.fire_step_host(None, None, None, 0.5, None, None) == E
    assert lib.fire_get_state(None, None, None, None, None) == E
    assert lib.fire_set_state(None, None, None, None, 0.0) == E
    assert lib.fire_set_kernel(None, 0, 1, 1) == E
    assert lib.fire_get_kernel(None, C.byref(i1), C.byref(i2), C.byref(i3)) == E
    assert lib.fire_adjoint(None, 10, 0.5, None, None, None, 5, C.byref(J), None, None, None,
                            None) == E
    assert lib.fire_adjoint_heat(None, 10, 0.5, None, None, None, 5, C.byref(J), None, None,
                                 None, None) == E
    assert lib.fire_autotune(None, None, None, 0.5, 2, C.byref(i1), C.byref(i2),
                             C.byref(i3)) == E
    assert lib.fire_default_kernel(pkg.FIRE_FP32, 10, 10, 10, 10, 0, C.byref(i1), C.byref(i2),
                                   C.byref(i3)) == E


GOOD_CLASS = {"fgi": 0.5, "weight": 7.0, "savr": 1e4, "fueldepthm": 0.3, "fueldens": 500.0,
              "fuelmce": 0.3, "se": 0.01}


@pytest.mark.parametrize("case", ["dx0", "dxnan", "dyneg", "sr0", "nx0", "prec", "band0",
                                  "epsneg", "epsnan", "psifarnan", "nxhuge", "ign_nan",
                                  "ign_radius", "drip_speed", "drip_tend", "classes65",
                                  "ign257"])
def test_init_rejects_each_invalid_argument_without_gpu(lib, case):
    """Every argument rule of fire_init answers FIRE_ERR_ARG before any device
    call (so this runs without a GPU), and leaves no context."""
    import paper_1102_1343_gb300 as pkg
    grid = dict(nx_atm=10, ny_atm=10, sr_x=10, sr_y=10, dx_atm=60.0, dy_atm=60.0,
                precision=pkg.FIRE_FP32, boundary_band=1, eps_visc=0.4, psi_far=0.0)
    ign = [dict(ax=300.0, ay=300.0, bx=300.0, by=300.0, t_start=0.0, radius=10.0, speed=0.0)]
    classes = [GOOD_CLASS]
    bad_grid = {"dx0": ("dx_atm", 0.0), "dxnan": ("dx_atm", float("nan")),
                "dyneg": ("dy_atm", -60.0), "sr0": ("sr_x", 0), "nx0": ("nx_atm", 0),
                "prec": ("precision", 7), "band0": ("boundary_band", 0),
                "epsneg": ("eps_visc", -0.1), "epsnan": ("eps_visc", float("nan")),
                "psifarnan": ("psi_far", float("nan")), "nxhuge": ("nx_atm", 1 << 28)}
    if case in bad_grid:
        k, v = bad_grid[case]
        grid[k] = v
    elif case == "ign_nan":
        ign[0]["ax"] = float("nan")
    elif case == "ign_radius":
        ign[0]["radius"] = -1.0
    elif case == "drip_speed":  # a drip torch needs a growth speed
        ign[0].update(vx=1.0, t_end=10.0)
    elif case == "drip_tend":  # and an end no earlier than its start
        ign[0].update(vx=1.0, speed=1.0, t_start=5.0, t_end=4.0)
    elif case == "classes65":
        classes = [GOOD_CLASS] * (pkg.FIRE_MAX_CLASSES + 1)
    elif case == "ign257":
        ign = ign * (pkg.FIRE_MAX_IGNITIONS + 1)
    g = pkg.make_grid(grid["nx_atm"], grid["ny_atm"], grid["sr_x"], grid["sr_y"],
                      grid["dx_atm"], grid["dy_atm"], grid["precision"], grid["boundary_band"],
                      grid["eps_visc"], grid["psi_far"])
    cls = pkg.make_classes(classes)
    igs = pkg.make_ignitions(ign)
    out = C.c_void_p()
    # nonzero dummies stand for the device pointers: the checks come first
    assert lib.fire_init(C.byref(out), C.byref(g), cls, len(classes), 1, None, None, 1, 1, igs,
                         len(ign), None) == pkg.FIRE_ERR_ARG, case
    assert out.value is None


def test_ensemble_create_checks_without_gpu(lib):
    """No members, more than FIRE_MAX_MEMBERS, or members of two precisions:
    FIRE_ERR_ARG before any device call."""
    import paper_1102_1343_gb300 as pkg
    cls = pkg.make_classes([GOOD_CLASS])

    def descs(precs):
        d = (pkg.fire_member_desc * max(1, len(precs)))()
        for k, prec in enumerate(precs):
            d[k].grid = pkg.make_grid(10, 10, 10, 10, 60.0, 60.0, prec)
            d[k].classes = C.cast(cls, C.POINTER(pkg.fire_fuel_class))
            d[k].n_classes = 1
            d[k].fuel_class_dev = d[k].dzdx_dev = d[k].dzdy_dev = 1
        return d
    out = C.c_void_p()
    E = pkg.FIRE_ERR_ARG
    assert lib.fire_ensemble_create(C.byref(out), 0, descs([]), None) == E
    n = pkg.FIRE_MAX_MEMBERS + 1
    assert lib.fire_ensemble_create(C.byref(out), n, descs([pkg.FIRE_FP32] * n), None) == E
    assert lib.fire_ensemble_create(C.byref(out), 2, descs([pkg.FIRE_FP32, pkg.FIRE_FP64]),
                                    None) == E
    assert lib.fire_ensemble_create(None, 1, descs([pkg.FIRE_FP32]), None) == E
    assert out.value is None


def test_absurd_mesh_is_out_of_memory_without_gpu(lib):
    """A mesh whose state fits on no device (6.9e10 nodes) is refused with
    FIRE_ERR_OOM before anything is allocated (no device needed)."""
    import paper_1102_1343_gb300 as pkg
    out = C.c_void_p()
    g = pkg.make_grid(26214, 26214, 10, 10, 60.0, 60.0)
    cls = pkg.make_classes([{"fgi": 0.5, "weight": 7.0, "savr": 1e4, "fueldepthm": 0.3,
                             "fueldens": 500.0, "fuelmce": 0.3, "se": 0.01}])
    assert lib.fire_init(C.byref(out), C.byref(g), cls, 1, 1, None, None, 1, 1, None, 0,
                         None) == pkg.FIRE_ERR_OOM
    assert out.value is None


@pytest.mark.parametrize("field", ["savr", "fueldepthm", "fueldens", "fuelmce", "se", "weight"])
def test_noalloc_checks_fuel_classes_like_fire_init(lib, field):
    """fire_step_noalloc refuses the fuel classes fire_init refuses (a
    Rothermel class with a non-positive sigma, depth, density, moisture of
    extinction or mineral content, or a non-positive weight), before any
    device call."""
    import paper_1102_1343_gb300 as pkg
    from paper_1102_1343_gb300 import synth
    bad = dict(synth.nominal_class(), **{field: 0.0})
    g = pkg.make_grid(4, 4, 10, 10, 60.0, 60.0)
    with pytest.raises(pkg.FireError) as e:
        pkg.fire_step_noalloc(g, [bad], 1, 2, 3, 4, 5, 6, None, 7, 8, 9, 10, 0.0, 0.5)
    assert e.value.code == pkg.FIRE_ERR_ARG
    out = C.c_void_p()
    assert lib.fire_init(C.byref(out), C.byref(g), pkg.make_classes([bad]), 1, 1, None, None, 1,
                         1, None, 0, None) == pkg.FIRE_ERR_ARG


def test_noalloc_binding_refuses_host_tensors(lib):
    """The binding checks torch tensors before the call: a host tensor never
    reaches the kernels (FIRE_ERR_ARG, no device needed)."""
    import torch

    import paper_1102_1343_gb300 as pkg
    from paper_1102_1343_gb300 import synth
    g = pkg.make_grid(4, 4, 10, 10, 60.0, 60.0)
    psi = torch.zeros(40 * 40, dtype=torch.float64)
    with pytest.raises(pkg.FireError) as e:
        pkg.fire_step_noalloc(g, [synth.nominal_class()], psi, 2, 3, 4, 5, 6, None, 7, 8, 9, 10,
                              0.0, 0.5)
    assert e.value.code == pkg.FIRE_ERR_ARG and "psi_in" in str(e.value)


def test_coupling_entry_points_check_arguments_without_gpu(lib):
    import paper_1102_1343_gb300 as pkg
    E = pkg.FIRE_ERR_ARG
    assert lib.fire_wind_at_height(pkg.FIRE_FP64, 0, 10, 1, 1, 1, 6.1, 1, None) == E
    assert lib.fire_wind_at_height(7, 5, 10, 1, 1, 1, 6.1, 1, None) == E
    assert lib.fire_wind_at_height(pkg.FIRE_FP32, 5, 10, None, 1, 1, 6.1, 1, None) == E
    assert lib.fire_heat_insertion(10, 100, 1, 1, 1, 1, 1, 0.0, 1004.0, 2.5e6, 1, 1, None) == E
    assert lib.fire_heat_insertion(10, 100, None, 1, 1, 1, 1, 50.0, 1004.0, 2.5e6, 1, 1,
                                   None) == E
    assert lib.fire_heat_insertion(10, 100, 1, 1, 1, 1, 1, 50.0, 1004.0, 2.5e6, None, None,
                                   None) == E
