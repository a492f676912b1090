"""Child process of test_bounds_check_gpu.py.

Runs small cases through every step-kernel variant (and the ensemble) on the
library named by the WRFFIRE_LIBRARY environment variable, or the normal one,
and saves each case's psi, t_i, F, last heat grids and status code, plus
whether the library is the bounds-checked build, to the .npz file argv[1].
Meshes: 230x170 nodes at refinement 10 with point ignitions, 65x55 at
refinement 5 (odd width: single-column loads and stores), two drip torches,
and a per-node fuel moisture (the per-node kernels).
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import torch  # noqa: E402

import paper_1102_1343_gb300 as pkg  # noqa: E402
from gpu_helpers import node_moisture  # noqa: E402
from paper_1102_1343_gb300 import synth  # noqa: E402

STEPS = 60


def meshes():
    a = synth.random_landscape(23, 17, seed=21, ignition="points", n_points=4, edge_margin=200.0,
                               steps=STEPS)
    b = synth.random_landscape(13, 11, sr=5, seed=22, ignition="line", steps=STEPS)
    c = synth.random_landscape(23, 17, seed=61, ignition="none", steps=STEPS)
    c.ignitions = [synth.drip_torch(300.0, 400.0, 3.0, 1.0, t_start=1.0, t_end=21.0,
                                    radius=15.0, speed=2.0),
                   synth.drip_torch(900.0, 300.0, -2.0, 2.5, t_start=10.25, t_end=25.0,
                                    radius=9.0, speed=4.0)]
    d = node_moisture(synth.random_landscape(23, 17, seed=23, ignition="points", n_points=4,
                                             edge_margin=200.0, steps=STEPS))
    return {"pts": a, "odd": b, "drip": c, "moist": d}


def run(w, prec, variant=None, scheme=0):
    m = pkg.FireModel.from_workload(w, precision=prec)
    if scheme:
        pkg.fire_set_fraction_scheme(m.ctx, scheme)
    if variant is not None:
        pkg.fire_set_kernel(m.ctx, *variant)
    u, v = m.wind(w.u, w.v)
    for _ in range(w.steps):
        hs, hl = m.step(u, v, w.dt)
    torch.cuda.synchronize()
    psi, tign, frac, _ = m.state()
    out = [psi.double().cpu().numpy(), tign.cpu().numpy(), frac.double().cpu().numpy(),
           hs.cpu().numpy(), hl.cpu().numpy()]
    code = m.status()
    m.close()
    return out, code


def run_ensemble(ws, prec):
    P = pkg.FIRE_FP64 if prec == "fp64" else pkg.FIRE_FP32
    dt_ = torch.float64 if prec == "fp64" else torch.float32
    keep, members, us, vs = [], [], [], []
    for w in ws:
        fuel = torch.as_tensor(w.fuel).cuda().contiguous()
        zx = torch.as_tensor(w.dzdx).to("cuda", dt_).contiguous()
        zy = torch.as_tensor(w.dzdy).to("cuda", dt_).contiguous()
        keep += [fuel, zx, zy]
        members.append(dict(grid=pkg.make_grid(w.nxa, w.nya, w.srx, w.sry, w.dx_atm, w.dy_atm, P,
                                               w.band, w.eps),
                            classes=w.classes, fuel_class_dev=fuel, dzdx_dev=zx, dzdy_dev=zy,
                            ignitions=w.ignitions))
        us.append(torch.as_tensor(w.u).to("cuda", dt_).contiguous())
        vs.append(torch.as_tensor(w.v).to("cuda", dt_).contiguous())
    ens = pkg.fire_ensemble_create(members)
    pkg.fire_ensemble_step(ens, STEPS, ws[0].dt, us, vs)
    code, _ = pkg.fire_ensemble_status(ens, len(ws))
    out = []
    for m, w in enumerate(ws):
        ctx = pkg.fire_ensemble_member(ens, m)
        psi = torch.empty((w.ny, w.nx), dtype=dt_, device="cuda")
        tign = torch.empty((w.ny, w.nx), dtype=torch.float64, device="cuda")
        frac = torch.empty_like(psi)
        pkg.fire_get_state(ctx, psi, tign, frac)
        torch.cuda.synchronize()
        out += [psi.double().cpu().numpy(), tign.cpu().numpy(), frac.double().cpu().numpy()]
    pkg.fire_ensemble_destroy(ens)
    return out, code


def main(path):
    pkg.load_library()
    res = {"checked": np.array(pkg.fire_bounds_checked())}
    ms = meshes()
    # variant, kx, ky: shapes valid at refinement 10 and 5
    f32 = {"default": None, "warp": (pkg.FIRE_KERNEL_WARP, 4, 2),
           "dense": (pkg.FIRE_KERNEL_WARP_DENSE, 4, 2), "warp4": (pkg.FIRE_KERNEL_WARP4, 8, 2),
           "march": (pkg.FIRE_KERNEL_MARCH, 8, 3), "tile": (pkg.FIRE_KERNEL_TILE, 2, 2)}
    f64 = {"default": None, "warp": (pkg.FIRE_KERNEL_WARP, 4, 2),
           "march": (pkg.FIRE_KERNEL_MARCH, 8, 3), "tile": (pkg.FIRE_KERNEL_TILE, 2, 2)}
    cases = []
    for mesh in ("pts", "odd", "drip", "moist"):
        cases += [(mesh, "fp32", name, var, 0) for name, var in f32.items()]
        cases += [(mesh, "fp64", name, var, 0) for name, var in f64.items()]
    cases += [("pts", "fp32", "linear", (pkg.FIRE_KERNEL_TILE, 2, 2), 1),
              ("pts", "fp64", "linear", (pkg.FIRE_KERNEL_TILE, 2, 2), 1)]
    for mesh, prec, name, var, scheme in cases:
        out, code = run(ms[mesh], prec, var, scheme)
        key = f"{mesh}_{prec}_{name}"
        for q, arr in enumerate(out):
            res[f"{key}_{q}"] = arr
        res[f"{key}_status"] = np.array(code)
    for prec in ("fp32", "fp64"):
        out, code = run_ensemble([ms["pts"], ms["odd"]], prec)
        for q, arr in enumerate(out):
            res[f"ens_{prec}_{q}"] = arr
        res[f"ens_{prec}_status"] = np.array(code)
    np.savez(path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
