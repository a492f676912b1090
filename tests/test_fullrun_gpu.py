"""The 2000x2000 line-fire case in full (1200 steps of 0.5 s) on the GPU in
FP64 and in FP32, against the FP64 oracle run on all host cores over the same
1200 steps.

FP64: psi, F, the ignition times of the nodes ignited in both, and every
step's two heat grids within 1e-10 norm-wise relative error.
FP32: ignition time within 0.1 s (nodes ignited in both), burnt area within
0.5 % by both definitions (#{psi <= 0} dx dy and sum (1 - F) dx dy), integrated
sensible heat within 1e-4 relative.

All three runs take the same inputs: the wind, terrain gradient and
multiplier are rounded to FP32 once (the FP32 path's inputs), and the FP64
runs take those values in double.  With WRFFIRE_ACCURACY_OUT set, the errors
are written there as JSON (the record the benchmark line reports).
"""
import json
import os

import numpy as np
import pytest

import oracle
from gpu_helpers import as_path_precision, rel_inf, state_np
from paper_1102_1343_gb300 import synth

pytestmark = pytest.mark.gpu


def test_line2000_full_run_fp32_and_fp64_against_oracle():
    import torch

    from paper_1102_1343_gb300 import build
    build.build()
    import paper_1102_1343_gb300 as pkg

    torch.cuda.set_device(0)
    w = as_path_precision(synth.line_fire_2000(), "fp32")
    area = w.dx * w.dy
    cell_area = w.dx_atm * w.dy_atm
    m64 = pkg.FireModel.from_workload(w, precision="fp64")
    m32 = pkg.FireModel.from_workload(w, precision="fp32")
    u64, v64 = m64.wind(w.u, w.v)
    u32, v32 = m32.wind(w.u, w.v)
    threads = oracle.set_threads(os.cpu_count() or 1)
    try:
        orc = oracle.OracleFire.from_workload(w)
        heat64 = 0.0
        Q = {"oracle": 0.0, "fp64": 0.0, "fp32": 0.0}
        for n in range(w.steps):
            hs64, hl64 = m64.step(u64, v64, w.dt)
            hs32, _ = m32.step(u32, v32, w.dt)
            hs_o, hl_o, _ = orc.step(w.u, w.v, w.dt)
            a, b = hs64.cpu().numpy(), hl64.cpu().numpy()
            heat64 = max(heat64, rel_inf(a, hs_o), rel_inf(b, hl_o))
            Q["oracle"] += hs_o.sum() * w.dt * cell_area
            Q["fp64"] += a.sum() * w.dt * cell_area
            Q["fp32"] += hs32.sum().item() * w.dt * cell_area
    finally:
        oracle.set_threads(1)
    torch.cuda.synchronize()
    assert m64.status() == pkg.FIRE_OK and m32.status() == pkg.FIRE_OK and orc.status == 0

    psi64, t64, f64, _ = state_np(m64)
    psi32, t32, f32, _ = state_np(m32)
    fin_o = np.isfinite(orc.tign)
    both64 = np.isfinite(t64) & fin_o
    both32 = np.isfinite(t32) & fin_o
    A_o, B_o = float((orc.psi <= 0).sum()) * area, float((1 - orc.frac).sum()) * area
    rec = {
        "workload": "line-fire-2000x2000 (200x200 atmos x10, 1 km line ignition), "
                    f"{w.steps} steps of {w.dt} s, inputs rounded to FP32 for all runs",
        "oracle_threads": threads,
        "ignited_nodes_oracle": int(fin_o.sum()),
        "burnt_area_oracle_m2": A_o,
        "fp64": {"psi_rel_inf": rel_inf(psi64, orc.psi), "frac_rel_inf": rel_inf(f64, orc.frac),
                 "tign_rel_inf": rel_inf(t64[both64], orc.tign[both64]),
                 "ignited_mismatch": int((np.isfinite(t64) != fin_o).sum()),
                 "heat_per_step_rel_inf_max": heat64,
                 "integrated_heat_rel": abs(Q["fp64"] - Q["oracle"]) / Q["oracle"]},
        "fp32": {"tign_max_abs_s": float(np.abs(t32[both32] - orc.tign[both32]).max()),
                 "ignited_mismatch": int((np.isfinite(t32) != fin_o).sum()),
                 "burnt_area_rel": abs(float((psi32 <= 0).sum()) * area - A_o) / A_o,
                 "burned_fuel_area_rel": abs(float((1 - f32).sum()) * area - B_o) / B_o,
                 "integrated_heat_rel": abs(Q["fp32"] - Q["oracle"]) / Q["oracle"],
                 "psi_rel_inf": rel_inf(psi32, orc.psi), "frac_max_abs": float(np.abs(f32 - orc.frac).max())},
        "tolerances": {"fp64_rel": 1e-10, "fp32_tign_s": 0.1, "fp32_area_rel": 0.005,
                       "fp32_heat_rel": 1e-4},
    }
    import bench  # the hash of the step-kernel sources the record belongs to
    rec["kernel_source_hash"] = bench.kernel_hash()
    print(json.dumps(rec, indent=1))
    out = os.environ.get("WRFFIRE_ACCURACY_OUT")
    if out:
        with open(out, "w") as f:
            json.dump(rec, f, indent=1)
    m64.close()
    m32.close()
    # the 1 km line (about 560 nodes at t = 0) has grown to several times that
    assert rec["ignited_nodes_oracle"] > 2000 and Q["oracle"] > 0
    e = rec["fp64"]
    assert e["psi_rel_inf"] <= 1e-10 and e["frac_rel_inf"] <= 1e-10, e
    assert e["tign_rel_inf"] <= 1e-10 and e["ignited_mismatch"] == 0, e
    assert e["heat_per_step_rel_inf_max"] <= 1e-10 and e["integrated_heat_rel"] <= 1e-10, e
    e = rec["fp32"]
    assert e["tign_max_abs_s"] <= 0.1, e
    assert e["burnt_area_rel"] <= 0.005 and e["burned_fuel_area_rel"] <= 0.005, e
    assert e["integrated_heat_rel"] <= 1e-4, e
