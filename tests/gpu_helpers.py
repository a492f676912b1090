"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare them."""
import numpy as np

import oracle
from paper_1102_1343_gb300 import synth


def rel_inf(a, b):
    """Norm-wise relative error ||a - b||_inf / ||b||_inf (absolute when b = 0)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    d = np.abs(a - b).max() if a.size else 0.0
    s = np.abs(b).max() if b.size else 0.0
    return d / s if s > 0 else d


def as_path_precision(w: synth.Workload, prec: str) -> synth.Workload:
    """The inputs as the CUDA path sees them: FP32 rounds the terrain gradient,
    the multiplier and the wind; the oracle then computes in FP64 from the
    same rounded values."""
    if prec == "fp64":
        return w
    import dataclasses
    r = lambda a: None if a is None else np.asarray(a, np.float32).astype(np.float64)
    return dataclasses.replace(w, dzdx=r(w.dzdx), dzdy=r(w.dzdy), u=r(w.u), v=r(w.v),
                               mult=r(w.mult), moisture=r(w.moisture))


def node_moisture(w, seed=5, amp=0.05, length=6.0):
    """Give w a per-node fuel moisture: each node's class moisture plus a
    smooth random field of +-amp (clipped at 0.01)."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    f = gaussian_filter(rng.standard_normal((w.ny, w.nx)), length, mode="reflect")
    f *= amp / max(np.abs(f).max(), 1e-12)
    w.moisture = np.maximum(0.01, np.array([c["fuelmc_g"] for c in w.classes])[w.fuel] + f)
    return w


def state_np(m):
    psi, tign, frac, t = m.state()
    return (psi.double().cpu().numpy(), tign.cpu().numpy(), frac.double().cpu().numpy(), t)


def compare_fp64(gpu, orc, tol=1e-10):
    """psi, F and the ignition times of the ignited nodes, norm-wise."""
    psi, tign, frac, _ = gpu
    e = {"psi": rel_inf(psi, orc.psi), "frac": rel_inf(frac, orc.frac)}
    fin_g, fin_o = np.isfinite(tign), np.isfinite(orc.tign)
    e["ignited_mismatch"] = int((fin_g != fin_o).sum())
    both = fin_g & fin_o
    e["tign"] = rel_inf(tign[both], orc.tign[both]) if both.any() else 0.0
    ok = e["psi"] <= tol and e["frac"] <= tol and e["tign"] <= tol and e["ignited_mismatch"] == 0
    return ok, e


def crop_step(w, psi, tign, frac, t, I0, J0, dt, r=1):
    """One oracle step on the atmospheric cells [I0-r, I0+r] x [J0-r, J0+r]
    starting from a given state.  The centre cell's nodes lie >= r*sr nodes
    from the crop edge, beyond the 3-node reach of one step, so its results
    equal those of a step on the whole domain.  Returns the crop oracle and
    the slices of the centre cell."""
    Ia, Ib, Ja, Jb = I0 - r, I0 + r + 1, J0 - r, J0 + r + 1
    xs = slice(Ia * w.srx, Ib * w.srx)
    ys = slice(Ja * w.sry, Jb * w.sry)
    sub = oracle.OracleFire(Ib - Ia, Jb - Ja, (w.srx, w.sry), w.dx_atm, w.classes,
                            w.fuel[ys, xs], w.dzdx[ys, xs], w.dzdy[ys, xs], [],
                            mult=None if w.mult is None else w.mult[ys, xs], eps=w.eps,
                            band=w.band, dy_atm=w.dy_atm)
    sub.set_state(psi[ys, xs], tign[ys, xs], frac[ys, xs], t)
    hs, hl, _ = sub.step(w.u[Ja:Jb, Ia:Ib + 1], w.v[Ja:Jb + 1, Ia:Ib], dt)
    cy = slice(r * w.sry, (r + 1) * w.sry)
    cx = slice(r * w.srx, (r + 1) * w.srx)
    return sub, hs[r, r], hl[r, r], (cy, cx), (ys, xs)


def check_step_on_cell(prec, sub, cy, cx, psi0, t0, psi1, tign1, frac1, hs, hl, hs_o, hl_o,
                       Hs_max, Hq_max, dt):
    """One GPU step against the oracle's crop step (crop_step) on one
    atmospheric cell: psi0 the crop's nodes before the step (the scale of
    the FP64 psi bound), psi1, tign1, frac1 the cell's nodes after it, hs / hl
    the GPU's heat of the cell.  FP64 within 1e-10;
    FP32 within the bounds of one step's rounding (psi 2e-6 relative, a
    crossing only where psi^{n+1} is within that of 0, t_i 1e-2 s, F 1e-4,
    heat the F bound times the largest heat factor / dt).  Returns whether
    the oracle has a burning node in the cell."""
    po, fo, to = sub.psi[cy, cx], sub.frac[cy, cx], sub.tign[cy, cx]
    if prec == "fp64":
        scale = max(np.abs(psi0).max(), 1.0)
        assert np.abs(psi1 - po).max() <= 1e-10 * scale
        assert np.abs(frac1 - fo).max() <= 1e-10
        assert np.array_equal(np.isfinite(tign1), np.isfinite(to))
        f = np.isfinite(to)
        assert np.abs(tign1[f] - to[f]).max(initial=0) <= 1e-10 * max(1.0, t0)
        assert abs(hs - hs_o) <= 1e-10 * max(abs(hs_o), 1.0)
        assert abs(hl - hl_o) <= 1e-10 * max(abs(hl_o), 1.0)
    else:
        # FP32 rounding of psi (relative 6e-8), of the spread rate
        # (fast pow/exp, ~1e-6) over one step
        tol_psi = 2e-6 * (1.0 + np.abs(po))
        assert np.all(np.abs(psi1 - po) <= tol_psi)
        # crossings may differ only where psi^{n+1} is within rounding of 0
        diff = np.isfinite(tign1) != np.isfinite(to)
        assert np.all(np.abs(po[diff]) <= tol_psi[diff])
        f = np.isfinite(tign1) & np.isfinite(to)
        assert np.abs(tign1[f] - to[f]).max(initial=0) <= 1e-2
        assert np.abs(frac1 - fo).max() <= 1e-4
        # heat: per-node F error bound times the largest heat factor / dt
        assert abs(hs - hs_o) <= 1e-4 * Hs_max / dt
        assert abs(hl - hl_o) <= 1e-4 * Hq_max / dt
    return bool((po <= 0).any())
