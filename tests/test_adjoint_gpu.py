"""GPU adjoint of the arrival-time misfit (fire_adjoint, FireAdjointFn)
against the oracle's reference adjoint and against central finite
differences of the GPU forward, FP64 and FP32."""

import numpy as np
import pytest

import oracle
from paper_1102_1343_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    from paper_1102_1343_gb300 import build
    build.build()
    import paper_1102_1343_gb300 as p
    p.load_library()
    assert torch.cuda.is_available()
    return p


def small_case(seed=7, dy_atm=None):
    """2 m cells, centred ignition, spread multiplier 3 (the front crosses
    several cells in 60 steps of 0.25 s); no ignition after t = 0."""
    w = synth.random_landscape(8, 8, sr=5, dx_atm=10.0, seed=seed, ignition="center", steps=60,
                               dt=0.25)
    if dy_atm is not None:
        w.dy_atm = dy_atm
    rng = np.random.default_rng(seed + 5)
    w.mult = 3.0 * (1.0 + 0.05 * rng.standard_normal((w.ny, w.nx)))
    return w


def with_node_moisture(w, seed=5):
    """A per-node fuel moisture: each node's class moisture plus a smooth
    random field of +-0.03 (clipped at 0.01)."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    f = gaussian_filter(rng.standard_normal((w.ny, w.nx)), 4.0, mode="reflect")
    f *= 0.03 / max(np.abs(f).max(), 1e-12)
    base = np.array([c["fuelmc_g"] for c in w.classes])[w.fuel]
    w.moisture = np.maximum(0.01, base + f)
    return w


def observations(w, nsteps):
    """Arrival times of an oracle 'truth' run: multiplier x1.2, moisture -0.02,
    wind x1.1 (NaN where the truth did not burn)."""
    classes = [dict(c, fuelmc_g=max(0.01, c["fuelmc_g"] - 0.02)) for c in w.classes]
    moist = None if w.moisture is None else np.maximum(0.01, w.moisture - 0.02)
    f = oracle.OracleFire.from_workload(w, classes=classes, mult=w.mult * 1.2, moisture=moist)
    for _ in range(nsteps):
        f.step(w.u * 1.1, w.v * 1.1, w.dt)
    return np.where(np.isfinite(f.tign), f.tign, np.nan)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def gpu_adjoint(pkg, w, prec, nsteps, tobs, ckpt):
    m = pkg.FireModel.from_workload(w, precision=prec)
    u, v = m.wind(w.u, w.v)
    J, gm, gM, gu, gv = m.adjoint(u, v, w.dt, nsteps, tobs, ckpt_every=ckpt)
    out = (J, gm.cpu().numpy(), gM.cpu().numpy(), gu.cpu().numpy(), gv.cpu().numpy())
    st = m.state()
    m.close()
    return out, st


@pytest.mark.parametrize("dy_atm,node_moisture", [(None, False), (14.0, False), (None, True)])
def test_fp64_matches_oracle_adjoint(pkg, dy_atm, node_moisture):
    """FP64 GPU adjoint against the oracle's reference adjoint; with a
    per-node moisture field the forward takes per-node coefficients and the
    moisture gradient is taken at each node's own moisture."""
    w = small_case(dy_atm=dy_atm)
    if node_moisture:
        w = with_node_moisture(w)
    nsteps = 60
    tobs = observations(w, nsteps)
    ref = oracle.OracleFire.from_workload(w)
    Jr, gmr, gMr, gur, gvr = ref.adjoint(w.u, w.v, w.dt, nsteps, tobs)
    assert Jr > 0
    (J, gm, gM, gu, gv), st = gpu_adjoint(pkg, w, "fp64", nsteps, tobs, ckpt=7)
    assert abs(J - Jr) <= 1e-10 * Jr
    for g, gr, name in ((gm, gmr, "mult"), (gM, gMr, "moist"), (gu, gur, "u"), (gv, gvr, "v")):
        e = rel(g, gr)
        print(f"fp64 d{name}: rel err {e:.2e}")
        assert e <= 1e-8, (name, e)
    # the call advanced the context like the forward steps: same state
    assert np.array_equal(st[1].cpu().numpy() == np.inf, ref.tign == np.inf)
    assert np.max(np.abs(st[0].cpu().numpy() - ref.psi)) <= 1e-10 * np.max(np.abs(ref.psi))


def test_checkpoint_interval_does_not_change_the_result(pkg):
    w = small_case(seed=9)
    nsteps = 40
    tobs = observations(w, nsteps)
    outs = [gpu_adjoint(pkg, w, "fp64", nsteps, tobs, ckpt=k)[0] for k in (1, 7, 40, 100)]
    for o in outs[1:]:
        assert o[0] == outs[0][0]
        for a, b in zip(o[1:], outs[0][1:]):
            assert np.array_equal(a, b)


def test_fp32_against_fp64_oracle(pkg):
    """FP32 state and partial derivatives, double adjoint fields: the gradient
    differs from the FP64 oracle's by the FP32 rounding of the forward states
    (relative 1e-7 per operation, amplified through the 1/(psi^n - psi^{n+1})
    of the ignition-time interpolation); bound 2e-3 in norm."""
    w = small_case(seed=7)
    nsteps = 60
    tobs = observations(w, nsteps)
    ref = oracle.OracleFire.from_workload(w)
    Jr, gmr, gMr, gur, gvr = ref.adjoint(w.u, w.v, w.dt, nsteps, tobs)
    (J, gm, gM, gu, gv), _ = gpu_adjoint(pkg, w, "fp32", nsteps, tobs, ckpt=20)
    print(f"fp32: J rel {abs(J - Jr) / Jr:.2e}")
    assert abs(J - Jr) <= 2e-3 * Jr
    for g, gr, name in ((gm, gmr, "mult"), (gM, gMr, "moist"), (gu, gur, "u"), (gv, gvr, "v")):
        e = rel(g, gr)
        print(f"fp32 d{name}: rel err {e:.2e}")
        assert e <= 2e-3, (name, e)


def test_fp64_gradient_matches_gpu_central_differences(pkg):
    """Directional derivatives of the GPU forward misfit (J-only calls) along
    random multiplier, wind, class-moisture and per-node moisture directions,
    away from switch points (same set of ignited nodes in the perturbed
    runs).  The per-node directions perturb a per-node moisture field set by
    fire_set_moisture (equal to the class moisture at the base point), so
    the per-node dJ/dM_f is checked node by node, not only summed over
    classes."""
    import torch
    w = small_case(seed=11)
    nsteps = 50
    tobs = observations(w, nsteps)
    m = pkg.FireModel.from_workload(w, precision="fp64")
    st0 = m.state()
    st0 = tuple(x.clone() if hasattr(x, "clone") else x for x in st0)
    u0, v0 = m.wind(w.u, w.v)
    mult0 = torch.as_tensor(w.mult).cuda().double()
    classes0 = [dict(c) for c in w.classes]
    J, gm, gM, gu, gv = m.adjoint(u0, v0, w.dt, nsteps, tobs)
    fuel = torch.as_tensor(w.fuel).cuda().long()
    gcls = torch.zeros(len(classes0), dtype=torch.float64, device="cuda").index_add_(
        0, fuel.flatten(), gM.flatten())
    ign0 = torch.isfinite(m.state()[1]).cpu().numpy()

    moist0 = torch.as_tensor(np.array([c["fuelmc_g"] for c in classes0])[w.fuel]).cuda()

    def J_at(mult, classes, u, v, moist=None):
        m.set_state(*st0)
        m.set_mult(mult)
        m.set_classes(classes)
        m.set_moisture(moist)
        Jv, *_ = m.adjoint(u, v, w.dt, nsteps, tobs, grads=False)
        ign = torch.isfinite(m.state()[1]).cpu().numpy()
        return Jv, ign

    rng = np.random.default_rng(3)
    checked = 0
    for q in range(4):
        dm = torch.as_tensor(rng.standard_normal((w.ny, w.nx))).cuda()
        du = torch.as_tensor(rng.standard_normal(w.u.shape)).cuda()
        dv = torch.as_tensor(rng.standard_normal(w.v.shape)).cuda()
        dc = rng.standard_normal(len(classes0)) * 0.01
        dM = torch.as_tensor(rng.standard_normal((w.ny, w.nx)) * 0.01).cuda()
        h = 1e-6
        cases = {
            "m": (lambda s: (mult0 + s * h * dm, classes0, u0, v0), float((gm * dm).sum())),
            "u": (lambda s: (mult0, classes0, u0 + s * h * du, v0), float((gu * du).sum())),
            "v": (lambda s: (mult0, classes0, u0, v0 + s * h * dv), float((gv * dv).sum())),
            "M": (lambda s: (mult0, [dict(c, fuelmc_g=c["fuelmc_g"] + s * h * dc[k])
                                     for k, c in enumerate(classes0)], u0, v0),
                  float(np.dot(gcls.cpu().numpy(), dc))),
            "M_node": (lambda s: (mult0, classes0, u0, v0, moist0 + s * h * dM),
                       float((gM * dM).sum())),
        }
        for name, (args, ad) in cases.items():
            Jp, ip = J_at(*args(1.0))
            Jm, im = J_at(*args(-1.0))
            if not (np.array_equal(ip, ign0) and np.array_equal(im, ign0)):
                continue
            fd = (Jp - Jm) / (2 * h)
            print(f"{name}: fd {fd:.6e} adjoint {ad:.6e}")
            assert abs(fd - ad) <= 1e-5 * max(abs(fd), 1e-3 * J), (name, q, fd, ad)
            checked += 1
    assert checked >= 15
    m.close()


def test_autograd_function(pkg):
    import torch
    w = small_case(seed=13)
    nsteps = 40
    tobs = torch.as_tensor(observations(w, nsteps)).cuda()
    m = pkg.FireModel.from_workload(w, precision="fp64")
    st0 = tuple(x.clone() if hasattr(x, "clone") else x for x in m.state())
    mult = torch.as_tensor(w.mult).cuda().double().requires_grad_(True)
    # the per-node moisture field at the class values (the same coefficients)
    moist = torch.as_tensor(np.array([c["fuelmc_g"] for c in w.classes])[w.fuel],
                            dtype=torch.float64).cuda().requires_grad_(True)
    u = torch.as_tensor(w.u).cuda().double().requires_grad_(True)
    v = torch.as_tensor(w.v).cuda().double().requires_grad_(True)
    J = pkg.FireAdjointFn.apply(m, st0, mult, moist, u, v, tobs, w.dt, nsteps, 10)
    (2.0 * J).backward()
    # against the raw entry point
    m2 = pkg.FireModel.from_workload(w, precision="fp64")
    J2, gm, gM, gu, gv = m2.adjoint(*m2.wind(w.u, w.v), w.dt, nsteps, tobs, ckpt_every=10)
    assert float(J.detach()) == J2
    assert torch.equal(mult.grad, 2.0 * gm)
    assert torch.equal(u.grad, 2.0 * gu) and torch.equal(v.grad, 2.0 * gv)
    assert torch.equal(moist.grad, 2.0 * gM)
    # a second evaluation from the same initial state gives the same J
    J3 = pkg.FireAdjointFn.apply(m, st0, mult.detach(), moist.detach(), u.detach(),
                                 v.detach(), tobs, w.dt, nsteps, 10)
    assert float(J3) == float(J.detach())
    m.close()
    m2.close()


@pytest.mark.parametrize("prec,nsteps,ckpt,grads", [("fp32", 30, 20, False),
                                                    ("fp32", 31, 1, False),
                                                    ("fp64", 30, 1, True),
                                                    ("fp32", 29, 1, True)])
def test_misfit_only_call_advances_like_run(pkg, prec, nsteps, ckpt, grads):
    """The adjoint call leaves the context where fire_run leaves it, also
    when every state is kept (its forward then launches the step kernel on
    the checkpoint slots itself)."""
    import torch
    w = small_case(seed=7)
    tobs = observations(w, nsteps)
    a = pkg.FireModel.from_workload(w, precision=prec)
    b = pkg.FireModel.from_workload(w, precision=prec)
    u, v = a.wind(w.u, w.v)
    J, *_ = a.adjoint(u, v, w.dt, nsteps, tobs, ckpt_every=ckpt, grads=grads)
    b.run(nsteps, u, v, w.dt)
    sa, sb = a.state(), b.state()
    for x, y in zip(sa[:3], sb[:3]):
        assert torch.equal(x, y)
    assert sa[3] == sb[3]
    ti = sb[1].cpu().numpy()
    ok = np.isfinite(ti) & np.isfinite(tobs)
    assert abs(J - 0.5 * np.sum((ti[ok] - tobs[ok]) ** 2)) <= 1e-12 * max(J, 1.0)
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_adjoint_edge_cases(pkg, prec):
    """One reverse step after 40 forward steps, against the oracle's adjoint
    from the same state (only the nodes that cross in that step carry a
    gradient; earlier ignition times are constants); a window with no
    observed node (J = 0 and every gradient exactly 0); no step at all
    (refused)."""
    w = small_case(seed=11)
    tobs = observations(w, 41)
    ref = oracle.OracleFire.from_workload(w)
    for _ in range(40):
        ref.step(w.u, w.v, w.dt)
    Jr, gmr, gMr, gur, gvr = ref.adjoint(w.u, w.v, w.dt, 1, tobs)
    m = pkg.FireModel.from_workload(w, precision=prec)
    u, v = m.wind(w.u, w.v)
    m.run(40, u, v, w.dt)
    J, gm, gM, gu, gv = m.adjoint(u, v, w.dt, 1, tobs)
    tol = 1e-8 if prec == "fp64" else 2e-3
    assert Jr > 0 and abs(J - Jr) <= (1e-10 if prec == "fp64" else 2e-3) * Jr
    assert np.abs(gmr).max() > 0
    for g, gr, name in ((gm, gmr, "mult"), (gM, gMr, "moist"), (gu, gur, "u"), (gv, gvr, "v")):
        assert rel(g.cpu().numpy(), gr) <= tol, name
    J0, *g0 = m.adjoint(u, v, w.dt, 5, np.full((w.ny, w.nx), np.nan))
    assert J0 == 0.0
    for g in g0:
        assert not bool(g.any())
    with pytest.raises(pkg.FireError) as e:
        m.adjoint(u, v, w.dt, 0, tobs)
    assert e.value.code == pkg.FIRE_ERR_ARG
    m.close()


@pytest.mark.parametrize("misfit", ["arrival", "heat"])
def test_fp32_adjoint_does_not_depend_on_the_forward_kernel(pkg, misfit):
    """The FP32 warp kernels (two-column, dense, four-column) give the same
    forward bits, so the adjoint over them gives the same J and gradients bit
    for bit (every state kept, and checkpoints every 7 steps)."""
    w = synth.random_landscape(23, 17, seed=12, ignition="points", n_points=4,
                               edge_margin=150.0, ignition_radius=25.0, steps=40)
    w.mult = 1.0 + 0.05 * np.random.default_rng(13).standard_normal((w.ny, w.nx))
    nsteps = 40
    obs = observations(w, nsteps) if misfit == "arrival" else heat_observations(w, nsteps)
    for ckpt in (1, 7):
        outs = []
        for var, kx in ((pkg.FIRE_KERNEL_WARP, 6), (pkg.FIRE_KERNEL_WARP_DENSE, 6),
                        (pkg.FIRE_KERNEL_WARP4, 12)):
            m = pkg.FireModel.from_workload(w, precision="fp32")
            pkg.fire_set_kernel(m.ctx, var, kx, 2)
            u, v = m.wind(w.u, w.v)
            f = m.adjoint if misfit == "arrival" else m.adjoint_heat
            J, *g = f(u, v, w.dt, nsteps, obs, ckpt_every=ckpt)
            outs.append((J, [x.cpu().numpy() for x in g]))
            m.close()
        assert outs[0][0] > 0
        for J, g in outs[1:]:
            assert J == outs[0][0], ckpt
            for a, b in zip(g, outs[0][1]):
                assert np.array_equal(a, b), ckpt


def test_pending_ignition_is_rejected(pkg):
    w = small_case(seed=7)
    w.ignitions = w.ignitions + [synth.point_ignition(30.0, 30.0, radius=4.0, t_start=2.0)]
    m = pkg.FireModel.from_workload(w, precision="fp64")
    u, v = m.wind(w.u, w.v)
    tobs = np.full((w.ny, w.nx), np.nan)
    with pytest.raises(pkg.FireError) as e:
        m.adjoint(u, v, w.dt, 20, tobs)
    assert e.value.code == pkg.FIRE_ERR_STATE
    m.close()


def test_full_size_fp64_matches_oracle(pkg):
    """The 510x510 adjoint workload (51 atmos cells x 10), 400 steps of 0.5 s,
    checkpoints every 20 steps, against the oracle's reference adjoint."""
    w, truth = synth.adjoint_case()
    f = oracle.OracleFire.from_workload(w, classes=truth["classes"], mult=truth["mult"])
    for _ in range(w.steps):
        f.step(w.u * truth["wind_scale"], w.v * truth["wind_scale"], w.dt)
    tobs = np.where(np.isfinite(f.tign), f.tign, np.nan)
    ref = oracle.OracleFire.from_workload(w)
    Jr, gmr, gMr, gur, gvr = ref.adjoint(w.u, w.v, w.dt, w.steps, tobs)
    assert Jr > 0
    (J, gm, gM, gu, gv), _ = gpu_adjoint(pkg, w, "fp64", w.steps, tobs, ckpt=20)
    assert abs(J - Jr) <= 1e-10 * Jr
    for g, gr, name in ((gm, gmr, "mult"), (gM, gMr, "moist"), (gu, gur, "u"), (gv, gvr, "v")):
        e = rel(g, gr)
        print(f"510x510 fp64 d{name}: rel err {e:.2e}")
        assert e <= 1e-8, (name, e)


def test_full_size_central_differences_32_directions(pkg):
    """The 510x510 adjoint workload (400 steps of 0.5 s, checkpoints every
    20, FP64): the gradient against central differences of the GPU forward
    misfit along 40 random directions (8 each of the multiplier, u, v, the
    class moisture and a per-node moisture field set by fire_set_moisture,
    equal to the class moisture at the base point), skipping directions
    whose perturbed runs change the set of ignited nodes (a switch point)."""
    import os
    import torch
    w, truth = synth.adjoint_case()
    threads = oracle.set_threads(len(os.sched_getaffinity(0)))
    try:
        f = oracle.OracleFire.from_workload(w, classes=truth["classes"], mult=truth["mult"])
        for _ in range(w.steps):
            f.step(w.u * truth["wind_scale"], w.v * truth["wind_scale"], w.dt)
    finally:
        oracle.set_threads(1)
    assert threads >= 1
    tobs = np.where(np.isfinite(f.tign), f.tign, np.nan)
    m = pkg.FireModel.from_workload(w, precision="fp64")
    st0 = m.state()
    st0 = tuple(x.clone() if hasattr(x, "clone") else x for x in st0)
    u0, v0 = m.wind(w.u, w.v)
    mult0 = torch.ones((w.ny, w.nx), dtype=torch.float64, device="cuda")
    classes0 = [dict(c) for c in w.classes]
    J, gm, gM, gu, gv = m.adjoint(u0, v0, w.dt, w.steps, tobs, ckpt_every=20)
    fuel = torch.as_tensor(w.fuel).cuda().long()
    gcls = torch.zeros(len(classes0), dtype=torch.float64, device="cuda").index_add_(
        0, fuel.flatten(), gM.flatten())
    ign0 = torch.isfinite(m.state()[1]).cpu().numpy()
    # a slow fire: by t = 200 s a handful of nodes around the centre ignited
    assert J > 0 and ign0.sum() >= 10

    moist0 = torch.as_tensor(np.array([c["fuelmc_g"] for c in classes0])[w.fuel]).cuda()

    def J_at(mult, classes, u, v, moist=None):
        m.set_state(*st0)
        m.set_mult(mult)
        m.set_classes(classes)
        m.set_moisture(moist)
        Jv, *_ = m.adjoint(u, v, w.dt, w.steps, tobs, ckpt_every=20, grads=False)
        return Jv, torch.isfinite(m.state()[1]).cpu().numpy()

    rng = np.random.default_rng(404)
    h = 1e-6
    checked, worst = 0, 0.0
    for q in range(8):
        dm = torch.as_tensor(rng.standard_normal((w.ny, w.nx))).cuda()
        du = torch.as_tensor(rng.standard_normal(w.u.shape)).cuda()
        dv = torch.as_tensor(rng.standard_normal(w.v.shape)).cuda()
        dc = rng.standard_normal(len(classes0)) * 0.01
        dM = torch.as_tensor(rng.standard_normal((w.ny, w.nx)) * 0.01).cuda()
        cases = {
            "m": (lambda s: (mult0 + s * h * dm, classes0, u0, v0), float((gm * dm).sum())),
            "u": (lambda s: (mult0, classes0, u0 + s * h * du, v0), float((gu * du).sum())),
            "v": (lambda s: (mult0, classes0, u0, v0 + s * h * dv), float((gv * dv).sum())),
            "M": (lambda s: (mult0, [dict(c, fuelmc_g=c["fuelmc_g"] + s * h * dc[k])
                                     for k, c in enumerate(classes0)], u0, v0),
                  float(np.dot(gcls.cpu().numpy(), dc))),
            "M_node": (lambda s: (mult0, classes0, u0, v0, moist0 + s * h * dM),
                       float((gM * dM).sum())),
        }
        for name, (args, ad) in cases.items():
            Jp, ip = J_at(*args(1.0))
            Jm, im = J_at(*args(-1.0))
            if not (np.array_equal(ip, ign0) and np.array_equal(im, ign0)):
                continue
            fd = (Jp - Jm) / (2 * h)
            err = abs(fd - ad) / max(abs(fd), 1e-3 * J)
            print(f"{name} {q}: fd {fd:.6e} adjoint {ad:.6e} rel {err:.1e}")
            assert err <= 1e-5, (name, q, fd, ad)
            worst = max(worst, err)
            checked += 1
    print("checked", checked, "of 40, worst rel", worst)
    assert checked >= 20
    m.close()


# ---------------------------------------------------------------------------
# heat misfit (fire_adjoint_heat)
# ---------------------------------------------------------------------------

def heat_observations(w, nsteps):
    """Sensible heat released per atmospheric cell over the run by an oracle
    'truth' run (multiplier x1.2, moisture -0.02, wind x1.1): the time
    integral of its heat flux output."""
    classes = [dict(c, fuelmc_g=max(0.01, c["fuelmc_g"] - 0.02)) for c in w.classes]
    moist = None if w.moisture is None else np.maximum(0.01, w.moisture - 0.02)
    f = oracle.OracleFire.from_workload(w, classes=classes, mult=w.mult * 1.2, moisture=moist)
    Q = np.zeros((w.nya, w.nxa))
    for _ in range(nsteps):
        hs, _, _ = f.step(w.u * 1.1, w.v * 1.1, w.dt)
        Q += hs * w.dt
    return Q


def gpu_adjoint_heat(pkg, w, prec, nsteps, qobs, ckpt):
    m = pkg.FireModel.from_workload(w, precision=prec)
    u, v = m.wind(w.u, w.v)
    J, gm, gM, gu, gv = m.adjoint_heat(u, v, w.dt, nsteps, qobs, ckpt_every=ckpt)
    out = (J, gm.cpu().numpy(), gM.cpu().numpy(), gu.cpu().numpy(), gv.cpu().numpy())
    m.close()
    return out


@pytest.mark.parametrize("variant", ["center", "anisotropic", "corner", "node_moisture"])
def test_heat_fp64_matches_oracle_adjoint(pkg, variant):
    w = small_case(dy_atm=14.0 if variant == "anisotropic" else None)
    if variant == "node_moisture":
        w = with_node_moisture(w)
    if variant == "corner":
        # the fire at the domain corner: the quadrature's ghosts carry t_i
        w.ignitions = [synth.point_ignition(1.0, 1.0, radius=7.0)]
    nsteps = 50
    qobs = heat_observations(w, nsteps)
    qobs[0, 0] = np.nan  # an unobserved cell
    ref = oracle.OracleFire.from_workload(w)
    Jr, gmr, gMr, gur, gvr = ref.adjoint_heat(w.u, w.v, w.dt, nsteps, qobs)
    assert Jr > 0
    J, gm, gM, gu, gv = gpu_adjoint_heat(pkg, w, "fp64", nsteps, qobs, ckpt=7)
    assert abs(J - Jr) <= 1e-10 * Jr
    for g, gr, name in ((gm, gmr, "mult"), (gM, gMr, "moist"), (gu, gur, "u"), (gv, gvr, "v")):
        e = rel(g, gr)
        print(f"heat {variant} fp64 d{name}: rel err {e:.2e}")
        assert e <= 1e-8, (name, e)


def test_heat_checkpoint_interval_and_misfit_only_call(pkg):
    w = small_case(seed=9)
    nsteps = 40
    qobs = heat_observations(w, nsteps)
    outs = [gpu_adjoint_heat(pkg, w, "fp64", nsteps, qobs, ckpt=k) for k in (1, 7, 40)]
    for o in outs[1:]:
        assert o[0] == outs[0][0]
        for a, b in zip(o[1:], outs[0][1:]):
            assert np.array_equal(a, b)
    m = pkg.FireModel.from_workload(w, precision="fp64")
    u, v = m.wind(w.u, w.v)
    J, *rest = m.adjoint_heat(u, v, w.dt, nsteps, qobs, grads=False)
    assert J == outs[0][0] and all(r is None for r in rest)
    m.close()


def test_heat_fp32_against_fp64_oracle(pkg):
    """FP32 state and partials: the heat-misfit gradient within 2e-3 of the
    FP64 oracle's in norm."""
    w = small_case(seed=13)
    nsteps = 50
    qobs = heat_observations(w, nsteps)
    ref = oracle.OracleFire.from_workload(w)
    Jr, gmr, gMr, gur, gvr = ref.adjoint_heat(w.u, w.v, w.dt, nsteps, qobs)
    J, gm, gM, gu, gv = gpu_adjoint_heat(pkg, w, "fp32", nsteps, qobs, ckpt=10)
    print("heat fp32 J", J, Jr)
    assert abs(J - Jr) <= 2e-3 * Jr
    for g, gr, name in ((gm, gmr, "mult"), (gM, gMr, "moist"), (gu, gur, "u"), (gv, gvr, "v")):
        e = rel(g, gr)
        print(f"heat fp32 d{name}: rel err {e:.2e}")
        assert e <= 2e-3, (name, e)


def test_heat_autograd_function(pkg):
    import torch
    w = small_case(seed=13)
    nsteps = 40
    qobs = torch.as_tensor(heat_observations(w, nsteps)).cuda()
    m = pkg.FireModel.from_workload(w, precision="fp64")
    st0 = tuple(x.clone() if hasattr(x, "clone") else x for x in m.state())
    mult = torch.as_tensor(w.mult).cuda().double().requires_grad_(True)
    moist = torch.as_tensor(np.array([c["fuelmc_g"] for c in w.classes])[w.fuel],
                            dtype=torch.float64).cuda().requires_grad_(True)
    u = torch.as_tensor(w.u).cuda().double().requires_grad_(True)
    v = torch.as_tensor(w.v).cuda().double().requires_grad_(True)
    J = pkg.FireHeatAdjointFn.apply(m, st0, mult, moist, u, v, qobs, w.dt, nsteps, 10)
    (0.5 * J).backward()
    m2 = pkg.FireModel.from_workload(w, precision="fp64")
    J2, gm, gM, gu, gv = m2.adjoint_heat(*m2.wind(w.u, w.v), w.dt, nsteps, qobs, ckpt_every=10)
    assert float(J.detach()) == J2 and J2 > 0
    assert torch.equal(mult.grad, 0.5 * gm)
    assert torch.equal(u.grad, 0.5 * gu) and torch.equal(v.grad, 0.5 * gv)
    assert torch.equal(moist.grad, 0.5 * gM)
    m.close()
    m2.close()
