"""The domain decomposition of one fire (paper_1102_1343_gb300/decomp.py) with
the CUDA step kernels as the per-patch engine, on one GPU: every patch of a
2x2 split is its own context on its extended mesh, and before each step its 3
halo node rows / columns are refreshed from the neighbours' own nodes (device
copies issued by the host between the steps; no kernel waits on another).
With a power-of-two refinement (8) the assembled patches equal the whole-mesh
run of the same kernel bit for bit: psi, t_i, F and every step's two heat
grids, in FP64 and FP32, also when every halo node deeper than the refreshed
ones holds random values before each step (also on a 3x3 split, whose
interior patch takes its halo from all eight neighbours), with the 2-D tile,
the warp-strip and the marching-strip kernels.  The ranks of a multi-GPU run
would do the same copies over NVLink or NCCL; this test covers the patch
arithmetic with the real kernels, tests/test_decomposition.py the exchange
between processes."""
import numpy as np
import pytest

from paper_1102_1343_gb300 import decomp, synth

pytestmark = pytest.mark.gpu

# kernels valid on every patch: 2-D tiles of 2x2 atmospheric cells, warp
# strips of 4x2 cells (32 columns), marching strips of 4x2 cells
KERNELS = {"tile": (0, 2, 2), "warp": (2, 4, 2), "march": (1, 4, 2)}


@pytest.fixture(scope="module")
def pkg():
    import torch
    from paper_1102_1343_gb300 import build
    build.build()
    import paper_1102_1343_gb300 as p
    p.load_library()
    assert torch.cuda.is_available()
    return p


def case():
    w = synth.random_landscape(12, 9, sr=8, seed=71, ignition="points", n_points=4,
                               edge_margin=100.0, steps=60)
    w.ignitions = w.ignitions + [synth.line_ignition(200.0, 250.0, 520.0, 290.0, radius=8.0,
                                                     t_start=2.0, speed=1.5),
                                 synth.point_ignition(5.0, 300.0, radius=9.0)]
    w.mult = 2.0 + np.random.default_rng(3).uniform(0.0, 1.0, (w.ny, w.nx))
    return w


def _shift(g, x0, y0):
    g = dict(g)
    for k in ("ax", "bx"):
        g[k] -= x0
    for k in ("ay", "by"):
        g[k] -= y0
    return g


def model(pkg, w, prec, psi_far, kernel, sl=None, x0=0.0, y0=0.0, nxa=None, nya=None):
    ey, ex = sl if sl is not None else (slice(None), slice(None))
    m = pkg.FireModel(nxa or w.nxa, nya or w.nya, (w.srx, w.sry), w.dx_atm, w.classes,
                      w.fuel[ey, ex], w.dzdx[ey, ex], w.dzdy[ey, ex],
                      [_shift(g, x0, y0) for g in w.ignitions], precision=prec,
                      mult=w.mult[ey, ex], eps=w.eps, band=w.band, psi_far=psi_far,
                      dy_atm=w.dy_atm)
    pkg.fire_set_kernel(m.ctx, *KERNELS[kernel])
    return m


@pytest.mark.parametrize("kernel", sorted(KERNELS))
@pytest.mark.parametrize("split", [(2, 2), (3, 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_patches_on_one_gpu_equal_the_whole_run(pkg, prec, split, kernel):
    import torch
    w = case()
    psi_far = float(np.hypot(w.nx * w.dx, w.ny * w.dy))
    whole = model(pkg, w, prec, psi_far, kernel)
    uw, vw = whole.wind(w.u, w.v)
    part = decomp.Partition(w.nxa, w.nya, w.srx, w.sry, *split)
    pats, models, winds, stale = [], [], [], []
    rng = np.random.default_rng(7)
    for r in range(part.size):
        p = part.patch(r)
        ey, ex = part.ext_nodes(p)
        x0, y0 = part.origin(p, w.dx_atm, w.dy_atm)
        m = model(pkg, w, prec, psi_far, kernel, (ey, ex), x0, y0, p.E_I1 - p.E_I0,
                  p.E_J1 - p.E_J0)
        ue, ve = part.ext_wind(p, w.u, w.v)
        pats.append(p)
        models.append(m)
        winds.append(m.wind(ue, ve))
        # halo nodes the exchange does not refresh (deeper than 3)
        st = np.ones((ey.stop - ey.start, ex.stop - ex.start), bool)
        st[part.own_in_ext(p)] = False
        for _, _, recv in part.exchange_plan(p):
            st[recv[0].start - ey.start:recv[0].stop - ey.start,
               recv[1].start - ex.start:recv[1].stop - ex.start] = False
        stale.append(torch.as_tensor(st, device="cuda"))
    for n in range(w.steps):
        hw = whole.step(uw, vw, w.dt)
        states = [m.state() for m in models]
        for r, p in enumerate(pats):
            ey, ex = part.ext_nodes(p)
            psi, tign, frac, t = states[r]
            psi, tign, frac = psi.clone(), tign.clone(), frac.clone()
            for peer, _, recv in part.exchange_plan(p):
                q = pats[peer]
                qy, qx = part.ext_nodes(q)
                src = (slice(recv[0].start - qy.start, recv[0].stop - qy.start),
                       slice(recv[1].start - qx.start, recv[1].stop - qx.start))
                dst = (slice(recv[0].start - ey.start, recv[0].stop - ey.start),
                       slice(recv[1].start - ex.start, recv[1].stop - ex.start))
                for f, g in zip((psi, tign, frac), states[peer][:3]):
                    f[dst] = g[src]
            k = int(stale[r].sum())
            psi[stale[r]] = torch.as_tensor(rng.uniform(-50.0, 50.0, k), device="cuda",
                                            dtype=psi.dtype)
            tign[stale[r]] = torch.as_tensor(
                np.where(rng.uniform(size=k) < 0.5, np.inf, rng.uniform(0.0, n * w.dt + 1e-3, k)),
                device="cuda", dtype=tign.dtype)
            frac[stale[r]] = torch.as_tensor(rng.uniform(0.0, 1.0, k), device="cuda",
                                             dtype=frac.dtype)
            models[r].set_state(psi, tign, frac, t)
        for r, p in enumerate(pats):
            hs, hl = models[r].step(*winds[r], w.dt)
            cells = part.own_cells_in_ext(p)
            assert torch.equal(hs[cells], hw[0][p.J0:p.J1, p.I0:p.I1]), (n, r)
            assert torch.equal(hl[cells], hw[1][p.J0:p.J1, p.I0:p.I1]), (n, r)
    psi_w, tign_w, frac_w, _ = whole.state()
    for r, p in enumerate(pats):
        psi, tign, frac, _ = models[r].state()
        own = part.own_in_ext(p)
        oy, ox = part.own_nodes(p)
        assert torch.equal(psi[own], psi_w[oy, ox]), r
        assert torch.equal(tign[own], tign_w[oy, ox]), r
        assert torch.equal(frac[own], frac_w[oy, ox]), r
    assert int(torch.isfinite(tign_w).sum()) > 100
    # the fire reached the domain's outer band (the boundary status of the
    # whole run), and some patch sees it on its own band nodes
    assert whole.status() == pkg.FIRE_ERR_BOUNDARY
    band_hit = False
    for r, p in enumerate(pats):
        psi = models[r].state()[0][part.own_in_ext(p)].cpu().numpy()
        band_hit |= bool((psi[part.boundary_mask(p, w.band)] < 0).any())
    assert band_hit
    for m in models + [whole]:
        m.close()
