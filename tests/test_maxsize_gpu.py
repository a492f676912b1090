"""The largest meshes of the step kernels' index arithmetic.

The warp kernels index the fire mesh with 32-bit offsets and take meshes of
up to 2^31 - 1 nodes; larger meshes go to the marching strips, whose offsets
are 64-bit.  On a mesh of 46340 x 46340 = 2,147,395,600 nodes (88,047 below
that limit) the default FP32 kernel is the warp kernel; on one of 46400 x
46340 = 2,150,176,000 nodes it is the marching-strip kernel, run here in FP32
and FP64.  Fires burn in the cells next to the far corner (the largest
offsets), next to the first ones, at the other two corners and in the
middle.  After a few steps, one more step is compared on atmospheric cells
around the fires, at the corners and at random, with the oracle stepped on
3x3-cell crops of the same state (the bounds of the full-size test in
test_parity_gpu.py).  The inputs are built on the device
(synth.large_landscape); inputs and state reach the host only as crops."""
import dataclasses

import numpy as np
import pytest

import oracle
from gpu_helpers import check_step_on_cell, crop_step
from paper_1102_1343_gb300 import synth

pytestmark = pytest.mark.gpu

LIMIT = 2**31 - 1  # nodes of the largest mesh with 32-bit offsets


@pytest.fixture(scope="module")
def pkg():
    import torch
    from paper_1102_1343_gb300 import build
    build.build()
    import paper_1102_1343_gb300 as p
    p.load_library()
    assert torch.cuda.is_available()
    return p


def sample_cells(nxa, nya, fires, rng, n_random=8):
    """The 3x3 cells around each fire, the four corner cells that have a full
    crop, and random cells (all at least one cell from the edge)."""
    cells = set()
    for I, J in fires:
        cells.update((I + a, J + b) for a in (-1, 0, 1) for b in (-1, 0, 1))
    cells.update([(1, 1), (nxa - 2, 1), (1, nya - 2), (nxa - 2, nya - 2)])
    while len(cells) < 9 * len(fires) + 4 + n_random:
        cells.add((int(rng.integers(1, nxa - 1)), int(rng.integers(1, nya - 1))))
    return sorted((I, J) for I, J in cells if 1 <= I <= nxa - 2 and 1 <= J <= nya - 2)


def crops(t, cells, sr):
    """Host copies (float64, uint8 kept) of the 3x3-cell crops of a device
    array around each cell."""
    out = {}
    for I, J in cells:
        c = t[(J - 1) * sr:(J + 2) * sr, (I - 1) * sr:(I + 2) * sr].cpu().numpy()
        out[I, J] = c if c.dtype == np.uint8 else c.astype(np.float64)
    return out


@pytest.mark.parametrize("kernel,nxa,nya,prec,warm", [("warp", 4634, 4634, "fp32", 16),
                                                      ("march", 4640, 4634, "fp32", 16),
                                                      ("march", 4640, 4634, "fp64", 2)])
def test_largest_meshes_sampled_cells(pkg, kernel, nxa, nya, prec, warm):
    import torch
    sr = 10
    n = nxa * sr * nya * sr
    assert (n <= LIMIT) == (kernel == "warp")
    # library state, inputs and one copy of the state (bytes per node)
    per_node = (57 + 17 + 32) if prec == "fp64" else (33 + 9 + 16)
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < 1.05 * per_node * n:
        pytest.skip(f"{per_node * n / 1e9:.0f} GB of device memory needed, {free / 1e9:.0f} free")
    fires = [(1, 1), (nxa - 3, nya - 3), (nxa - 3, 2), (2, nya - 3), (nxa // 2, nya // 2)]
    w = synth.large_landscape(nxa, nya, sr=sr, seed=83, ignition_cells=fires,
                              dtype="float64" if prec == "fp64" else "float32")
    cells = sample_cells(nxa, nya, fires, np.random.default_rng(5))
    fuel_c = crops(w.fuel, cells, sr)
    zx_c, zy_c = crops(w.dzdx, cells, sr), crops(w.dzdy, cells, sr)
    P = pkg.FIRE_FP64 if prec == "fp64" else pkg.FIRE_FP32
    grid = pkg.make_grid(nxa, nya, sr, sr, w.dx_atm, w.dy_atm, P, w.band, w.eps)
    stream = torch.cuda.current_stream()
    ctx = pkg.fire_init(grid, w.classes, w.fuel, None, None, w.dzdx, w.dzdy, w.ignitions,
                        stream.cuda_stream)
    try:
        torch.cuda.synchronize()
        w = dataclasses.replace(w, fuel=None, dzdx=None, dzdy=None)  # the library holds copies
        torch.cuda.empty_cache()
        want = pkg.FIRE_KERNEL_WARP if kernel == "warp" else pkg.FIRE_KERNEL_MARCH
        assert pkg.fire_get_kernel(ctx)[0] == want
        if n > LIMIT:  # the 32-bit kernels refuse the mesh
            with pytest.raises(pkg.FireError):
                pkg.fire_set_kernel(ctx, pkg.FIRE_KERNEL_WARP, 6, 4)
        dt_ = torch.float64 if prec == "fp64" else torch.float32
        u = torch.as_tensor(w.u).to("cuda", dt_).contiguous()
        v = torch.as_tensor(w.v).to("cuda", dt_).contiguous()
        # the wind as the path sees it (rounded to FP32 on the FP32 path)
        uh, vh = u.double().cpu().numpy(), v.double().cpu().numpy()
        hs = torch.zeros((nya, nxa), dtype=torch.float64, device="cuda")
        hl = torch.zeros_like(hs)
        for _ in range(warm):
            pkg.fire_step(ctx, u, v, w.dt, hs, hl)

        def state_crops():
            psi = torch.empty((nya * sr, nxa * sr), dtype=dt_, device="cuda")
            tign = torch.empty((nya * sr, nxa * sr), dtype=torch.float64, device="cuda")
            frac = torch.empty_like(psi)
            t = pkg.fire_get_state(ctx, psi, tign, frac)
            out = crops(psi, cells, sr), crops(tign, cells, sr), crops(frac, cells, sr), t
            del psi, tign, frac
            torch.cuda.empty_cache()
            return out

        psi0, tign0, frac0, t0 = state_crops()
        pkg.fire_step(ctx, u, v, w.dt, hs, hl)
        torch.cuda.synchronize()
        psi1, tign1, frac1, _ = state_crops()
        hs_g, hl_g = hs.cpu().numpy(), hl.cpu().numpy()
        assert pkg.fire_status(ctx) == pkg.FIRE_OK
    finally:
        pkg.fire_destroy(ctx)
    Hs_max = max(oracle.fuel_coefficients(c)[7] for c in w.classes)
    Hq_max = max(oracle.fuel_coefficients(c)[8] for c in w.classes)
    burning = 0
    for I, J in cells:
        wc = dataclasses.replace(w, nxa=3, nya=3, fuel=fuel_c[I, J], dzdx=zx_c[I, J],
                                 dzdy=zy_c[I, J], u=uh[J - 1:J + 2, I - 1:I + 3],
                                 v=vh[J - 1:J + 3, I - 1:I + 2], ignitions=[])
        sub, hs_o, hl_o, (cy, cx), _ = crop_step(wc, psi0[I, J], tign0[I, J], frac0[I, J], t0,
                                                 1, 1, w.dt)
        burning += check_step_on_cell(prec, sub, cy, cx, psi0[I, J], t0, psi1[I, J][cy, cx],
                                      tign1[I, J][cy, cx], frac1[I, J][cy, cx], hs_g[J, I],
                                      hl_g[J, I], hs_o, hl_o, Hs_max, Hq_max, w.dt)
    # every fire burns in the cell it was lit in
    assert burning >= len(fires)
