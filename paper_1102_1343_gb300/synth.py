"""Seeded synthetic inputs shaped like the paper's workloads.

This module produces inputs only: wind on the staggered atmospheric grid,
terrain gradients, fuel-class maps and tables, ignitions.  It holds none of the
fire model's arithmetic and is shared by the tests, the benchmark and the
oracle's callers.  Everything is deterministic in the seed
(``numpy.random.default_rng``).

The paper's runs use WRF winds and FireFlux / Landfire / NED data, which are
not available here; these generators stand in for them with the structure the
paper describes: a fire mesh refined 10x from a 60 m atmospheric mesh
(Sect. "Fire subgrid refinement ratios"), smooth winds, hills, patchy fuel maps
at roughly 30 m data resolution, point and line ignitions (Sect. "Ignition").
"""
from __future__ import annotations

import dataclasses

import numpy as np

BASE_SEED = 1102


@dataclasses.dataclass
class Workload:
    """One fire-step workload: grids, fuels, terrain, wind, ignitions."""
    name: str
    nxa: int
    nya: int
    srx: int
    sry: int
    dx_atm: float
    dy_atm: float
    classes: list            # fuel classes: dicts of Table 1 identifiers (SI units)
    fuel: np.ndarray         # uint8 [ny][nx] class index per fire node
    dzdx: np.ndarray         # float64 [ny][nx]
    dzdy: np.ndarray         # float64 [ny][nx]
    u: np.ndarray            # float64 [nya][nxa+1], x-faces
    v: np.ndarray            # float64 [nya+1][nxa], y-faces
    ignitions: list          # dicts {ax, ay, bx, by, t_start, radius, speed}
    dt: float
    steps: int
    eps: float = 0.4
    band: int = 1
    moisture: np.ndarray | None = None   # optional per-node M_f
    mult: np.ndarray | None = None       # optional per-node spread multiplier

    @property
    def nx(self):
        return self.nxa * self.srx

    @property
    def ny(self):
        return self.nya * self.sry

    @property
    def dx(self):
        return self.dx_atm / self.srx

    @property
    def dy(self):
        return self.dy_atm / self.sry


# ---------------------------------------------------------------------------
# fuel classes (Table 1 identifiers, SI units as in Table 1)
# ---------------------------------------------------------------------------

def nominal_class(**over) -> dict:
    """A grass-like class with nominal Table 1 values (SI).

    The 13 Anderson categories of namelist.fire are not available; these values
    are chosen in the usual ranges (sigma 3500 1/ft, rho_P 32 lb/ft^3,
    S_T 0.0555, S_E 0.010, h 8000 BTU/lb)."""
    c = dict(windrf=0.36, weight=7.0, weight_is_tf=0.0, fgi=0.166, fueldepthm=0.305,
             savr=3500.0 / 0.3048, fuelmce=0.12, fueldens=32.0 * 0.45359237 / 0.3048 ** 3,
             st=0.0555, se=0.010, cmbcnst=18.608e6, fuelmc_g=0.08, chaparral=0.0)
    c.update(over)
    return c


def random_classes(rng, n=13, chaparral_index=None) -> list:
    """n synthetic classes: load 0.1-2 kg/m^2, moisture 0.04-0.2.

    The remaining Table 1 values are drawn from ranges (sigma 1500-2500 1/ft,
    depth 0.3-1.0 m, wind reduction 0.1-0.2) whose head-fire rates stay below
    about 2 m/s for winds up to 13 m/s on slopes up to 0.4, so that the
    explicit scheme stays stable at dt = 0.5 s on a 6 m mesh.  The chaparral
    rule (6 m/s in any wind above 4.6 m/s) is only used when chaparral_index
    is given."""
    out = []
    for k in range(n):
        c = nominal_class(
            windrf=float(rng.uniform(0.1, 0.2)),
            weight=float(rng.uniform(7.0, 180.0)),
            fgi=float(rng.uniform(0.1, 2.0)),
            fueldepthm=float(rng.uniform(0.3, 1.0)),
            savr=float(rng.uniform(1500.0, 2500.0)) / 0.3048,
            fuelmce=float(rng.uniform(0.25, 0.40)),
            fuelmc_g=float(rng.uniform(0.04, 0.2)),
            chaparral=1.0 if k == chaparral_index else 0.0,
        )
        out.append(c)
    return out


# ---------------------------------------------------------------------------
# fields
# ---------------------------------------------------------------------------

def smooth_wind(rng, nxa, nya, mean=(5.0, 0.0), std=1.5, sigma_cells=5.0):
    """Staggered wind: mean + white noise Gaussian-filtered (sigma in atmos
    cells), centred and rescaled to the given standard deviation (centring
    matters on meshes not much larger than the filter, where the filtered
    noise is nearly constant)."""
    from scipy.ndimage import gaussian_filter

    def field(shape, m):
        w = gaussian_filter(rng.standard_normal(shape), sigma=sigma_cells, mode="reflect")
        w = w - w.mean()
        s = w.std()
        if s > 0:
            w = w * (std / s)
        return m + w

    u = field((nya, nxa + 1), mean[0])
    v = field((nya + 1, nxa), mean[1])
    return u, v


def constant_wind(nxa, nya, U=0.0, V=0.0):
    return (np.full((nya, nxa + 1), float(U)), np.full((nya + 1, nxa), float(V)))


def hills_gradient(rng, nx, ny, dx, dy, n_hills=20, s_range=(200.0, 800.0), max_slope=0.4):
    """Analytic gradient of a sum of Gaussian hills, rescaled to max |grad z|.

    z = sum_k h_k exp(-|x - c_k|^2 / (2 s_k^2)); each hill is separable, so
    the gradient is a rank-n_hills product evaluated with two matmuls."""
    Lx, Ly = nx * dx, ny * dy
    cx = rng.uniform(0.0, Lx, n_hills)
    cy = rng.uniform(0.0, Ly, n_hills)
    s = rng.uniform(s_range[0], s_range[1], n_hills)
    h = rng.uniform(0.5, 1.0, n_hills)
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    ex = np.exp(-((x[None, :] - cx[:, None]) ** 2) / (2 * s[:, None] ** 2))   # [K, nx]
    ey = np.exp(-((y[None, :] - cy[:, None]) ** 2) / (2 * s[:, None] ** 2))   # [K, ny]
    dex = -(x[None, :] - cx[:, None]) / s[:, None] ** 2 * ex
    dey = -(y[None, :] - cy[:, None]) / s[:, None] ** 2 * ey
    dzdx = (ey.T * h[None, :]) @ dex
    dzdy = (dey.T * h[None, :]) @ ex
    m = 0.0
    step = max(1, (1 << 24) // max(1, nx))
    for j0 in range(0, ny, step):   # chunked to bound temporaries
        m = max(m, float(np.sqrt(dzdx[j0:j0 + step] ** 2 + dzdy[j0:j0 + step] ** 2).max()))
    if m > 0:
        scale = max_slope / m
        dzdx *= scale
        dzdy *= scale
    return dzdx, dzdy


def voronoi_fuel(rng, nx, ny, dx, n_classes=13, n_sites=400, data_res=30.0):
    """Fuel-class map: Voronoi patches on a data grid of ~30 m pixels (like
    Landfire), each patch one random class, replicated to the fire mesh."""
    from scipy.ndimage import distance_transform_edt
    b = max(1, int(round(data_res / dx)))
    cy, cx = -(-ny // b), -(-nx // b)
    n_sites = max(1, min(n_sites, cx * cy))
    flat = rng.choice(cx * cy, size=n_sites, replace=False)
    site_cls = rng.integers(0, n_classes, size=n_sites).astype(np.uint8)
    mask = np.ones((cy, cx), dtype=bool)
    mask.flat[flat] = False
    label = np.zeros((cy, cx), dtype=np.int32)
    label.flat[flat] = np.arange(n_sites, dtype=np.int32)
    idx = distance_transform_edt(mask, return_distances=False, return_indices=True)
    coarse = site_cls[label[idx[0], idx[1]]]
    fine = np.repeat(np.repeat(coarse, b, axis=0), b, axis=1)[:ny, :nx]
    return np.ascontiguousarray(fine)


def point_ignition(x, y, radius=10.0, t_start=0.0, speed=0.0):
    return dict(ax=float(x), ay=float(y), bx=float(x), by=float(y), t_start=float(t_start),
                radius=float(radius), speed=float(speed))


def line_ignition(ax, ay, bx, by, radius=10.0, t_start=0.0, speed=0.0):
    return dict(ax=float(ax), ay=float(ay), bx=float(bx), by=float(by),
                t_start=float(t_start), radius=float(radius), speed=float(speed))


def drip_torch(ax, ay, vx, vy, t_start, t_end, radius, speed):
    """A drip torch leaving (ax, ay) at t_start with velocity (vx, vy) m/s
    until t_end, its fire growing at `speed` to `radius` around the line it
    has laid."""
    return dict(ax=float(ax), ay=float(ay), bx=float(ax), by=float(ay), t_start=float(t_start),
                radius=float(radius), speed=float(speed), vx=float(vx), vy=float(vy),
                t_end=float(t_end))


# ---------------------------------------------------------------------------
# the workloads
# ---------------------------------------------------------------------------

def plain_circle(nxa=10, nya=10, sr=10, dx_atm=60.0, steps=120, dt=0.5, U=3.0, V=0.0,
                 radius=10.0, fgi=0.5, Mf=0.08, Tf=60.0) -> Workload:
    """Plain FP64 case: flat terrain, one uniform fuel (load 0.5 kg/m^2,
    moisture 0.08, burn time 60 s), constant wind (3, 0) m/s, circular ignition
    of radius 10 m at the centre at t = 0; 10x10 atmos cells of 60 m refined 10x
    to a 100x100 fire mesh of 6 m; 120 steps of 0.5 s."""
    nx, ny = nxa * sr, nya * sr
    dx = dx_atm / sr
    cls = [nominal_class(fgi=fgi, fuelmc_g=Mf, weight=Tf, weight_is_tf=1.0)]
    u, v = constant_wind(nxa, nya, U, V)
    z = np.zeros((ny, nx))
    ign = [point_ignition(nx * dx / 2, ny * dx / 2, radius=radius)]
    return Workload("circle-fp64-100x100", nxa, nya, sr, sr, dx_atm, dx_atm, cls,
                    np.zeros((ny, nx), np.uint8), z, z.copy(), u, v, ign, dt, steps)


def random_landscape(nxa, nya, sr=10, dx_atm=60.0, seed=BASE_SEED, steps=1200, dt=0.5,
                     ignition="line", n_points=50, edge_margin=2000.0, wind_mean=(5.0, 0.0),
                     wind_scale=1.0, moisture_shift=0.0, name=None,
                     ignition_radius=10.0) -> Workload:
    """Random landscape: smooth wind (mean 5 m/s, std 1.5 m/s, 300 m filter
    length), 20 Gaussian hills with max slope 0.4, 13 Voronoi fuel classes
    (load 0.1-2 kg/m^2, moisture 0.04-0.2, one chaparral), and either a 1 km
    line ignition perpendicular to the wind at x = 3 km ("line"), n random
    point ignitions at least edge_margin from the edges ("points"), one
    central point ("center") or none ("none").  Sizes are free so the same recipe serves the
    2000x2000 and 8200x8200 meshes and small parity cases."""
    rng = np.random.default_rng(seed)
    srx = sry = sr
    nx, ny = nxa * srx, nya * sry
    dx = dx_atm / srx
    Lx, Ly = nx * dx, ny * dx
    u, v = smooth_wind(rng, nxa, nya, mean=wind_mean, std=1.5,
                       sigma_cells=300.0 / dx_atm)
    u, v = u * wind_scale, v * wind_scale
    dzdx, dzdy = hills_gradient(rng, nx, ny, dx, dx)
    classes = random_classes(rng)
    if moisture_shift:
        for c in classes:
            c["fuelmc_g"] = max(0.01, c["fuelmc_g"] + moisture_shift)
    fuel = voronoi_fuel(rng, nx, ny, dx, n_classes=len(classes))
    if ignition == "line":
        x0 = min(3000.0, 0.25 * Lx)
        half = min(500.0, 0.25 * Ly)
        ign = [line_ignition(x0, Ly / 2 - half, x0, Ly / 2 + half, radius=10.0)]
    elif ignition == "points":
        m = min(edge_margin, 0.25 * min(Lx, Ly))
        xs = rng.uniform(m, Lx - m, n_points)
        ys = rng.uniform(m, Ly - m, n_points)
        ign = [point_ignition(a, b, radius=ignition_radius) for a, b in zip(xs, ys)]
    elif ignition == "center":
        ign = [point_ignition(Lx / 2, Ly / 2, radius=10.0)]
    elif ignition == "none":
        ign = []
    else:
        raise ValueError(ignition)
    return Workload(name or f"landscape-{nx}x{ny}", nxa, nya, srx, sry, dx_atm, dx_atm,
                    classes, fuel, dzdx, dzdy, u, v, ign, dt, steps)


def atmos_columns(rng, shape, nz=20, top=3000.0, stretch=1.6, z0_range=(0.02, 0.5),
                  ustar_range=(0.2, 0.6), noise=0.3):
    """Synthetic atmospheric columns at the points of `shape` (the u- or
    v-points of the staggered grid, or the mass points): face heights above
    the terrain zw [nz+1][...] (0 at the surface, stretched toward the top,
    varied by a few per cent from column to column), cell-centre heights z
    [nz][...], roughness heights z0 [...] and a wind component [nz][...]
    following a logarithmic profile u*/0.4 ln(z/z0) (u* per point, either
    sign) plus noise.  Stand-ins for WRF's geopotential heights and winds,
    which are not available here."""
    shape = tuple(shape)
    k = np.arange(nz + 1, dtype=np.float64).reshape((nz + 1,) + (1,) * len(shape))
    base = top * (k / nz) ** stretch
    wobble = 1.0 + 0.03 * rng.standard_normal(shape)
    zw = base * wobble
    z = 0.5 * (zw[1:] + zw[:-1])
    z0 = rng.uniform(*z0_range, size=shape)
    ustar = rng.uniform(*ustar_range, size=shape) * rng.choice([-1.0, 1.0], size=shape)
    u = ustar / 0.4 * np.log(np.maximum(z, 1e-3) / z0) + noise * rng.standard_normal(z.shape)
    return zw, z, z0, u


def air_columns(rng, shape, zw):
    """Density [nz][...] (kg m^-3, exponential with an 8 km scale height) at
    the cell centres of face heights zw, and the dry-air column mass mu [...]
    (Pa) for the heat insertion."""
    z = 0.5 * (zw[1:] + zw[:-1])
    rho = 1.2 * np.exp(-z / 8000.0) * (1.0 + 0.01 * rng.standard_normal(z.shape))
    mu = 9.0e4 * (1.0 + 0.02 * rng.standard_normal(tuple(shape)))
    return rho, mu


def line_fire_2000(seed=BASE_SEED) -> Workload:
    """FP32-vs-FP64 forward case: 200x200 atmos -> 2000x2000 fire mesh, 1 km
    line ignition, 1200 steps of 0.5 s."""
    return random_landscape(200, 200, seed=seed, steps=1200, ignition="line",
                            name="line-fire-2000x2000")


def points_fire_8200(seed=BASE_SEED) -> Workload:
    """Large forward case: 820x820 atmos -> 8200x8200 fire mesh (the stated
    8192 rounded to a multiple of the refinement 10), 50 point ignitions,
    2000 steps."""
    return random_landscape(820, 820, seed=seed, steps=2000, ignition="points",
                            n_points=50, name="points-fire-8200x8200")


def burning_fire_8200(seed=BASE_SEED) -> Workload:
    """The large mesh in a heavily burning state: the 8200x8200 recipe with
    50 point ignitions of radius 3 km (centres at least 3.5 km from the edges),
    so that about half of the domain is burnt from t = 0 and its cells run the
    fuel-fraction quadrature and the ignition-time path every step."""
    return random_landscape(820, 820, seed=seed, steps=2000, ignition="points", n_points=50,
                            edge_margin=3500.0, ignition_radius=3000.0,
                            name="burning-fire-8200x8200")


def large_landscape(nxa, nya, sr=10, dx_atm=60.0, seed=BASE_SEED, dtype="float32",
                    device="cuda", ignition_cells=(), steps=20, dt=0.5, patch_nodes=50,
                    n_hills=20, max_slope=0.4, row_chunk=2048, name=None) -> Workload:
    """The landscape recipe on meshes too large to build on the host (billions
    of fire nodes).  fuel, dzdx and dzdy of the returned workload are torch
    tensors on `device` (uint8, and `dtype` for the gradients), built there in
    chunks of rows; the wind and the classes are numpy and Python values made
    as in random_landscape.  The terrain is the same sum of Gaussian hills
    (hills_gradient, evaluated chunk by chunk); the fuel map is random classes
    on square patches of patch_nodes nodes (a Voronoi map needs a distance
    transform of the whole data grid).  Point ignitions of radius 10 m at the
    centres of the atmospheric cells (I, J) of ignition_cells."""
    import torch
    rng = np.random.default_rng(seed)
    nx, ny = nxa * sr, nya * sr
    dx = dx_atm / sr
    u, v = smooth_wind(rng, nxa, nya, std=1.5, sigma_cells=300.0 / dx_atm)
    classes = random_classes(rng)
    Lx, Ly = nx * dx, ny * dx
    dev = torch.device(device)
    f64 = torch.float64

    def col(a):
        return torch.as_tensor(a, dtype=f64, device=dev)[:, None]

    cx, cy = col(rng.uniform(0.0, Lx, n_hills)), col(rng.uniform(0.0, Ly, n_hills))
    s2 = col(rng.uniform(200.0, 800.0, n_hills)) ** 2
    h = torch.as_tensor(rng.uniform(0.5, 1.0, n_hills), dtype=f64, device=dev)[None, :]
    x = (torch.arange(nx, dtype=f64, device=dev) + 0.5) * dx
    ex = torch.exp(-((x[None, :] - cx) ** 2) / (2 * s2))  # [K, nx]
    dex = -(x[None, :] - cx) / s2 * ex
    dzdx = torch.empty((ny, nx), dtype=getattr(torch, dtype), device=dev)
    dzdy = torch.empty_like(dzdx)
    m = 0.0
    for j0 in range(0, ny, row_chunk):
        j1 = min(ny, j0 + row_chunk)
        y = (torch.arange(j0, j1, dtype=f64, device=dev) + 0.5) * dx
        ey = torch.exp(-((y[None, :] - cy) ** 2) / (2 * s2))  # [K, rows]
        dey = -(y[None, :] - cy) / s2 * ey
        gx = (ey.T * h) @ dex
        gy = (dey.T * h) @ ex
        m = max(m, float(torch.sqrt(gx * gx + gy * gy).max()))
        dzdx[j0:j1] = gx
        dzdy[j0:j1] = gy
        del gx, gy
    if m > 0:
        dzdx.mul_(max_slope / m)
        dzdy.mul_(max_slope / m)
    p = patch_nodes
    coarse = rng.integers(0, len(classes), size=(-(-ny // p), -(-nx // p))).astype(np.uint8)
    fuel = torch.as_tensor(coarse, device=dev).repeat_interleave(p, 0)[:ny]
    fuel = fuel.repeat_interleave(p, 1)[:, :nx].contiguous()
    ign = [point_ignition((I + 0.5) * dx_atm, (J + 0.5) * dx_atm, radius=10.0)
           for I, J in ignition_cells]
    return Workload(name or f"large-landscape-{nx}x{ny}", nxa, nya, sr, sr, dx_atm, dx_atm,
                    classes, fuel, dzdx, dzdy, u, v, ign, dt, steps)


def ensemble_sizes(n_members=64, seed=BASE_SEED, lo=26, hi=205):
    """Atmos sizes per member for the batched ensemble: fire meshes uniform in
    260^2..2050^2 (multiples of the refinement 10)."""
    rng = np.random.default_rng(seed + 999)
    return [int(a) for a in rng.integers(lo, hi + 1, size=n_members)]


def ensemble_member(k, nxa, seed=BASE_SEED, steps=600) -> Workload:
    """Member k: the landscape recipe at its own size, wind scaled by a
    member factor in [0.8, 1.2] and fuel moisture shifted by [-0.03, 0.03]."""
    rng = np.random.default_rng(seed + 1000 + k)
    ws = float(rng.uniform(0.8, 1.2))
    ms = float(rng.uniform(-0.03, 0.03))
    return random_landscape(nxa, nxa, seed=seed, steps=steps, ignition="center",
                            wind_scale=ws, moisture_shift=ms, name=f"member{k}-{nxa * 10}")


def smooth_field(rng, ny, nx, sigma_nodes):
    """Gaussian-filtered white noise, centred and scaled to max |f| = 1."""
    from scipy.ndimage import gaussian_filter
    f = gaussian_filter(rng.standard_normal((ny, nx)), sigma=sigma_nodes, mode="reflect")
    f = f - f.mean()
    m = np.abs(f).max()
    return f / m if m > 0 else f


def adjoint_case(nxa=51, sr=10, seed=BASE_SEED, steps=400, dt=0.5):
    """Adjoint workload: the landscape recipe on an nxa x nxa atmospheric mesh
    (51 -> 510x510 fire mesh) with one central point ignition, and the
    perturbations of the synthetic 'truth' run whose arrival times serve as
    observations: multiplier 1 + 0.2 f (f a smooth field of 300 m length,
    max |f| = 1), fuel moisture + 0.02 in every class, wind x 1.1.
    Returns (workload, truth) with truth = dict(mult, classes, wind_scale)."""
    w = random_landscape(nxa, nxa, sr=sr, seed=seed, steps=steps, dt=dt, ignition="center",
                         name=f"adjoint-{nxa * sr}x{nxa * sr}")
    rng = np.random.default_rng(seed + 77)
    mult = 1.0 + 0.2 * smooth_field(rng, w.ny, w.nx, 300.0 / w.dx)
    classes = [dict(c) for c in w.classes]
    for c in classes:
        c["fuelmc_g"] = c["fuelmc_g"] + 0.02
    return w, dict(mult=mult, classes=classes, wind_scale=1.1)


def wind_arrays_like(w: Workload, dtype=np.float64):
    return np.ascontiguousarray(w.u, dtype=dtype), np.ascontiguousarray(w.v, dtype=dtype)
