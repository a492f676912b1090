"""The coupling steps on the GPU (fire_wind_at_height, fire_heat_insertion)
against the oracle, alone and around the fire step: 3-D columns -> wind at
6.1 m on the staggered grid -> fire steps -> heat sources in the
atmospheric tendencies."""
import json
import os

import numpy as np
import pytest

import oracle
from gpu_helpers import compare_fp64, rel_inf, state_np
from paper_1102_1343_gb300 import synth

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
ZF = GOLD["midflame_height_m"]["z_f"]


@pytest.fixture(scope="module")
def pkg():
    import torch
    from paper_1102_1343_gb300 import build
    build.build()
    import paper_1102_1343_gb300 as p
    p.load_library()
    assert torch.cuda.is_available()
    return p


def cuda(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype).contiguous()


@pytest.mark.parametrize("shape", [(20, 31), (21, 30), (1, 1), (3, 700)])
def test_wind_at_height_matches_oracle(pkg, shape):
    """u-points (20 x 31), v-points (21 x 30), a single column and a long
    row; FP64 to rounding, FP32 within its rounding of the logarithms."""
    import torch
    rng = np.random.default_rng(11)
    zw, z, z0, u = synth.atmos_columns(rng, shape, nz=20)
    for zf in (ZF, 0.01, 250.0, 1e5):
        want = oracle.wind_at_height(u, z, z0, zf)
        got = pkg.fire_wind_at_height(cuda(u, torch.float64), cuda(z, torch.float64),
                                      cuda(z0, torch.float64), zf).cpu().numpy()
        assert np.allclose(got, want, rtol=1e-13, atol=1e-13)
        u32, z32, r32 = (np.asarray(a, np.float32).astype(np.float64) for a in (u, z, z0))
        want32 = oracle.wind_at_height(u32, z32, r32, float(np.float32(zf)))
        got32 = pkg.fire_wind_at_height(cuda(u, torch.float32), cuda(z, torch.float32),
                                        cuda(z0, torch.float32), zf).cpu().numpy()
        assert np.allclose(got32, want32, rtol=2e-5, atol=2e-5 * max(1.0, np.abs(u).max()))


def test_heat_insertion_matches_oracle(pkg):
    import torch
    rng = np.random.default_rng(12)
    shape = (17, 23)
    zw, z, z0, _ = synth.atmos_columns(rng, shape, nz=25)
    rho, mu = synth.air_columns(rng, shape, zw)
    hs = rng.uniform(0.0, 4e4, shape)
    hl = rng.uniform(0.0, 1e4, shape)
    base = rng.standard_normal(rho.shape)
    for zext in (30.0, 200.0):
        a, b = oracle.heat_insertion(hs, hl, zw, rho, mu, zext, rth=base, rqv=-base)
        f = torch.float64
        rth, rqv = cuda(base, f), cuda(-base, f)
        pkg.fire_heat_insertion(cuda(hs, f), cuda(hl, f), cuda(zw, f), cuda(rho, f), cuda(mu, f),
                                zext, rth, rqv)
        assert np.allclose(rth.cpu().numpy(), a, rtol=1e-13, atol=1e-13 * np.abs(a).max())
        assert np.allclose(rqv.cpu().numpy(), b, rtol=1e-13, atol=1e-13 * np.abs(b).max())
        only = cuda(base, f)
        pkg.fire_heat_insertion(cuda(hs, f), None, cuda(zw, f), cuda(rho, f), cuda(mu, f), zext,
                                only, None)
        assert torch.equal(only, rth)


def test_coupled_steps_fp64_match_oracle(pkg):
    """3-D synthetic columns on the u- and v-points -> the 6.1 m wind on the
    GPU -> 60 fire steps -> the heat sources of the last step inserted into
    the tendencies, all against the same chain in the oracle."""
    import torch
    w = synth.random_landscape(24, 18, seed=81, ignition="line", steps=60)
    rng = np.random.default_rng(82)
    _, zu, z0u, u3 = synth.atmos_columns(rng, w.u.shape, nz=18)
    _, zv, z0v, v3 = synth.atmos_columns(rng, w.v.shape, nz=18)
    u3 = u3 + 3.0  # a mean westerly on top of the log profile
    zw, _, _, _ = synth.atmos_columns(rng, (w.nya, w.nxa), nz=18)
    rho, mu = synth.air_columns(rng, (w.nya, w.nxa), zw)
    f = torch.float64
    u6 = pkg.fire_wind_at_height(cuda(u3, f), cuda(zu, f), cuda(z0u, f), ZF)
    v6 = pkg.fire_wind_at_height(cuda(v3, f), cuda(zv, f), cuda(z0v, f), ZF)
    uo = oracle.wind_at_height(u3, zu, z0u, ZF)
    vo = oracle.wind_at_height(v3, zv, z0v, ZF)
    assert rel_inf(u6.cpu().numpy(), uo) <= 1e-13 and rel_inf(v6.cpu().numpy(), vo) <= 1e-13
    m = pkg.FireModel.from_workload(w, precision="fp64")
    orc = oracle.OracleFire.from_workload(w)
    for _ in range(w.steps):
        hs, hl = m.step(u6, v6, w.dt)
        hs_o, hl_o, _ = orc.step(uo, vo, w.dt)
    ok, e = compare_fp64(state_np(m), orc)
    assert ok, e
    assert rel_inf(hs.cpu().numpy(), hs_o) <= 1e-10 and hs_o.max() > 0
    rth = torch.zeros(rho.shape, dtype=f, device="cuda")
    rqv = torch.zeros_like(rth)
    pkg.fire_heat_insertion(hs, hl, cuda(zw, f), cuda(rho, f), cuda(mu, f), 50.0, rth, rqv)
    a, b = oracle.heat_insertion(hs_o, hl_o, zw, rho, mu, 50.0)
    assert rel_inf(rth.cpu().numpy(), a) <= 1e-10 and rel_inf(rqv.cpu().numpy(), b) <= 1e-10
    m.close()
