"""The adaptive choice between the two FP32 warp-strip kernels
(fire_set_adaptive, fire_adaptive_info): the default strips while under
0.5 % of the nodes have psi <= 0, the dense variant with strips of at most 6
atmospheric rows from there on (back below 0.25 %).  The two kernels give
the same bits, so a run that switches mid-way equals a run that does not;
the counted fraction is the state's own; explicit kernel choices turn the
adaptive choice off."""
import numpy as np
import pytest

from gpu_helpers import state_np
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


def fires(radius, steps=200, n_points=20):
    """2000x2000 nodes (fire_init's default there: warp strips 60 x 10
    nodes), n_points fires of the given radius."""
    return synth.random_landscape(200, 200, seed=57, ignition="points", n_points=n_points,
                                  edge_margin=1500.0, ignition_radius=radius, steps=steps)


def burnt(m):
    return float((m.state()[0] <= 0).double().mean())


def test_burning_and_sparse_states_at_init(pkg):
    w = fires(150.0)
    m = pkg.FireModel.from_workload(w, precision="fp32")
    on, counts, f = pkg.fire_adaptive_info(m.ctx)
    assert on and counts == 1
    assert f == burnt(m) and f >= 0.005
    sms = m.torch.cuda.get_device_properties(0).multi_processor_count
    default = pkg.fire_default_kernel("fp32", w.nxa, w.nya, 10, 10, sms)
    assert default[0] == pkg.FIRE_KERNEL_WARP
    assert pkg.fire_get_kernel(m.ctx) == (pkg.FIRE_KERNEL_WARP_DENSE, default[1], min(default[2], 6))
    m.close()
    w = fires(10.0)
    m = pkg.FireModel.from_workload(w, precision="fp32")
    on, counts, f = pkg.fire_adaptive_info(m.ctx)
    assert on and 0 < f < 0.0025 and f == burnt(m)
    assert pkg.fire_get_kernel(m.ctx) == tuple(default)
    m.close()


def test_switch_during_a_run_changes_no_bit(pkg):
    """Fires of 106 m (0.49 % burnt at the start) grow past 0.5 %: the run
    through fire_run (graph replays, the choice made between them; the host
    waits between calls, so that the counts have landed when they are read)
    switches to the dense kernel and ends with the same psi, t_i, F and heat
    grids as a run with the choice turned off."""
    import torch
    w = fires(106.0)
    runs = []
    for adaptive in (True, False):
        m = pkg.FireModel.from_workload(w, precision="fp32")
        start = pkg.fire_get_kernel(m.ctx)
        if not adaptive:
            pkg.fire_set_adaptive(m.ctx, False)
        assert start[0] == pkg.FIRE_KERNEL_WARP and pkg.fire_adaptive_info(m.ctx)[2] < 0.005
        u, v = m.wind(w.u, w.v)
        for _ in range(3):
            m.step(u, v, w.dt)
        m.run(7, u, v, w.dt)
        for _ in range(19):  # the host waits between the calls, so each count lands
            torch.cuda.synchronize()
            hs, hl = m.run(10, u, v, w.dt)
        torch.cuda.synchronize()
        end = pkg.fire_get_kernel(m.ctx)
        on, counts, f = pkg.fire_adaptive_info(m.ctx)
        if adaptive:
            assert burnt(m) >= 0.005 and f >= 0.005 and counts >= 3
            assert end == (pkg.FIRE_KERNEL_WARP_DENSE, start[1], min(start[2], 6))
        else:
            assert not on and end == start
        runs.append(state_np(m)[:3] + (hs.cpu().numpy(), hl.cpu().numpy()))
        assert m.status() == pkg.FIRE_OK
        m.close()
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


def test_explicit_choices_turn_it_off(pkg):
    w = fires(10.0, steps=5)
    m = pkg.FireModel.from_workload(w, precision="fp32")
    u, v = m.wind(w.u, w.v)
    pkg.fire_set_kernel(m.ctx, pkg.FIRE_KERNEL_MARCH, 24, 2)
    assert not pkg.fire_adaptive_info(m.ctx)[0]
    with pytest.raises(pkg.FireError):
        pkg.fire_set_adaptive(m.ctx, True)  # not on warp strips
    pkg.fire_set_kernel(m.ctx, pkg.FIRE_KERNEL_WARP_DENSE, 6, 4)
    pkg.fire_set_adaptive(m.ctx, True)  # the current strips become the default shape
    assert pkg.fire_adaptive_info(m.ctx)[0]
    assert pkg.fire_get_kernel(m.ctx) == (pkg.FIRE_KERNEL_WARP, 6, 4)
    m.autotune(u, v, w.dt)
    assert not pkg.fire_adaptive_info(m.ctx)[0]
    m.close()
    m = pkg.FireModel.from_workload(w, precision="fp64")
    assert not pkg.fire_adaptive_info(m.ctx)[0]
    with pytest.raises(pkg.FireError):
        pkg.fire_set_adaptive(m.ctx, True)
    m.close()
