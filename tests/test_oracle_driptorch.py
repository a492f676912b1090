"""Pins of the oracle's drip-torch ignition (Sect. "Ignition", the paragraph
after eq. (ignition-min)): a torch leaves a at t_g with velocity v until t_h;
at every step start t in [t_g, t_h + r_g/S_g] the ignition line is the
segment [a, a + v (min{t, t_h} - t_g)], psi_g = dist - min{r_g, S_g (t - t_g)}
and psi := min(psi, psi_g).

On a fuel that does not spread (no load: S = 0, so the level-set step leaves
psi unchanged) the ignition alone shapes the fire, which gives closed forms:
the final level set is the signed distance to the laid line minus r_g (a
stadium), and nodes reached as the torch passes get the time the torch's
fire front reaches them."""
import numpy as np
import pytest

import oracle
from paper_1102_1343_gb300 import synth


def still_workload(nxa=20, nya=12, steps=40, dt=0.5, ignitions=()):
    """6 m mesh, flat, one fuel class without load (no spread), calm."""
    w = synth.plain_circle(nxa=nxa, nya=nya, steps=steps, dt=dt, U=0.0)
    w.classes = [synth.nominal_class(fgi=0.0, weight=60.0, weight_is_tf=1.0)]
    w.ignitions = list(ignitions)
    return w


def run(w):
    o = oracle.OracleFire.from_workload(w)
    for _ in range(w.steps):
        o.step(w.u, w.v, w.dt)
    return o


def node_xy(w):
    x = (np.arange(w.nx) + 0.5) * w.dx
    y = (np.arange(w.ny) + 0.5) * w.dy
    return np.meshgrid(x, y)


def seg_dist(X, Y, a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    d = b - a
    L2 = d @ d
    s = np.zeros_like(X) if L2 == 0 else np.clip(((X - a[0]) * d[0] + (Y - a[1]) * d[1]) / L2,
                                                 0.0, 1.0)
    return np.hypot(X - a[0] - s * d[0], Y - a[1] - s * d[1])


@pytest.mark.parametrize("b", [None, (500.0, 400.0)])
def test_laid_line_is_a_stadium(orc, b):
    """After the window the level set is dist(x, [a, a + v (t_h - t_g)]) - r_g
    wherever that is below psi_far, node by node, and t_i is set exactly
    where it is <= 0.  The segment's end b plays no part in a drip torch (the
    line runs from a along v): a far-away b gives the same stadium."""
    tor = synth.drip_torch(40.0, 33.0, 7.0, 2.5, t_start=0.5, t_end=8.0, radius=9.0, speed=5.0)
    if b is not None:
        tor = dict(tor, bx=b[0], by=b[1])
    w = still_workload(ignitions=[tor])
    o = run(w)
    X, Y = node_xy(w)
    a = (40.0, 33.0)
    b = (40.0 + 7.0 * 7.5, 33.0 + 2.5 * 7.5)
    want = seg_dist(X, Y, a, b) - 9.0
    near = want < 0.5 * o.psi_far
    assert near.sum() > 100
    assert np.allclose(o.psi[near], want[near], rtol=0, atol=1e-12)
    assert np.array_equal(np.isfinite(o.tign), want <= 1e-12)
    assert np.all(o.tign[np.isfinite(o.tign)] <= w.steps * w.dt)


def test_arrival_times_along_the_path(orc):
    """Torch along a node row at 12 m/s (one 6 m node per 0.5 s step), r_g =
    6 m, S_g = 24 m/s (the radius is capped from the second step on): the
    node L metres down the path (L >= 12 m) is first covered at the step
    where psi_g = 0 exactly, at t_g + (L - r_g)/|v|; a node 6 m beside the
    path is covered when the torch passes it, at t_g + L/|v|.  (Both are
    step starts: the nearest point was laid at that instant, and the arrival
    from it, t_p + dist/S_g, is capped at the step start.)"""
    a = (3.0 + 6 * 10, 3.0 + 6 * 20)
    tor = synth.drip_torch(a[0], a[1], 12.0, 0.0, t_start=0.0, t_end=10.0, radius=6.0,
                           speed=24.0)
    w = still_workload(nxa=12, nya=6, steps=30, ignitions=[tor])
    o = run(w)
    i0, j0 = 10, 20
    # the torch stops at t_h = 10 s, 120 m down the path
    for m in range(2, 22):
        L = 6.0 * m
        assert o.tign[j0, i0 + m] == pytest.approx((L - 6.0) / 12.0, abs=1e-13), m
        if L <= 120.0:
            assert o.tign[j0 + 1, i0 + m] == pytest.approx(L / 12.0, abs=1e-13), m
            assert o.tign[j0 - 1, i0 + m] == pytest.approx(L / 12.0, abs=1e-13), m
    # beyond the end of the laid line plus r_g nothing is ignited
    assert not np.isfinite(o.tign[j0, i0 + 22:]).any()
    assert not np.isfinite(o.tign[j0 + 1, i0 + 21:]).any()
    # behind the start the nearest point is a, laid at t_g: covered at the
    # step start 0.5 s (R = 6 m), reached by the S_g front at 6/24 = 0.25 s
    assert o.tign[j0, i0 - 1] == pytest.approx(0.25, abs=1e-13)


def test_torch_that_does_not_move_is_a_growing_point(orc):
    """t_h = t_g: the segment stays the point a, the radius min{r_g, S_g (t -
    t_g)} grows at S_g over the same window as a fixed point ignition: the
    same level set and, up to rounding, the same arrival times t_g +
    dist/S_g."""
    tor = synth.drip_torch(300.0, 200.0, 5.0, -3.0, t_start=1.0, t_end=1.0, radius=40.0,
                           speed=2.0)
    fix = synth.point_ignition(300.0, 200.0, radius=40.0, t_start=1.0, speed=2.0)
    wa = still_workload(steps=45, ignitions=[tor])
    wb = still_workload(steps=45, ignitions=[fix])
    a, b = run(wa), run(wb)
    assert np.array_equal(a.psi, b.psi)
    fa, fb = np.isfinite(a.tign), np.isfinite(b.tign)
    assert np.array_equal(fa, fb) and fa.sum() > 100
    assert np.allclose(a.tign[fa], b.tign[fb], rtol=0, atol=1e-12)


def test_window_ends_after_the_torch_and_the_radius(orc):
    """No application after t_h + r_g/S_g: a later level set is unchanged
    once the window has closed (the fuel does not spread)."""
    tor = synth.drip_torch(40.0, 33.0, 10.0, 0.0, t_start=0.0, t_end=2.0, radius=8.0, speed=4.0)
    w = still_workload(steps=9, ignitions=[tor])  # last step start 4.0 = 2.0 + 8/4
    o = run(w)
    p9, t9 = o.psi.copy(), o.tign.copy()
    for _ in range(10):
        o.step(w.u, w.v, w.dt)
    assert np.array_equal(o.psi, p9) and np.array_equal(o.tign, t9, equal_nan=True)
    X, Y = node_xy(w)
    want = seg_dist(X, Y, (40.0, 33.0), (60.0, 33.0)) - 8.0
    near = want < 0.5 * o.psi_far
    assert np.allclose(o.psi[near], want[near], rtol=0, atol=1e-12)
