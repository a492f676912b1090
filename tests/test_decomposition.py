"""The multi-GPU domain decomposition of one fire (paper_1102_1343_gb300/
decomp.py), emulated with gloo ranks on the CPU: each rank advances its
patch extended by one atmospheric cell, refreshing the 3 halo node rows /
columns next to its patch from the neighbours before every step, and the
boundary status is OR-ed over the ranks.  The per-patch engine is the oracle
run on the extended patch.  The assembled patches must equal the unsplit run:
bitwise with a power-of-two refinement (8: every node coordinate and wind
weight is then exact, so a patch computes the same bits as the whole mesh),
within rounding with the paper's refinement 10 (the interpolation weight
(j + 1/2)/10 rounds differently at different offsets).  Unmeasured on
hardware: every run of this project has one GPU."""
import os
import socket

import numpy as np
import pytest

from paper_1102_1343_gb300 import decomp, synth


def case(sr, boundary=False):
    w = synth.random_landscape(12, 9, sr=sr, seed=71, ignition="points", n_points=4,
                               edge_margin=100.0, steps=60)
    w.ignitions = w.ignitions + [synth.line_ignition(200.0, 250.0, 520.0, 290.0, radius=8.0,
                                                     t_start=2.0, speed=1.5)]
    if boundary:  # a fire next to the domain edge: the boundary status
        w.ignitions = w.ignitions + [synth.point_ignition(5.0, 300.0, radius=9.0)]
    w.mult = 2.0 + np.random.default_rng(3).uniform(0.0, 1.0, (w.ny, w.nx))
    return w


def psi_far(w):
    return float(np.hypot(w.nx * w.dx, w.ny * w.dy))


def _shift(g, x0, y0):
    g = dict(g)
    for k in ("ax", "bx"):
        g[k] -= x0
    for k in ("ay", "by"):
        g[k] -= y0
    return g


def _rank(rank, world, px, py, sr, boundary, port, q, width, poison):
    import torch.distributed as dist

    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = case(sr, boundary)
        part = decomp.Partition(w.nxa, w.nya, w.srx, w.sry, px, py)
        p = part.patch(rank)
        ey, ex = part.ext_nodes(p)
        x0, y0 = part.origin(p, w.dx_atm, w.dy_atm)
        orc = oracle.OracleFire(p.E_I1 - p.E_I0, p.E_J1 - p.E_J0, (w.srx, w.sry), w.dx_atm,
                                w.classes, w.fuel[ey, ex], w.dzdx[ey, ex], w.dzdy[ey, ex],
                                [_shift(g, x0, y0) for g in w.ignitions], mult=w.mult[ey, ex],
                                eps=w.eps, band=w.band, psi_far=psi_far(w), dy_atm=w.dy_atm)
        ue, ve = part.ext_wind(p, w.u, w.v)
        own, cells = part.own_in_ext(p), part.own_cells_in_ext(p)
        band = part.boundary_mask(p, w.band)
        heat, status = [], 0
        # halo nodes the exchange does not refresh (deeper than `width`)
        stale = np.ones((ey.stop - ey.start, ex.stop - ex.start), bool)
        stale[own] = False
        for _, _, recv in part.exchange_plan(p, width):
            stale[recv[0].start - ey.start:recv[0].stop - ey.start,
                  recv[1].start - ex.start:recv[1].stop - ex.start] = False
        rng = np.random.default_rng(100 + rank)
        for n in range(w.steps):
            decomp.exchange_halos(part, rank, [orc.psi, orc.tign, orc.frac], (ey.start, ex.start),
                                  width)
            if poison:  # finite garbage where the step must not look
                k = int(stale.sum())
                orc.psi[stale] = rng.uniform(-50.0, 50.0, k)
                orc.tign[stale] = np.where(rng.uniform(size=k) < 0.5, np.inf,
                                           rng.uniform(0.0, n * w.dt + 1e-3, k))
                orc.frac[stale] = rng.uniform(0.0, 1.0, k)
            hs, hl, st = orc.step(ue, ve, w.dt)
            mine = (st & oracle.STATUS_NONFINITE) | (
                oracle.STATUS_BOUNDARY if (orc.psi[own][band] < 0).any() else 0)
            status |= decomp.reduce_status(mine)
            heat.append((hs[cells].copy(), hl[cells].copy()))
        q.put((rank, orc.psi[own].copy(), orc.tign[own].copy(), orc.frac[own].copy(), heat,
               status))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def run_split(px, py, sr, boundary, width=decomp.HALO_NODES, poison=False):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = px * py
    port = _free_port()
    procs = [ctx.Process(target=_rank,
                         args=(r, world, px, py, sr, boundary, port, q, width, poison))
             for r in range(world)]
    for pr in procs:
        pr.start()
    out = {}
    for _ in range(world):
        r, *res = q.get(timeout=300)
        out[r] = res
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    w = case(sr, boundary)
    part = decomp.Partition(w.nxa, w.nya, w.srx, w.sry, px, py)
    psi = np.full((w.ny, w.nx), np.nan)
    tign, frac = psi.copy(), psi.copy()
    hs = [np.full((w.nya, w.nxa), np.nan) for _ in range(w.steps)]
    hl = [h.copy() for h in hs]
    statuses = set()
    for r, (ps, ti, fr, heat, st) in out.items():
        p = part.patch(r)
        oy, ox = part.own_nodes(p)
        psi[oy, ox], tign[oy, ox], frac[oy, ox] = ps, ti, fr
        for n, (a, b) in enumerate(heat):
            hs[n][p.J0:p.J1, p.I0:p.I1] = a
            hl[n][p.J0:p.J1, p.I0:p.I1] = b
        statuses.add(st)
    assert len(statuses) == 1  # every rank holds the reduced status
    return w, psi, tign, frac, hs, hl, statuses.pop()


def run_whole(w):
    import oracle
    o = oracle.OracleFire.from_workload(w, psi_far=psi_far(w))
    hs, hl, status = [], [], 0
    for _ in range(w.steps):
        a, b, st = o.step(w.u, w.v, w.dt)
        hs.append(a)
        hl.append(b)
        status |= st
    return o, hs, hl, status


@pytest.mark.parametrize("px,py,boundary,poison", [(1, 2, False, False), (2, 1, True, False),
                                                   (2, 2, False, False), (2, 2, True, True),
                                                   (3, 3, True, True)])
def test_split_run_is_bitwise_the_whole_run(orc, px, py, boundary, poison):
    """Refinement 8: patches of 1x2, 2x1 (with fire at the domain edge), 2x2
    and 3x3 ranks (an interior patch exchanging with all eight neighbours)
    give the whole run's psi, t_i, F, every step's heat grids and status,
    bit for bit; also when every halo node deeper than the 3 refreshed ones
    holds random values before each step (the step's reach is 3 nodes)."""
    w, psi, tign, frac, hs, hl, st = run_split(px, py, 8, boundary, poison=poison)
    o, hs_o, hl_o, st_o = run_whole(w)
    assert np.array_equal(psi, o.psi)
    assert np.array_equal(tign, o.tign)
    assert np.array_equal(frac, o.frac)
    for n in range(w.steps):
        assert np.array_equal(hs[n], hs_o[n]) and np.array_equal(hl[n], hl_o[n]), n
    assert st == st_o
    assert (st_o & oracle_boundary()) == (oracle_boundary() if boundary else 0)
    assert np.isfinite(o.tign).sum() > 100


def oracle_boundary():
    import oracle
    return oracle.STATUS_BOUNDARY


def test_split_run_matches_with_refinement_10(orc):
    """The paper's refinement 10 on 2x2 ranks: equal to the whole run within
    rounding (the wind weights of a patch differ in their last bit)."""
    w, psi, tign, frac, hs, hl, st = run_split(2, 2, 10, False)
    o, hs_o, hl_o, st_o = run_whole(w)
    scale = np.abs(o.psi).max()
    assert np.abs(psi - o.psi).max() <= 1e-10 * scale
    assert np.abs(frac - o.frac).max() <= 1e-10
    fin = np.isfinite(o.tign)
    assert np.array_equal(np.isfinite(tign), fin)
    assert np.abs(tign[fin] - o.tign[fin]).max() <= 1e-10 * w.steps * w.dt
    for n in range(w.steps):
        assert np.abs(hs[n] - hs_o[n]).max() <= 1e-10 * max(1.0, np.abs(hs_o[n]).max())
    assert st == st_o


def test_a_thinner_halo_is_not_enough(orc):
    """The step's reach: psi^{n+1} and t_i read psi two nodes out (stage 2
    reads psi* one node away, which read psi^n one further), the fuel
    fraction three (the quadrature reads psi^{n+1} one node out).  With
    only 2 halo rows / columns refreshed and the rest of the halo random,
    psi and t_i stay exact while F and the heat fluxes do not."""
    w, psi, tign, frac, hs, hl, st = run_split(2, 2, 8, False, width=2, poison=True)
    o, hs_o, hl_o, _ = run_whole(w)
    assert np.array_equal(psi, o.psi) and np.array_equal(tign, o.tign)
    assert not np.array_equal(frac, o.frac)
    assert any(not np.array_equal(a, b) for a, b in zip(hs, hs_o))


def test_partition_and_exchange_plan():
    """Patches tile the mesh; a halo region received from a peer is what
    that peer sends; corner neighbours exchange a 3 x 3 block; a refinement
    below 6 is refused."""
    part = decomp.Partition(12, 9, 8, 8, 3, 2)
    cover = np.zeros((72, 96), int)
    for p in part.patches:
        oy, ox = part.own_nodes(p)
        cover[oy, ox] += 1
    assert (cover == 1).all()
    for p in part.patches:
        for peer, send, recv in part.exchange_plan(p):
            back = {r: (s, rv) for r, s, rv in part.exchange_plan(part.patch(peer))}
            assert back[p.rank][0] == recv and back[p.rank][1] == send
            hy, hx = recv[0].stop - recv[0].start, recv[1].stop - recv[1].start
            q = part.patch(peer)
            if q.px != p.px and q.py != p.py:
                assert (hy, hx) == (3, 3)
            # received nodes lie inside this patch's extended range
            ey, ex = part.ext_nodes(p)
            assert ey.start <= recv[0].start and recv[0].stop <= ey.stop
            assert ex.start <= recv[1].start and recv[1].stop <= ex.stop
    with pytest.raises(ValueError):
        decomp.Partition(12, 9, 5, 5, 2, 2)


def test_ensemble_members_shard_without_communication():
    sizes = [int(s) ** 2 for s in synth.ensemble_sizes(64)]
    shards = decomp.shard_members(sizes, 4)
    assert sorted(k for s in shards for k in s) == list(range(64))
    loads = [sum(sizes[k] for k in s) for s in shards]
    assert max(loads) <= 1.05 * sum(sizes) / 4 + max(sizes)
