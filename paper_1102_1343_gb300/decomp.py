"""Domain decomposition of one fire over several GPUs: the host-side plan.

The fire step (Sect. 5) is a stencil: one step moves information at most 3
fire nodes (stage 1 reads psi^n one node away, stage 2 reads psi* one node
away, the quadrature reads psi^{n+1} and t_i one node away).  So the fire mesh
splits into rectangular patches of whole atmospheric cells (as WRF splits its
domain into patches, Sect. "Parallel structure"), each rank advancing its
patch extended by a halo:

* the halo is one atmospheric cell wide on every side that borders another
  patch (so the extended patch is again a mesh of whole atmospheric cells
  with its own staggered wind); the rank computes the whole extended patch
  (redundant work in the halo) and keeps its own cells;
* before each step the 3 node rows / columns of the halo next to the patch
  are refreshed from the neighbours that own them (psi, t_i and F); deeper
  halo nodes hold stale values that cannot reach the patch within one step;
* the heat fluxes of the patch's own atmospheric cells are exact and stay on
  the rank (no communication);
* the boundary check of Sect. 3.1 applies to the whole domain's outer band:
  each rank tests its own nodes in that band and the status is OR-ed over
  the ranks (an all-reduce of one integer); the per-patch engine's own
  boundary flag, raised at the extended patch's edge, is not used.

Nothing here computes the fire model: the per-patch step is a callable (the
CUDA library on a GPU rank; in the tests, any engine that advances a mesh
given its staggered wind).  Point-to-point exchange uses torch.distributed
send/recv (NCCL between GPUs, gloo on the CPU).
"""
from __future__ import annotations

import dataclasses

import numpy as np

HALO_NODES = 3  # reach of one fire step in nodes (two Heun stages + quadrature)


@dataclasses.dataclass(frozen=True)
class Patch:
    """Patch of rank `rank` at grid position (px, py): its own atmospheric
    cells [I0, I1) x [J0, J1) and the extended range [E_I0, E_I1) x
    [E_J0, E_J1) it computes (one halo cell toward each neighbour)."""
    rank: int
    px: int
    py: int
    I0: int
    I1: int
    J0: int
    J1: int
    E_I0: int
    E_I1: int
    E_J0: int
    E_J1: int


class Partition:
    """nx_atm x ny_atm atmospheric cells refined sr_x x sr_y, split into a
    grid of px x py patches of whole atmospheric cells (rank = py_index * px
    + px_index).  Every patch needs at least one atmospheric cell and the
    refinement must give the halo cell at least HALO_NODES nodes; a halo node
    within HALO_NODES of the patch then lies in the half of its cell next to
    the patch, so its wind comes from atmospheric rows the extended patch
    holds (refinements >= 6, e.g. the paper's 10)."""

    def __init__(self, nx_atm, ny_atm, sr_x, sr_y, px, py):
        if px < 1 or py < 1 or px > nx_atm or py > ny_atm:
            raise ValueError("each patch needs at least one atmospheric cell")
        if min(sr_x, sr_y) < 2 * HALO_NODES:
            raise ValueError(f"refinement must be at least {2 * HALO_NODES}")
        self.nxa, self.nya, self.srx, self.sry = nx_atm, ny_atm, sr_x, sr_y
        self.px, self.py = px, py
        xs = np.linspace(0, nx_atm, px + 1).round().astype(int)
        ys = np.linspace(0, ny_atm, py + 1).round().astype(int)
        self.patches = []
        for j in range(py):
            for i in range(px):
                I0, I1, J0, J1 = int(xs[i]), int(xs[i + 1]), int(ys[j]), int(ys[j + 1])
                self.patches.append(Patch(j * px + i, i, j, I0, I1, J0, J1,
                                          I0 - (1 if i > 0 else 0), I1 + (1 if i < px - 1 else 0),
                                          J0 - (1 if j > 0 else 0), J1 + (1 if j < py - 1 else 0)))

    @property
    def size(self):
        return self.px * self.py

    def patch(self, rank) -> Patch:
        return self.patches[rank]

    # fire-node slices (global) of a patch's own and extended ranges
    def own_nodes(self, p: Patch):
        return (slice(p.J0 * self.sry, p.J1 * self.sry), slice(p.I0 * self.srx, p.I1 * self.srx))

    def ext_nodes(self, p: Patch):
        return (slice(p.E_J0 * self.sry, p.E_J1 * self.sry),
                slice(p.E_I0 * self.srx, p.E_I1 * self.srx))

    def own_in_ext(self, p: Patch):
        """The own nodes as a slice of the extended patch's arrays."""
        oy, ox = (p.J0 - p.E_J0) * self.sry, (p.I0 - p.E_I0) * self.srx
        return (slice(oy, oy + (p.J1 - p.J0) * self.sry), slice(ox, ox + (p.I1 - p.I0) * self.srx))

    def own_cells_in_ext(self, p: Patch):
        """The own atmospheric cells as a slice of the extended patch's grid."""
        return (slice(p.J0 - p.E_J0, p.J1 - p.E_J0), slice(p.I0 - p.E_I0, p.I1 - p.E_I0))

    def ext_wind(self, p: Patch, u, v):
        """The staggered wind of the extended patch: u [ny][nx+1] on x-faces,
        v [ny+1][nx] on y-faces, sub-arrays of the global ones."""
        return (u[p.E_J0:p.E_J1, p.E_I0:p.E_I1 + 1], v[p.E_J0:p.E_J1 + 1, p.E_I0:p.E_I1])

    def origin(self, p: Patch, dx_atm, dy_atm):
        """Position (m) of the extended patch's corner in the domain."""
        return p.E_I0 * dx_atm, p.E_J0 * dy_atm

    # ---- halo exchange plan: (peer, region to send, region to receive),
    # each region a pair of global node slices.  p sends the peer its own
    # nodes within `width` of the peer's own nodes and receives the peer's
    # own nodes within `width` of its own (side and corner neighbours)
    def exchange_plan(self, p: Patch, width=HALO_NODES):
        nx, ny = self.nxa * self.srx, self.nya * self.sry
        (oy, ox) = self.own_nodes(p)
        plan = []
        for q in self.patches:
            if q.rank == p.rank or abs(q.px - p.px) > 1 or abs(q.py - p.py) > 1:
                continue
            (qy, qx) = self.own_nodes(q)
            send = (_inter(oy, _dilate(qy, width, ny)), _inter(ox, _dilate(qx, width, nx)))
            recv = (_inter(qy, _dilate(oy, width, ny)), _inter(qx, _dilate(ox, width, nx)))
            if None in send or None in recv:
                continue
            plan.append((q.rank, send, recv))
        return plan

    def boundary_mask(self, p: Patch, band: int):
        """Own nodes of p that lie in the domain's outer band (Sect. 3.1)."""
        (oy, ox) = self.own_nodes(p)
        nx, ny = self.nxa * self.srx, self.nya * self.sry
        yy = np.arange(oy.start, oy.stop)[:, None]
        xx = np.arange(ox.start, ox.stop)[None, :]
        return (xx < band) | (xx >= nx - band) | (yy < band) | (yy >= ny - band)


def _dilate(a: slice, w: int, n: int) -> slice:
    return slice(max(0, a.start - w), min(n, a.stop + w))


def _inter(a: slice, b: slice):
    s = slice(max(a.start, b.start), min(a.stop, b.stop))
    return s if s.start < s.stop else None


def exchange_halos(part: Partition, rank: int, fields, ext_origin, width=HALO_NODES):
    """Refresh the halo of this rank's extended arrays from the neighbours'
    own nodes.  fields: list of 2-D numpy arrays (or CPU tensors) over the
    extended patch; ext_origin: (row, col) of the extended patch's first node
    in the domain.  Blocking point-to-point torch.distributed send/recv, in
    an order that cannot deadlock (lower rank sends first to each peer)."""
    import torch
    import torch.distributed as dist
    p = part.patch(rank)
    r0, c0 = ext_origin

    def local(sl):
        return (slice(sl[0].start - r0, sl[0].stop - r0), slice(sl[1].start - c0, sl[1].stop - c0))

    for peer, send, recv in part.exchange_plan(p, width):
        out = [torch.from_numpy(np.ascontiguousarray(f[local(send)])) for f in fields]
        inn = [torch.empty(((recv[0].stop - recv[0].start), (recv[1].stop - recv[1].start)),
                           dtype=torch.from_numpy(np.asarray(f[:1, :1])).dtype) for f in fields]
        for k in range(len(fields)):
            if rank < peer:
                dist.send(out[k], peer)
                dist.recv(inn[k], peer)
            else:
                dist.recv(inn[k], peer)
                dist.send(out[k], peer)
        for f, x in zip(fields, inn):
            f[local(recv)] = x.numpy()


def reduce_status(status: int) -> int:
    """OR of the ranks' status bits (an all-reduce of one integer)."""
    import torch
    import torch.distributed as dist
    # the OR from the per-bit maxima (MAX is reduced by every backend)
    bits = torch.tensor([(int(status) >> b) & 1 for b in range(8)], dtype=torch.int64)
    dist.all_reduce(bits, op=dist.ReduceOp.MAX)
    return int(sum(int(x) << b for b, x in enumerate(bits.tolist())))


def shard_members(sizes, world):
    """Ensemble members spread over `world` ranks without communication:
    largest first onto the least-loaded rank (sizes = nodes per member).
    Returns, per rank, the list of member indices."""
    load = [0] * world
    out = [[] for _ in range(world)]
    for k in sorted(range(len(sizes)), key=lambda k: -sizes[k]):
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(k)
        load[r] += sizes[k]
    return [sorted(x) for x in out]
