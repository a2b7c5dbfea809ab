"""Slabs of a domain split along z: partition, ghost-plane messages, exchange.

The paper runs one GPU and names multi-GPU runs as future work (Sec. 4 and
5).  The fused update of a node reads the stored moments of the nodes one
step away and the phase field of the nodes up to two steps away (its
gradient and Hessian stencils at the neighbours), so a domain cut into slabs
along z needs, before each step, one plane of the ten moment fields and two
planes of phi from each neighbouring slab; nothing else crosses a cut.

A slab is a single-grid context whose z faces toward its neighbours have
the "halo" rule (its ghost planes are written by ``tslb_halo_unpack``); the
faces of the whole domain stay where they are (the inlet on the first slab,
the outflow on the last).  The message of one side is ``tslb_halo_values``
values: the ten moment fields of one plane, then phi of two planes in
increasing z (``send_planes`` / ``ghost_planes`` below name the planes).

The exchange is point to point between z neighbours with
``torch.distributed`` (NCCL between GPUs, gloo between CPU processes); the
same functions drive the library's contexts on GPUs and, in the tests, FP64
oracle slabs on CPU ranks.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, Optional, Tuple

from . import inputs

MOMENT_FIELDS = 10  # rho - 1, u (3), P (6): one plane per message
PHI_PLANES = 2      # phi: two planes per message


@dataclasses.dataclass
class Slab:
    """Planes [z0, z1) of a domain of nz planes, held by `rank` of `world`;
    `lower` / `upper`: the rank holding the slab across the -z / +z cut, or
    None where the slab ends at a face of the domain."""

    rank: int
    world: int
    nz: int
    z0: int
    z1: int
    lower: Optional[int]
    upper: Optional[int]

    @property
    def planes(self) -> int:
        return self.z1 - self.z0


def partition(nz: int, world: int, rank: int, periodic_z: bool = False) -> Slab:
    """Balanced split of nz planes over `world` ranks (the first nz % world
    slabs one plane thicker); every slab has at least two planes.  With a
    periodic z axis the first and last slabs are neighbours."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    if nz < 2 * world:
        raise ValueError("every slab needs at least two planes")
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    z1 = z0 + base + (1 if rank < extra else 0)
    lower = rank - 1 if rank > 0 else (world - 1 if periodic_z and world > 1 else None)
    upper = rank + 1 if rank < world - 1 else (0 if periodic_z and world > 1 else None)
    return Slab(rank, world, nz, z0, z1, lower, upper)


def send_planes(planes: int, side: int) -> Tuple[int, Tuple[int, int]]:
    """Local planes a slab of `planes` planes sends through `side` (0: -z, 1:
    +z): (the plane of the moment fields, the two planes of phi)."""
    if side == 0:
        return 0, (0, 1)
    return planes - 1, (planes - 2, planes - 1)


def ghost_planes(planes: int, side: int) -> Tuple[int, Tuple[int, int]]:
    """Local ghost planes a message received through `side` fills: (the
    moment plane, the two phi planes); -1, -2 lie below the slab, planes,
    planes + 1 above it."""
    if side == 0:
        return -1, (-2, -1)
    return planes, (planes, planes + 1)


def slab_workload(w: inputs.Workload, slab: Slab) -> inputs.Workload:
    """The slab's own grid: the planes [z0, z1) of `w`, its z faces toward
    neighbouring slabs with the halo rule, every other face as in `w`."""
    faces = list(w.faces)
    if slab.lower is not None:
        faces[4] = "halo"
    if slab.upper is not None:
        faces[5] = "halo"
    return dataclasses.replace(w, name=f"{w.name}_slab{slab.rank}", nz=slab.planes, faces=tuple(faces))


def exchange(slab: Slab, pack: Callable[[int], object], unpack: Callable[[int, object], None],
             new_buffer: Callable[[], object], dist) -> None:
    """One exchange of ghost planes with the z neighbours.  pack(side) gives
    the message for the neighbour on that side, new_buffer() an empty message
    to receive into, unpack(side, message) stores the neighbour's message.
    The sends are posted in side order 0, 1 and the receives in side order 1,
    0, so that between any pair of ranks the k-th send of one matches the
    k-th receive of the other even where both cuts join the same two ranks
    (a periodic z axis split in two)."""
    ops, recvd = [], []
    for side, peer in ((0, slab.lower), (1, slab.upper)):
        if peer is not None:
            ops.append(dist.P2POp(dist.isend, pack(side), peer, tag=side))
    for side, peer in ((1, slab.upper), (0, slab.lower)):
        if peer is not None:
            buf = new_buffer()
            # the neighbour sent it through its opposite side
            ops.append(dist.P2POp(dist.irecv, buf, peer, tag=1 - side))
            recvd.append((side, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for side, buf in recvd:
        unpack(side, buf)


class SlabSimulation:
    """One slab of a jet or droplet domain split along z, on this rank's GPU:
    a library context for the slab (halo faces toward the neighbours) and the
    exchange of ghost planes before every step (torch.distributed, NCCL)."""

    def __init__(self, workload: inputs.Workload, slab: Slab, dist, **sim_kw):
        import torch

        from . import Simulation, tslb_halo_values
        self.workload, self.slab, self.dist = workload, slab, dist
        self.local = slab_workload(workload, slab)
        sim_kw.setdefault("graph_steps", 1)
        self.sim = Simulation(self.local, **sim_kw)
        self.values = tslb_halo_values(self.sim.ctx)
        dtype = torch.float32 if self.sim.options.storage == 0 else torch.int16
        self._dtype = dtype
        self._send = {side: torch.empty(self.values, dtype=dtype, device="cuda") for side in (0, 1)}

    def set_state(self, rho, u, phi, pi=None):
        """The whole domain's rho[nz, ny, nx], u[3, nz, ny, nx], phi (numpy or
        torch); this slab takes its planes."""
        z0, z1 = self.slab.z0, self.slab.z1
        self.sim.set_state(rho[z0:z1], u[:, z0:z1], phi[z0:z1], None if pi is None else pi[:, z0:z1])

    def exchange(self):
        import torch

        from . import tslb_halo_pack, tslb_halo_unpack
        ctx = self.sim.ctx

        def pack(side):
            tslb_halo_pack(ctx, side, self._send[side].data_ptr(), 1)
            self.sim.stream.synchronize()
            return self._send[side]

        def unpack(side, buf):
            tslb_halo_unpack(ctx, side, buf.data_ptr(), 1)
            self.sim.stream.synchronize()

        exchange(self.slab, pack, unpack, lambda: torch.empty(self.values, dtype=self._dtype, device="cuda"),
                 self.dist)

    def step(self, n: int = 1):
        for _ in range(int(n)):
            self.exchange()
            self.sim.step(1)

    def sums(self):
        """Total mass and phase field of the whole domain (FP64, summed over ranks)."""
        import torch
        m, p = self.sim.sums()
        t = torch.tensor([m, p], dtype=torch.float64, device="cuda")
        self.dist.all_reduce(t)
        return float(t[0]), float(t[1])

    def fields_numpy(self):
        return self.sim.fields_numpy()

    def close(self):
        self.sim.close()


def exchange_in_process(sims) -> None:
    """The ghost-plane exchange between the slabs of one domain held as
    contexts of one process (sims[k] holds slab k, in z order; a periodic z
    axis joins the last and the first): device-to-device copies, no
    communicator."""
    import torch

    from . import tslb_halo_pack, tslb_halo_unpack, tslb_halo_values
    n = len(sims)
    msgs = {}
    for k, s in enumerate(sims):
        vals = tslb_halo_values(s.ctx)
        dtype = torch.float32 if s.options.storage == 0 else torch.int16
        for side in (0, 1):
            if s.workload.faces[4 + side] == "halo":
                buf = torch.empty(vals, dtype=dtype, device="cuda")
                tslb_halo_pack(s.ctx, side, buf.data_ptr(), 1)
                msgs[(k, side)] = buf
    for s in sims:
        s.stream.synchronize()
    for k, s in enumerate(sims):
        if s.workload.faces[4] == "halo":
            tslb_halo_unpack(s.ctx, 0, msgs[((k - 1) % n, 1)].data_ptr(), 1)
        if s.workload.faces[5] == "halo":
            tslb_halo_unpack(s.ctx, 1, msgs[((k + 1) % n, 0)].data_ptr(), 1)
    for s in sims:
        s.stream.synchronize()
