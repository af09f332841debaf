"""Spatial domain decomposition: the mesh cut into slabs along x, one per rank.

The upwind common flux (paper Sec. 2.1, Eq. 9) is the only coupling between elements: the moments,
the conservative Maxwellian and the BGK relaxation are local to a point. So a slab needs, per RK
stage, only the element layers of its x-neighbour slabs next to the two shared faces. Each stage of a
step then runs as: pack the slab's own two x-face element layers of the stage source, exchange them
with the neighbouring ranks (point-to-point, torch.distributed: NCCL between GPUs, gloo on CPU), set
the received layers as the halos of the exchange faces, run the stage.

`slab_config` cuts a workload into its slabs; `SlabStepper` drives any subdomain object that has
    stage(dt, s), pack_halo(face, s) -> tensor, set_halo(face, tensor), halo_like(face) -> tensor
through the stages. `GpuSlab` is that object for a libbgk context (bgk_stage, bgk_halo_pack,
bgk_set_halo on device tensors). Only argument marshalling and message passing are here; the halos
are packed and read by the library's own copies and kernels.
"""
from __future__ import annotations

from . import workloads as W

EXCHANGE = 3  # boundary kind of a face shared with another slab (BGK_BC_EXCHANGE)
LO, HI = 0, 1  # the slab's x-faces (face index 2 d + side with d = 0)


def slab_range(ne_x: int, rank: int, world: int):
    """Elements [e0, e1) along x of slab `rank`: as even as possible, the first slabs one larger."""
    q, r = divmod(ne_x, world)
    e0 = rank * q + min(rank, r)
    return e0, e0 + q + (1 if rank < r else 0)


def slab_config(c: dict, rank: int, world: int) -> dict:
    """The slab of workload config c (a mesh_kwargs-style dict with optional bc, bc_state) owned by
    `rank`: its x-extent and element count, and exchange faces where it meets another slab (also
    across a periodic x-wrap). The global x-faces keep their own kinds at the outer slabs."""
    ne = list(c["nelem"])
    if world > ne[0]:
        raise ValueError(f"{world} slabs need at least {world} elements along x, not {ne[0]}")
    e0, e1 = slab_range(ne[0], rank, world)
    h = (c["hi"][0] - c["lo"][0]) / ne[0]
    bc = [list(b) for b in c.get("bc", ((W.PERIODIC, W.PERIODIC),) * 3)]
    periodic_x = bc[0][0] == W.PERIODIC and bc[0][1] == W.PERIODIC
    if world > 1:
        if rank > 0 or periodic_x:
            bc[0][0] = EXCHANGE
        if rank < world - 1 or periodic_x:
            bc[0][1] = EXCHANGE
    out = dict(c)
    out["nelem"] = tuple([e1 - e0] + ne[1:])
    out["lo"] = tuple([c["lo"][0] + e0 * h] + list(c["lo"][1:]))
    out["hi"] = tuple([c["lo"][0] + e1 * h] + list(c["hi"][1:]))
    out["bc"] = tuple(tuple(b) for b in bc)
    out["x_range"] = (e0, e1)
    return out


class SlabStepper:
    """SSP-RK3 steps of one slab with the halo exchange before every stage."""

    def __init__(self, slab, rank: int, world: int, bc_x, dist=None):
        self.slab, self.rank, self.world, self.dist = slab, rank, world, dist
        self.left = (rank - 1) % world
        self.right = (rank + 1) % world
        self.has = [bc_x[LO] == EXCHANGE, bc_x[HI] == EXCHANGE]
        self.recv = [slab.halo_like(f) if self.has[f] else None for f in (LO, HI)]

    def exchange(self, stage: int):
        """Send this slab's lo-face layer to the left neighbour (its hi halo) and its hi-face layer to
        the right one (its lo halo); receive the neighbours' layers into this slab's halos. The send
        and receive order per peer is the same on both sides, so it also matches when left and right
        are one rank (two slabs on a periodic x)."""
        if not (self.has[LO] or self.has[HI]):
            return
        dist = self.dist
        send = [self.slab.pack_halo(f, stage) if self.has[f] else None for f in (LO, HI)]
        ops = []
        if self.has[LO]:
            ops.append(dist.P2POp(dist.isend, send[LO], self.left))
        if self.has[HI]:
            ops.append(dist.P2POp(dist.isend, send[HI], self.right))
        if self.has[HI]:
            ops.append(dist.P2POp(dist.irecv, self.recv[HI], self.right))
        if self.has[LO]:
            ops.append(dist.P2POp(dist.irecv, self.recv[LO], self.left))
        for r in dist.batch_isend_irecv(ops):
            r.wait()
        for f in (LO, HI):
            if self.has[f]:
                self.slab.set_halo(f, self.recv[f])

    def step(self, dt: float, nsteps: int = 1):
        for _ in range(nsteps):
            for s in range(3):
                self.exchange(s)
                self.slab.stage(dt, s)


class GpuSlab:
    """A libbgk context as a slab: halos are device tensors in the library's tile layout
    [velocity tile][face element][node][lane] (FP32). The context's stream must be torch's current
    stream (the messages are ordered on it)."""

    def __init__(self, solver, torch):
        self.s = solver
        self.torch = torch
        self.nhalo = solver.halo_floats()
        self.send = [self.halo_like(f) for f in (LO, HI)]

    def halo_like(self, face):
        return self.torch.empty(self.nhalo, dtype=self.torch.float32, device="cuda")

    def pack_halo(self, face, stage):
        self.s.halo_pack(stage, self.send[LO] if face == LO else None, self.send[HI] if face == HI else None)
        return self.send[face]

    def set_halo(self, face, t):
        self.s.set_halo(face, t)

    def stage(self, dt, s):
        self.s.stage(dt, s)
