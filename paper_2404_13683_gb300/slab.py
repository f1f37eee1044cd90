"""Z-slab decomposition of one model over several GPUs.

The paper closes (Section 4) with the remark that the method extends to many
GPUs.  The explicit step needs, at a node, only the nodes of the eight
elements around it, so the node planes k = 0..nz split into contiguous slabs,
one per rank.  A rank's mesh holds the element layers around its own planes:
its own planes [z0, z1) plus one halo node plane on each side that has a
neighbour.  After every step each rank sends u^n of its lowest own plane to
the rank below and of its highest own plane to the rank above, and writes the
two planes it receives into its halo planes (``vfe_pack_plane`` /
``vfe_unpack_plane``); the next step then forms K u on its own planes exactly
as the whole mesh would.  Its own update, the source and the receivers on its
planes need nothing else, so one exchange of a node plane each way per step
is the only exchange (3 (nx+1)(ny+1) doubles per neighbour).  On the
tensor-core path the slabs also agree on the fixed-point unit of the state:
one all-reduce MAX of an 8-byte bound per step (``vfe_get_scale_bound`` /
``vfe_set_scale_bound``), and the slabs without the source size the unit for
its increment too (``vfe_set_source_bound``).

The decomposition (plane ranges, the sub-model each rank builds, which local
plane goes where) is independent of the engine that steps a slab: ``run_slab``
takes any object with ``step()``, ``pack(k, buf)``, ``unpack(k, buf)`` and a
transport for the exchange (torch.distributed point-to-point operations, over
NCCL on GPUs or gloo on CPUs).
"""
from __future__ import annotations

import numpy as np


def plane_ranges(nz: int, world: int):
    """Own node planes [z0, z1) of each rank: node planes 0..nz in ``world``
    contiguous ranges as equal as possible (each at least one plane)."""
    planes = nz + 1
    if world < 1 or world > planes:
        raise ValueError("need 1 <= world <= nz + 1 (%d planes, %d ranks)" % (planes, world))
    cuts = [planes * r // world for r in range(world + 1)]
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


class Slab:
    """Rank ``rank``'s part of ``workload`` split over ``world`` ranks.

    Attributes: ``z0, z1`` (own global node planes), ``e0`` (global index of
    the slab mesh's node plane 0 and element layer 0), ``lo_halo`` / ``hi_halo``
    (local halo planes or None), ``lo_own`` / ``hi_own`` (local own planes
    sent down / up), ``receivers`` (indices into the workload's receiver list
    of the receivers on own planes, in the slab mesh's order), ``workload``
    (the slab mesh's workload dictionary)."""

    def __init__(self, workload, world: int, rank: int, dt: float):
        nx, ny, nz = workload["shape"]
        self.world, self.rank = world, rank
        self.z0, self.z1 = plane_ranges(nz, world)[rank]
        # node planes [e0, e1] and element layers [e0, e1) of the slab mesh
        self.e0 = max(self.z0 - 1, 0)
        e1 = min(self.z1, nz)
        if e1 <= self.e0:   # a top slab that is only the plane nz
            self.e0 = e1 - 1
        self.nz_local = e1 - self.e0
        self.ranges = plane_ranges(nz, world)
        self.global_source = workload.get("source")
        self.lo_halo = 0 if rank > 0 else None
        self.hi_halo = self.nz_local if rank < world - 1 else None
        self.lo_own = self.z0 - self.e0
        self.hi_own = self.z1 - 1 - self.e0
        mat = np.asarray(workload["material_ids"]).reshape(nz, ny, nx)[self.e0:e1]
        rec = np.asarray(workload["receivers"], dtype=np.int64).reshape(-1, 3)
        own = np.flatnonzero((rec[:, 2] >= self.z0) & (rec[:, 2] < self.z1))
        self.receivers = own
        local_rec = rec[own].copy()
        local_rec[:, 2] -= self.e0
        src = workload.get("source")
        if src is not None and not (self.z0 <= src["ijk"][2] < self.z1):
            src = None
        elif src is not None:
            i, j, k = src["ijk"]
            src = dict(src, ijk=(i, j, k - self.e0))
        w = dict(workload)
        w.update(shape=(nx, ny, self.nz_local), material_ids=np.ascontiguousarray(mat.reshape(-1)),
                 receivers=local_rec.astype(np.int32).reshape(-1, 3), source=src, dt=float(dt),
                 name="%s_slab%d_of_%d" % (workload.get("name", "mesh"), rank, world))
        # only the lowest slab holds the model's bottom plane; a halo plane is
        # overwritten by the exchange after every step, so it is left free
        w["fix_bottom"] = int(workload.get("fix_bottom", 1)) if rank == 0 else 0
        self.workload = w

    def plane_values(self):
        nx, ny, _ = self.workload["shape"]
        return 3 * (nx + 1) * (ny + 1)


def exchange(slab: Slab, engine, dist, bufs):
    """One exchange after a step: own boundary planes to the neighbours,
    their planes into the halo planes.  ``bufs`` holds four tensors of
    ``slab.plane_values()`` doubles on the transport's device (send down, send
    up, receive from below, receive from above)."""
    send_lo, send_hi, recv_lo, recv_hi = bufs
    ops = []
    if slab.lo_halo is not None:
        engine.pack(slab.lo_own, send_lo)
        ops += [dist.P2POp(dist.isend, send_lo, slab.rank - 1),
                dist.P2POp(dist.irecv, recv_lo, slab.rank - 1)]
    if slab.hi_halo is not None:
        engine.pack(slab.hi_own, send_hi)
        ops += [dist.P2POp(dist.isend, send_hi, slab.rank + 1),
                dist.P2POp(dist.irecv, recv_hi, slab.rank + 1)]
    engine.before_exchange()
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    if slab.lo_halo is not None:
        engine.unpack(slab.lo_halo, recv_lo)
    if slab.hi_halo is not None:
        engine.unpack(slab.hi_halo, recv_hi)
    engine.sync_scale(dist)


def run_slab(slab: Slab, engine, dist, nsteps: int, make_buffer):
    """Advance the slab ``nsteps`` steps with an exchange after each.
    ``make_buffer(n)`` returns a tensor of n doubles on the transport's
    device."""
    n = slab.plane_values()
    bufs = [make_buffer(n) for _ in range(4)]
    for _ in range(nsteps):
        engine.step()
        exchange(slab, engine, dist, bufs)


def source_scale(slab: Slab, engine, dist):
    """dt^2 / m at the model's source node, from the slab that holds it (a
    broadcast over the group; None without a source)."""
    import torch
    src = slab.global_source
    if src is None:
        return None
    owner = next(r for r, (z0, z1) in enumerate(slab.ranges) if z0 <= src["ijk"][2] < z1)
    t = torch.zeros(1, dtype=torch.float64, device=engine.device)
    if slab.rank == owner:
        t[0] = engine.source_scale()
    if dist is not None:
        dist.broadcast(t, owner)
    return float(t[0])


class GpuSlabEngine:
    """A slab stepped by the library on the current CUDA device; the
    exchange runs on the mesh's stream (the torch stream the mesh was created
    with), so NCCL point-to-point operations queue behind the step."""

    device = "cuda"

    def __init__(self, slab: Slab, torch, path=None, stages=5, stencil=True):
        from . import vfe
        self.vfe, self.torch = vfe, torch
        self.stream = torch.cuda.Stream()
        self.mesh = vfe.Mesh(slab.workload, path=vfe.VFE_PATH_TC if path is None else path,
                             stages=stages, dt=slab.workload["dt"],
                             stream=self.stream.cuda_stream, stencil=stencil)
        if self.vfe.vfe_plane_values(self.mesh.handle) != slab.plane_values():
            raise RuntimeError("slab plane size mismatch")
        self.bound = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.slab = slab

    def source_scale(self):
        return self.vfe.vfe_get_source_scale(self.mesh.handle)

    def set_source_bound(self, dt2_over_m):
        """The model's source lies in another slab: size the fixed-point unit
        for its increment (dt2_over_m from that slab)."""
        src = self.slab.global_source
        if src is not None and self.slab.workload["source"] is None:
            self.vfe.vfe_set_source_bound(self.mesh.handle, src["dir"], src["f0"], src["t0"],
                                          src["amp"], dt2_over_m)

    def bound_word(self):
        self.vfe.vfe_get_scale_bound(self.mesh.handle, self.bound.data_ptr())
        return self.bound

    def set_bound_word(self, t):
        self.vfe.vfe_set_scale_bound(self.mesh.handle, t.data_ptr())

    def sync_scale(self, dist):
        if dist is None:
            return
        b = self.bound_word()
        dist.all_reduce(b, op=dist.ReduceOp.MAX)
        self.set_bound_word(b)

    def step(self):
        self.mesh.step(1)

    def pack(self, k, buf):
        self.vfe.vfe_pack_plane(self.mesh.handle, k, buf.data_ptr())

    def unpack(self, k, buf):
        self.vfe.vfe_unpack_plane(self.mesh.handle, k, buf.data_ptr())

    def before_exchange(self):
        # NCCL runs on torch's current stream: make it the mesh's stream
        self.torch.cuda.set_stream(self.stream)

    def close(self):
        self.mesh.close()
