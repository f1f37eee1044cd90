"""The z-slab decomposition (paper_2404_13683_gb300/slab.py) on CPU ranks
(gloo): each rank steps its slab with the FP64 oracle as the engine and
exchanges its boundary node planes after every step; the own planes of all
ranks must equal the single-rank oracle run bit for bit (the same element
sums in the same order at every own node).  No GPU is used."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2404_13683_gb300 import slab as S  # noqa: E402
from paper_2404_13683_gb300 import workloads as W  # noqa: E402

NSTEPS = 7


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _model():
    mesh = W.random_mesh(123, shape=(9, 7, 11), n_mat=3, void_frac=0.1)
    return mesh


def _initial_state(mesh):
    u0 = W.random_displacement(mesh, 5)
    return u0, 0.97 * u0


class OracleSlabEngine:
    """Steps a slab with the oracle (one call per step, from the state)."""

    def __init__(self, slab, orc, u_global, um_global):
        self.orc, self.slab = orc, slab
        nx, ny, nzl = slab.workload["shape"]
        per = 3 * (nx + 1) * (ny + 1)
        lo, hi = slab.e0 * per, (slab.e0 + nzl + 1) * per
        self.u = u_global[lo:hi].copy()
        self.um = um_global[lo:hi].copy()
        self.per = per

    def step(self):
        w = self.slab.workload
        _, u, um = self.orc.run(0, w, w["dt"], 1, u0=self.u, um1=self.um, return_state=True,
                                fix_bottom=w["fix_bottom"])
        self.u, self.um = u, um

    def pack(self, k, buf):
        buf.copy_(torch.from_numpy(self.u[k * self.per:(k + 1) * self.per]))

    def unpack(self, k, buf):
        self.u[k * self.per:(k + 1) * self.per] = buf.numpy()

    def before_exchange(self):
        pass

    def sync_scale(self, dist):
        pass


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    oracle.build()
    mesh = _model()
    dt = oracle.dt(0, mesh, 0.5)
    u0, um0 = _initial_state(mesh)
    slab = S.Slab(mesh, world, rank, dt)
    eng = OracleSlabEngine(slab, oracle, u0, um0)
    S.run_slab(slab, eng, dist, NSTEPS, lambda n: torch.zeros(n, dtype=torch.float64))
    per = eng.per
    out[rank] = (slab.z0, slab.z1,
                 eng.u[slab.lo_own * per:(slab.hi_own + 1) * per].copy(),
                 eng.um[slab.lo_own * per:(slab.hi_own + 1) * per].copy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_equal_single_rank_bit_for_bit(orc, world):
    mesh = _model()
    dt = orc.dt(0, mesh, 0.5)
    u0, um0 = _initial_state(mesh)
    _, uref, umref = orc.run(0, mesh, dt, NSTEPS, u0=u0, um1=um0, return_state=True)
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    nx, ny, nz = mesh["shape"]
    per = 3 * (nx + 1) * (ny + 1)
    covered = 0
    for r in range(world):
        z0, z1, u, um = out[r]
        assert np.array_equal(u, uref[z0 * per:z1 * per]), r
        assert np.array_equal(um, umref[z0 * per:z1 * per]), r
        covered += z1 - z0
    assert covered == nz + 1


def test_plane_ranges_and_halos():
    assert S.plane_ranges(10, 1) == [(0, 11)]
    assert S.plane_ranges(10, 3) == [(0, 3), (3, 7), (7, 11)]
    mesh = _model()
    nz = mesh["shape"][2]
    for world in (1, 2, 4, nz + 1):
        slabs = [S.Slab(mesh, world, r, 1e-3) for r in range(world)]
        assert slabs[0].lo_halo is None and slabs[-1].hi_halo is None
        for a, b in zip(slabs, slabs[1:]):
            assert a.z1 == b.z0
            # the plane a sends up is b's lower halo, and back
            assert a.e0 + a.hi_own == b.e0 + b.lo_halo == b.z0 - 1
            assert b.e0 + b.lo_own == a.e0 + a.hi_halo == a.z1
        recs = np.concatenate([s.receivers for s in slabs])
        assert sorted(recs.tolist()) == list(range(len(mesh["receivers"])))
        assert sum(s.workload["source"] is not None for s in slabs) == 1
    with pytest.raises(ValueError):
        S.plane_ranges(3, 5)
