"""The z-slab decomposition on one GPU: the slabs of one model stepped one
after another with the node-plane exchange (vfe_pack_plane /
vfe_unpack_plane) after every step, against the whole model stepped as one
mesh.  The FP64 path gives the same bits (the same element sums at every own
node); the tensor-core path keeps each slab's own fixed-point unit, so a
received plane is rounded once into it, and matches to the FP64-equivalent
bound, as do both against the oracle."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import slab as S
from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import PATHS, oracle_source, rel_l2, rel_max

pytestmark = pytest.mark.gpu


def _model():
    nx, ny, nz = 40, 36, 30
    k = np.arange(nz)[:, None, None] * np.ones((nz, ny, nx), dtype=np.int64)
    mat = np.where(k >= 18, 0, np.where(k >= 9, 1, 2))
    mat[12:16, 10:20, 5:30] = 3
    mat[nz - 2:, :, :20] = -1
    table = [[1800.0, 700.0, 2000.0], [2600.0, 1100.0, 2200.0], [3000.0, 1400.0, 2300.0],
             [1500.0, 500.0, 1900.0]]
    rec = [(5, 5, 14), (20, 18, 15), (30, 30, 29), (12, 8, 3), (33, 2, 22)]
    return W._mesh((nx, ny, nz), 1.0, mat, table, W._source((20, 18, 15), 80.0), rec, 60,
                   "slab_test_40x36x30")


def _run_slabs(mesh, world, nsteps, path, dt, stencil=True):
    import torch
    slabs = [S.Slab(mesh, world, r, dt) for r in range(world)]
    engines = [S.GpuSlabEngine(s, torch, path=path, stencil=stencil) for s in slabs]
    # the slabs without the source size the fixed-point unit for it too
    scale = next(e.source_scale() for s, e in zip(slabs, engines) if s.workload["source"])
    for e in engines:
        e.set_source_bound(scale)
    bufs = [torch.empty(s.plane_values(), dtype=torch.float64, device="cuda") for s in slabs]
    for _ in range(nsteps):
        for e in engines:
            e.step()
        # each slab's own boundary planes into its neighbours' halo planes
        for r in range(world - 1):
            lo, hi = slabs[r], slabs[r + 1]
            engines[r].pack(lo.hi_own, bufs[r])
            engines[r].mesh.synchronize()
            engines[r + 1].unpack(hi.lo_halo, bufs[r])
            engines[r + 1].mesh.synchronize()
            engines[r + 1].pack(hi.lo_own, bufs[r + 1])
            engines[r + 1].mesh.synchronize()
            engines[r].unpack(lo.hi_halo, bufs[r + 1])
            engines[r].mesh.synchronize()
        # one fixed-point unit for all slabs: the maximum of their bounds
        for e in engines:
            e.bound_word()
            e.mesh.synchronize()
        top = torch.stack([e.bound.clone() for e in engines]).max(dim=0).values
        torch.cuda.synchronize()
        for e in engines:
            e.set_bound_word(top)
            e.mesh.synchronize()
    nx, ny, nz = mesh["shape"]
    per = 3 * (nx + 1) * (ny + 1)
    u = np.zeros(per * (nz + 1))
    traces = np.zeros((nsteps, len(mesh["receivers"]), 3))
    for s, e in zip(slabs, engines):
        ul, _ = vfe.vfe_get_state(e.mesh.handle)
        u[s.z0 * per:s.z1 * per] = ul[s.lo_own * per:(s.hi_own + 1) * per]
        if len(s.receivers):
            traces[:, s.receivers] = e.mesh.traces()
        e.close()
    return u, traces


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("path", ["fp64", "tc"])
def test_slabs_match_whole_mesh(orc, world, path):
    mesh = _model()
    nsteps = 60
    dt = orc.dt(0, mesh, 0.5)
    with vfe.Mesh(mesh, path=PATHS[path], dt=dt) as m:
        m.step(nsteps)
        u_one, _ = vfe.vfe_get_state(m.handle)
        tr_one = m.traces()
    u_sl, tr_sl = _run_slabs(mesh, world, nsteps, PATHS[path], dt)
    ref = orc.run(0, mesh, dt, nsteps, source=oracle_source(mesh),
                  receivers=W.receiver_nodes(mesh))
    if path == "fp64":
        assert np.array_equal(u_sl, u_one)
        assert np.array_equal(tr_sl, tr_one)
        assert rel_l2(tr_sl, ref) <= 1e-12
    else:
        assert rel_max(u_sl, u_one) <= 1e-12
        assert rel_l2(tr_sl, tr_one) <= 1e-9
        assert rel_l2(tr_sl, ref) <= 1e-9


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_with_node_corrections_match_whole_mesh(orc, world):
    """Slabs and the whole mesh with per-node corrections (stencil=2: the
    layer, inclusion and void interfaces and the faces, including each
    slab's halo planes, corrected in the stencil kernel's runs)."""
    mesh = _model()
    nsteps = 40
    dt = orc.dt(0, mesh, 0.5)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, dt=dt, stencil=2) as m:
        m.step(nsteps)
        u_one, _ = vfe.vfe_get_state(m.handle)
        tr_one = m.traces()
    u_sl, tr_sl = _run_slabs(mesh, world, nsteps, vfe.VFE_PATH_TC, dt, stencil=2)
    ref = orc.run(0, mesh, dt, nsteps, source=oracle_source(mesh),
                  receivers=W.receiver_nodes(mesh))
    assert rel_max(u_sl, u_one) <= 1e-12
    assert rel_l2(tr_sl, tr_one) <= 1e-9
    assert rel_l2(tr_sl, ref) <= 1e-9
