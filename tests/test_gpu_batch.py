"""Batched stepping of several meshes (the many-case use): one fused element
kernel launch per step and stage count, plus each mesh's node-stencil launch
on side streams; bit-identical to stepping each mesh alone, and against the
oracle."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import TRACE_TOL, oracle_source, rel_l2

pytestmark = pytest.mark.gpu


def _models():
    ms = [W.random_mesh(70 + i, shape=s, void_frac=0.05)
          for i, s in enumerate([(9, 8, 7), (20, 17, 12), (31, 33, 9), (16, 16, 16), (5, 40, 6)])]
    ms += W.config4(seed=9, n_models=3, n_min=24, n_max=40)
    return ms


def test_batch_equals_individual_runs():
    models = _models()
    nsteps = 23
    alone = []
    for w in models:   # the same kernels per node as in the batch
        with vfe.Mesh(w) as m:
            m.step(nsteps)
            alone.append((vfe.vfe_get_state(m.handle), m.traces()))
    meshes = [vfe.Mesh(w) for w in models]
    with vfe.Batch(meshes) as b:
        b.step(10)
        b.step(13)   # odd count: the single-step path and the parity swap
        b.synchronize()
        for m, (state, tr) in zip(meshes, alone):
            u, um = vfe.vfe_get_state(m.handle)
            assert np.array_equal(u, state[0]) and np.array_equal(um, state[1])
            assert np.array_equal(m.traces(), tr)
    for m in meshes:
        m.close()


def test_batch_vs_oracle(orc):
    models = _models()[:3]
    meshes = [vfe.Mesh(w) for w in models]
    with vfe.Batch(meshes) as b:
        b.step(30)
        b.synchronize()
        for w, m in zip(models, meshes):
            dt = orc.dt(0, w, 0.5)
            ref = orc.run(0, w, dt, 30, source=oracle_source(w), receivers=W.receiver_nodes(w))
            assert rel_l2(m.traces(), ref) <= TRACE_TOL["tc"]
    for m in meshes:
        m.close()


def test_batch_element_kernel_only_meshes_equal_individual_runs():
    """Meshes without the stencil kernel: every column-plane in the fused
    element launch, bit-identical to each mesh alone."""
    models = _models()[:4]
    alone = []
    for w in models:
        with vfe.Mesh(w, stencil=False) as m:
            m.step(9)
            alone.append(m.traces())
    meshes = [vfe.Mesh(w, stencil=False) for w in models]
    with vfe.Batch(meshes) as b:
        b.step(9)
        b.synchronize()
        for m, tr in zip(meshes, alone):
            assert np.array_equal(m.traces(), tr)
    for m in meshes:
        m.close()


def test_batch_rejects_mixed_paths():
    w = W.random_mesh(80, shape=(4, 4, 4))
    a = vfe.Mesh(w, path=vfe.VFE_PATH_TC)
    b = vfe.Mesh(w, path=vfe.VFE_PATH_FP64)
    with pytest.raises(vfe.VfeError):
        vfe.Batch([a, b])
    a.close()
    b.close()


def test_batch_fewer_stages_equals_individual_runs():
    """The batched kernel with three digit stages: bit-identical to each mesh
    stepped alone with three stages."""
    models = _models()[:4]
    alone = []
    for w in models:
        with vfe.Mesh(w, stages=3) as m:
            m.step(11)
            alone.append(m.traces())
    meshes = [vfe.Mesh(w, stages=3) for w in models]
    with vfe.Batch(meshes) as b:
        b.step(11)
        b.synchronize()
        for m, tr in zip(meshes, alone):
            assert np.array_equal(m.traces(), tr)
    for m in meshes:
        m.close()


def test_batch_with_node_corrections_equals_individual_runs():
    """Meshes with per-node corrections (stencil=2: every column-plane but
    the source and receiver planes in the stencil kernel, the interface,
    void and face nodes corrected after it, on the batch's side streams)
    beside meshes without: bit-identical to each mesh alone."""
    models = [W.config3(shape=(48, 44, 24)), W.random_mesh(75, shape=(21, 18, 11), void_frac=0.15),
              _models()[2], _models()[5]]
    opts = [2, 2, 1, 2]
    nsteps = 11
    alone = []
    for w, st in zip(models, opts):
        with vfe.Mesh(w, stencil=st) as m:
            m.step(nsteps)
            alone.append((vfe.vfe_get_state(m.handle), m.traces()))
    meshes = [vfe.Mesh(w, stencil=st) for w, st in zip(models, opts)]
    with vfe.Batch(meshes) as b:
        b.step(nsteps)
        b.synchronize()
        for m, (state, tr) in zip(meshes, alone):
            u, um = vfe.vfe_get_state(m.handle)
            assert np.array_equal(u, state[0]) and np.array_equal(um, state[1])
            assert np.array_equal(m.traces(), tr)
    for m in meshes:
        m.close()
