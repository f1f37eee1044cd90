"""Tensor-core path with fewer digit stages, run-to-run determinism and the
digit-stage autotuner.

Each dropped low stage removes one 11-bit digit of the integer split of
Eq. int8comp1, so the node values carry 11 bits less and the error of K u
grows by about 2^11 per stage (the same rule as the paper's 7 bits per INT8
stage, Section 3, Table 3)."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import autotune, vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import KU_TOL, PATHS, rel_max

pytestmark = pytest.mark.gpu


def ku_stage_bound(stages):
    """Relative K u error allowed with `stages` digit stages.  The dropped
    balanced digits change a node value q (|q| < 2^51 at the column's scale)
    by at most 1024 * sum_{s < 5 - stages} 2^(11 s) < 2^(11 (5 - stages) - 1),
    i.e. 2^(11 (5 - stages) - 51) of the column's largest value; K's row sums
    of magnitudes turn that into at most a small multiple of max|K u| for the
    smooth random fields used here (factor 32 allowed)."""
    return max(KU_TOL, 32.0 * 2.0 ** (11 * (5 - stages) - 51))


@pytest.mark.parametrize("stages", [1, 2, 3, 4])
def test_ku_fewer_stages_within_bound(orc, stages):
    mesh = W.random_mesh(40 + stages, shape=(17, 16, 6), void_frac=0.1)
    u = W.random_displacement(mesh, 21)
    ref = orc.ku(0, mesh, u)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, stages=stages, source=False,
                  receivers=False) as m:
        f = m.internal_force(u)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, stages=5, source=False, receivers=False) as m:
        f5 = m.internal_force(u)
    err = rel_max(f, ref)
    assert err <= ku_stage_bound(stages), (stages, err)
    # a dropped stage is visible: the result differs from the full split
    if stages <= 3:
        assert rel_max(f, f5) > 1e3 * rel_max(f5, ref)


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_steps_are_deterministic(path):
    """No atomics on the data path: two runs give bit-identical states and
    traces."""
    mesh = W.random_mesh(33, shape=(31, 17, 9), void_frac=0.05)
    out = []
    for _ in range(2):
        with vfe.Mesh(mesh, path=PATHS[path]) as m:
            m.step(37)
            out.append((vfe.vfe_get_state(m.handle), m.traces()))
    (a, ta), (b, tb) = out
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(ta, tb)


def test_autotuner_choice_meets_tolerance():
    mesh = W.random_mesh(3, shape=(20, 18, 10), void_frac=0.05)
    best, report = autotune.choose_stages(mesh, tol=1e-6, steps=60)
    assert set(report) == {2, 3, 4, 5}
    assert report[5]["rel_l2"] <= 1e-12
    assert report[best]["rel_l2"] <= 1e-6
    assert report[2]["rel_l2"] >= report[4]["rel_l2"]


def test_autotuner_launch_config():
    """The launch-configuration search (stages x node-stencil x CTAs per
    launch) returns a candidate within the tolerance, and every candidate
    stays FP64-equivalent at five stages."""
    from tests.test_gpu_stencil import layered
    mesh = layered((40, 36, 16), void_top=2)   # uniform runs; receivers near the source
    choice, report = autotune.choose_config(mesh, tol=1e-6, steps=60, stages=(3, 5),
                                            stencil=(True, False), ctas=(0, 38))
    assert len(report) == 8
    assert choice["rel_l2"] <= 1e-6
    assert (choice["stages"], choice["stencil"], choice["ctas"]) in report
    for (st, sc, ct), r in report.items():
        if st == 5:
            assert r["rel_l2"] <= 1e-9, (sc, ct)


def test_batch_with_mixed_stage_counts_equals_individual_runs():
    """One batch whose meshes use different digit stage counts (one fused
    launch per count): each mesh bit-identical to its run alone."""
    models = [W.random_mesh(90 + i, shape=s, void_frac=0.05)
              for i, s in enumerate([(9, 8, 7), (20, 17, 12), (16, 16, 16), (31, 33, 9)])]
    stages = [5, 3, 4, 5]
    alone = []
    for w, st in zip(models, stages):
        with vfe.Mesh(w, stages=st) as m:
            m.step(37)
            alone.append(m.traces())
    meshes = [vfe.Mesh(w, stages=st) for w, st in zip(models, stages)]
    with vfe.Batch(meshes) as b:
        b.step(37)   # one 32-step graph, one 2-step graph, one single step
        b.synchronize()
        for m, tr in zip(meshes, alone):
            assert np.array_equal(m.traces(), tr)
    for m in meshes:
        m.close()
