"""GPU parity of the central-difference step (Eq. eqtimehistory) against
the FP64 oracle: one step from a given state, source-only steps, and full
receiver traces of the 32^3 two-layer workload."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import PATHS, TRACE_TOL, oracle_source, rel_l2, rel_max

pytestmark = pytest.mark.gpu


def _random_state(orc, mesh, seed, kind=0):
    mass = orc.node_mass(kind, mesh)
    nx, ny, nz = mesh["shape"]
    free = mass > 0
    free[: (nx + 1) * (ny + 1)] = False
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1e-3, 1e-3, 3 * len(mass)) * np.repeat(free, 3)
    um = u + rng.uniform(-1e-5, 1e-5, len(u)) * np.repeat(free, 3)
    return u, um


@pytest.mark.parametrize("path", ["tc", "fp64"])
@pytest.mark.parametrize("nsteps", [1, 2, 7])
def test_steps_from_state(orc, path, nsteps):
    mesh = W.random_mesh(5, shape=(17, 16, 6), void_frac=0.1)
    u, um = _random_state(orc, mesh, 3)
    dt = orc.dt(0, mesh, 0.5)
    _, uo, umo = orc.run(0, mesh, dt, nsteps, u0=u, um1=um, return_state=True)
    with vfe.Mesh(mesh, path=PATHS[path], source=False, receivers=False) as m:
        assert m.dt == pytest.approx(dt, rel=1e-13)
        vfe.vfe_set_state(m.handle, u, um)
        m.step(nsteps)
        ug, ugm = vfe.vfe_get_state(m.handle)
    assert rel_max(ug, uo) <= 1e-13
    assert rel_max(ugm, umo) <= 1e-13


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_source_only_steps(orc, path):
    mesh = W.random_mesh(6, shape=(9, 8, 7), void_frac=0.0)
    dt = orc.dt(0, mesh, 0.5)
    src = oracle_source(mesh)
    rec = W.receiver_nodes(mesh)
    tro = orc.run(0, mesh, dt, 12, source=src, receivers=rec)
    with vfe.Mesh(mesh, path=PATHS[path]) as m:
        m.step(12)
        tr = m.traces()
    assert tr.shape == tro.shape
    assert rel_l2(tr, tro) <= TRACE_TOL[path]


@pytest.mark.parametrize("path,kind", [("fp64", 0), ("fp64", 1), ("tc", 0)])
def test_config1_traces(orc, path, kind):
    mesh = W.config1()
    dt = orc.dt(kind, mesh, 0.5)
    tro = orc.run(kind, mesh, dt, mesh["nsteps"], source=oracle_source(mesh),
                  receivers=W.receiver_nodes(mesh))
    with vfe.Mesh(mesh, path=PATHS[path], kind=kind) as m:
        m.step(mesh["nsteps"])
        tr = m.traces()
    assert rel_l2(tr, tro) <= TRACE_TOL[path]


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_corner_fixed_traces(orc, path):
    """The experiment's boundary condition (the four bottom corner points
    fixed, Section 3): traces against the oracle."""
    mesh = W.random_mesh(44, shape=(19, 17, 9), void_frac=0.0)
    dt = orc.dt(0, mesh, 0.5)
    tro = orc.run(0, mesh, dt, 40, source=oracle_source(mesh), receivers=W.receiver_nodes(mesh),
                  fix_bottom=2)
    with vfe.Mesh(mesh, path=PATHS[path], fix_bottom=2) as m:
        m.step(40)
        tr = m.traces()
    assert rel_l2(tr, tro) <= TRACE_TOL[path]
