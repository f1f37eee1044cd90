"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times: the whole state after steps of the 128x128x64 model against the oracle,
and K u of the 512x512x256 topographic model (67 M elements) at sampled nodes
against the oracle evaluated one node at a time."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import KU_TOL, PATHS, oracle_source, rel_max

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_config2_state_after_steps(orc, path):
    mesh = W.config2()
    n = 20
    dt = orc.dt(0, mesh, 0.5)
    _, uo, umo = orc.run(0, mesh, dt, n, source=oracle_source(mesh),
                         receivers=W.receiver_nodes(mesh), return_state=True)
    with vfe.Mesh(mesh, path=PATHS[path]) as m:
        m.step(n)
        u, um = vfe.vfe_get_state(m.handle)
    tol = 1e-12 if path == "fp64" else 1e-9
    assert rel_max(u, uo) <= tol
    assert rel_max(um, umo) <= tol


@pytest.fixture(scope="module")
def config3():
    return W.config3()


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_config3_ku_sampled(orc, config3, path):
    mesh = config3
    u = W.random_displacement(mesh, 21)
    nn = len(u) // 3
    rng = np.random.default_rng(4)
    sel = rng.choice(nn, 3000, replace=False)
    ref = orc.ku_nodes(0, mesh, u, sel)
    with vfe.Mesh(mesh, path=PATHS[path], source=False, receivers=False) as m:
        f = m.internal_force(u).reshape(-1, 3)
    assert rel_max(f[sel], ref) <= KU_TOL
    # void cells above the topography: nodes with no solid element feel no force
    assert np.isfinite(f).all()
