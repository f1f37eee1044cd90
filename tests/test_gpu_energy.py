"""Energy drift of the GPU paths.  Unforced, the central-difference scheme
(Eq. eqtimehistory) keeps E_{n+1/2} = 1/2 v^T M v + 1/2 u^{n+1 T} K u^n,
v = (u^{n+1} - u^n)/dt, constant; the FP64 path keeps it to round-off, and the
tensor-core path's drift (its K u is FP64-equivalent, its state a 64-bit fixed
point) is measured here over 2,000 steps.  The energy is evaluated on the CPU
with the oracle's K u."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import PATHS

pytestmark = pytest.mark.gpu

# worst |E - E_0| / E_0 over 2,000 steps (both paths measure below 1e-15:
# the round-off of evaluating E)
DRIFT_TOL = {"fp64": 1e-13, "tc": 1e-13}


def _energy(orc, mesh, dt, u_new, u_old, mass, free):
    v = (u_new - u_old) / dt
    m3 = np.repeat(mass * free, 3)
    return 0.5 * np.sum(m3 * v * v) + 0.5 * u_new @ orc.ku(0, mesh, u_old)


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_energy_drift(orc, path):
    mesh = W.random_mesh(41, shape=(14, 13, 9), void_frac=0.1)
    mass = orc.node_mass(0, mesh)
    nx, ny, nz = mesh["shape"]
    free = mass > 0
    free[: (nx + 1) * (ny + 1)] = False
    rng = np.random.default_rng(8)
    u = rng.uniform(-1e-3, 1e-3, 3 * len(mass)) * np.repeat(free, 3)
    um = u + rng.uniform(-1e-5, 1e-5, len(u)) * np.repeat(free, 3)
    energies = []
    with vfe.Mesh(mesh, path=PATHS[path], source=False, receivers=False) as m:
        dt = m.dt
        vfe.vfe_set_state(m.handle, u, um)
        for _ in range(40):
            m.step(50)
            un, uo = vfe.vfe_get_state(m.handle)
            energies.append(_energy(orc, mesh, dt, un, uo, mass, free))
    e = np.array(energies)
    e0 = _energy(orc, mesh, dt, u, um, mass, free)
    assert e0 > 0
    drift = float(np.abs(e - e0).max() / e0)
    assert drift <= DRIFT_TOL[path], drift
