"""The experiment's boundary condition (Section 3: the four corner points of
the bottom face fixed in x, y and z) in the oracle's run, against stepping
the brute-force dense assembly in the test: the free-DOF update of
Eq. eqtimehistory with exactly those four nodes (and massless ones) held."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import workloads as W
from tests.test_oracle_mesh import _dense_K


@pytest.mark.parametrize("shape", [(3, 2, 3), (2, 4, 2)])
def test_corner_fixed_run_matches_dense_stepping(orc, shape):
    mesh = W.random_mesh(60 + sum(shape), shape=shape, void_frac=0.0)
    nx, ny, nz = shape
    K = _dense_K(orc, 0, mesh)
    mass = orc.node_mass(0, mesh)
    dt = orc.dt(0, mesh, 0.5)
    fixed = np.zeros(len(mass), dtype=bool)
    for i in (0, nx):
        for j in (0, ny):
            fixed[W.node_index(shape, i, j, 0)] = True
    free3 = np.repeat(~fixed & (mass > 0), 3)
    rng = np.random.default_rng(8)
    u = rng.uniform(-1e-3, 1e-3, 3 * len(mass)) * free3
    um = u + rng.uniform(-1e-5, 1e-5, len(u)) * free3
    a, b = u.copy(), um.copy()
    for _ in range(6):
        n = 2 * a - b - dt * dt / np.repeat(mass, 3) * (K @ a)
        n[~free3] = 0.0
        a, b = n, a
    _, uo, umo = orc.run(0, mesh, dt, 6, u0=u, um1=um, return_state=True, fix_bottom=2)
    assert np.abs(uo - a).max() <= 1e-12 * np.abs(a).max()
    assert np.abs(umo - b).max() <= 1e-12 * np.abs(b).max()
    # the bottom face moves except at its corners
    bottom = [W.node_index(shape, i, j, 0) for i in range(nx + 1) for j in range(ny + 1)]
    moving = [n for n in bottom if not fixed[n]]
    assert np.abs(uo.reshape(-1, 3)[moving]).max() > 0
    assert np.abs(uo.reshape(-1, 3)[fixed]).max() == 0
