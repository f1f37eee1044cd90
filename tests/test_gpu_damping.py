"""Rayleigh damping C = alpha M + beta K (Section 3) on both GPU paths against
the oracle's damped run (the same explicit discretisation: mass term with the
central velocity, stiffness term with the backward velocity)."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import PATHS, TRACE_TOL, oracle_source, rel_l2, rel_max

pytestmark = pytest.mark.gpu


def _mesh():
    return W.random_mesh(17, shape=(21, 17, 11), void_frac=0.05)


def _coefficients(mesh, dt, h=0.04):
    """Rayleigh coefficients for ratio h around the source frequency, kept
    well inside the stability bound (beta / dt <= 0.5 at half the critical
    step)."""
    f0 = mesh["source"]["f0"]
    alpha, beta = vfe.vfe_rayleigh_coefficients(h, 0.5 * f0, 2.0 * f0)
    beta = min(beta, 0.5 * dt)
    return alpha, beta


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_damped_traces_match_oracle(orc, path):
    mesh = _mesh()
    dt = orc.dt(0, mesh, 0.5)
    alpha, beta = _coefficients(mesh, dt)
    n = 60
    ref = orc.run(0, mesh, dt, n, source=oracle_source(mesh), receivers=W.receiver_nodes(mesh),
                  alpha=alpha, beta=beta)
    und = orc.run(0, mesh, dt, n, source=oracle_source(mesh), receivers=W.receiver_nodes(mesh))
    assert rel_l2(ref, und) > 1e-3   # the damping is visible
    with vfe.Mesh(mesh, path=PATHS[path]) as m:
        m.set_damping(alpha, beta)
        m.step(n)
        tr = m.traces()
    assert rel_l2(tr, ref) <= TRACE_TOL[path]


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_damped_steps_from_state_and_switch_on(orc, path):
    """Damped steps from a given state, and damping switched on after
    undamped steps (the library rebuilds w^n from the state it holds)."""
    mesh = _mesh()
    dt = orc.dt(0, mesh, 0.5)
    alpha, beta = _coefficients(mesh, dt, h=0.1)
    mass = orc.node_mass(0, mesh)
    nx, ny, nz = mesh["shape"]
    free = mass > 0
    free[: (nx + 1) * (ny + 1)] = False
    rng = np.random.default_rng(5)
    u = rng.uniform(-1e-3, 1e-3, 3 * len(mass)) * np.repeat(free, 3)
    um = u + rng.uniform(-1e-5, 1e-5, len(u)) * np.repeat(free, 3)
    _, u1, um1 = orc.run(0, mesh, dt, 6, u0=u, um1=um, return_state=True)
    _, u2, um2 = orc.run(0, mesh, dt, 9, u0=u1, um1=um1, return_state=True, alpha=alpha,
                         beta=beta)
    with vfe.Mesh(mesh, path=PATHS[path], source=False, receivers=False) as m:
        vfe.vfe_set_state(m.handle, u, um)
        m.step(6)
        m.set_damping(alpha, beta)
        m.step(9)
        ug, ugm = vfe.vfe_get_state(m.handle)
    assert rel_max(ug, u2) <= 1e-12
    assert rel_max(ugm, um2) <= 1e-12


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_zero_damping_is_the_undamped_step(path):
    mesh = _mesh()
    out = []
    for damp in (False, True):
        with vfe.Mesh(mesh, path=PATHS[path]) as m:
            if damp:
                m.set_damping(0.0, 0.0)
            m.step(25)
            out.append(m.traces())
    assert np.array_equal(out[0], out[1])


def test_damping_rejections(orc):
    mesh = _mesh()
    with vfe.Mesh(mesh) as m:
        dt = m.dt
        for a, b in ((-1.0, 0.0), (0.0, -1.0), (0.0, 10.0 * dt), (4.0 / dt, 0.0)):
            with pytest.raises(vfe.VfeError) as e:
                m.set_damping(a, b)
            assert e.value.code == vfe.VFE_EINVAL
        m.set_damping(*_coefficients(mesh, dt))
        with pytest.raises(vfe.VfeError):
            vfe.Batch([m])
        data = np.zeros((3, m.n_rec, 3))
        with pytest.raises(vfe.VfeError) as e:
            vfe.vfe_misfit_gradient(m.handle, data, 1)
        assert e.value.code == vfe.VFE_ESTATE


def test_damped_tc_matches_damped_fp64_long():
    """300 damped steps: the tensor-core path stays within its trace bar of the
    FP64 path, with damping and a forced source together."""
    mesh = W.random_mesh(23, shape=(40, 33, 20), void_frac=0.02)
    out = {}
    for path in ("tc", "fp64"):
        with vfe.Mesh(mesh, path=PATHS[path]) as m:
            alpha, beta = _coefficients(mesh, m.dt, h=0.05)
            m.set_damping(alpha, beta)
            s = mesh["source"]
            t = np.arange(300) * m.dt
            a = (np.pi * s["f0"] * (t - s["t0"])) ** 2
            rows = (s["amp"] * (1 - 2 * a) * np.exp(-a))[:, None] * np.array([0.3, 0.4, 0.866])[None, :]
            m.step_forced(rows[:150])
            m.step_forced(rows[150:])
            out[path] = m.traces()
    assert np.linalg.norm(out["fp64"]) > 0
    assert rel_l2(out["tc"], out["fp64"]) <= 1e-8
