"""Pins of the oracle's Rayleigh-damped run.  Section 3 uses Rayleigh damping
C = alpha M + beta K without a time discretisation; oracle_run_damped takes
the mass term with the central velocity and the stiffness term with the
backward velocity:
    (1 + a) u^{n+1} = 2 u^n - (1 - a) u^{n-1} - dt^2 M^-1 (K w^n - F^n),
    a = alpha dt / 2,  w^n = u^n + (beta / dt) (u^n - u^{n-1}).
Pinned here: no damping reproduces the undamped run bit for bit; on a single
free element started on an eigenmode of M^-1 K the motion stays on that mode
and its amplitude follows the scalar form of the same recurrence; for small
time steps the modal decay rate is Rayleigh's damping ratio
h(w) = alpha / (2 w) + beta w / 2."""
import ctypes

import numpy as np
import pytest

from paper_2404_13683_gb300 import workloads as W


def _one_element(vp=2000.0, vs=800.0, rho=2100.0, h=1.0):
    return {"name": "one", "shape": (1, 1, 1), "h": h,
            "material_ids": np.zeros(1, dtype=np.int32),
            "material_table": np.array([[vp, vs, rho]]), "source": None,
            "receivers": np.zeros((0, 3), dtype=np.int32), "nsteps": 1}


def _modes(orc, mesh):
    vp, vs, rho = mesh["material_table"][0]
    G, kap = rho * vs * vs, rho * (vp * vp - 4.0 / 3.0 * vs * vs)
    K = orc.element_stiffness(0, mesh["h"], kap, G)
    m = rho * mesh["h"] ** 3 / 8.0
    lam, phi = np.linalg.eigh(K / m)
    return lam, phi


def _damped_direct(orc, mesh, dt, nsteps, u0, um1, alpha, beta, receivers):
    """oracle_run_damped called directly (also with alpha = beta = 0)."""
    L = orc.lib()
    nx, ny, nz = mesh["shape"]
    mat = np.ascontiguousarray(mesh["material_ids"], dtype=np.int32)
    tab = np.ascontiguousarray(mesh["material_table"], dtype=np.float64)
    rec = np.ascontiguousarray(receivers, dtype=np.int64)
    tr = np.zeros((nsteps, len(rec), 3))
    uo, umo = np.zeros_like(u0), np.zeros_like(u0)
    sdir = np.zeros(3)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = L.oracle_run_damped(0, nx, ny, nz, mesh["h"], p(mat), p(tab), len(tab), 1, dt, nsteps,
                             -1, p(sdir), 1.0, 0.0, 0.0, float(alpha), float(beta), len(rec),
                             p(rec), p(u0), p(um1), p(tr), p(uo), p(umo))
    assert rc == 0
    return tr, uo, umo


def test_no_damping_is_the_undamped_run(orc):
    mesh = W.random_mesh(31, shape=(4, 3, 5), void_frac=0.1)
    dt = orc.dt(0, mesh, 0.5)
    rng = np.random.default_rng(3)
    nn = (4 + 1) * (3 + 1) * (5 + 1)
    u0 = rng.uniform(-1e-3, 1e-3, 3 * nn)
    um1 = u0 + rng.uniform(-1e-5, 1e-5, 3 * nn)
    rec = np.arange(0, nn, 7)
    tr, uo, umo = _damped_direct(orc, mesh, dt, 25, u0, um1, 0.0, 0.0, rec)
    tr0, uo0, umo0 = orc.run(0, mesh, dt, 25, receivers=rec, u0=u0, um1=um1, return_state=True)
    assert np.array_equal(tr, tr0) and np.array_equal(uo, uo0) and np.array_equal(umo, umo0)


@pytest.mark.parametrize("which", [-1, 12])
@pytest.mark.parametrize("a,b", [(0.05, 0.0), (0.0, 0.2), (0.04, 0.1)])
def test_eigenmode_follows_the_scalar_recurrence(orc, which, a, b):
    mesh = _one_element()
    lam, phi = _modes(orc, mesh)
    dt = 0.5 * 2.0 / np.sqrt(lam.max())
    alpha, beta = 2.0 * a / dt, b * dt
    lk, vk = lam[which], phi[:, which]
    assert lk > 1e-6 * lam.max()
    n = 30
    tr = orc.run(0, mesh, dt, n, receivers=np.arange(8), fix_bottom=False, u0=vk, um1=vk,
                 alpha=alpha, beta=beta)
    x = [1.0, 1.0]   # x^{-1}, x^0
    for _ in range(n):
        xn, xp = x[-1], x[-2]
        x.append((2 * xn - (1 - a) * xp - dt * dt * lk * (xn + b * (xn - xp))) / (1 + a))
    expect = np.array(x[2:])[:, None] * vk[None, :]
    assert np.abs(tr.reshape(n, 24) - expect).max() <= 1e-12 * np.abs(vk).max()


@pytest.mark.parametrize("alpha_frac,beta_frac", [(1.0, 0.0), (0.0, 1.0), (0.5, 0.5)])
def test_decay_rate_is_rayleigh_ratio(orc, alpha_frac, beta_frac):
    """Small dt: the modal amplitude decays as exp(-h(w) w t).  Writing the
    modal recurrence as x_{n+1} = T x_n - D x_{n-1}, the quadratic form
    x_n^2 - T x_n x_{n-1} + D x_{n-1}^2 shrinks by exactly D per step, so it
    measures the decay without the phase ripple."""
    mesh = _one_element()
    lam, phi = _modes(orc, mesh)
    lk, vk = lam[-1], phi[:, -1]
    w = np.sqrt(lk)
    dt = 0.01 * 2.0 / w
    h_target = 0.02
    alpha, beta = alpha_frac * h_target * 2.0 * w, beta_frac * h_target * 2.0 / w
    h = alpha / (2 * w) + beta * w / 2
    n = 2000   # about six periods
    _, uo, umo = orc.run(0, mesh, dt, n, fix_bottom=False, u0=vk, um1=vk,
                         return_state=True, alpha=alpha, beta=beta)
    a, b, c = 0.5 * alpha * dt, beta / dt, dt * dt * lk
    T, D = (2.0 - c * (1.0 + b)) / (1.0 + a), (1.0 - a - c * b) / (1.0 + a)
    q = lambda xn, xp: xn * xn - T * xn * xp + D * xp * xp
    rate = -np.log(q(uo @ vk, umo @ vk) / q(1.0, 1.0)) / (2 * w * n * dt)
    assert rate == pytest.approx(h, rel=0.01)
