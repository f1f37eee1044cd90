"""Pins of the oracle's time integration: CFL bound, energy conservation of the
central-difference scheme, the element dispersion relation (axis-aligned
closed form) and a time-domain plane-wave check against the Bloch symbol."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import workloads as W
from tests.closed_forms import OV_ALPHA, V_ALPHA, element_closed_form, sign


@pytest.mark.parametrize("kind,alpha", [(0, OV_ALPHA), (1, V_ALPHA)])
@pytest.mark.parametrize("vp,vs", [(3.5, 1.0), (2.5, 1.0), (2000.0, 800.0)])
def test_element_max_eig_vs_lapack(orc, kind, alpha, vp, vs):
    rho, ds = 1.7, 0.9
    G, kap = rho * vs * vs, rho * (vp * vp - 4.0 / 3.0 * vs * vs)
    K = element_closed_form(alpha, ds, kap - 2 * G / 3, G)
    lmax = np.linalg.eigvalsh(K / (rho * ds ** 3 / 8)).max()
    assert orc.element_max_eig(kind, ds, kap, G, rho) == pytest.approx(lmax, rel=1e-12)


def test_dt_is_half_critical(orc):
    mesh = W.config1()
    dt = orc.dt(0, mesh, 0.5)
    crit = []
    for vp, vs, rho in mesh["material_table"]:
        G, kap = rho * vs * vs, rho * (vp * vp - 4 / 3 * vs * vs)
        crit.append(2.0 / np.sqrt(orc.element_max_eig(0, 1.0, kap, G, rho)))
    assert dt == pytest.approx(0.5 * min(crit), rel=1e-15)


def _energy(orc, kind, mesh, dt, u_next, u_now, mass, free):
    v = (u_next - u_now) / dt
    m3 = np.repeat(mass, 3) * np.repeat(free, 3)
    return 0.5 * np.sum(m3 * v * v) + 0.5 * u_next @ orc.ku(kind, mesh, u_now)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("fix_bottom", [True, False])
def test_energy_conserved(orc, kind, fix_bottom):
    mesh = W.random_mesh(21, shape=(4, 3, 4), void_frac=0.15)
    dt = orc.dt(kind, mesh, 0.5)
    mass = orc.node_mass(kind, mesh)
    nx, ny, nz = mesh["shape"]
    free = mass > 0
    if fix_bottom:
        free[: (nx + 1) * (ny + 1)] = False
    rng = np.random.default_rng(4)
    u = rng.uniform(-1e-3, 1e-3, 3 * len(mass)) * np.repeat(free, 3)
    um = u + rng.uniform(-1e-5, 1e-5, len(u)) * np.repeat(free, 3)
    energies = []
    for _ in range(40):
        _, un, uc = orc.run(kind, mesh, dt, 1, fix_bottom=fix_bottom, u0=u, um1=um,
                            return_state=True)
        energies.append(_energy(orc, kind, mesh, dt, un, uc, mass, free))
        um, u = uc, un
    e = np.array(energies)
    assert e[0] > 0
    assert np.abs(e - e[0]).max() <= 1e-11 * e[0]


def _bloch(K, kvec, ds):
    D = np.zeros((3, 3), dtype=complex)
    for a in range(8):
        for b in range(8):
            dx = np.array([(sign(b, m) - sign(a, m)) * ds / 2 for m in range(3)])
            D += K[3 * a:3 * a + 3, 3 * b:3 * b + 3] * np.exp(1j * kvec @ dx)
    return D


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("ppw", [5, 10, 20])
def test_axis_dispersion_closed_form(orc, kind, ppw):
    """Waves along an axis: c_h/c = sin(kh/2)/(kh/2) for both elements."""
    ds, rho, vp, vs = 1.0, 2000.0, 2500.0, 1000.0
    G, kap = rho * vs * vs, rho * (vp * vp - 4 / 3 * vs * vs)
    K = orc.element_stiffness(kind, ds, kap, G)
    kh = 2 * np.pi / ppw
    D = _bloch(K, np.array([kh / ds, 0, 0]), ds)
    w2 = np.sort(np.linalg.eigvalsh(D).real) / (rho * ds ** 3)
    ratio = np.sin(kh / 2) / (kh / 2)
    cs, cp = np.sqrt(w2[0]) / (kh / ds), np.sqrt(w2[2]) / (kh / ds)
    assert cs / vs == pytest.approx(ratio, rel=1e-12)
    assert cp / vp == pytest.approx(ratio, rel=1e-12)


@pytest.mark.parametrize("kind", [0, 1])
def test_plane_wave_time_domain(orc, kind):
    """An exact discrete plane wave (Bloch eigenvector, fully discrete omega)
    propagates unchanged at nodes the boundary cannot reach in n steps."""
    n = 10
    shape = (2 * n + 6,) * 3
    nx, ny, nz = shape
    mesh = {"shape": shape, "h": 1.0, "material_ids": np.zeros(nx * ny * nz, np.int32),
            "material_table": np.array([[2500.0, 1000.0, 2000.0]])}
    vp, vs, rho = mesh["material_table"][0]
    G, kap = rho * vs * vs, rho * (vp * vp - 4 / 3 * vs * vs)
    K = orc.element_stiffness(kind, 1.0, kap, G)
    kvec = 2 * np.pi / 8.0 * np.array([1.0, 0.6, 0.3])
    D = _bloch(K, kvec, 1.0)
    w2, V = np.linalg.eigh(D)
    dt = orc.dt(kind, mesh, 0.5)
    for mode in (0, 2):
        lam = w2[mode].real / rho
        omega = 2.0 / dt * np.arcsin(dt / 2 * np.sqrt(lam))
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1),
                              indexing="ij")
        x = np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)], axis=1).astype(float)
        def field(t):
            ph = np.exp(1j * (x @ kvec - omega * t))
            return np.real(ph[:, None] * V[:, mode][None, :]).reshape(-1)
        tr, un, _ = orc.run(kind, mesh, dt, n, fix_bottom=False, u0=field(0.0),
                            um1=field(-dt), return_state=True)
        exact = field(n * dt).reshape(-1, 3)
        got = un.reshape(-1, 3)
        inner = ((i >= n + 1) & (i <= nx - n - 1) & (j >= n + 1) & (j <= ny - n - 1)
                 & (k >= n + 1) & (k <= nz - n - 1)).reshape(-1)
        assert inner.sum() > 0
        err = np.abs(got[inner] - exact[inner]).max()
        assert err <= 1e-11, (mode, err)
        # and a wrong omega (the semi-discrete one) is visibly off
        wrong = np.sqrt(lam)
        ph = np.exp(1j * (x @ kvec - wrong * n * dt))
        bad = np.real(ph[:, None] * V[:, mode][None, :])
        assert np.abs(got[inner] - bad[inner]).max() > 100 * max(err, 1e-14)


def test_ovfem_less_dispersive_diagonal(orc):
    """Section 2's claim: OVFEM suppresses dispersion relative to VFEM; along a
    diagonal at 5 points per wavelength the OVFEM phase error is smaller for
    the P wave."""
    ds, rho, vp, vs = 1.0, 2000.0, 2500.0, 1000.0
    G, kap = rho * vs * vs, rho * (vp * vp - 4 / 3 * vs * vs)
    kh = 2 * np.pi / 5
    kvec = kh * np.ones(3) / np.sqrt(3)
    errs = []
    for kind in (0, 1):
        D = _bloch(orc.element_stiffness(kind, ds, kap, G), kvec, ds)
        w2 = np.sort(np.linalg.eigvalsh(D).real) / rho
        errs.append(abs(np.sqrt(w2[2]) / kh / vp - 1.0))
    assert errs[0] < errs[1]


def test_source_first_steps(orc):
    """From rest, u^1 = dt^2/m F^0 at the source node only, and u^2 follows
    Eq. eqtimehistory with K u^1 (checked against the oracle's own K u)."""
    mesh = W.random_mesh(31, shape=(3, 3, 3), void_frac=0.0)
    dt = orc.dt(0, mesh, 0.5)
    src = {"node": W.node_index(mesh["shape"], 1, 2, 2), "dir": [0.2, -0.3, 0.9],
           "f0": 7.0, "t0": 0.05, "amp": 3.0}
    mass = orc.node_mass(0, mesh)
    nn = len(mass)
    rec = np.arange(nn)
    tr = orc.run(0, mesh, dt, 2, source=src, receivers=rec, fix_bottom=True)
    F0 = 3.0 * orc.ricker(0.0, 7.0, 0.05) * np.array([0.2, -0.3, 0.9])
    u1 = np.zeros((nn, 3)); u1[src["node"]] = dt * dt / mass[src["node"]] * F0
    assert np.allclose(tr[0], u1, rtol=1e-15, atol=0)
    F1 = 3.0 * orc.ricker(dt, 7.0, 0.05) * np.array([0.2, -0.3, 0.9])
    f = orc.ku(0, mesh, u1.reshape(-1)).reshape(-1, 3)
    u2 = 2 * u1 - dt * dt / mass[:, None] * f
    u2[src["node"]] += dt * dt / mass[src["node"]] * F1
    nxy = (mesh["shape"][0] + 1) * (mesh["shape"][1] + 1)
    u2[:nxy] = 0.0
    assert np.allclose(tr[1], u2, rtol=1e-13, atol=1e-13 * np.abs(u2).max())


def test_ricker_closed_form(orc):
    for t in (0.0, 0.05, 0.1, 0.137):
        a = (np.pi * 10.0 * (t - 0.1)) ** 2
        assert orc.ricker(t, 10.0, 0.1) == pytest.approx((1 - 2 * a) * np.exp(-a), rel=1e-15)
