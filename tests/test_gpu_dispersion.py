"""Measured dispersion of the GPU paths.  An exact discrete plane wave (the
Bloch eigenvector of the element stencil with the fully discrete frequency
omega = (2/dt) asin((dt/2) sqrt(lambda)), Section 2's element and Eq.
eqtimehistory) is started on a homogeneous block and stepped on the GPU; at the
nodes no boundary can reach, the computed field must be that wave, and the
phase advance fitted from it gives the measured phase velocity, whose ratio to
the continuum velocity is the dispersion error.  The Bloch matrix comes from
the hand-derived closed form of the element, not from the oracle."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from tests.closed_forms import OV_ALPHA, V_ALPHA, element_closed_form, sign
from tests.gpu_common import PATHS

pytestmark = pytest.mark.gpu

VP, VS, RHO = 2500.0, 1000.0, 2000.0
NSTEP = 10


def _bloch(K, kvec):
    D = np.zeros((3, 3), dtype=complex)
    for a in range(8):
        for b in range(8):
            dx = np.array([(sign(b, m) - sign(a, m)) / 2.0 for m in range(3)])
            D += K[3 * a:3 * a + 3, 3 * b:3 * b + 3] * np.exp(1j * kvec @ dx)
    return D


def _block():
    n = 2 * NSTEP + 6
    return {"name": "homogeneous", "shape": (n, n, n), "h": 1.0,
            "material_ids": np.zeros(n ** 3, dtype=np.int32),
            "material_table": np.array([[VP, VS, RHO]]), "source": None,
            "receivers": None, "nsteps": NSTEP, "fix_bottom": 0}


def _measure(path, kind, kvec, mode):
    """Step the plane wave NSTEP times on the GPU; return (worst interior
    deviation from the exact discrete wave / amplitude, fitted omega, exact
    discrete omega, continuum omega)."""
    mesh = _block()
    n = mesh["shape"][0]
    G, kap = RHO * VS * VS, RHO * (VP * VP - 4.0 / 3.0 * VS * VS)
    K = element_closed_form(OV_ALPHA if kind == vfe.VFE_OVFEM else V_ALPHA, 1.0,
                            kap - 2.0 * G / 3.0, G)
    w2, V = np.linalg.eigh(_bloch(K, kvec))
    lam = w2[mode].real / RHO
    k, j, i = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    x = np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)], axis=1).astype(float)
    e = np.exp(1j * (x @ kvec))[:, None] * V[:, mode][None, :]   # [nodes][3]
    inner = ((i > NSTEP) & (i < n - NSTEP) & (j > NSTEP) & (j < n - NSTEP)
             & (k > NSTEP) & (k < n - NSTEP)).reshape(-1)
    with vfe.Mesh(mesh, path=PATHS[path], kind=kind, source=False, receivers=False) as m:
        dt = m.dt
        omega = 2.0 / dt * np.arcsin(0.5 * dt * np.sqrt(lam))
        field = lambda t: np.real(e * np.exp(-1j * omega * t)).reshape(-1)
        vfe.vfe_set_state(m.handle, field(0.0), field(-dt))
        dev, phases = 0.0, []
        # u(t) = Re(e) cos(omega t) + Im(e) sin(omega t) on the inner nodes:
        # fit (cos, sin) after every step and unwrap the phase
        basis = np.stack([np.real(e[inner]).reshape(-1), np.imag(e[inner]).reshape(-1)], axis=1)
        for s in range(1, NSTEP + 1):
            m.step(1)
            u, _ = vfe.vfe_get_state(m.handle)
            ui = u.reshape(-1, 3)[inner].reshape(-1)
            dev = max(dev, float(np.abs(ui - field(s * dt).reshape(-1, 3)[inner].reshape(-1)).max()))
            c, sn = np.linalg.lstsq(basis, ui, rcond=None)[0]
            phases.append(np.arctan2(sn, c))
    ph = np.unwrap(np.concatenate([[0.0], phases]))
    omega_fit = np.polyfit(np.arange(NSTEP + 1) * dt, ph, 1)[0]
    amp = float(np.abs(e).max())
    c0 = VP if mode == 2 else VS
    return dev / amp, omega_fit, omega, c0 * np.linalg.norm(kvec)


# the worst deviation of either path from the exact wave after ten steps,
# relative to the wave's amplitude (both measure below 1e-14)
DEV_TOL = {"tc": 1e-13, "fp64": 1e-13}


@pytest.mark.parametrize("path", ["tc", "fp64"])
@pytest.mark.parametrize("ppw", [5.0, 10.0])
@pytest.mark.parametrize("mode", [0, 2])   # slowest shear mode, P mode
def test_plane_wave_phase_velocity(path, ppw, mode):
    kvec = 2 * np.pi / ppw * np.array([1.0, 0.6, 0.3]) / np.linalg.norm([1.0, 0.6, 0.3])
    dev, omega_fit, omega, omega_c = _measure(path, vfe.VFE_OVFEM, kvec, mode)
    assert dev <= DEV_TOL[path]
    # the measured phase velocity is the discrete one ...
    assert omega_fit == pytest.approx(omega, rel=1e-12)
    # ... whose error against the continuum is several per cent at 5 points per
    # wavelength and about a quarter of that at 10 (a second-order scheme)
    err = abs(omega_fit / omega_c - 1.0)
    lo, hi = (0.02, 0.1) if ppw == 5.0 else (0.005, 0.025)
    assert lo < err < hi


def test_ovfem_less_dispersive_than_vfem_measured():
    """Section 2's claim, measured on the GPU (FP64 path, both elements): along
    a diagonal at 5 points per wavelength the P wave of the orthogonal element
    travels closer to the continuum velocity than that of the trilinear one."""
    kvec = 2 * np.pi / 5.0 * np.ones(3) / np.sqrt(3.0)
    errs = {}
    for kind in (vfe.VFE_OVFEM, vfe.VFE_VFEM):
        dev, omega_fit, omega, omega_c = _measure("fp64", kind, kvec, 2)
        assert dev <= DEV_TOL["fp64"]
        errs[kind] = abs(omega_fit / omega_c - 1.0)
    assert errs[vfe.VFE_OVFEM] < errs[vfe.VFE_VFEM]
