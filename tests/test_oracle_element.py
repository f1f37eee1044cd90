"""Pins of the oracle's element matrices (Section 2: VFEM and OVFEM)."""
import numpy as np
import pytest

from tests.closed_forms import (OV_ALPHA, V_ALPHA, element_closed_form, rigid_modes)


@pytest.mark.parametrize("kind,alpha", [(0, OV_ALPHA), (1, V_ALPHA)])
@pytest.mark.parametrize("ds,kappa,G", [(1.0, 1.0, 0.0), (1.0, 0.0, 1.0), (0.37, 7.1e9, 2.3e9),
                                        (2e-3, 2.5e10, 1.1e10)])
def test_element_matches_closed_form(orc, kind, alpha, ds, kappa, G):
    K = orc.element_stiffness(kind, ds, kappa, G)
    ref = element_closed_form(alpha, ds, kappa - 2.0 * G / 3.0, G)
    scale = np.abs(ref).max()
    assert np.abs(K - ref).max() <= 1e-14 * scale


def test_elements_differ_off_axis(orc):
    # a transposed or dropped alpha-dependent factor would make them agree
    Ko = orc.element_stiffness(0, 1.0, 3.0, 1.0)
    Kv = orc.element_stiffness(1, 1.0, 3.0, 1.0)
    assert np.abs(Ko - Kv).max() > 0.01 * np.abs(Ko).max()


@pytest.mark.parametrize("kind", [0, 1])
def test_symmetric_psd_rank18_rigid_null(orc, kind):
    ds = 0.8
    K = orc.element_stiffness(kind, ds, 5.0e9, 1.7e9)
    assert np.abs(K - K.T).max() <= 1e-15 * np.abs(K).max()
    w = np.linalg.eigvalsh(K)
    tol = 1e-12 * w.max()
    assert w.min() > -tol
    assert int((w > tol).sum()) == 18
    R = rigid_modes(ds)
    assert np.abs(R @ K).max() <= 1e-13 * np.abs(K).max()


@pytest.mark.parametrize("kind", [0, 1])
def test_mass_diagonal_total(orc, kind):
    ds, rho = 0.6, 2100.0
    m = orc.element_node_mass(kind, ds, rho)
    assert m * 8 == pytest.approx(rho * ds ** 3, rel=1e-15)


def test_uniaxial_strain_energy(orc):
    # Uniform strain eps_xx = e: u_x = e*x.  Energy = 1/2 (lambda+2G) e^2 V for
    # both elements (the constant-strain patch test).
    from tests.closed_forms import node_positions
    ds, kap, G, e = 1.3, 4.0, 1.5, 0.01
    x = node_positions(ds)
    u = np.zeros(24); u[0::3] = e * x[:, 0]
    for kind in (0, 1):
        K = orc.element_stiffness(kind, ds, kap, G)
        energy = 0.5 * u @ K @ u
        lam = kap - 2 * G / 3
        assert energy == pytest.approx(0.5 * (lam + 2 * G) * e * e * ds ** 3, rel=1e-13)
