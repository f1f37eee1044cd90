"""Pin of the oracle's adjoint-state gradient: dJ/dG_e against central finite
differences of the oracle's own misfit (each perturbed element gets its own
material with G +- delta at fixed kappa and rho; dt held fixed)."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import workloads as W


def with_element_G(mesh, e, dG):
    """Copy of mesh in which element e has shear modulus G_e + dG (kappa fixed)."""
    tab = mesh["material_table"].copy()
    m = int(mesh["material_ids"][e])
    vp, vs, rho = tab[m]
    G = rho * vs * vs
    kap = rho * (vp * vp - 4.0 / 3.0 * vs * vs)
    G2 = G + dG
    row = [np.sqrt((kap + 4.0 / 3.0 * G2) / rho), np.sqrt(G2 / rho), rho]
    ids = mesh["material_ids"].copy()
    ids[e] = len(tab)
    return dict(mesh, material_ids=ids, material_table=np.vstack([tab, row])), G


def problem(seed=3, shape=(6, 5, 5), nsteps=40):
    mesh = W.random_mesh(seed, shape=shape, void_frac=0.0)
    s = mesh["source"]
    src = {"node": W.source_node(mesh), "dir": [0.3, -0.2, 1.0], "f0": s["f0"] * 20,
           "t0": 0.004, "amp": 1e6}
    rec = W.receiver_nodes(mesh)
    return mesh, src, rec, nsteps


def misfit(orc, mesh, dt, n, src, rec, data):
    tr = orc.run(0, mesh, dt, n, source=src, receivers=rec)
    return 0.5 * float(np.sum((tr - data) ** 2))


@pytest.mark.parametrize("kind,fix_bottom", [(0, 1), (1, 1), (0, 2)])
def test_adjoint_gradient_matches_finite_differences(orc, kind, fix_bottom):
    """Both elements with the bottom plane fixed, and the orthogonal element
    with only the four bottom corner points fixed (the experiment's support)."""
    mesh, src, rec, n = problem()
    dt = orc.dt(kind, mesh, 0.5)
    # "observed" data from a model with a softer block
    obs = dict(mesh, material_table=mesh["material_table"] * np.array([1.0, 0.9, 1.0]))
    data = orc.run(kind, obs, dt, n, source=src, receivers=rec, fix_bottom=fix_bottom)
    grad, J = orc.misfit_gradient(kind, mesh, dt, n, src, rec, data, fix_bottom=fix_bottom)
    assert J > 0
    tr = orc.run(kind, mesh, dt, n, source=src, receivers=rec, fix_bottom=fix_bottom)
    assert J == pytest.approx(0.5 * np.sum((tr - data) ** 2), rel=1e-12)
    rng = np.random.default_rng(7)
    ne = mesh["material_ids"].size
    checked = 0
    for e in rng.choice(ne, 12, replace=False):
        mp, G = with_element_G(mesh, e, 0.0)
        d = 1e-4 * G
        jp = misfit_kind(orc, kind, with_element_G(mesh, e, +d)[0], dt, n, src, rec, data,
                         fix_bottom)
        jm = misfit_kind(orc, kind, with_element_G(mesh, e, -d)[0], dt, n, src, rec, data,
                         fix_bottom)
        fd = (jp - jm) / (2 * d)
        scale = np.abs(grad).max()
        assert abs(fd - grad[e]) <= 1e-5 * scale, (e, fd, grad[e])
        checked += 1
    assert checked == 12


def misfit_kind(orc, kind, mesh, dt, n, src, rec, data, fix_bottom=1):
    tr = orc.run(kind, mesh, dt, n, source=src, receivers=rec, fix_bottom=fix_bottom)
    return 0.5 * float(np.sum((tr - data) ** 2))


def test_adjoint_gradient_zero_at_data(orc):
    mesh, src, rec, n = problem(seed=4)
    dt = orc.dt(0, mesh, 0.5)
    data = orc.run(0, mesh, dt, n, source=src, receivers=rec)
    grad, J = orc.misfit_gradient(0, mesh, dt, n, src, rec, data)
    assert J == 0.0 and np.abs(grad).max() == 0.0
