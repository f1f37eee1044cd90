"""Pins of the oracle's mesh-level operations: brute-force dense assembly vs
element-by-element K u, rigid modes, symmetry, node masses, sampled nodes."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import workloads as W


def _dense_K(orc, kind, mesh):
    """Dense global stiffness assembled in the test with its own indexing."""
    nx, ny, nz = mesh["shape"]
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    K = np.zeros((3 * nn, 3 * nn))
    tab = mesh["material_table"]
    mats = mesh["material_ids"].reshape(nz, ny, nx)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                m = mats[k, j, i]
                if m < 0:
                    continue
                vp, vs, rho = tab[m]
                G = rho * vs * vs
                kap = rho * (vp * vp - 4.0 / 3.0 * vs * vs)
                Ke = orc.element_stiffness(kind, mesh["h"], kap, G)
                dofs = []
                for a in range(8):
                    n = W.node_index(mesh["shape"], i + (a & 1), j + ((a >> 1) & 1), k + (a >> 2))
                    dofs += [3 * n, 3 * n + 1, 3 * n + 2]
                K[np.ix_(dofs, dofs)] += Ke
    return K


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("seed,shape", [(1, (1, 1, 1)), (2, (2, 3, 2)), (3, (3, 2, 4))])
def test_ebe_equals_dense(orc, kind, seed, shape):
    mesh = W.random_mesh(seed, shape=shape, void_frac=0.25)
    u = W.random_displacement(mesh, seed)
    K = _dense_K(orc, kind, mesh)
    f = orc.ku(kind, mesh, u)
    assert np.abs(f - K @ u).max() <= 1e-12 * np.abs(K @ u).max()
    assert np.abs(K - K.T).max() <= 1e-12 * np.abs(K).max()


@pytest.mark.parametrize("kind", [0, 1])
def test_rigid_translation_and_rotation(orc, kind):
    mesh = W.random_mesh(7, shape=(4, 3, 5), void_frac=0.2)
    nx, ny, nz = mesh["shape"]
    h = mesh["h"]
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    x = np.stack([i.reshape(-1), j.reshape(-1), k.reshape(-1)], axis=1) * h
    ref = np.abs(orc.ku(kind, mesh, W.random_displacement(mesh, 1))).max()
    for c in range(3):
        u = np.zeros_like(x); u[:, c] = 1e-3
        assert np.abs(orc.ku(kind, mesh, u.reshape(-1))).max() <= 1e-11 * ref * 1e3
    w = np.array([0.3, -0.2, 0.5]) * 1e-3
    u = np.cross(np.broadcast_to(w, x.shape), x)
    assert np.abs(orc.ku(kind, mesh, u.reshape(-1))).max() <= 1e-9 * ref


def test_ku_nodes_matches_full(orc):
    mesh = W.random_mesh(11, shape=(5, 4, 3), void_frac=0.2)
    u = W.random_displacement(mesh, 2)
    f = orc.ku(0, mesh, u).reshape(-1, 3)
    sel = np.array([0, 7, 19, 33, len(f) - 1])
    fs = orc.ku_nodes(0, mesh, u, sel)
    assert np.allclose(fs, f[sel], rtol=0, atol=1e-12 * np.abs(f).max())


def test_ku_tc_matches_fp64(orc):
    mesh = W.random_mesh(12, shape=(4, 4, 4), void_frac=0.1)
    u = W.random_displacement(mesh, 3)
    f64 = orc.ku(0, mesh, u)
    f8 = orc.ku(0, mesh, u, tc_stages=8)
    f4 = orc.ku(0, mesh, u, tc_stages=4)
    s = np.abs(f64).max()
    assert np.abs(f8 - f64).max() <= 1e-13 * s
    assert 1e-12 * s < np.abs(f4 - f64).max() <= 1e-6 * s


def test_node_mass_total(orc):
    mesh = W.random_mesh(13, shape=(3, 5, 2), void_frac=0.3)
    m = orc.node_mass(0, mesh)
    tab = mesh["material_table"]
    ids = mesh["material_ids"]
    total = sum(tab[i][2] for i in ids if i >= 0) * mesh["h"] ** 3
    assert m.sum() == pytest.approx(total, rel=1e-13)
    assert (m >= 0).all()
