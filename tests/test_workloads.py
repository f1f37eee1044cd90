"""The seeded synthetic workloads match their stated recipes: sizes, layer
boundaries, material ranges, void fraction, sources, receivers and lengths.
They stand in for the paper's rebar model (Section 3), whose data and
constants are not published."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import workloads as W


def _vs_vp_rho(w):
    t = np.asarray(w["material_table"])
    return t[:, 1], t[:, 0], t[:, 2]


def _mat3(w):
    nx, ny, nz = w["shape"]
    return np.asarray(w["material_ids"]).reshape(nz, ny, nx)


def test_config1():
    w = W.config1()
    assert w["shape"] == (32, 32, 32) and w["h"] == 1.0 and w["nsteps"] == 300
    m = _mat3(w)
    assert (m[20:] == 0).all() and (m[:20] == 1).all()          # soft top 12 cells
    assert w["material_table"].tolist() == [[700.0, 200.0, 1800.0], [2000.0, 800.0, 2100.0]]
    assert w["source"]["ijk"] == (16, 16, 16) and w["source"]["f0"] == 10.0
    assert len(w["receivers"]) == 16 and (w["receivers"][:, 2] == 32).all()


def test_config2():
    w = W.config2()
    assert w["shape"] == (128, 128, 64) and w["nsteps"] == 2000
    assert w["material_ids"].size == 1048576
    vs, vp, rho = _vs_vp_rho(w)
    assert len(vs) == 23                                          # 3 layers + 20 ellipsoids
    assert ((vs[3:] >= 150) & (vs[3:] <= 1200)).all()
    assert ((vp[3:] / vs[3:] >= 2.0) & (vp[3:] / vs[3:] <= 3.0)).all()
    assert ((rho[3:] >= 1600) & (rho[3:] <= 2300)).all()
    m = _mat3(w)
    layered = np.where(np.arange(64) >= 48, 0, np.where(np.arange(64) >= 32, 1, 2))
    outside = m < 3                                               # cells no ellipsoid covers
    assert (m[outside] == np.broadcast_to(layered[:, None, None], m.shape)[outside]).all()
    assert 0.02 < (m >= 3).mean() < 0.5
    assert w["source"]["ijk"] == (64, 64, 32) and w["source"]["f0"] == 5.0
    assert len(w["receivers"]) == 64 and (w["receivers"][:, 2] == 64).all()


def test_config3_recipe_at_reduced_size():
    nx, ny, nz = 128, 128, 64
    w = W.config3(shape=(nx, ny, nz))
    vs, vp, rho = _vs_vp_rho(w)
    assert len(vs) == 10
    assert vs[0] == pytest.approx(200.0) and vs[-1] == pytest.approx(2000.0)
    assert np.allclose(vp, 2.2 * vs)
    m = _mat3(w)
    void = m < 0
    # void only above the surface: along k every column is solid then void
    assert (np.diff(void.astype(np.int8), axis=0) >= 0).all()
    assert 0.05 < void.mean() < 0.2
    # the layers dip: along x at a fixed depth below the top the layer index changes
    assert len(np.unique(m[nz // 4, ny // 2][m[nz // 4, ny // 2] >= 0])) > 1
    # every receiver sits on a node touching a solid element
    for i, j, k in w["receivers"]:
        below = m[k - 1, max(j - 1, 0):j + 1, max(i - 1, 0):i + 1]
        assert (below >= 0).any()
    assert w["nsteps"] == 5000


def test_config4():
    models = W.config4()
    assert len(models) == 64
    for w in models:
        n = w["shape"][0]
        assert w["shape"] == (n, n, n) and 32 <= n <= 128
        vs, vp, rho = _vs_vp_rho(w)
        assert len(vs) == 3 and np.allclose(vp, 2.5 * vs)
        assert ((vs >= 200) & (vs <= 1000)).all()
        assert 3.0 <= w["source"]["f0"] <= 10.0 and w["nsteps"] == 1000
    assert len({w["shape"][0] for w in models}) > 10              # uneven sizes


def test_config5_anomaly():
    obs, bg = W.config5(anomaly=True), W.config5(anomaly=False)
    n = 96
    assert obs["shape"] == bg["shape"] == (n, n, n) and obs["nsteps"] == 1500
    vs, _, _ = _vs_vp_rho(obs)
    assert vs[2] == pytest.approx(0.7 * vs[1])                    # the anomaly: Vs -30 %
    mo, mb = _mat3(obs), _mat3(bg)
    assert not (mb == 2).any()
    sphere = mo == 2
    r = n / 8.0                                                   # radius 12 cells
    kk, jj, ii = np.nonzero(sphere)
    d = np.sqrt((ii + 0.5 - n / 2) ** 2 + (jj + 0.5 - n / 2) ** 2 + (kk + 0.5 - n / 2) ** 2)
    assert d.max() <= r and sphere.sum() == pytest.approx(4.0 / 3.0 * np.pi * r ** 3, rel=0.05)
    assert (mo[~sphere] == mb[~sphere]).all()
    assert len(obs["receivers"]) == 36 and (obs["receivers"][:, 2] == n).all()


def test_paper_rebar_geometry():
    w = W.paper_rebar()
    ds = w["h"]
    assert ds == 2e-3 and w["dt"] == 5e-8 and w["nsteps"] == 16384 and w["fix_bottom"] == 2
    m = _mat3(w)
    nz, ny, nx = m.shape
    kk, ii = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    r = np.hypot((ii + 0.5) * ds - 0.160, (kk + 0.5) * ds - 0.100)
    steel = (m == 1).all(axis=1)                                  # the bar runs along y
    assert ((m == 1) == (m == 1)[:, :1, :]).all()
    assert (steel == (r <= 0.015)).all()
    vs, vp, rho = _vs_vp_rho(w)
    assert (vp[1], vs[1], rho[1]) == (5900.0, 3200.0, 7850.0)
    assert 100e3 <= w["source"]["f0"] <= 125e3
