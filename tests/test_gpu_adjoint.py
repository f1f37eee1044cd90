"""GPU adjoint-state gradient (vfe_misfit_gradient) against the FP64 CPU
adjoint of the oracle and against central finite differences, plus the
torch.autograd wrapper."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import adjoint, vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import PATHS

pytestmark = pytest.mark.gpu


def small_problem(n=12, nsteps=80):
    obs = W.config5(anomaly=True, n=n, nsteps=nsteps)
    bg = W.config5(anomaly=False, n=n, nsteps=nsteps)
    return obs, bg


def _oracle_data(orc, w, dt, n):
    s = w["source"]
    src = {"node": W.source_node(w), "dir": s["dir"], "f0": s["f0"], "t0": s["t0"], "amp": s["amp"]}
    return orc.run(0, w, dt, n, source=src, receivers=W.receiver_nodes(w)), src


@pytest.mark.parametrize("path,tol", [("fp64", 1e-10), ("tc", 1e-6)])
@pytest.mark.parametrize("checkpoint", [7, 100])
def test_gradient_matches_oracle_adjoint(orc, path, tol, checkpoint):
    obs, bg = small_problem()
    n = bg["nsteps"]
    dt = orc.dt(0, obs, 0.5)
    data, src = _oracle_data(orc, obs, dt, n)
    g_ref, J_ref = orc.misfit_gradient(0, bg, dt, n, src, W.receiver_nodes(bg), data)
    with vfe.Mesh(bg, path=PATHS[path], dt=dt) as m:
        g, J = vfe.vfe_misfit_gradient(m.handle, data, checkpoint)
    assert J == pytest.approx(J_ref, rel=tol)
    assert np.abs(g - g_ref).max() <= tol * np.abs(g_ref).max()


def test_gradient_with_node_corrections_matches_oracle_adjoint(orc):
    """The TC gradient with every column-plane but the source and receiver
    planes in the stencil kernel (stencil=2: per-node material, the layer
    interface and face nodes corrected), forward and adjoint runs."""
    obs, bg = small_problem(n=16, nsteps=60)
    n = bg["nsteps"]
    dt = orc.dt(0, obs, 0.5)
    data, src = _oracle_data(orc, obs, dt, n)
    g_ref, J_ref = orc.misfit_gradient(0, bg, dt, n, src, W.receiver_nodes(bg), data)
    with vfe.Mesh(bg, path=vfe.VFE_PATH_TC, dt=dt, stencil=2) as m:
        g, J = vfe.vfe_misfit_gradient(m.handle, data, 20)
    assert J == pytest.approx(J_ref, rel=1e-6)
    assert np.abs(g - g_ref).max() <= 1e-6 * np.abs(g_ref).max()


def test_gradient_matches_finite_differences():
    obs, bg = small_problem(n=12, nsteps=60)
    with vfe.Mesh(obs, path=vfe.VFE_PATH_FP64) as m:
        dt = m.dt
        m.step(bg["nsteps"])
        data = m.traces()
    with vfe.Mesh(bg, path=vfe.VFE_PATH_FP64, dt=dt) as m:
        g, J = vfe.vfe_misfit_gradient(m.handle, data, 20)
    rng = np.random.default_rng(5)
    ne = bg["material_ids"].size
    for e in rng.choice(ne, 20, replace=False):
        tab = bg["material_table"]
        mm = int(bg["material_ids"][e])
        vp, vs, rho = tab[mm]
        G = rho * vs * vs
        js = []
        for sgn in (1.0, -1.0):
            w = dict(bg, material_ids=bg["material_ids"].copy())
            G2 = G * (1 + sgn * 1e-4)
            kap = rho * (vp * vp - 4.0 / 3.0 * vs * vs)
            w["material_table"] = np.vstack([tab, [np.sqrt((kap + 4 / 3 * G2) / rho),
                                                   np.sqrt(G2 / rho), rho]])
            w["material_ids"][e] = len(tab)
            with vfe.Mesh(w, path=vfe.VFE_PATH_FP64, dt=dt) as mp:
                mp.step(bg["nsteps"])
                js.append(0.5 * float(np.sum((mp.traces() - data) ** 2)))
        fd = (js[0] - js[1]) / (2e-4 * G)
        assert abs(fd - g[e]) <= 1e-5 * np.abs(g).max(), (e, fd, g[e])


def test_autograd_function():
    torch = pytest.importorskip("torch")
    obs, bg = small_problem(n=12, nsteps=40)
    with vfe.Mesh(obs, path=vfe.VFE_PATH_TC) as m:
        dt = m.dt
        m.step(bg["nsteps"])
        data = m.traces()
    G = torch.tensor(adjoint.shear_moduli(bg), dtype=torch.float64, requires_grad=True)
    J = adjoint.ShearModulusMisfit.apply(G, bg, data, vfe.VFE_PATH_TC, 10, dt)
    J.backward()
    _, g_e, g_m = adjoint.misfit_and_gradient(bg, data, vfe.VFE_PATH_TC, 10, dt)
    assert np.allclose(G.grad.numpy(), g_m, rtol=1e-12, atol=0)
    assert J.item() > 0 and np.isfinite(G.grad.numpy()).all()


def per_element_workload(w, G):
    """The model with one material per solid element, shear modulus G[e] at
    its material's bulk modulus and density: the oracle's form of
    per-element moduli (it takes any number of materials)."""
    tab = np.asarray(w["material_table"], dtype=np.float64)
    mat = np.asarray(w["material_ids"])
    vp, vs, rho = tab[:, 0], tab[:, 1], tab[:, 2]
    kap = rho * (vp * vp - 4.0 / 3.0 * vs * vs)
    solid = mat >= 0
    r, k, g = rho[mat[solid]], kap[mat[solid]], np.asarray(G)[solid]
    new_tab = np.stack([np.sqrt((k + 4.0 / 3.0 * g) / r), np.sqrt(g / r), r], axis=1)
    new_mat = -np.ones_like(mat)
    new_mat[solid] = np.arange(int(solid.sum()))
    return dict(w, material_ids=new_mat.astype(np.int32), material_table=new_tab)


def _random_element_G(w, seed):
    tab = np.asarray(w["material_table"])
    mat = np.asarray(w["material_ids"])
    G = tab[:, 2] * tab[:, 1] ** 2
    rng = np.random.default_rng(seed)
    return G[np.maximum(mat, 0)] * rng.uniform(0.7, 1.3, size=mat.size)


@pytest.mark.parametrize("path,tol", [("fp64", 1e-12), ("tc", 1e-9)])
def test_per_element_moduli_forward(orc, path, tol):
    _, bg = small_problem(n=12, nsteps=60)
    G = _random_element_G(bg, 1)
    pe = per_element_workload(bg, G)
    dt = orc.dt(0, bg, 0.5)
    ref, src = _oracle_data(orc, pe, dt, bg["nsteps"])
    with vfe.Mesh(bg, path=PATHS[path], dt=dt) as m:
        vfe.vfe_set_shear_moduli(m.handle, G)
        m.step(bg["nsteps"])
        tr = m.traces()
        vfe.vfe_set_shear_moduli(m.handle, None)   # back to the materials' moduli
    assert np.linalg.norm(tr - ref) <= tol * np.linalg.norm(ref)


@pytest.mark.parametrize("path,tol", [("fp64", 1e-10), ("tc", 1e-6)])
def test_per_element_gradient_matches_oracle_adjoint(orc, path, tol):
    obs, bg = small_problem(n=12, nsteps=50)
    dt = orc.dt(0, obs, 0.5)
    data, src = _oracle_data(orc, obs, dt, bg["nsteps"])
    G = _random_element_G(bg, 2)
    pe = per_element_workload(bg, G)
    g_ref, J_ref = orc.misfit_gradient(0, pe, dt, bg["nsteps"], src, W.receiver_nodes(bg), data)
    J, g_e, _ = adjoint.misfit_and_gradient(bg, data, PATHS[path], 10, dt, element_G=G)
    assert J == pytest.approx(J_ref, rel=tol)
    assert np.abs(g_e - g_ref).max() <= tol * np.abs(g_ref).max()


@pytest.mark.parametrize("path", ["fp64", "tc"])
def test_element_autograd_matches_finite_differences(path):
    """ElementShearMisfit through torch.autograd: G.grad against central
    finite differences of the function's own forward on 20 elements."""
    torch = pytest.importorskip("torch")
    obs, bg = small_problem(n=12, nsteps=40)
    with vfe.Mesh(obs, path=vfe.VFE_PATH_FP64) as m:
        dt = m.dt
        m.step(bg["nsteps"])
        data = m.traces()
    G0 = _random_element_G(bg, 3)
    G = torch.tensor(G0, dtype=torch.float64, requires_grad=True)
    J = adjoint.ElementShearMisfit.apply(G, bg, data, dt, PATHS[path], 10)
    J.backward()
    g = G.grad.numpy()
    assert np.isfinite(g).all() and J.item() > 0
    rng = np.random.default_rng(6)
    solid = np.flatnonzero(np.asarray(bg["material_ids"]) >= 0)
    for e in rng.choice(solid, 20, replace=False):
        h = 1e-4 * G0[e]
        js = []
        for sgn in (1.0, -1.0):
            Gp = torch.tensor(G0, dtype=torch.float64)
            Gp[e] += sgn * h
            js.append(float(adjoint.ElementShearMisfit.apply(Gp, bg, data, dt, PATHS[path], 10)))
        fd = (js[0] - js[1]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-5 * np.abs(g).max(), (e, fd, g[e])


def test_misfit_needs_a_time_step():
    _, bg = small_problem(n=8, nsteps=4)
    with pytest.raises(ValueError):
        adjoint.misfit_and_gradient(bg, np.zeros((4, 36, 3)), dt=None)
