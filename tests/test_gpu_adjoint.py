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
