"""Steps driven by a caller-supplied force series at the source node
(vfe_step_forced), the form in which Section 3's experiment prescribes its
point force: against the device-evaluated wavelet and against the oracle."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import PATHS, TRACE_TOL, rel_l2

pytestmark = pytest.mark.gpu


def ricker_rows(n, dt, f0, t0, amp, direction):
    """F^k = amp (1 - 2 a) exp(-a) dir, a = pi^2 f0^2 (k dt - t0)^2 (the wavelet
    of vfe_set_source), computed on the host."""
    t = np.arange(n) * dt
    a = (np.pi * f0 * (t - t0)) ** 2
    return amp * ((1.0 - 2.0 * a) * np.exp(-a))[:, None] * np.asarray(direction)[None, :]


def _mesh():
    return W.random_mesh(12, shape=(20, 18, 10), void_frac=0.05)


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_forced_rows_reproduce_the_wavelet_run(path):
    mesh = _mesh()
    s = mesh["source"]
    n, n1 = 48, 17
    with vfe.Mesh(mesh, path=PATHS[path]) as m:
        m.step(n)
        ref = m.traces()
        rows = ricker_rows(n, m.dt, s["f0"], s["t0"], s["amp"], s["dir"])
    with vfe.Mesh(mesh, path=PATHS[path]) as m:   # two forced calls
        m.step_forced(rows[:n1])
        m.step_forced(rows[n1:])
        tr2 = m.traces()
    with vfe.Mesh(mesh, path=PATHS[path]) as m:   # forced, then the wavelet again
        m.step_forced(rows[:n1])
        m.step(n - n1)
        tr3 = m.traces()
    assert rel_l2(tr2, ref) <= 1e-12
    assert rel_l2(tr3, ref) <= 1e-12


@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_forced_rows_match_oracle(orc, path):
    """A different wavelet (amplitude, direction, frequency and delay) given as
    rows: the oracle runs the same force through its own wavelet."""
    mesh = _mesh()
    s = mesh["source"]
    f0, t0, amp = 1.3 * s["f0"], 0.9 * s["t0"], 2.5
    direction = (0.6, 0.0, 0.8)
    n = 40
    dt = orc.dt(0, mesh, 0.5)
    src = {"node": W.source_node(mesh), "dir": direction, "f0": f0, "t0": t0, "amp": amp}
    ref = orc.run(0, mesh, dt, n, source=src, receivers=W.receiver_nodes(mesh))
    with vfe.Mesh(mesh, path=PATHS[path]) as m:
        m.step_forced(ricker_rows(n, m.dt, f0, t0, amp, direction))
        tr = m.traces()
    assert rel_l2(tr, ref) <= TRACE_TOL[path]


def test_forced_rejects_bad_calls():
    mesh = _mesh()
    with vfe.Mesh(mesh, source=False) as m:
        with pytest.raises(vfe.VfeError) as e:
            m.step_forced(np.zeros((3, 3)))
        assert e.value.code == vfe.VFE_ESTATE
    with vfe.Mesh(mesh) as m:
        bad = np.zeros((4, 3))
        bad[2, 1] = np.nan
        with pytest.raises(vfe.VfeError) as e:
            m.step_forced(bad)
        assert e.value.code == vfe.VFE_EINVAL
        m.step_forced(np.zeros((0, 3)))   # no steps: a no-op
        m.synchronize()
        for bad_dir, f0 in (((np.nan, 0.0, 1.0), 5.0), ((0.0, np.inf, 1.0), 5.0),
                            ((0.0, 0.0, 1.0), 0.0), ((0.0, 0.0, 1.0), np.inf)):
            with pytest.raises(vfe.VfeError) as e:
                vfe.vfe_set_source(m.handle, 1, 1, 1, bad_dir, f0, 0.0, 1.0)
            assert e.value.code == vfe.VFE_EINVAL


def test_streamed_rows_equal_traces():
    """vfe_get_trace_rows_async: each step's receiver row copied to page-locked
    host memory behind the step, without waiting, equals the recorded traces
    once the mesh is synchronised; the same checks on the row range as the
    synchronous read."""
    torch = pytest.importorskip("torch")
    mesh = _mesh()
    n = 30
    with vfe.Mesh(mesh) as m:
        out = torch.zeros((n, m.n_rec, 3), dtype=torch.float64, pin_memory=True).numpy()
        s = mesh["source"]
        rows = ricker_rows(n, m.dt, s["f0"], s["t0"], s["amp"], s["dir"])
        for k in range(n):
            if k % 2:
                m.step(1)
            else:
                m.step_forced(rows[k:k + 1])
            vfe.vfe_get_trace_rows_async(m.handle, k, 1, m.n_rec, out[k])
        m.synchronize()
        assert np.abs(out).max() > 0
        assert np.array_equal(out, m.traces())
        with pytest.raises(vfe.VfeError) as e:
            vfe.vfe_get_trace_rows_async(m.handle, n, 1, m.n_rec, out[0])
        assert e.value.code == vfe.VFE_EINVAL
        with pytest.raises(ValueError):   # the host buffer is too small for two rows
            vfe.vfe_get_trace_rows_async(m.handle, 0, 2, m.n_rec, out[0])
