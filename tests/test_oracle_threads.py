"""The oracle's multi-threaded loops (eight colours of element parity) against
its one-thread loops: the same sums in another order, so they agree to
rounding, and the colour order makes the result independent of the thread
count."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import oracle_source


@pytest.fixture
def threads(orc):
    yield orc
    orc.set_threads(1)


@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 1), (7, 5, 6), (16, 9, 11), (33, 2, 4)])
def test_coloured_ku_matches_sequential(threads, shape):
    orc = threads
    mesh = W.random_mesh(40 + sum(shape), shape=shape, void_frac=0.2)
    u = W.random_displacement(mesh, 3)
    orc.set_threads(1)
    f1 = orc.ku(0, mesh, u)
    if orc.set_threads(4) == 1:
        pytest.skip("oracle built without OpenMP")
    f4 = orc.ku(0, mesh, u)
    orc.set_threads(3)
    f3 = orc.ku(0, mesh, u)
    # at most eight contributions per node added in another order
    assert np.abs(f4 - f1).max() <= 8 * np.finfo(float).eps * np.abs(f1).max()
    assert np.array_equal(f3, f4)
    # the TC integer expansion goes through the same colour loop
    orc.set_threads(1)
    g1 = orc.ku(0, mesh, u, tc_stages=8)
    orc.set_threads(4)
    g4 = orc.ku(0, mesh, u, tc_stages=8)
    assert np.abs(g4 - g1).max() <= 8 * np.finfo(float).eps * np.abs(g1).max()


def test_threaded_run_matches_sequential(threads):
    orc = threads
    mesh = W.random_mesh(77, shape=(11, 9, 7), void_frac=0.1)
    dt = orc.dt(0, mesh, 0.5)
    src, rec = oracle_source(mesh), W.receiver_nodes(mesh)
    orc.set_threads(1)
    t1, u1, _ = orc.run(0, mesh, dt, 60, source=src, receivers=rec, return_state=True)
    if orc.set_threads(4) == 1:
        pytest.skip("oracle built without OpenMP")
    t4, u4, _ = orc.run(0, mesh, dt, 60, source=src, receivers=rec, return_state=True)
    assert np.linalg.norm(t4 - t1) <= 1e-13 * np.linalg.norm(t1)
    assert np.abs(u4 - u1).max() <= 1e-13 * np.abs(u1).max()
