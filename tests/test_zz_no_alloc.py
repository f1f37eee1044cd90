"""The allocation-free K u entry point (vfe_internal_force_noalloc).

Callers that cannot allocate device memory -- a host framework that owns the
whole memory pool, a real-time loop that must not hit cudaMalloc's implicit
synchronisation -- get the tensor-core K u through this call, which keeps its
temporaries in a fixed device array declared by the library.  This file runs
last so that a failure here cannot hide the other tests, and it passes both on
its own and after them: the array keeps the previous call's contents, so two
calls in a row must each give the right answer.  The result is checked
against the FP64 oracle and against the allocating entry point.
"""
import ctypes

import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import KU_TOL, rel_max

pytestmark = pytest.mark.gpu


def _noalloc_rc(handle, u):
    lib = vfe.load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = np.full_like(u, np.nan)
    rc = lib.vfe_internal_force_noalloc(handle, u.ctypes.data_as(ctypes.c_void_p),
                                        f.ctypes.data_as(ctypes.c_void_p))
    return rc, f


def _noalloc_via_cabi(handle, u):
    rc, f = _noalloc_rc(handle, u)
    assert rc == vfe.VFE_OK, vfe.vfe_last_error()
    return f


@pytest.mark.parametrize("stencil", [1, 2])   # 2: per-node corrections in the stencil kernel
@pytest.mark.parametrize("shape", [(17, 16, 6), (33, 31, 9)])
def test_noalloc_matches_oracle_and_internal_force_twice(orc, shape, stencil):
    mesh = W.random_mesh(300 + sum(shape), shape=shape, void_frac=0.1)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False,
                  stencil=stencil) as m:
        for seed, scale in ((1, 1e-3), (2, 7e-9)):
            u = W.random_displacement(mesh, seed, scale=scale)
            want = orc.ku(0, mesh, u)
            got = _noalloc_via_cabi(m.handle, u)
            assert rel_max(got, want) <= KU_TOL
            assert rel_max(got, m.internal_force(u)) <= KU_TOL


def test_noalloc_rejects_non_finite_input():
    mesh = W.random_mesh(311, shape=(9, 8, 5), void_frac=0.0)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False) as m:
        for bad in (np.nan, np.inf, -np.inf):
            u = W.random_displacement(mesh, 3)
            u[17] = bad
            rc, _ = _noalloc_rc(m.handle, u)
            assert rc == vfe.VFE_EINVAL
            assert "non-finite" in vfe.vfe_last_error()
        # the array keeps working after a rejected call
        u = W.random_displacement(mesh, 4)
        assert rel_max(_noalloc_via_cabi(m.handle, u), m.internal_force(u)) <= KU_TOL


def test_noalloc_reports_the_kernel_status_word():
    """A status bit set on the device (here injected from the host, as a
    kernel sets it when a bounded wait gives up) makes the call fail instead
    of returning an unwritten f."""
    mesh = W.random_mesh(312, shape=(9, 8, 5), void_frac=0.0)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False) as m:
        assert vfe.load().vfe_debug_inject_status(m.handle, 1) == vfe.VFE_OK
        rc, _ = _noalloc_rc(m.handle, W.random_displacement(mesh, 5))
        assert rc == vfe.VFE_ETIMEOUT, vfe.vfe_last_error()
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False) as m:
        assert vfe.load().vfe_debug_inject_status(m.handle, 4) == vfe.VFE_OK
        rc, _ = _noalloc_rc(m.handle, W.random_displacement(mesh, 5))
        assert rc == vfe.VFE_ECUDA, vfe.vfe_last_error()


def test_noalloc_keeps_the_callers_current_device():
    import torch
    mesh = W.random_mesh(313, shape=(6, 5, 4), void_frac=0.0)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False) as m:
        before = torch.cuda.current_device()
        _noalloc_via_cabi(m.handle, W.random_displacement(mesh, 6))
        assert torch.cuda.current_device() == before


def test_noalloc_rejects_oversized_mesh():
    mesh = W.config2()
    mesh = dict(mesh, shape=(160, 160, 64),
                material_ids=np.zeros(160 * 160 * 64, dtype=np.int32))
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False) as m:
        u = np.zeros(3 * 161 * 161 * 65)
        rc, _ = _noalloc_rc(m.handle, u)
        assert rc == vfe.VFE_EINVAL
        assert "no-alloc scratch" in vfe.vfe_last_error()
