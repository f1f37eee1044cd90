"""The allocation-free K u entry point (vfe_internal_force_noalloc).

Callers that cannot allocate device memory -- a host framework that owns the
whole memory pool, a real-time loop that must not hit cudaMalloc's implicit
synchronisation -- get the tensor-core K u through this call, which keeps its
temporaries in a fixed device array declared by the library.  This file runs
last so that a failure here cannot hide the other tests, and it passes both on
its own and after them: the array keeps the previous call's contents, so two
calls in a row must each give the right answer.
"""
import ctypes

import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.gpu_common import KU_TOL, rel_max

pytestmark = pytest.mark.gpu


def _noalloc_via_cabi(handle, u):
    lib = vfe.load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    f = np.empty_like(u)
    rc = lib.vfe_internal_force_noalloc(handle, u.ctypes.data_as(ctypes.c_void_p),
                                        f.ctypes.data_as(ctypes.c_void_p))
    assert rc == vfe.VFE_OK, vfe.vfe_last_error()
    return f


@pytest.mark.parametrize("shape", [(17, 16, 6), (33, 31, 9)])
def test_noalloc_matches_internal_force_twice(shape):
    mesh = W.random_mesh(300 + sum(shape), shape=shape, void_frac=0.1)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False) as m:
        for seed, scale in ((1, 1e-3), (2, 7e-9)):
            u = W.random_displacement(mesh, seed, scale=scale)
            ref = m.internal_force(u)
            got = _noalloc_via_cabi(m.handle, u)
            assert rel_max(got, ref) <= KU_TOL


def test_noalloc_rejects_oversized_mesh():
    mesh = W.config2()
    mesh = dict(mesh, shape=(160, 160, 64),
                material_ids=np.zeros(160 * 160 * 64, dtype=np.int32))
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False) as m:
        u = np.zeros(3 * 161 * 161 * 65)
        lib = vfe.load()
        f = np.empty_like(u)
        rc = lib.vfe_internal_force_noalloc(m.handle, u.ctypes.data_as(ctypes.c_void_p),
                                            f.ctypes.data_as(ctypes.c_void_p))
        assert rc == vfe.VFE_EINVAL
        assert "no-alloc scratch" in vfe.vfe_last_error()
