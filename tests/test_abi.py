"""CPU checks of the C-ABI library: it builds, loads, exports every entry point
declared in include/vfe.h, and rejects bad arguments before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "vfe.h")).read()
    return sorted(set(re.findall(r"\b(vfe_[a-z_]+)\s*\(", text)))


def test_header_matches_binding():
    assert set(_declared()) == set(vfe.EXPORTS)


def test_library_exports_every_declared_symbol():
    lib = vfe.load()
    for name in _declared():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_default_options():
    o = vfe.vfe_default_options()
    assert (o.element_kind, o.path, o.stages, o.fix_bottom) == (vfe.VFE_OVFEM, vfe.VFE_PATH_TC, 5, 1)
    assert o.cfl_fraction == 0.5 and o.dt == 0.0


@pytest.mark.parametrize("kw,msg", [
    (dict(nx=0), "grid"),
    (dict(h=-1.0), "h must"),
    (dict(table=[[100.0, 90.0, 2000.0]]), "material 0"),
    (dict(table=[[1000.0, 500.0, 0.0]]), "material 0"),
    (dict(ids_fill=5), "out of range"),
    (dict(ids_fill=-1), "no solid"),
    (dict(opt=dict(path=vfe.VFE_PATH_TC, element_kind=vfe.VFE_VFEM)), "orthogonal"),
    (dict(opt=dict(stages=6)), "stages"),
    (dict(opt=dict(stages=0)), "stages"),
    (dict(opt=dict(cfl_fraction=1.5)), "cfl"),
    (dict(opt=dict(dt=1.0)), "stability limit"),
])
def test_create_mesh_validation(kw, msg):
    nx = kw.get("nx", 2)
    ids = np.full(nx * 2 * 2, kw.get("ids_fill", 0), dtype=np.int32)
    table = kw.get("table", [[1000.0, 500.0, 2000.0]])
    opt = vfe.vfe_default_options(**kw.get("opt", {}))
    with pytest.raises(vfe.VfeError) as ei:
        vfe.vfe_create_mesh(nx, 2, 2, kw.get("h", 1.0), ids, table, opt)
    assert ei.value.code == vfe.VFE_EINVAL
    assert msg in str(ei.value)


def test_null_mesh_rejected():
    lib = vfe.load()
    assert lib.vfe_step(None, 1) == vfe.VFE_EINVAL
    assert lib.vfe_destroy(None) == vfe.VFE_OK
    assert "NULL" in vfe.vfe_last_error()


def test_workload_generators_are_seeded():
    a, b = W.config2(), W.config2()
    assert np.array_equal(a["material_ids"], b["material_ids"])
    assert a["material_ids"].size == 128 * 128 * 64
    assert len(a["material_table"]) == 23 and len(a["receivers"]) == 64
    c = W.config1()
    assert c["material_ids"].size == 32 ** 3 and len(c["receivers"]) == 16
    r1, r2 = W.random_mesh(4), W.random_mesh(4)
    assert np.array_equal(r1["material_ids"], r2["material_ids"])
    assert (r1["material_ids"] >= -1).all()


def test_every_entry_point_rejects_null_handles():
    """Every call that takes a mesh or batch rejects NULL with VFE_EINVAL and a
    message, before touching the GPU (destroy calls accept NULL)."""
    import ctypes
    lib = vfe.load()
    d, i64, i32 = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int()
    buf = np.zeros(64)
    p = buf.ctypes.data_as(ctypes.c_void_p)
    calls = {
        "vfe_set_source": lambda: lib.vfe_set_source(None, 0, 0, 0, p, 1.0, 0.0, 1.0),
        "vfe_set_receivers": lambda: lib.vfe_set_receivers(None, 0, None),
        "vfe_internal_force": lambda: lib.vfe_internal_force(None, p, p),
        "vfe_internal_force_noalloc": lambda: lib.vfe_internal_force_noalloc(None, p, p),
        "vfe_step": lambda: lib.vfe_step(None, 1),
        "vfe_step_forced": lambda: lib.vfe_step_forced(None, 1, p),
        "vfe_set_damping": lambda: lib.vfe_set_damping(None, 0.0, 0.0),
        "vfe_synchronize": lambda: lib.vfe_synchronize(None),
        "vfe_get_traces": lambda: lib.vfe_get_traces(None, p, ctypes.byref(i64)),
        "vfe_get_trace_rows": lambda: lib.vfe_get_trace_rows(None, 0, 1, p),
        "vfe_get_trace_rows_async": lambda: lib.vfe_get_trace_rows_async(None, 0, 1, p),
        "vfe_get_dt": lambda: lib.vfe_get_dt(None, ctypes.byref(d)),
        "vfe_get_sizes": lambda: lib.vfe_get_sizes(None, ctypes.byref(i64), ctypes.byref(i64)),
        "vfe_get_step_count": lambda: lib.vfe_get_step_count(None, ctypes.byref(i64)),
        "vfe_get_state": lambda: lib.vfe_get_state(None, p, p),
        "vfe_set_state": lambda: lib.vfe_set_state(None, p, p),
        "vfe_debug_tc_partials": lambda: lib.vfe_debug_tc_partials(
            None, p, 1, p, p, ctypes.byref(i32), ctypes.byref(i32)),
        "vfe_misfit_gradient": lambda: lib.vfe_misfit_gradient(None, 1, p, 1, p, ctypes.byref(d)),
        "vfe_batch_step": lambda: lib.vfe_batch_step(None, 1),
        "vfe_batch_synchronize": lambda: lib.vfe_batch_synchronize(None),
        "vfe_create_batch": lambda: lib.vfe_create_batch(1, None, None),
    }
    for name, call in calls.items():
        assert call() == vfe.VFE_EINVAL, name
        assert vfe.vfe_last_error(), name
    assert lib.vfe_destroy(None) == vfe.VFE_OK
    assert lib.vfe_destroy_batch(None) == vfe.VFE_OK
