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
