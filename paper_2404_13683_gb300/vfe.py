"""Thin Python binding of the C ABI in ``include/vfe.h``.

Functions keep the C names and only marshal arguments (numpy arrays in,
numpy arrays out).  Every step of the solver runs in the CUDA library
``libvfe.so``; if that library cannot be loaded this module raises instead of
falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

VFE_OK = 0
VFE_EINVAL = -1
VFE_ENOMEM = -2
VFE_ECUDA = -3
VFE_ETIMEOUT = -4
VFE_ESTATE = -5

VFE_OVFEM = 0
VFE_VFEM = 1
VFE_PATH_FP64 = 0
VFE_PATH_TC = 1

# every entry point declared in include/vfe.h
EXPORTS = (
    "vfe_default_options", "vfe_create_mesh", "vfe_destroy", "vfe_set_source",
    "vfe_set_receivers", "vfe_internal_force", "vfe_step", "vfe_synchronize",
    "vfe_get_traces", "vfe_get_dt", "vfe_get_sizes", "vfe_get_step_count",
    "vfe_get_launches_per_step",
    "vfe_get_state", "vfe_set_state", "vfe_last_error", "vfe_debug_tc_partials",
    "vfe_get_trace_rows", "vfe_internal_force_noalloc",
    "vfe_create_batch", "vfe_batch_step", "vfe_batch_synchronize", "vfe_destroy_batch",
    "vfe_misfit_gradient", "vfe_step_forced", "vfe_set_damping", "vfe_rayleigh_coefficients",
    "vfe_get_trace_rows_async", "vfe_debug_inject_status", "vfe_debug_stencil_partials",
    "vfe_plane_values", "vfe_pack_plane", "vfe_unpack_plane", "vfe_get_scale_bound",
    "vfe_set_scale_bound", "vfe_get_source_scale", "vfe_set_source_bound",
    "vfe_set_shear_moduli",
)


class VfeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("vfe error %d: %s" % (code, msg))
        self.code = code


class vfe_options(ctypes.Structure):
    _fields_ = [("element_kind", ctypes.c_int), ("path", ctypes.c_int), ("stages", ctypes.c_int),
                ("fix_bottom", ctypes.c_int), ("dt", ctypes.c_double),
                ("cfl_fraction", ctypes.c_double), ("device", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("stencil", ctypes.c_int), ("ctas", ctypes.c_int)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build: bool = True) -> ctypes.CDLL:
    """Load ``libvfe.so`` (building it with nvcc first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if build:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError("libvfe.so is missing; run paper_2404_13683_gb300.build.build()")
    L = ctypes.CDLL(_build.LIB)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    L.vfe_default_options.argtypes = [ctypes.POINTER(vfe_options)]
    L.vfe_default_options.restype = None
    L.vfe_create_mesh.argtypes = [I, I, I, D, P, P, I, ctypes.POINTER(vfe_options),
                                  ctypes.POINTER(ctypes.c_void_p)]
    L.vfe_destroy.argtypes = [P]
    L.vfe_set_source.argtypes = [P, I, I, I, P, D, D, D]
    L.vfe_set_receivers.argtypes = [P, I, P]
    L.vfe_internal_force.argtypes = [P, P, P]
    L.vfe_internal_force_noalloc.argtypes = [P, P, P]
    L.vfe_create_batch.argtypes = [I, P, ctypes.POINTER(ctypes.c_void_p)]
    L.vfe_misfit_gradient.argtypes = [P, I, P, I, P, ctypes.POINTER(D)]
    L.vfe_batch_step.argtypes = [P, I]
    L.vfe_batch_synchronize.argtypes = [P]
    L.vfe_destroy_batch.argtypes = [P]
    L.vfe_step.argtypes = [P, I]
    L.vfe_step_forced.argtypes = [P, I, P]
    L.vfe_set_damping.argtypes = [P, D, D]
    L.vfe_rayleigh_coefficients.argtypes = [D, D, D, ctypes.POINTER(D), ctypes.POINTER(D)]
    L.vfe_synchronize.argtypes = [P]
    L.vfe_get_traces.argtypes = [P, P, ctypes.POINTER(I64)]
    L.vfe_get_trace_rows.argtypes = [P, I64, I64, P]
    L.vfe_get_trace_rows_async.argtypes = [P, I64, I64, P]
    L.vfe_get_dt.argtypes = [P, ctypes.POINTER(D)]
    L.vfe_get_sizes.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I64)]
    L.vfe_get_step_count.argtypes = [P, ctypes.POINTER(I64)]
    L.vfe_get_launches_per_step.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
    L.vfe_get_state.argtypes = [P, P, P]
    L.vfe_set_state.argtypes = [P, P, P]
    L.vfe_last_error.argtypes = []
    L.vfe_last_error.restype = ctypes.c_char_p
    L.vfe_debug_tc_partials.argtypes = [P, P, I, P, P, ctypes.POINTER(I), ctypes.POINTER(I)]
    L.vfe_debug_inject_status.argtypes = [P, I]
    L.vfe_plane_values.argtypes = [P, ctypes.POINTER(I64)]
    L.vfe_pack_plane.argtypes = [P, I, P]
    L.vfe_unpack_plane.argtypes = [P, I, P]
    L.vfe_get_scale_bound.argtypes = [P, P]
    L.vfe_set_scale_bound.argtypes = [P, P]
    L.vfe_get_source_scale.argtypes = [P, ctypes.POINTER(D)]
    L.vfe_set_source_bound.argtypes = [P, P, D, D, D, D]
    L.vfe_set_shear_moduli.argtypes = [P, P]
    L.vfe_debug_stencil_partials.argtypes = [P, P, P, P, ctypes.POINTER(I), ctypes.POINTER(I)]
    for name in EXPORTS:
        if name not in ("vfe_default_options", "vfe_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(rc):
    if rc != VFE_OK:
        raise VfeError(rc, load().vfe_last_error().decode(errors="replace"))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def vfe_last_error() -> str:
    return load().vfe_last_error().decode(errors="replace")


def vfe_default_options(**kw) -> vfe_options:
    o = vfe_options()
    load().vfe_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def vfe_create_mesh(nx, ny, nz, h, material_ids, material_table, opt=None):
    ids = np.ascontiguousarray(material_ids, dtype=np.int32).reshape(-1)
    tab = np.ascontiguousarray(material_table, dtype=np.float64).reshape(-1, 3)
    if ids.size != nx * ny * nz:
        raise ValueError("material_ids must have nx*ny*nz entries")
    out = ctypes.c_void_p()
    _check(load().vfe_create_mesh(int(nx), int(ny), int(nz), float(h), _p(ids), _p(tab),
                                  len(tab), ctypes.byref(opt) if opt is not None else None,
                                  ctypes.byref(out)))
    return out


def vfe_destroy(mesh):
    _check(load().vfe_destroy(mesh))


def vfe_set_source(mesh, i, j, k, direction, f0_hz, t0_s, amp):
    d = np.ascontiguousarray(direction, dtype=np.float64)
    _check(load().vfe_set_source(mesh, int(i), int(j), int(k), _p(d), float(f0_hz), float(t0_s),
                                 float(amp)))


def vfe_set_receivers(mesh, ijk):
    a = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    _check(load().vfe_set_receivers(mesh, len(a), _p(a) if len(a) else None))


def vfe_get_sizes(mesh):
    nn, ne = ctypes.c_int64(), ctypes.c_int64()
    _check(load().vfe_get_sizes(mesh, ctypes.byref(nn), ctypes.byref(ne)))
    return nn.value, ne.value


def vfe_internal_force(mesh, u):
    nn, _ = vfe_get_sizes(mesh)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    if u.size != 3 * nn:
        raise ValueError("u must have 3*n_nodes entries")
    f = np.empty_like(u)
    _check(load().vfe_internal_force(mesh, _p(u), _p(f)))
    return f


def vfe_internal_force_noalloc(mesh, u):
    nn, _ = vfe_get_sizes(mesh)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    if u.size != 3 * nn:
        raise ValueError("u must have 3*n_nodes entries")
    f = np.empty_like(u)
    _check(load().vfe_internal_force_noalloc(mesh, _p(u), _p(f)))
    return f


def vfe_step(mesh, n):
    _check(load().vfe_step(mesh, int(n)))


def vfe_step_forced(mesh, force):
    """Advance len(force) steps with the source-node force rows ``force``
    ([n][3] FP64; a page-locked array is passed through without a copy)."""
    if isinstance(force, np.ndarray) and force.dtype == np.float64 and force.flags.c_contiguous:
        f = force
    else:
        f = np.ascontiguousarray(force, dtype=np.float64)
    f = f.reshape(-1, 3)
    _check(load().vfe_step_forced(mesh, int(f.shape[0]), f.ctypes.data_as(ctypes.c_void_p)))


def vfe_set_damping(mesh, alpha, beta):
    _check(load().vfe_set_damping(mesh, float(alpha), float(beta)))


def vfe_rayleigh_coefficients(h, f1_hz, f2_hz):
    """(alpha, beta) giving damping ratio h at f1 and f2."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().vfe_rayleigh_coefficients(float(h), float(f1_hz), float(f2_hz),
                                            ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def vfe_synchronize(mesh):
    _check(load().vfe_synchronize(mesh))


def vfe_get_traces(mesh, n_rec=None):
    rows = ctypes.c_int64()
    _check(load().vfe_get_traces(mesh, None, ctypes.byref(rows)))
    if n_rec is None:
        raise ValueError("n_rec is required")
    out = np.zeros((rows.value, n_rec, 3))
    if rows.value and n_rec:
        _check(load().vfe_get_traces(mesh, _p(out), ctypes.byref(rows)))
    return out


def vfe_get_trace_rows(mesh, first, count, n_rec, out=None):
    if out is None:
        out = np.zeros((count, n_rec, 3))
    _check(load().vfe_get_trace_rows(mesh, int(first), int(count), _p(out)))
    return out


def vfe_get_trace_rows_async(mesh, first, count, n_rec, out):
    """Queue the copy of rows [first, first+count) into ``out`` (a C-contiguous
    float64 array of at least count x n_rec x 3 values, ideally page-locked,
    kept alive and unread until the next synchronising call)."""
    if not (isinstance(out, np.ndarray) and out.dtype == np.float64 and out.flags.c_contiguous):
        raise ValueError("out must be a C-contiguous float64 array")
    if out.size < int(count) * int(n_rec) * 3:
        raise ValueError("out holds %d values, the rows need %d" % (out.size, count * n_rec * 3))
    _check(load().vfe_get_trace_rows_async(mesh, int(first), int(count),
                                           out.ctypes.data_as(ctypes.c_void_p)))
    return out


def vfe_get_dt(mesh):
    v = ctypes.c_double()
    _check(load().vfe_get_dt(mesh, ctypes.byref(v)))
    return v.value


def vfe_get_step_count(mesh):
    v = ctypes.c_int64()
    _check(load().vfe_get_step_count(mesh, ctypes.byref(v)))
    return v.value


def vfe_get_launches_per_step(mesh):
    v = ctypes.c_int()
    _check(load().vfe_get_launches_per_step(mesh, ctypes.byref(v)))
    return v.value


def vfe_get_state(mesh):
    nn, _ = vfe_get_sizes(mesh)
    u = np.zeros(3 * nn)
    up = np.zeros(3 * nn)
    _check(load().vfe_get_state(mesh, _p(u), _p(up)))
    return u, up


def vfe_set_state(mesh, u, u_prev):
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    up = np.ascontiguousarray(u_prev, dtype=np.float64).reshape(-1)
    _check(load().vfe_set_state(mesh, _p(u), _p(up)))


def vfe_debug_tc_partials(mesh, u, element_ids):
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    ids = np.ascontiguousarray(element_ids, dtype=np.int64).reshape(-1)
    out = np.zeros((len(ids), 48), dtype=np.int64)
    sh, fb = ctypes.c_int(), ctypes.c_int()
    _check(load().vfe_debug_tc_partials(mesh, _p(u), len(ids), _p(ids), _p(out),
                                        ctypes.byref(sh), ctypes.byref(fb)))
    return out, sh.value, fb.value


def vfe_misfit_gradient(mesh, data, checkpoint_every=100):
    """(dJ/dG per element, J) for a run of len(data) steps from rest."""
    data = np.ascontiguousarray(data, dtype=np.float64)
    nsteps = data.shape[0]
    _, ne = vfe_get_sizes(mesh)
    grad = np.zeros(ne)
    J = ctypes.c_double()
    _check(load().vfe_misfit_gradient(mesh, int(nsteps), _p(data), int(checkpoint_every),
                                      _p(grad), ctypes.byref(J)))
    return grad, J.value


def vfe_debug_stencil_partials(mesh, u):
    """(out [nodes][9] int64: P, S^G q, q'; covered [nodes] bool; shift; frac
    bits) of the node-stencil kernel for u."""
    nn, _ = vfe_get_sizes(mesh)
    u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
    out = np.zeros((nn, 9), dtype=np.int64)
    cov = np.zeros(nn, dtype=np.int8)
    sh, F = ctypes.c_int(), ctypes.c_int()
    _check(load().vfe_debug_stencil_partials(mesh, _p(u), _p(out), _p(cov), ctypes.byref(sh),
                                             ctypes.byref(F)))
    return out, cov.astype(bool), sh.value, F.value


def vfe_plane_values(mesh):
    n = ctypes.c_int64()
    _check(load().vfe_plane_values(mesh, ctypes.byref(n)))
    return n.value


def vfe_pack_plane(mesh, k, dev_ptr):
    """Queue the copy of u^n of node plane k to the device address dev_ptr."""
    _check(load().vfe_pack_plane(mesh, int(k), ctypes.c_void_p(int(dev_ptr))))


def vfe_unpack_plane(mesh, k, dev_ptr):
    """Queue the write of the device array at dev_ptr into u^n of plane k."""
    _check(load().vfe_unpack_plane(mesh, int(k), ctypes.c_void_p(int(dev_ptr))))


def vfe_get_scale_bound(mesh, dev_ptr):
    _check(load().vfe_get_scale_bound(mesh, ctypes.c_void_p(int(dev_ptr))))


def vfe_set_scale_bound(mesh, dev_ptr):
    _check(load().vfe_set_scale_bound(mesh, ctypes.c_void_p(int(dev_ptr))))


def vfe_get_source_scale(mesh):
    v = ctypes.c_double()
    _check(load().vfe_get_source_scale(mesh, ctypes.byref(v)))
    return v.value


def vfe_set_source_bound(mesh, direction, f0, t0, amp, dt2_over_m):
    d = np.ascontiguousarray(direction, dtype=np.float64)
    _check(load().vfe_set_source_bound(mesh, _p(d), float(f0), float(t0), float(amp),
                                       float(dt2_over_m)))


def vfe_set_shear_moduli(mesh, G):
    """Per-element shear moduli (None: the materials' own)."""
    if G is None:
        _check(load().vfe_set_shear_moduli(mesh, None))
        return
    g = np.ascontiguousarray(G, dtype=np.float64).reshape(-1)
    _, ne = vfe_get_sizes(mesh)
    if g.size != ne:
        raise ValueError("G must have one value per element")
    _check(load().vfe_set_shear_moduli(mesh, _p(g)))


def vfe_create_batch(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h
                                             for h in handles])
    out = ctypes.c_void_p()
    _check(load().vfe_create_batch(len(handles), ctypes.cast(arr, ctypes.c_void_p),
                                   ctypes.byref(out)))
    return out


def vfe_batch_step(batch, n):
    _check(load().vfe_batch_step(batch, int(n)))


def vfe_batch_synchronize(batch):
    _check(load().vfe_batch_synchronize(batch))


def vfe_destroy_batch(batch):
    _check(load().vfe_destroy_batch(batch))


class Batch:
    """Several ``Mesh`` objects advanced by one fused launch per step."""

    def __init__(self, meshes):
        self.meshes = list(meshes)
        self.handle = vfe_create_batch([m.handle for m in self.meshes])

    def step(self, n):
        vfe_batch_step(self.handle, n)

    def synchronize(self):
        vfe_batch_synchronize(self.handle)

    def close(self):
        if self.handle:
            vfe_destroy_batch(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """Owning wrapper over a ``vfe_mesh*`` built from a workload dictionary
    (see ``workloads.py``).  ``stencil``: the tensor-core path's node-stencil
    option (``vfe_options.stencil``): True or 1 (default; per-node
    corrections on meshes of 8 Mi elements or more), 2 (per-node
    corrections on any mesh), False or 0 (the element kernel everywhere)."""

    def __init__(self, workload, path=VFE_PATH_TC, kind=VFE_OVFEM, stages=5, dt=None,
                 fix_bottom=None, stream=None, device=0, source=True, receivers=True,
                 stencil=True, ctas=0):
        nx, ny, nz = workload["shape"]
        if dt is None:
            dt = float(workload.get("dt", 0.0))
        if fix_bottom is None:   # the workload's boundary condition, else the bottom plane
            fix_bottom = workload.get("fix_bottom", 1)
        opt = vfe_default_options(element_kind=kind, path=path, stages=stages, dt=dt,
                                  fix_bottom=int(fix_bottom), device=device,
                                  stream=stream or 0,
                                  stencil=int(stencil) if stencil is not True else 1,
                                  ctas=int(ctas))
        self.handle = vfe_create_mesh(nx, ny, nz, workload["h"], workload["material_ids"],
                                      workload["material_table"], opt)
        self.workload = workload
        self.n_rec = 0
        if source and workload.get("source") is not None:
            s = workload["source"]
            vfe_set_source(self.handle, *s["ijk"], s["dir"], s["f0"], s["t0"], s["amp"])
        if receivers and workload.get("receivers") is not None:
            self.set_receivers(workload["receivers"])

    def set_receivers(self, ijk):
        ijk = np.asarray(ijk, dtype=np.int32).reshape(-1, 3)
        vfe_set_receivers(self.handle, ijk)
        self.n_rec = len(ijk)

    def step(self, n):
        vfe_step(self.handle, n)

    def step_forced(self, force):
        vfe_step_forced(self.handle, force)

    def set_damping(self, alpha, beta):
        vfe_set_damping(self.handle, alpha, beta)

    def synchronize(self):
        vfe_synchronize(self.handle)

    def traces(self):
        return vfe_get_traces(self.handle, self.n_rec)

    def internal_force(self, u):
        return vfe_internal_force(self.handle, u)

    @property
    def dt(self):
        return vfe_get_dt(self.handle)

    def close(self):
        if self.handle:
            vfe_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
