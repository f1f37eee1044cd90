"""Plain FP64 CPU oracle for the voxel finite-element wave step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never imports,
links or runs it, and it shares no code with the CUDA path.

The C sources (``vfe_oracle.c``) follow arXiv 2404.13683, Section 2 (VFEM,
OVFEM, TCOVFEM and the central-difference update); this module only builds the
shared library with gcc and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vfe_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OVFEM = 0
VFEM = 1
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (plain C, -O2, no architecture flags;
    OpenMP for the optional multi-threaded loops, dropped if the compiler
    lacks it)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "vfe_oracle.h"))):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        try:
            subprocess.check_call(base[:5] + ["-fopenmp"] + base[5:],
                                  stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_model() -> str:
    """The host CPU's model name (from /proc/cpuinfo; '' if unknown)."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":", 1)[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def set_threads(n: int) -> int:
    """Threads for the element loop of ``ku`` and the runs (see
    ``oracle_set_threads`` in vfe_oracle.h); returns the count in effect."""
    return int(lib().oracle_set_threads(int(n)))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, i, p, i64 = ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64
        L.oracle_element_stiffness.argtypes = [i, d, d, d, p]
        L.oracle_element_node_mass.argtypes = [i, d, d]
        L.oracle_element_node_mass.restype = d
        L.oracle_kint8.argtypes = [d, p]
        L.oracle_ku_element_tc_fp64.argtypes = [d, d, d, p, p]
        L.oracle_ku_element_tc_int.argtypes = [d, d, d, i, p, p]
        L.oracle_node_mass.argtypes = [i, i, i, i, d, p, p, i, p]
        L.oracle_ku.argtypes = [i, i, i, i, d, p, p, i, i, p, p]
        L.oracle_ku_nodes.argtypes = [i, i, i, i, d, p, p, i, p, i, p, p]
        L.oracle_element_max_eig.argtypes = [i, d, d, d, d]
        L.oracle_element_max_eig.restype = d
        L.oracle_dt.argtypes = [i, i, i, i, d, p, p, i, d]
        L.oracle_dt.restype = d
        L.oracle_ricker.argtypes = [d, d, d]
        L.oracle_ricker.restype = d
        L.oracle_run.argtypes = [i, i, i, i, d, p, p, i, i, d, i, i64, p, d, d, d,
                                 i, p, p, p, p, p, p]
        L.oracle_run_damped.argtypes = [i, i, i, i, d, p, p, i, i, d, i, i64, p, d, d, d, d, d,
                                        i, p, p, p, p, p, p]
        L.oracle_set_threads.argtypes = [i]
        L.oracle_set_threads.restype = i
        L.oracle_get_threads.argtypes = []
        L.oracle_get_threads.restype = i
        L.oracle_misfit_gradient.argtypes = [i, i, i, i, d, p, p, i, i, d, i, i64, p, d, d, d,
                                             i, p, p, p, p]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise ValueError("oracle %s failed (%d)" % (what, rc))


def element_stiffness(kind: int, ds: float, kappa: float, G: float) -> np.ndarray:
    K = np.zeros((24, 24))
    _check(lib().oracle_element_stiffness(kind, ds, kappa, G, _ptr(K)), "element_stiffness")
    return K


def element_node_mass(kind: int, ds: float, rho: float) -> float:
    return lib().oracle_element_node_mass(kind, ds, rho)


def kint8(ds: float = 1.0) -> np.ndarray:
    K = np.zeros((24, 48))
    _check(lib().oracle_kint8(ds, _ptr(K)), "kint8")
    return K


def ku_element_tc_fp64(ds, kappa, G, ue):
    ue = _f64(ue); fe = np.zeros(24)
    _check(lib().oracle_ku_element_tc_fp64(ds, kappa, G, _ptr(ue), _ptr(fe)), "tc_fp64")
    return fe


def ku_element_tc_int(ds, kappa, G, M, ue):
    ue = _f64(ue); fe = np.zeros(24)
    _check(lib().oracle_ku_element_tc_int(ds, kappa, G, M, _ptr(ue), _ptr(fe)), "tc_int")
    return fe


def _mesh_args(mesh):
    mat = np.ascontiguousarray(mesh["material_ids"], dtype=np.int32)
    tab = _f64(mesh["material_table"])
    return mat, tab


def node_mass(kind, mesh):
    mat, tab = _mesh_args(mesh)
    nx, ny, nz = mesh["shape"]
    m = np.zeros((nx + 1) * (ny + 1) * (nz + 1))
    _check(lib().oracle_node_mass(kind, nx, ny, nz, mesh["h"], _ptr(mat), _ptr(tab),
                                  len(tab), _ptr(m)), "node_mass")
    return m


def ku(kind, mesh, u, tc_stages: int = 0):
    mat, tab = _mesh_args(mesh)
    nx, ny, nz = mesh["shape"]
    u = _f64(u).reshape(-1)
    f = np.zeros_like(u)
    _check(lib().oracle_ku(kind, nx, ny, nz, mesh["h"], _ptr(mat), _ptr(tab), len(tab),
                           tc_stages, _ptr(u), _ptr(f)), "ku")
    return f


def ku_nodes(kind, mesh, u, nodes):
    mat, tab = _mesh_args(mesh)
    nx, ny, nz = mesh["shape"]
    u = _f64(u).reshape(-1)
    sel = np.ascontiguousarray(nodes, dtype=np.int64)
    f = np.zeros(3 * len(sel))
    _check(lib().oracle_ku_nodes(kind, nx, ny, nz, mesh["h"], _ptr(mat), _ptr(tab), len(tab),
                                 _ptr(u), len(sel), _ptr(sel), _ptr(f)), "ku_nodes")
    return f.reshape(-1, 3)


def element_max_eig(kind, ds, kappa, G, rho):
    return lib().oracle_element_max_eig(kind, ds, kappa, G, rho)


def dt(kind, mesh, cfl_fraction=0.5):
    mat, tab = _mesh_args(mesh)
    nx, ny, nz = mesh["shape"]
    v = lib().oracle_dt(kind, nx, ny, nz, mesh["h"], _ptr(mat), _ptr(tab), len(tab), cfl_fraction)
    if v <= 0:
        raise ValueError("oracle dt failed")
    return v


def ricker(t, f0, t0):
    return lib().oracle_ricker(t, f0, t0)


def run(kind, mesh, dt_, nsteps, source=None, receivers=(), fix_bottom=True,
        u0=None, um1=None, return_state=False, alpha=0.0, beta=0.0):
    """Central-difference run; returns traces [nsteps, n_rec, 3] (and state).
    alpha, beta != 0 run oracle_run_damped (Rayleigh damping C = alpha M + beta K)."""
    mat, tab = _mesh_args(mesh)
    nx, ny, nz = mesh["shape"]
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    rec = np.ascontiguousarray(receivers, dtype=np.int64).reshape(-1)
    tr = np.zeros((max(nsteps, 0), len(rec), 3))
    if source is None:
        src_node, sdir, f0, t0, amp = -1, np.zeros(3), 1.0, 0.0, 0.0
    else:
        src_node, sdir, f0, t0, amp = (int(source["node"]), _f64(source["dir"]),
                                       float(source["f0"]), float(source["t0"]),
                                       float(source["amp"]))
    sdir = _f64(sdir)
    u0 = None if u0 is None else _f64(u0).reshape(-1)
    um1 = None if um1 is None else _f64(um1).reshape(-1)
    uo = np.zeros(3 * nn) if return_state else None
    umo = np.zeros(3 * nn) if return_state else None
    if alpha or beta:
        _check(lib().oracle_run_damped(kind, nx, ny, nz, mesh["h"], _ptr(mat), _ptr(tab),
                                       len(tab), int(fix_bottom), dt_, nsteps, src_node,
                                       _ptr(sdir), f0, t0, amp, float(alpha), float(beta),
                                       len(rec), _ptr(rec) if len(rec) else None, _ptr(u0),
                                       _ptr(um1), _ptr(tr) if len(rec) else None, _ptr(uo),
                                       _ptr(umo)), "run_damped")
    else:
        _check(lib().oracle_run(kind, nx, ny, nz, mesh["h"], _ptr(mat), _ptr(tab), len(tab),
                                int(fix_bottom), dt_, nsteps, src_node, _ptr(sdir), f0, t0, amp,
                                len(rec), _ptr(rec) if len(rec) else None, _ptr(u0), _ptr(um1),
                                _ptr(tr) if len(rec) else None, _ptr(uo), _ptr(umo)), "run")
    if return_state:
        return tr, uo, umo
    return tr


def misfit_gradient(kind, mesh, dt_, nsteps, source, receivers, data, fix_bottom=True):
    """(dJ/dG per element, J) of the receiver misfit against ``data``."""
    mat, tab = _mesh_args(mesh)
    nx, ny, nz = mesh["shape"]
    rec = np.ascontiguousarray(receivers, dtype=np.int64).reshape(-1)
    data = _f64(data).reshape(-1)
    grad = np.zeros(nx * ny * nz)
    J = ctypes.c_double()
    if source is None:
        src_node, sdir, f0, t0, amp = -1, np.zeros(3), 1.0, 0.0, 0.0
    else:
        src_node, sdir, f0, t0, amp = (int(source["node"]), _f64(source["dir"]),
                                       float(source["f0"]), float(source["t0"]),
                                       float(source["amp"]))
    sdir = _f64(sdir)
    _check(lib().oracle_misfit_gradient(kind, nx, ny, nz, mesh["h"], _ptr(mat), _ptr(tab), len(tab),
                                        int(fix_bottom), dt_, nsteps, src_node, _ptr(sdir), f0, t0,
                                        amp, len(rec), _ptr(rec), _ptr(data), _ptr(grad),
                                        ctypes.byref(J)), "misfit_gradient")
    return grad, J.value
