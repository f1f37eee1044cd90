"""Helpers shared by the GPU parity tests (test infrastructure)."""
import numpy as np

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W

PATHS = {"tc": vfe.VFE_PATH_TC, "fp64": vfe.VFE_PATH_FP64}

# Tolerances.  FP64 path: relative L2 of traces <= 1e-12, K u <= 1e-13.
# TC path: K u is FP64-equivalent (55-bit integer split, then 64-bit fixed
# point): <= 1e-13 of max|K u|; traces <= 1e-6 relative L2 (the stated bar),
# and in practice ~1e-14.
KU_TOL = 1e-13
TRACE_TOL = {"fp64": 1e-12, "tc": 1e-6}


def rel_max(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_source(mesh):
    s = mesh["source"]
    return {"node": W.source_node(mesh), "dir": s["dir"], "f0": s["f0"], "t0": s["t0"],
            "amp": s["amp"]}
