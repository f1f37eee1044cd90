"""Choose the number of integer digit stages of the tensor-core path.

Each 11-bit stage adds one tensor-core product per element and one more word
to recombine, and about 11 bits of precision (Section 3 of the paper: 7 bits
per INT8 stage, M = 4 ~ FP32, M = 8 >= FP64).  ``choose_stages`` runs a short
simulation of a model with every stage count through the C ABI, compares the
receiver traces with the five-stage run (FP64-equivalent) and returns the
fastest count that stays within the tolerance.
"""
from __future__ import annotations

import time

import numpy as np

from . import vfe


def _run(workload, stages, steps):
    m = vfe.Mesh(workload, path=vfe.VFE_PATH_TC, stages=stages)
    try:
        m.step(2)
        m.synchronize()
        t0 = time.perf_counter()
        m.step(steps - 2)
        m.synchronize()
        el = time.perf_counter() - t0
        return m.traces(), el / max(steps - 2, 1)
    finally:
        m.close()


def choose_stages(workload, tol=1e-6, steps=200, candidates=(2, 3, 4, 5)):
    """Return (stages, report): the fastest stage count whose traces agree with
    the five-stage run to ``tol`` relative L2, and per-count error and time."""
    ref, tref = _run(workload, 5, steps)
    den = float(np.linalg.norm(ref))
    report = {5: {"rel_l2": 0.0, "s_per_step": tref}}
    for s in candidates:
        if s == 5:
            continue
        tr, t = _run(workload, s, steps)
        err = float(np.linalg.norm(tr - ref)) / den if den > 0 else 0.0
        report[s] = {"rel_l2": err, "s_per_step": t}
    ok = [s for s, r in report.items() if r["rel_l2"] <= tol]
    best = min(ok, key=lambda s: (report[s]["s_per_step"], -s))
    return best, report
