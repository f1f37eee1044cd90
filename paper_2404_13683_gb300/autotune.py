"""Choose the launch configuration of the tensor-core path for a model.

The knobs, each a trade of work against precision or overhead:

* the number of 11-bit integer digit stages (Eq. int8comp1): each stage adds
  tensor-core products and one more word to recombine, and about 11 bits of
  precision (the paper's rule: 7 bits per INT8 stage, M = 4 ~ FP32, M = 8 >=
  FP64);
* the node-stencil kernel on the uniform node planes, or the element kernel
  everywhere;
* the work bricks: how many CTAs the (15 x 15 node column x plane range)
  bricks are cut into per launch (fewer, longer bricks start fewer pipelines;
  more use more SMs).

``choose_config`` runs a short simulation of the model with every candidate
through the C ABI, compares the receiver traces with the five-stage run
(FP64-equivalent), and returns the fastest candidate within the tolerance
together with the measurements (the record to keep per model).
"""
from __future__ import annotations

import itertools
import time

import numpy as np

from . import vfe


def _run(workload, steps, stages=5, stencil=True, ctas=0):
    m = vfe.Mesh(workload, path=vfe.VFE_PATH_TC, stages=stages, stencil=stencil, ctas=ctas)
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


def choose_config(workload, tol=1e-6, steps=200, stages=(3, 4, 5), stencil=(True, False),
                  ctas=(0,)):
    """Return (choice, report): choice = {"stages", "stencil", "ctas",
    "s_per_step", "rel_l2"} of the fastest candidate whose traces agree with
    the five-stage element-kernel run to ``tol`` relative L2; report maps every
    candidate (stages, stencil, ctas) to its error and time."""
    ref, _ = _run(workload, steps, 5, False, 0)
    den = float(np.linalg.norm(ref))
    report = {}
    for st, sc, ct in itertools.product(stages, stencil, ctas):
        tr, t = _run(workload, steps, st, sc, ct)
        err = float(np.linalg.norm(tr - ref)) / den if den > 0 else 0.0
        report[(st, sc, ct)] = {"rel_l2": err, "s_per_step": t}
    ok = [k for k, r in report.items() if r["rel_l2"] <= tol]
    if not ok:
        raise RuntimeError("no candidate meets the tolerance %g" % tol)
    best = min(ok, key=lambda k: (report[k]["s_per_step"], -k[0]))
    choice = {"stages": best[0], "stencil": best[1], "ctas": best[2]}
    choice.update(report[best])
    return choice, report


def choose_stages(workload, tol=1e-6, steps=200, candidates=(2, 3, 4, 5)):
    """Return (stages, report): the fastest stage count whose traces agree with
    the five-stage run to ``tol`` relative L2, and per-count error and time."""
    choice, report = choose_config(workload, tol, steps, stages=tuple(candidates),
                                   stencil=(True,), ctas=(0,))
    return choice["stages"], {k[0]: v for k, v in report.items()}
