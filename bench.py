#!/usr/bin/env python
"""Benchmark of the explicit voxel FE wave step (arXiv 2404.13683, OVFEM).

One bench "step" is one time step of the whole hot path -- f = K u over every
element (integer-split tensor-core products) plus the central-difference
update, source and receiver recording -- on the 512 x 512 x 256 model of ten
dipping layers under a random topographic surface (67,108,864 voxels of which
the cells above the surface are void, 67,634,433 nodes, ``workloads.config3``),
the largest of the layered-ground workloads that fits one GPU.

Prints one JSON line (rank 0).  ``value`` is element*steps/s over all ranks;
ranks run independent replicas (the path needs no exchange on one GPU).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (test infrastructure) on the
same workload, on every host core, and prints the same line with
``"impl": "reference"``.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "element·steps/s, INT8-TC vs FP64 path on 1 GB300 at ≤1e-6 rel trace error"
UNIT = "element*steps/s"
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2
PROFILES = {"config3": os.path.join(ROOT, "profiles", "tc_step_kernels_config3_512x512x256.txt")}
# the sources of the kernels of one tensor-core step (the roofline's unit)
KERNEL_SRCS = [os.path.join(ROOT, "paper_2404_13683_gb300", "csrc", f)
               for f in ("vfe_tc.cu", "vfe_stencil.cu", "vfe_tc_common.cuh")]


def parse():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--stages", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--stencil", type=int, choices=[0, 1, 2], default=1,
                    help="TC path node-stencil option: 1 (default: per-node corrections on "
                         "meshes of 8 Mi elements or more), 2 (on every mesh), 0 (element "
                         "kernel only)")
    ap.add_argument("--damping", type=float, default=0.0,
                    help="Rayleigh damping ratio h over the source band (100-125 kHz on "
                         "paper_rebar, f0 * [0.89, 1.11] otherwise); 0 = undamped")
    ap.add_argument("--trace-steps", type=int, default=2000,
                    help="length of the untimed TC vs FP64 path trace comparison "
                         "(capped by the workload's own length)")
    ap.add_argument("--workload", default="config3",
                    choices=["config1", "config2", "config3", "config4", "config5",
                             "paper_rebar"],
                    help="config3 (default: 512x512x256, the largest single-GPU model) is the "
                         "headline; config2 (128x128x64) and the others are reported in the "
                         "design notes")
    ap.add_argument("--decomp", choices=["replicas", "slab"], default="replicas",
                    help="with --gpus N > 1: independent replicas (default, weak scaling) or "
                         "one model split into N z-slabs with a node-plane exchange per step "
                         "(strong scaling)")
    ap.add_argument("--shape", default=None,
                    help="NX,NY,NZ: the config3 generator at another size (for profiling a "
                         "smaller model of the same kind; the headline is 512,512,256)")
    return ap.parse_args()


def make_workload(args, W):
    if args.workload == "config3" and args.shape:
        nx, ny, nz = (int(v) for v in args.shape.split(","))
        return W.config3(shape=(nx, ny, nz))
    return {"config1": W.config1, "config2": W.config2, "config3": W.config3,
            "paper_rebar": W.paper_rebar}[args.workload]()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


DESCRIPTIONS = {
    "config1": "two horizontal layers",
    "config2": "layered ground (3 layers) + 20 ellipsoidal inclusions",
    "config3": "10 dipping layers under a random topographic surface (void above)",
    "paper_rebar": "concrete block with a steel rebar shaped like the paper's ultrasonic model",
}


def ricker_rows(n, dt, source):
    """The source wavelet of the workload sampled at t = k dt on the host:
    F^k = amp (1 - 2 a) exp(-a) dir, a = (pi f0 (k dt - t0))^2 ([n][3] FP64)."""
    t = np.arange(n) * dt
    a = (np.pi * source["f0"] * (t - source["t0"])) ** 2
    return (source["amp"] * (1.0 - 2.0 * a) * np.exp(-a))[:, None] * \
        np.asarray(source["dir"], dtype=np.float64)[None, :]


def paper_err(obs, ref, rel_floor=0.0, return_channels=False):
    """The paper's trace error (Section 3, accuracy comparison): the mean over
    channels (receiver x component) of sum_t (obs - ref)^2 / sum_t ref^2,
    over the channels whose reference peak exceeds rel_floor times the
    strongest channel's peak (and is not zero).  A channel the wave has not
    reached holds only the scheme's leading-edge tail, far below the signal;
    rel_floor leaves such channels out."""
    o = obs.reshape(obs.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    den = (r * r).sum(axis=0)
    peak = np.abs(r).max(axis=0)
    keep = (den > 0) & (peak > rel_floor * peak.max())
    if not keep.any():
        return (None, 0) if return_channels else None
    err = float((((o - r) ** 2).sum(axis=0)[keep] / den[keep]).mean())
    return (err, int(keep.sum())) if return_channels else err


def channel_errors(obs, ref):
    """Per-channel (receiver x component) errors of obs against ref: the
    largest |obs - ref| relative to the channel's own peak |ref| and to the
    strongest channel's peak, the number of channels whose reference is
    identically zero, and the largest |obs - ref| over all channels relative
    to the strongest peak (the bound the fixed-point state is held to)."""
    o = obs.reshape(obs.shape[0], -1)
    r = ref.reshape(ref.shape[0], -1)
    d = np.abs(o - r).max(axis=0)
    peak = np.abs(r).max(axis=0)
    top = float(peak.max()) if peak.size else 0.0
    live = peak > 0
    return {"channels": int(peak.size), "zero_reference": int((~live).sum()),
            "max_err_over_own_peak": float((d[live] / peak[live]).max()) if live.any() else None,
            "max_err_over_strongest_peak": float(d.max() / top) if top > 0 else None,
            "weakest_channel_peak_over_strongest": float(peak[live].min() / top)
            if live.any() else None}


# tensor-core work per element and step: N = 48 outputs x K = 32 inputs
# (24 data + 8 bias rows) x 2 ops per multiply-add, for each digit stage
def tc_ops_per_element(stages):
    return 2 * 48 * 32 * stages


def workload_config(mesh, stages, path_name):
    nx, ny, nz = mesh["shape"]
    kind = next((v for k, v in DESCRIPTIONS.items() if mesh["name"].startswith(k)), "")
    return {"workload": "%s %s, OVFEM, %s path" % (mesh["name"], kind, path_name),
            "elements": nx * ny * nz, "nodes": (nx + 1) * (ny + 1) * (nz + 1),
            "materials": int(len(mesh["material_table"])), "receivers": int(len(mesh["receivers"])),
            "tc_digit_stages": stages, "tc_digit_bits": 11,
            "l2": "flushed (512 MiB write) between timed steps", "step": "one time step"}


# --------------------------------------------------------------------------
# clocks (nvidia-smi sampled during the timed region)
# --------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = os.path.join("/tmp", "vfe_clocks_%d_%d.csv" % (os.getpid(), gpu))

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.25)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return None
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 7:
                    rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# --------------------------------------------------------------------------
# roofline bookkeeping for one time step (the dominant unit: all its kernels)
# --------------------------------------------------------------------------
def algorithmic_bytes_per_step(mesh, damped=False):
    """HBM bytes one time step must move at minimum: read u^n, u^{n-1} and the
    per-node update multiplier, write u^{n+1} (3 x int64 each), read each
    element's int32 material id.  With Rayleigh damping the stiffness acts on
    the state w^n, which is read as well and written for the next step
    (2 x 24 bytes more per node)."""
    nx, ny, nz = mesh["shape"]
    nodes = (nx + 1) * (ny + 1) * (nz + 1)
    per_node = 24 + 24 + 24 + 8 + (48 if damped else 0)
    return nodes * per_node + nx * ny * nz * 4


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_code_hash(paths=KERNEL_SRCS):
    """First 16 hex digits of the SHA-256 of the kernel sources with comments
    and whitespace removed (so a comment edit keeps its profile)."""
    import re
    src = ""
    for path in paths:
        with open(path) as f:
            src += f.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", "", src)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def profiled_counters(workload):
    """DRAM bytes and warp instructions per launch from the committed ncu
    summary of this workload, if it was taken on the current kernel code
    (else None)."""
    if workload not in PROFILES:
        return None
    try:
        with open(PROFILES[workload]) as f:
            text = f.read()
        sha = kernel_code_hash()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_code_sha256_16", "").split(" ")[0] != sha:
        return None
    try:
        out = {"dram_bytes": float(vals["dram_bytes_per_launch"].split()[0]),
               "warp_instructions": None}
    except (KeyError, ValueError, IndexError):
        return None
    try:
        out["warp_instructions"] = float(vals["smsp__inst_executed.sum"].split()[0])
    except (KeyError, ValueError, IndexError):
        pass
    return out


# warp-instruction issue rate of a GB300: 152 SMs x 4 schedulers, one warp
# instruction per scheduler per cycle, at the 2,070 MHz maximum SM clock
ISSUE_PEAK_WARP_INST_PER_S = 152 * 4 * 2.070e9


# --------------------------------------------------------------------------
# replicas across ranks: each rank advances its own copy of the model, so the
# job's throughput is the work of all ranks over the slowest rank's time
# --------------------------------------------------------------------------
def reduce_max(x, dist, device):
    """Max of a per-rank float over all ranks (identity without a group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, elements, steps, seconds_max):
    """element*steps/s of the whole job (weak scaling: fixed work per rank)."""
    return world * elements * steps / seconds_max


# --------------------------------------------------------------------------
# our implementation
# --------------------------------------------------------------------------
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2404_13683_gb300 import build as vbuild
    if rank == 0:
        vbuild.build()
    if dist is not None:
        dist.barrier()
    from paper_2404_13683_gb300 import vfe, workloads as W

    if args.workload == "config4":
        return run_batch(args, torch, dist, world, rank, local, vfe, W)
    if args.decomp == "slab":
        return run_slabs(args, torch, dist, world, rank, local, vfe, W)
    if args.workload == "config5":
        return run_adjoint(args, torch, dist, world, rank, local, vfe, W)
    mesh = make_workload(args, W)
    ne = int(mesh["material_ids"].size)
    # a dedicated stream: the library launches on it and the events are
    # recorded on it (torch's default stream is the legacy NULL stream)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    def timed_steps(m, steps, warmup):
        for _ in range(warmup):
            m.step(1)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for k in range(steps):
            flush.zero_()                       # evict L2 between timed steps
            ev[k][0].record(stream)
            m.step(1)                           # prologue + tc_step_kernel
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        m.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        return float(np.sum(ms)), ms

    def damp(mm):
        if args.damping > 0:
            f0 = mesh["source"]["f0"]
            band = (100e3, 125e3) if mesh["name"].startswith("paper_rebar") else (0.89 * f0, 1.11 * f0)
            alpha, beta = vfe.vfe_rayleigh_coefficients(args.damping, *band)
            mm.set_damping(alpha, beta)
        return mm

    # --- the TC path (headline)
    m = damp(vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, stages=args.stages,
                      stream=stream.cuda_stream, device=local, stencil=args.stencil))
    with ClockSampler(local) as clk:
        total_ms, per = timed_steps(m, args.steps, args.warmup)
    clocks = clk.summary()
    total_ms = reduce_max(total_ms, dist, "cuda")
    ms_step = total_ms / args.steps
    value = replica_throughput(world, ne, args.steps, total_ms * 1e-3)
    launches_per_step = vfe.vfe_get_launches_per_step(m.handle)
    m.close()

    # --- e2e: the public API on host buffers -- each step is vfe_step_forced(1)
    # with that step's source-node force uploaded from page-locked host memory,
    # then the device-to-host copy of that step's receiver row into page-locked
    # memory, queued behind the step (vfe_get_trace_rows_async); the timed
    # region ends when every row has arrived (vfe_synchronize).  The model
    # itself is uploaded once by vfe_create_mesh.
    m = damp(vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, stages=args.stages, device=local,
                      stencil=args.stencil))
    ntot = args.warmup + args.steps
    force = torch.empty((ntot, 3), dtype=torch.float64, pin_memory=True).numpy()
    force[:] = ricker_rows(ntot, m.dt, mesh["source"])
    rows = torch.zeros((ntot, m.n_rec, 3), dtype=torch.float64, pin_memory=True).numpy()
    for k in range(args.warmup):
        m.step_forced(force[k:k + 1])
        vfe.vfe_get_trace_rows_async(m.handle, k, 1, m.n_rec, rows[k])
    m.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(args.warmup, ntot):
        m.step_forced(force[k:k + 1])
        vfe.vfe_get_trace_rows_async(m.handle, k, 1, m.n_rec, rows[k])
    m.synchronize()
    e2e_s = time.perf_counter() - t0
    streamed_ok = bool(np.array_equal(rows, m.traces()))   # every row arrived intact
    m.close()
    e2e_value = replica_throughput(world, ne, args.steps, reduce_max(e2e_s, dist, "cuda"))

    # --- the plain FP64 CUDA-core path on the same workload, and the trace
    # agreement of the two GPU paths over the same steps
    cfg = workload_config(mesh, args.stages, "TC (exact 11-bit integer digits on tcgen05)")
    if args.stencil != 1:
        cfg["stencil_option"] = args.stencil
    if args.damping > 0:
        cfg["rayleigh_damping_ratio"] = args.damping
    if not args.no_fp64:
        nf = max(3, min(args.steps, 20))
        mf = damp(vfe.Mesh(mesh, path=vfe.VFE_PATH_FP64, stream=stream.cuda_stream,
                           device=local))
        f_ms, _ = timed_steps(mf, nf, min(args.warmup, 3))
        mf.close()
        f_value = ne * nf / (f_ms * 1e-3)
        cfg["fp64_path_value"] = f_value
        cfg["speedup_vs_fp64_path"] = (value / world) / f_value
        # the workload's full length (at most 2,000 steps) on both paths from
        # rest (untimed)
        nt = min(int(mesh["nsteps"]), args.trace_steps)
        trs = []
        for path in (vfe.VFE_PATH_TC, vfe.VFE_PATH_FP64):
            mp = damp(vfe.Mesh(mesh, path=path, stages=args.stages, stream=stream.cuda_stream,
                               device=local, stencil=args.stencil))
            mp.step(nt)
            trs.append(mp.traces())
            mp.close()
        num = float(np.linalg.norm(trs[0] - trs[1]))
        den = float(np.linalg.norm(trs[1]))
        cfg["trace_rel_l2_tc_vs_fp64_path"] = num / den if den > 0 else None
        # the paper's Err over every channel, and over the channels whose
        # reference peak exceeds 1e-6 of the strongest one (a channel the wave
        # has not reached holds only the scheme's leading-edge tail)
        cfg["trace_err_paper_all_channels"] = paper_err(trs[0], trs[1])
        err, nch = paper_err(trs[0], trs[1], rel_floor=1e-6, return_channels=True)
        cfg["trace_err_paper_tc_vs_fp64_path"] = err
        cfg["trace_err_channels"] = "%d of %d (reference peak above 1e-6 of the strongest)" % (
            nch, trs[1][0].size)
        cfg["trace_channels"] = channel_errors(trs[0], trs[1])
        cfg["trace_max_abs_fp64_path"] = float(np.abs(trs[1]).max())
        cfg["trace_steps_compared"] = nt

    # --- roofline of the dominant kernel
    peaks, peak_src = measured_peaks()
    abytes = algorithmic_bytes_per_step(mesh, damped=args.damping > 0)
    achieved = abytes / (ms_step * 1e-3) / 1e9
    prof = profiled_counters(args.workload) if args.damping == 0 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
            "frac": achieved / float(peaks["hbm_gbs"]),
            "traffic": prof["dram_bytes"] if prof else None,
            "algorithmic_bytes_per_launch": abytes, "peak_source": peak_src,
            "kernel": "one time step: tc_prologue_kernel, then tc_step_kernel (the source "
                      "and receiver planes, and the non-uniform ones on meshes below 8 Mi "
                      "elements) and tc_stencil_kernel (every other column-plane, per-node "
                      "material) as programmatic dependents that overlap, then "
                      "stencil_fix_kernel (nodes with elements of another material, void or "
                      "outside the mesh); duration = the step's CUDA-event time"}
    # the tensor pipe's share: fp16-digit multiply-adds per second against the
    # measured dense bf16 rate (fp16 runs at the same rate)
    tc_tops = tc_ops_per_element(args.stages) * ne / (ms_step * 1e-3) / 1e12
    tc_peak = float(peaks.get("bf16_tflops", 1900.0))
    roof["tensor"] = {"achieved": tc_tops, "peak": tc_peak, "unit": "TFLOP/s",
                      "frac": tc_tops / tc_peak}
    if prof and prof["warp_instructions"]:
        # the kernel is limited by instruction issue, not HBM: the same launch
        # against the GPU's warp-instruction issue rate
        ach_i = prof["warp_instructions"] / (ms_step * 1e-3)
        roof["issue"] = {"achieved": ach_i, "peak": ISSUE_PEAK_WARP_INST_PER_S,
                         "unit": "warp instructions/s", "frac": ach_i / ISSUE_PEAK_WARP_INST_PER_S,
                         "warp_instructions_per_launch": prof["warp_instructions"]}

    # --- the CPU oracle on a bounded sample (rank 0, one GPU only)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(mesh)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "int64", "data": "synthetic", "config": cfg,
                "roofline": roof, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * 8,
                        "d2h_bytes_per_step": int(len(mesh["receivers"]) * 3 * 8),
                        "rows_streamed_intact": streamed_ok,
                        "note": "per step: vfe_step_forced(1) with that step's source force "
                                "(3 doubles) from page-locked host memory, then "
                                "vfe_get_trace_rows_async of that step's receiver row into "
                                "page-locked memory; timed until vfe_synchronize returns; the "
                                "model is uploaded once by vfe_create_mesh"},
                "gpu_launches": launches_per_step * args.steps, "clocks": clocks,
                "parallelism": "replicas x%d" % world if world > 1 else "1 GPU"}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def run_slabs(args, torch, dist, world, rank, local, vfe, W):
    """One model split into `world` z-slabs (slab.py): every step, each rank
    steps its slab, exchanges its boundary node planes with its neighbours
    (NCCL send/recv on the mesh's stream) and all ranks agree on the
    fixed-point unit (one 8-byte all-reduce).  value = the model's
    element*steps per second (strong scaling)."""
    from paper_2404_13683_gb300 import slab as S
    mesh = make_workload(args, W)
    ne = int(mesh["material_ids"].size)
    # the model's time step: the minimum over the slabs' critical steps
    probe = S.Slab(mesh, world, rank, 0.0)
    w = dict(probe.workload)
    w.pop("dt")
    with vfe.Mesh(w, path=vfe.VFE_PATH_TC, stages=args.stages, device=local) as m:
        dt_local = m.dt
    t = torch.tensor([dt_local], dtype=torch.float64, device="cuda")
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
    slab = S.Slab(mesh, world, rank, float(t.item()))
    eng = S.GpuSlabEngine(slab, torch, stages=args.stages)
    eng.set_source_bound(S.source_scale(slab, eng, dist))
    bufs = [torch.zeros(slab.plane_values(), dtype=torch.float64, device="cuda")
            for _ in range(4)]

    def one_step():
        eng.step()
        if dist is not None:
            S.exchange(slab, eng, dist, bufs)

    for _ in range(args.warmup):
        one_step()
    torch.cuda.synchronize()
    eng.mesh.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(eng.stream)
    for _ in range(args.steps):
        one_step()
    e1.record(eng.stream)
    torch.cuda.synchronize()
    eng.mesh.synchronize()
    ms = reduce_max(e0.elapsed_time(e1), dist, "cuda")
    eng.close()
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": ne * args.steps / (ms * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "%s split into %d z-slabs (node-plane exchange per step)"
                                   % (mesh["name"], world), "elements": ne,
                       "slab_planes": S.plane_ranges(mesh["shape"][2], world),
                       "timing": "CUDA events on rank 0's mesh stream, max over ranks; L2 not "
                                 "flushed (the exchange separates the steps)"},
            "parallelism": "slab x%d" % world}), flush=True)


def run_batch(args, torch, dist, world, rank, local, vfe, W):
    """The 64-model many-case batch: one fused launch per step for all models
    (replayed as graphs of 32 steps), timed with CUDA events on the batch's
    stream from the first to the last step."""
    models = W.config4()
    ne = sum(int(m["material_ids"].size) for m in models)
    meshes = [vfe.Mesh(w, stages=args.stages, device=local) for w in models]
    batch = vfe.Batch(meshes)
    batch.step(max(args.warmup, 2))
    batch.synchronize()
    if dist is not None:
        dist.barrier()
    # a few hundred steps, at least the requested ones (each replay is 32 steps)
    nsteps = max(args.steps, 320)
    t0 = time.perf_counter()
    with ClockSampler(local) as clk:
        batch.step(nsteps)
        batch.synchronize()
    el = reduce_max(time.perf_counter() - t0, dist, "cuda")
    clocks = clk.summary()
    batch.close()
    for m in meshes:
        m.close()
    if rank == 0:
        print(json.dumps({"metric": METRIC, "value": replica_throughput(world, ne, nsteps, el),
                          "unit": UNIT, "n_gpus": world, "steps": nsteps,
                          "warmup": args.warmup, "ms_per_step": el / nsteps * 1e3,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                          "dtype": "int64", "data": "synthetic", "clocks": clocks,
                          "config": {"workload": "config4: 64 cubic models n in [32,128], "
                                                 "batched (one fused launch per step)",
                                     "elements": ne, "models": len(models),
                                     "tc_digit_stages": args.stages,
                                     "timing": "wall clock around the graph replays and the "
                                               "final synchronisation"}}),
              flush=True)


def run_adjoint(args, torch, dist, world, rank, local, vfe, W):
    """The structure-estimation gradient on the 96^3 model: dJ/dG per element
    of the receiver misfit, by the adjoint run with checkpoints every 100
    steps (forward with checkpoints, then the adjoint backward in time with
    recomputed segments), on the background model against data from the
    model with the anomaly.  Timed against a plain forward run of the same
    length; both paths, and the agreement of their gradients."""
    obs, bg = W.config5(anomaly=True), W.config5(anomaly=False)
    ne = int(bg["material_ids"].size)
    nt = int(bg["nsteps"])
    with vfe.Mesh(obs, device=local) as m:   # the observed data (untimed)
        dt = m.dt
        m.step(nt)
        data = m.traces()
    res = {}
    for name, path in (("tc", vfe.VFE_PATH_TC), ("fp64", vfe.VFE_PATH_FP64)):
        with vfe.Mesh(bg, path=path, dt=dt, stages=args.stages, device=local) as m:
            m.step(20)   # warm-up: graphs, tensor maps
            m.synchronize()
        with vfe.Mesh(bg, path=path, dt=dt, stages=args.stages, device=local) as m:
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
            m.step(nt)
            m.synchronize()
            fwd = reduce_max(time.perf_counter() - t0, dist, "cuda")
        with vfe.Mesh(bg, path=path, dt=dt, stages=args.stages, device=local) as m:
            vfe.vfe_misfit_gradient(m.handle, data[:40], 10)   # warm-up
        with vfe.Mesh(bg, path=path, dt=dt, stages=args.stages, device=local) as m:
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
            g, J = vfe.vfe_misfit_gradient(m.handle, data, 100)
            grad_s = reduce_max(time.perf_counter() - t0, dist, "cuda")
        res[name] = {"forward_s": fwd, "gradient_s": grad_s, "J": J, "g": g}
    tc, f64 = res["tc"], res["fp64"]
    if rank == 0:
        value = replica_throughput(world, ne, nt, tc["gradient_s"])
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": nt,
            "warmup": 1, "ms_per_step": tc["gradient_s"] / nt * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": {"workload": "config5: 96^3, two layers, misfit gradient dJ/dG per "
                                   "element (checkpoints every 100 steps) against data "
                                   "from the model with a spherical anomaly",
                       "elements": ne, "receivers": int(len(bg["receivers"])),
                       "value_counts": "elements x forward steps per second of the "
                                       "whole gradient computation",
                       "tc_forward_s": tc["forward_s"], "tc_gradient_s": tc["gradient_s"],
                       "tc_gradient_over_forward": tc["gradient_s"] / tc["forward_s"],
                       "fp64_forward_s": f64["forward_s"], "fp64_gradient_s": f64["gradient_s"],
                       "fp64_gradient_over_forward": f64["gradient_s"] / f64["forward_s"],
                       "gradient_speedup_vs_fp64_path": f64["gradient_s"] / tc["gradient_s"],
                       "misfit_rel_diff_tc_vs_fp64": abs(tc["J"] - f64["J"]) / abs(f64["J"]),
                       "gradient_rel_l2_tc_vs_fp64": float(np.linalg.norm(tc["g"] - f64["g"])
                                                           / np.linalg.norm(f64["g"])),
                       "timing": "wall clock around the synchronous call"}}), flush=True)


# --------------------------------------------------------------------------
# the CPU oracle (reference arm and cpu_baseline)
# --------------------------------------------------------------------------
def _oracle_runner(mesh, threads):
    """A function n -> seconds that runs the FP64 CPU oracle n time steps of
    the workload from rest (source, receivers and fixed nodes as the GPU runs
    use them) on the given number of threads, and the threads in effect."""
    import oracle
    from paper_2404_13683_gb300 import workloads as W
    oracle.build()
    used = oracle.set_threads(threads)
    dt = float(mesh["dt"]) if "dt" in mesh else oracle.dt(0, mesh, 0.5)
    s = mesh["source"]
    src = {"node": W.source_node(mesh), "dir": s["dir"], "f0": s["f0"], "t0": s["t0"],
           "amp": s["amp"]}
    rec = W.receiver_nodes(mesh)
    fix = int(mesh.get("fix_bottom", 1))

    def run(n):
        oracle.set_threads(used)
        t0 = time.perf_counter()
        oracle.run(0, mesh, dt, n, source=src, receivers=rec, fix_bottom=fix)
        return time.perf_counter() - t0
    return run, used


def _oracle_rate(run, ne, target_s):
    """element*steps/s of the oracle over about target_s seconds of steps,
    and the steps timed.  A run of 0 steps (allocation, node masses, fixed
    nodes) is timed too and subtracted, so only the time steps count."""
    setup = run(0)
    one = max(run(1) - setup, 1e-3)
    n = max(1, int(round(target_s / one)))
    el = run(n) - setup
    return ne * n / max(el, 1e-9), n


def cpu_baseline(mesh, target_s=12.0):
    """The oracle on every host core (the value) and on one core, each on a
    bounded sample of whole time steps of the workload."""
    import oracle
    ne = int(mesh["material_ids"].size)
    run_all, cores = _oracle_runner(mesh, oracle.host_cores())
    v_all, n_all = _oracle_rate(run_all, ne, target_s)
    run_one, _ = _oracle_runner(mesh, 1)
    v_one, n_one = _oracle_rate(run_one, ne, 0.0)
    oracle.set_threads(1)
    return {"value": v_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "cpu": oracle.cpu_model(),
            "sample": "%d time steps of the full %s model from rest (element-by-element FP64 "
                      "K u in eight colours of element parity, and the update, plain C with "
                      "OpenMP on %d threads); setup (allocation, node masses) excluded"
                      % (n_all, mesh["name"], cores),
            "single_thread": {"value": v_one, "cores": 1,
                              "sample": "%d time step(s), the plain sequential element loop"
                                        % n_one}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2404_13683_gb300 import workloads as W
    if args.workload not in ("config2", "config3", "paper_rebar"):
        args.workload = "config3"
    mesh = make_workload(args, W)
    ne = int(mesh["material_ids"].size)
    run, cores = _oracle_runner(mesh, oracle.host_cores())
    setup = run(0)
    if args.warmup > 0:
        run(args.warmup)
    el = run(args.steps) - setup
    value = ne * args.steps / el
    cfg = workload_config(mesh, args.stages, "FP64 CPU oracle")
    # the oracle runs on the host: no digit stages, no GPU cache to flush
    for key in ("tc_digit_stages", "tc_digit_bits", "l2"):
        cfg.pop(key, None)
    cfg["host"] = "%d threads of the host CPU (%s), plain C with OpenMP (oracle/vfe_oracle.c)" % (
        cores, oracle.cpu_model())
    sample = ("%d time steps of the full %s model from rest, timed as one oracle run; its "
              "setup (allocation, node masses), timed by a run of 0 steps, is subtracted"
              % (args.steps, mesh["name"]))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
