"""Seeded synthetic inputs shaped like the paper's workloads.

This module only builds meshes (material ids and a {Vp, Vs, rho} table),
source descriptions and receiver lists.  It holds none of the method's
arithmetic (no moduli, element matrices, masses or time steps), so both the
CUDA path and the CPU oracle can consume its output.

The paper's own model (a rebar in concrete, Section 3) has no public data and
its material constants are not given, so layered-ground models of the sizes
below stand in for it:

* ``config1``: 32^3 voxels, h = 1 m, two layers, 300 steps, 16 receivers.
* ``config2``: 128x128x64, three layers plus 20 seeded ellipsoidal inclusions,
  2,000 steps, 64 receivers (the benchmark workload).
* ``config3``: 512x512x256, ten dipping layers, seeded smoothed topography
  (cells above it are void), 5,000 steps.
* ``config4``: 64 independent cubic models, n ~ U{32..128} (seeded), three
  random layers each, random source node and frequency (3-10 Hz), 1,000
  steps each -- the many-case batch.
* ``config5``: 96^3, two layers and a hidden spherical low-velocity anomaly
  (diameter 12 cells, Vs -30 %) at the centre, 36 surface receivers (6 x 6),
  1,500 steps -- the adjoint-gradient workload (``anomaly=False`` gives the
  background model whose misfit gradient is sought).
* ``paper_rebar``: the shape of the paper's experiment (Section 3): a
  324 x 128 x 384 mm concrete block at ds = 2 mm (162 x 64 x 192 voxels) with a
  steel rebar of radius 15 mm along y at x = 160, z = 100 mm, the source and
  the eight observation points of Table 1, dt = 5e-8 s, 16,384 steps, the four
  bottom corner points fixed (``fix_bottom`` = 2).  The
  paper gives no material constants; typical concrete (Vp 4000, Vs 2400,
  rho 2300) and steel (5900, 3200, 7850) values stand in.
* ``random_mesh``: small random meshes with voids for parity tests.
"""
from __future__ import annotations

import numpy as np


def node_index(shape, i, j, k):
    nx, ny, _ = shape
    return int(i) + (nx + 1) * (int(j) + (ny + 1) * int(k))


def _mesh(shape, h, mat, table, source, receivers, nsteps, name):
    nx, ny, nz = shape
    mat = np.ascontiguousarray(mat.reshape(nz, ny, nx).reshape(-1), dtype=np.int32)
    return {
        "name": name,
        "shape": (int(nx), int(ny), int(nz)),
        "h": float(h),
        "material_ids": mat,
        "material_table": np.ascontiguousarray(table, dtype=np.float64).reshape(-1, 3),
        "source": source,
        "receivers": np.ascontiguousarray(receivers, dtype=np.int32).reshape(-1, 3),
        "nsteps": int(nsteps),
    }


def _source(ijk, f0, t0=None, amp=1.0, direction=(0.0, 0.0, 1.0)):
    return {"ijk": tuple(int(v) for v in ijk), "dir": tuple(float(v) for v in direction),
            "f0": float(f0), "t0": float(1.0 / f0 if t0 is None else t0), "amp": float(amp)}


def config1():
    """32^3, top 12 cells (k >= 20) soft layer, 10 Hz Ricker at the centre."""
    nx = ny = nz = 32
    k = np.arange(nz)[:, None, None] * np.ones((nz, ny, nx), dtype=np.int64)
    mat = np.where(k >= 20, 0, 1)
    table = [[700.0, 200.0, 1800.0], [2000.0, 800.0, 2100.0]]
    rec = [(i, j, nz) for j in (4, 12, 20, 28) for i in (4, 12, 20, 28)]
    return _mesh((nx, ny, nz), 1.0, mat, table, _source((16, 16, 16), 10.0, 0.1), rec, 300,
                 "config1_32x32x32")


def config2(seed: int = 2):
    """128x128x64, 3 layers + 20 ellipsoids (seeded), 5 Hz Ricker, 2,000 steps."""
    nx, ny, nz = 128, 128, 64
    rng = np.random.default_rng(seed)
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mat = np.where(kk >= 48, 0, np.where(kk >= 32, 1, 2)).astype(np.int64)
    table = [[700.0, 200.0, 1800.0], [1400.0, 500.0, 1950.0], [2000.0, 800.0, 2100.0]]
    xc, yc, zc = ii + 0.5, jj + 0.5, kk + 0.5
    for e in range(20):
        c = rng.uniform([0, 0, 0], [nx, ny, nz])
        ax = rng.uniform(4.0, 16.0, size=3)
        vs = rng.uniform(150.0, 1200.0)
        vp = vs * rng.uniform(2.0, 3.0)
        rho = rng.uniform(1600.0, 2300.0)
        inside = (((xc - c[0]) / ax[0]) ** 2 + ((yc - c[1]) / ax[1]) ** 2
                  + ((zc - c[2]) / ax[2]) ** 2) <= 1.0
        table.append([vp, vs, rho])
        mat[inside] = len(table) - 1
    rec = [(8 + 16 * a, 8 + 16 * b, nz) for b in range(8) for a in range(8)]
    return _mesh((nx, ny, nz), 1.0, mat, table, _source((64, 64, 32), 5.0), rec, 2000,
                 "config2_128x128x64")


def config3(seed: int = 3, shape=(512, 512, 256)):
    """Ten dipping layers, smoothed random topography (void above), 5,000 steps."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    field = rng.standard_normal((ny, nx))
    sigma = 32.0 * nx / 512.0
    fy = np.fft.fftfreq(ny)[:, None]
    fx = np.fft.fftfreq(nx)[None, :]
    smooth = np.real(np.fft.ifft2(np.fft.fft2(field) * np.exp(-2.0 * (np.pi * sigma) ** 2
                                                              * (fx ** 2 + fy ** 2))))
    smooth = smooth / np.max(np.abs(smooth))
    relief = 32.0 * nz / 256.0
    surface = np.round(224.0 * nz / 256.0 + relief * smooth).astype(np.int64)  # first void k
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    depth = (nz - kk - 0.5) + (ii + 0.5 - nx / 2.0) * np.tan(np.radians(10.0))
    layer = np.clip(np.floor(depth * 10.0 / nz), 0, 9).astype(np.int64)
    mat = np.where(kk >= surface[None, :, :], -1, layer)
    table = []
    for l in range(10):
        vs = 200.0 + 1800.0 * l / 9.0
        table.append([2.2 * vs, vs, 1700.0 + 800.0 * l / 9.0])
    src = (nx // 2, ny // 2, nz // 2)
    rec = []
    for b in range(8):
        for a in range(8):
            i, j = nx // 16 + a * nx // 8, ny // 16 + b * ny // 8
            rec.append((i, j, int(min(surface[j, i], surface[j, max(i - 1, 0)],
                                      surface[max(j - 1, 0), i],
                                      surface[max(j - 1, 0), max(i - 1, 0)]))))
    return _mesh((nx, ny, nz), 1.0, mat, table, _source(src, 5.0), rec, 5000,
                 "config3_%dx%dx%d" % (nx, ny, nz))


def config4(seed: int = 4, n_models: int = 64, n_min: int = 32, n_max: int = 128):
    """Many-case batch: independent cubic three-layer models of uneven sizes."""
    rng = np.random.default_rng(seed)
    models = []
    for i in range(n_models):
        n = int(rng.integers(n_min, n_max + 1))
        vs = rng.uniform(200.0, 1000.0, size=3)
        table = [[2.5 * v, v, float(rng.uniform(1700.0, 2300.0))] for v in vs]
        b1, b2 = sorted(rng.integers(1, n, size=2))
        k = np.arange(n)[:, None, None] * np.ones((n, n, n), dtype=np.int64)
        mat = np.where(k >= b2, 0, np.where(k >= b1, 1, 2))
        src = (int(rng.integers(1, n)), int(rng.integers(1, n)), int(rng.integers(1, n)))
        rec = [(n // 4 + a * n // 2, n // 4 + b * n // 2, n) for b in range(2) for a in range(2)]
        models.append(_mesh((n, n, n), 1.0, mat, table,
                            _source(src, float(rng.uniform(3.0, 10.0))), rec, 1000,
                            "config4_model%02d_%d" % (i, n)))
    return models


def config5(anomaly: bool = True, n: int = 96, nsteps: int = 1500):
    """Two layers with (or without) a spherical low-velocity anomaly."""
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    table = [[1500.0, 600.0, 1900.0], [2500.0, 1000.0, 2100.0], [2500.0, 700.0, 2100.0]]
    mat = np.where(kk >= n // 2, 0, 1)
    if anomaly:
        r = n / 8.0
        c = n / 2.0
        sphere = ((ii + 0.5 - c) ** 2 + (jj + 0.5 - c) ** 2 + (kk + 0.5 - c) ** 2) <= r * r
        mat = np.where(sphere, 2, mat)
    step = n // 6
    rec = [(step // 2 + a * step, step // 2 + b * step, n) for b in range(6) for a in range(6)]
    return _mesh((n, n, n), 1.0, mat, table, _source((n // 2, n // 2, n), 20.0), rec, nsteps,
                 "config5_%d%s" % (n, "_anomaly" if anomaly else "_background"))


def paper_rebar():
    """Concrete block with a rebar, sized like the paper's ultrasonic model."""
    ds = 2e-3
    nx, ny, nz = 162, 64, 192
    kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    xc, zc = (ii + 0.5) * ds, (kk + 0.5) * ds
    rebar = (xc - 0.160) ** 2 + (zc - 0.100) ** 2 <= 0.015 ** 2
    mat = np.where(rebar, 1, 0)
    table = [[4000.0, 2400.0, 2300.0], [5900.0, 3200.0, 7850.0]]
    src = _source((78, 36, 192), 112.5e3, 4.096e-4)
    rec = [(int(round(x / 2.0)), 30, 192) for x in (26, 60, 108, 144, 180, 216, 264, 300)]
    w = _mesh((nx, ny, nz), ds, mat, table, src, rec, 16384, "paper_rebar_162x64x192")
    w["dt"] = 5e-8
    w["fix_bottom"] = 2   # the four bottom corner points fixed, as in the experiment
    return w


def random_mesh(seed: int, shape=None, n_mat: int = 3, void_frac: float = 0.1, h=None):
    """Small random mesh with random materials and void cells (parity tests)."""
    rng = np.random.default_rng(seed)
    if shape is None:
        shape = tuple(int(v) for v in rng.integers(2, 9, size=3))
    nx, ny, nz = shape
    h = float(rng.uniform(0.5, 2.0)) if h is None else float(h)
    vs = rng.uniform(150.0, 1500.0, size=n_mat)
    table = np.stack([vs * rng.uniform(1.8, 3.5, size=n_mat), vs,
                      rng.uniform(1500.0, 2600.0, size=n_mat)], axis=1)
    mat = rng.integers(0, n_mat, size=(nz, ny, nx))
    mat[rng.random((nz, ny, nx)) < void_frac] = -1
    src = (int(rng.integers(0, nx + 1)), int(rng.integers(0, ny + 1)), int(rng.integers(1, nz + 1)))
    rec = [(int(rng.integers(0, nx + 1)), int(rng.integers(0, ny + 1)), int(rng.integers(0, nz + 1)))
           for _ in range(5)]
    return _mesh((nx, ny, nz), h, mat, table, _source(src, float(rng.uniform(3, 12))),
                 rec, 50, "random_%d" % seed)


def random_displacement(mesh, seed: int, scale: float = 1e-3):
    """Seeded random nodal displacement [N*3] (uniform in +-scale)."""
    nx, ny, nz = mesh["shape"]
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=3 * (nx + 1) * (ny + 1) * (nz + 1))


def receiver_nodes(mesh):
    return np.array([node_index(mesh["shape"], *r) for r in mesh["receivers"]], dtype=np.int64)


def source_node(mesh):
    return node_index(mesh["shape"], *mesh["source"]["ijk"])
