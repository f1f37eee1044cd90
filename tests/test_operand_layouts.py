"""A CPU model of how tcgen05.mma (kind::f16, no swizzle) reads its shared-
memory operands from (start, LBO, SBO) descriptors, used on two layouts.

1. The element-path layout of tc_step_kernel: node-digit blocks of 8 nodes x
   8 K-rows (3 components at x-shift 0 and 1, two magic-bias rows), A
   MN-major with SBO = 128 B and LBO = 256 B (the dy = 1 corner is the next
   node row), B K-major with N groups at 128 B and K groups at 768 B.  The
   model must reproduce P = K^kappa q_e and Q = K^G' q_e per element (plus the
   magic bias), as the GPU tests show the kernel does bit for bit.
2. The node-pair layout for uniform-material regions: an M row is a pair of
   adjacent x-nodes, K rows are 4 x-shifts x 3 components, one MMA per
   neighbour row (dy, dz) and digit stage.  The model must reproduce both
   nodes' 27-point integer stencils (Eq. GE:TC summed over a node's eight
   elements) exactly, with every partial sum exact in fp32.
"""
import importlib.util
import os
from fractions import Fraction

import numpy as np

from tests.closed_forms import OV_ALPHA, element_closed_form

MAGIC_A, MAGIC_B = 128.0, 12288.0


def read_mn_major(img, start, lbo, sbo, rows, K=16):
    """A[m][k]: core matrices of 8 K-rows x 8 MN-elements (16 B per K-row),
    MN groups of 8 at sbo bytes, K groups of 8 at lbo bytes."""
    m = np.arange(rows)[:, None]
    k = np.arange(K)[None, :]
    off = start + (m // 8) * sbo + (k // 8) * lbo + (k % 8) * 16 + (m % 8) * 2
    return img[off // 2]


def read_k_major(img, start, lbo, sbo, rows, K=16):
    """B[n][k]: core matrices of 8 N-rows x 8 K-values (16 B per N-row), N
    groups of 8 at sbo bytes, K groups of 8 at lbo bytes."""
    n = np.arange(rows)[:, None]
    k = np.arange(K)[None, :]
    off = start + (n // 8) * sbo + (k // 8) * lbo + (n % 8) * 16 + (k % 8) * 2
    return img[off // 2]


def _int_parts():
    Kk = element_closed_form(OV_ALPHA, 1, 1, 0, exact=True)
    Kg = element_closed_form(OV_ALPHA, 1, Fraction(-2, 3), 1, exact=True)
    return (np.array([[int(256 * v) for v in r] for r in Kk]),
            np.array([[int(384 * v) for v in r] for r in Kg]))


def _stencils():
    spec = importlib.util.spec_from_file_location(
        "node_stencil", os.path.join(os.path.dirname(__file__), "test_node_stencil.py"))
    ns = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(ns)
    Ik, Ig = _int_parts()
    return ns._node_stencil(Ik.tolist()), ns._node_stencil(Ig.tolist())


def test_element_path_layout():
    Ik, Ig = _int_parts()
    rng = np.random.default_rng(0)
    nodes = 17                                    # 16 elements + 1 per tile row
    q = rng.integers(-1024, 1024, size=(2, nodes, nodes, 3))   # planes L, L+1: [z][y][x][c]
    plane_bytes = nodes * 2 * 128                 # 17 node rows x 2 x-chunks x 128 B
    img = np.zeros(2 * plane_bytes // 2)
    for z in range(2):
        for row in range(nodes):
            for chunk in range(2):
                b = z * plane_bytes + (row * 2 + chunk) * 128
                for c in range(3):
                    for i in range(8):
                        x = 8 * chunk + i
                        img[(b + c * 16 + i * 2) // 2] = q[z, row, x, c]
                        img[(b + (3 + c) * 16 + i * 2) // 2] = q[z, row, x + 1, c] if x + 1 < nodes else 0
                for line in (6, 7):
                    img[(b + line * 16) // 2:(b + line * 16 + 16) // 2] = MAGIC_A
    # B: 48 outputs n = 12 corner-group + 6 dx + 3 part + component; K = 8 kg + l
    bop = np.zeros(48 * 32)
    for kg in range(4):
        for ng in range(6):
            for r in range(8):
                n = 8 * ng + r
                go, rem = n // 12, n % 12
                dxo, part, co = rem // 6, (rem % 6) // 3, rem % 3
                ao = dxo + 2 * (go & 1) + 4 * (go >> 1)
                for l in range(8):
                    if l >= 6:
                        v = MAGIC_B
                    else:
                        col = 3 * (l // 3 + 2 * (kg & 1) + 4 * (kg >> 1)) + l % 3
                        v = (Ik if part == 0 else Ig)[3 * ao + co, col]
                    bop[((kg * 6 + ng) * 8 + r) * 8 + l] = v
    bias = 8 * MAGIC_A * MAGIC_B                  # 1.5 2^23: the accumulator's start
    assert bias == 1.5 * 2 ** 23
    for mt in range(2):
        D = sum(read_mn_major(img, ks * plane_bytes + 16 * mt * 128, 256, 128, 128)
                @ read_k_major(bop, ks * 2 * 6 * 128, 6 * 128, 128, 48).T for ks in range(2))
        for m in range(128):
            ex, ey = m % 16, 8 * mt + m // 16
            qe = np.array([q[a >> 2, ey + ((a >> 1) & 1), ex + (a & 1), c]
                           for a in range(8) for c in range(3)])
            P, Q = Ik @ qe, Ig @ qe
            want = []
            for n in range(48):
                go, rem = n // 12, n % 12
                dxo, part, co = rem // 6, (rem % 6) // 3, rem % 3
                ao = dxo + 2 * (go & 1) + 4 * (go >> 1)
                want.append((P if part == 0 else Q)[3 * ao + co])
            assert np.array_equal(D[m] - bias, np.array(want, dtype=float)), (mt, m)


def test_node_pair_layout():
    Sk, Sg = _stencils()
    rng = np.random.default_rng(2)
    n = 18                                        # 16 owned-tile nodes + a halo node each side
    q = rng.integers(-1024, 1024, size=(3, n, n, 3))   # planes z-1, z, z+1
    row_bytes = 256                               # 8 pairs x 16 K-rows x 2 B per node row
    plane_bytes = n * row_bytes
    img = np.zeros(3 * plane_bytes // 2)
    for z in range(3):
        for y in range(n):
            b = z * plane_bytes + y * row_bytes
            for d in range(4):                    # x-shift d - 1 from the pair's first node
                for c in range(3):
                    for p in range(8):
                        img[(b + (3 * d + c) * 16 + p * 2) // 2] = q[z, y, 1 + 2 * p + d - 1, c]
    groups = [(dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1)]
    bimg = np.zeros(len(groups) * 16 * 16)
    for gi, (dy, dz) in enumerate(groups):
        for col in range(12):                     # (node j, part, component)
            j, part, co = col // 6, (col % 6) // 3, col % 3
            for k in range(12):
                d, c = k // 3, k % 3
                ox = (d - 1) - j
                if abs(ox) <= 1:
                    v = (Sk if part == 0 else Sg)[(ox, dy, dz)][co, c]
                    off = gi * 512 + (col // 8) * 128 + (k // 8) * 256 + (col % 8) * 16 + (k % 8) * 2
                    bimg[off // 2] = v
    D = sum(read_mn_major(img, (1 + dz) * plane_bytes + (1 + dy) * row_bytes, 128, 256, 128)
            @ read_k_major(bimg, gi * 512, 256, 128, 16).T for gi, (dy, dz) in enumerate(groups))
    assert np.abs(D).max() < 2 ** 24
    for m in range(128):
        p, y = m % 8, m // 8
        for j in range(2):
            x = 2 * p + j
            P = sum(blk @ q[1 + oz, 1 + y + oy, 1 + x + ox] for (ox, oy, oz), blk in Sk.items())
            Q = sum(blk @ q[1 + oz, 1 + y + oy, 1 + x + ox] for (ox, oy, oz), blk in Sg.items())
            assert np.array_equal(D[m, 6 * j:6 * j + 3], P)
            assert np.array_equal(D[m, 6 * j + 3:6 * j + 6], Q)
        assert not D[m, 12:].any()
