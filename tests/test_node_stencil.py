"""The node-level form of Eq. GE:TC on a uniform material: summed over the
eight elements around a node, the integer matrices K^kappa = 256/ds K_e(1, 0)
and K^G' = 384/ds K_e(0, 1) (the paper's K-bar^G + 128 I, Section 2) become
one 27-point integer stencil per part, and K u at the node is
ds (kappa/256 S^kappa u + G/384 S^G' u).  Checked against the oracle's
element-by-element K u, with the bounds that keep fp32 tensor-core partial
sums exact for 11-bit (and 12-bit) digits."""
from fractions import Fraction

import numpy as np

from paper_2404_13683_gb300 import workloads as W
from tests.closed_forms import OV_ALPHA, element_closed_form


def _integer_parts():
    Kk = element_closed_form(OV_ALPHA, 1, 1, 0, exact=True)
    Kg = element_closed_form(OV_ALPHA, 1, Fraction(-2, 3), 1, exact=True)
    Ik = [[int(256 * v) for v in row] for row in Kk]
    Ig = [[int(384 * v) for v in row] for row in Kg]
    assert all(256 * v == Ik[i][j] for i, row in enumerate(Kk) for j, v in enumerate(row))
    assert all(384 * v == Ig[i][j] for i, row in enumerate(Kg) for j, v in enumerate(row))
    assert Ig[0][0] == 245   # the paper's K-bar^G diagonal 117 plus 128
    return Ik, Ig


def _node_stencil(I):
    """S[(ox, oy, oz)][i][j]: output component i of a node, input component j
    of the node at offset o, summed over the node's eight elements."""
    S = {}
    for e in range(8):
        o = (-(e & 1), -((e >> 1) & 1), -((e >> 2) & 1))   # the element's corner offset
        a = -o[0] - 2 * o[1] - 4 * o[2]                     # the node's local index in it
        for b in range(8):
            off = (o[0] + (b & 1), o[1] + ((b >> 1) & 1), o[2] + ((b >> 2) & 1))
            blk = S.setdefault(off, np.zeros((3, 3), dtype=np.int64))
            for i in range(3):
                for j in range(3):
                    blk[i, j] += I[3 * a + i][3 * b + j]
    return S


def test_stencil_bounds():
    Ik, Ig = _integer_parts()
    for I, max_entry, row_l1 in ((Ik, 392, 1536), (Ig, 1960, 4176)):
        S = _node_stencil(I)
        assert len(S) == 27
        allv = np.stack(list(S.values()))
        assert np.abs(allv).max() == max_entry
        rows = np.abs(allv).sum(axis=(0, 2))
        assert (rows == row_l1).all()
        assert (allv != 0).sum() == 153
        # fp32 holds every integer below 2^24: 11- and 12-bit balanced digits
        assert row_l1 * 1024 < 2 ** 24 and row_l1 * 2048 < 2 ** 24


def test_stencil_reproduces_element_by_element_ku(orc):
    """On a uniform mesh, every interior node's K u from the two stencils
    equals the oracle's element-by-element K u."""
    Ik, Ig = _integer_parts()
    Sk, Sg = _node_stencil(Ik), _node_stencil(Ig)
    n = 5
    mesh = W.random_mesh(3, shape=(n, n, n), n_mat=1, void_frac=0.0)
    vp, vs, rho = mesh["material_table"][0]
    G, kap = rho * vs * vs, rho * (vp * vp - 4.0 / 3.0 * vs * vs)
    ds = mesh["h"]
    u = W.random_displacement(mesh, 5).reshape(-1, 3)
    ref = orc.ku(0, mesh, u.reshape(-1)).reshape(-1, 3)
    nid = lambda i, j, k: i + (n + 1) * (j + (n + 1) * k)
    for k in range(1, n):
        for j in range(1, n):
            for i in range(1, n):
                P = np.zeros(3)
                Q = np.zeros(3)
                for (ox, oy, oz), blk in Sk.items():
                    v = u[nid(i + ox, j + oy, k + oz)]
                    P += blk @ v
                    Q += Sg[(ox, oy, oz)] @ v
                c = nid(i, j, k)
                f = ds * (kap / 256.0 * P + G / 384.0 * Q)
                assert np.abs(f - ref[c]).max() <= 1e-12 * np.abs(ref).max()


def _mask_parts(I, mask):
    """{offset: 3x3} of the rows of the node summed over the elements of the
    octant mask (bit o: element origin (i - (o & 1), j - (o >> 1 & 1),
    k - (o >> 2)) of node (i, j, k))."""
    S = {}
    for e in range(8):
        if not (mask >> e) & 1:
            continue
        o = (-(e & 1), -((e >> 1) & 1), -((e >> 2) & 1))
        a = -o[0] - 2 * o[1] - 4 * o[2]
        for b in range(8):
            off = (o[0] + (b & 1), o[1] + ((b >> 1) & 1), o[2] + ((b >> 2) & 1))
            blk = S.setdefault(off, np.zeros((3, 3), dtype=np.int64))
            for i in range(3):
                for j in range(3):
                    blk[i, j] += I[3 * a + i][3 * b + j]
    return S


def test_mask_table_size_and_bounds():
    """The correction table's rows (the offsets each of the 255 octant masks
    reaches) number 5,023, the value the library's operand buffer is laid
    out for, and every subset row L1 norm of K^kappa and of K-bar^G = K^G' -
    128 I stays below 4,096, so that the corrections' int64 sums of q' (below
    2^51) cannot overflow."""
    import os
    import re
    Ik, Ig = _integer_parts()
    Igb = [[Ig[r][c] - (128 if r == c else 0) for c in range(24)] for r in range(24)]
    rows, worst = 0, 0
    for mask in range(256):
        Sk, Sg = _mask_parts(Ik, mask), _mask_parts(Igb, mask)
        rows += len(Sk)
        if Sk:
            worst = max(worst, max(np.abs(np.stack(list(S.values()))).sum(axis=(0, 2)).max()
                                   for S in (Sk, Sg)))
    assert worst == 3152 and worst < 4096   # the largest: all eight elements, K-bar^G
    hdr = os.path.join(os.path.dirname(__file__), "..", "paper_2404_13683_gb300", "csrc",
                       "vfe_internal.h")
    with open(hdr) as f:
        m = re.search(r"#define ST_MASK_ROWS (\d+)", f.read())
    assert m and int(m.group(1)) == rows == 5023


def test_reference_material_plus_corrections_is_element_by_element_ku(orc):
    """The per-node form the tensor-core path uses on large meshes: each
    node's K u is the full node stencil with the node's reference material
    (the most frequent among its eight elements, first in octant order on a
    tie) plus, per other value among its elements (another material, or
    absent: void or outside the mesh), the mask's rows with the difference
    of the multipliers.  Checked at every node with a solid element of a
    random mesh (four materials, 25% voids, faces) against the oracle's
    element-by-element K u."""
    Ik, Ig = _integer_parts()
    mesh = W.random_mesh(12, shape=(6, 5, 4), n_mat=4, void_frac=0.25, h=1.0)
    nx, ny, nz = mesh["shape"]
    tab = mesh["material_table"]
    kap = tab[:, 2] * (tab[:, 0] ** 2 - 4.0 / 3.0 * tab[:, 1] ** 2)
    G = tab[:, 2] * tab[:, 1] ** 2
    mat = mesh["material_ids"].reshape(nz, ny, nx)
    ds = mesh["h"]
    u = W.random_displacement(mesh, 13).reshape(-1, 3)
    ref = orc.ku(0, mesh, u.reshape(-1)).reshape(-1, 3)
    nid = lambda i, j, k: i + (nx + 1) * (j + (ny + 1) * k)

    def elem(i, j, k):
        if 0 <= i < nx and 0 <= j < ny and 0 <= k < nz:
            return int(mat[k, j, i])
        return -1

    def apply(S, i, j, k):   # neighbours outside the mesh hold zero
        out = np.zeros(3)
        for (ox, oy, oz), blk in S.items():
            a, b, c = i + ox, j + oy, k + oz
            if 0 <= a <= nx and 0 <= b <= ny and 0 <= c <= nz:
                out += blk @ u[nid(a, b, c)]
        return out

    full_k, full_g = _mask_parts(Ik, 255), _mask_parts(Ig, 255)
    checked = corrected = 0
    for k in range(nz + 1):
        for j in range(ny + 1):
            for i in range(nx + 1):
                v = [elem(i - (o & 1), j - ((o >> 1) & 1), k - (o >> 2)) for o in range(8)]
                solid = [x for x in v if x >= 0]
                if not solid:
                    continue
                r = max(solid, key=lambda x: (v.count(x), -v.index(x)))
                f = ds * (kap[r] / 256.0 * apply(full_k, i, j, k) + G[r] / 384.0 * apply(full_g, i, j, k))
                for val in sorted(set(v) - {r}):
                    mask = sum(1 << o for o in range(8) if v[o] == val)
                    ka, ga = (kap[val], G[val]) if val >= 0 else (0.0, 0.0)
                    f = f + ds * ((ka - kap[r]) / 256.0 * apply(_mask_parts(Ik, mask), i, j, k) +
                                  (ga - G[r]) / 384.0 * apply(_mask_parts(Ig, mask), i, j, k))
                    corrected += 1
                assert np.abs(f - ref[nid(i, j, k)]).max() <= 1e-12 * np.abs(ref).max()
                checked += 1
    assert checked > 100 and corrected > 100
