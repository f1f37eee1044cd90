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
