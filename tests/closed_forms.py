"""Hand-derived closed forms used to pin the oracle (test helpers only).

Both voxel elements share one closed form.  With local node signs s^a in
{-1,1}^3 (a = dx + 2dy + 4dz, s = 2d - 1),

  S_kl(a,b) = (1/16) s^a_k s^b_l  prod_{m not in {k,l}} (1 + alpha s^a_m s^b_m)
  K_{(a,i),(b,j)} = ds [ lambda S_ij + G S_ji + G delta_ij sum_k S_kk ],

alpha = 3/4 for the orthogonal element (Heaviside phi, seven psi bases:
sum over psi of (psi grad phi^a)(psi grad phi^b)/Gram gives the products
(1 + 3/4 ...)) and alpha = 1/3 for the trilinear element (exact 2x2x2 Gauss
of products of (1 + s r) factors).  Derived by hand from the definitions in
arXiv 2404.13683, Section 2; independent of the oracle's quadrature code.
"""
from fractions import Fraction

import numpy as np


def sign(a, k):
    return 1 if (a >> k) & 1 else -1


def s_matrix(alpha, a, b, k, l):
    v = Fraction(1, 16) * sign(a, k) * sign(b, l)
    for m in range(3):
        if m != k and m != l:
            v *= 1 + alpha * sign(a, m) * sign(b, m)
    return v


def element_closed_form(alpha, ds, lam, G, exact=False):
    """24x24 element matrix; Fractions if exact else float64."""
    K = [[0] * 24 for _ in range(24)]
    for a in range(8):
        for b in range(8):
            S = [[s_matrix(alpha, a, b, k, l) for l in range(3)] for k in range(3)]
            tr = S[0][0] + S[1][1] + S[2][2]
            for i in range(3):
                for j in range(3):
                    K[3 * a + i][3 * b + j] = ds * (lam * S[i][j] + G * S[j][i]
                                                   + (G * tr if i == j else 0))
    if exact:
        return K
    return np.array([[float(x) for x in row] for row in K])


OV_ALPHA = Fraction(3, 4)
V_ALPHA = Fraction(1, 3)


def kint8_exact():
    """K^INT8 = (256/ds K_e|kappa=1,G=0 , 384/ds K_e|kappa=0,G=1 - 128 I)."""
    Kk = element_closed_form(OV_ALPHA, 1, 1, 0, exact=True)          # lambda = kappa = 1
    Kg = element_closed_form(OV_ALPHA, 1, Fraction(-2, 3), 1, exact=True)  # lambda = -2/3 G
    out = [[0] * 48 for _ in range(24)]
    for m in range(24):
        for n in range(24):
            out[m][n] = 256 * Kk[m][n]
            out[m][24 + n] = 384 * Kg[m][n] - (128 if m == n else 0)
    return out


def node_positions(ds):
    return np.array([[ds / 2 * sign(a, k) for k in range(3)] for a in range(8)])


def rigid_modes(ds):
    """6 rigid-body modes (3 translations, 3 rotations) as 24-vectors."""
    x = node_positions(ds)
    modes = []
    for c in range(3):
        t = np.zeros(24); t[c::3] = 1.0; modes.append(t)
    for axis in range(3):
        w = np.zeros(3); w[axis] = 1.0
        r = np.cross(np.broadcast_to(w, x.shape), x)
        modes.append(r.reshape(-1))
    return np.array(modes)
