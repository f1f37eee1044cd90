"""Pins of the TCOVFEM integer reformulation (Section 2, K^INT8, Eq. GE:TC,
Eqs. intscaling, intcomp1-3, int8comp1-2) in the oracle."""
from fractions import Fraction

import numpy as np
import pytest

from tests.closed_forms import OV_ALPHA, element_closed_form, kint8_exact


def test_kint8_equals_exact_integers(orc):
    ref = np.array([[float(v) for v in row] for row in kint8_exact()])
    assert all(v.denominator == 1 for row in kint8_exact() for v in row)
    for ds in (1.0, 0.37, 2e-3):
        K = orc.kint8(ds)
        assert np.abs(K - ref).max() < 1e-9, ds       # independent of ds


def test_kint8_int8_range(orc):
    K = np.round(orc.kint8(1.0)).astype(int)
    Kk, Kg = K[:, :24], K[:, 24:]
    assert Kk.min() == -49 and Kk.max() == 49 and (np.diag(Kk) == 49).all()
    assert Kg.min() == -77 and Kg.max() == 117 and (np.diag(Kg) == 117).all()
    assert np.abs(K).sum(axis=1).max() == 1130
    assert -128 <= K.min() and K.max() <= 127


def test_ge_tc_identity_exact():
    # Eq. GE:TC in exact rationals: K_e u = kappa ds/256 (K^INT8 ubar + 256/3 G/kappa u)
    rng = np.random.default_rng(5)
    Ki = kint8_exact()
    kappa, G, ds = Fraction(7, 2), Fraction(5, 4), Fraction(3, 10)
    Ke = element_closed_form(OV_ALPHA, ds, kappa - Fraction(2, 3) * G, G, exact=True)
    u = [Fraction(float(v)) for v in rng.uniform(-1, 1, 24)]
    ubar = u + [Fraction(2, 3) * G / kappa * v for v in u]
    for m in range(24):
        lhs = sum(Ke[m][n] * u[n] for n in range(24))
        rhs = kappa * ds / 256 * (sum(Ki[m][n] * ubar[n] for n in range(48))
                                  + Fraction(256, 3) * G / kappa * u[m])
        assert lhs == rhs


def _exact_ku(ds, kappa, G, ue):
    Ke = element_closed_form(OV_ALPHA, Fraction(ds), Fraction(kappa) - Fraction(2, 3) * Fraction(G),
                             Fraction(G), exact=True)
    uf = [Fraction(float(v)) for v in ue]
    return [sum(Ke[m][n] * uf[n] for n in range(24)) for m in range(24)]


@pytest.mark.parametrize("seed", range(4))
def test_tc_fp64_matches_definition(orc, seed):
    rng = np.random.default_rng(seed)
    ds, kappa, G = 2e-3, rng.uniform(1e9, 3e10), rng.uniform(1e8, 1e10)
    ue = rng.uniform(-1e-6, 1e-6, 24)
    f = orc.ku_element_tc_fp64(ds, kappa, G, ue)
    K = orc.element_stiffness(0, ds, kappa, G)
    ref = K @ ue
    assert np.abs(f - ref).max() <= 1e-13 * np.abs(ref).max()


def _int_error_bound(ds, kappa, G, ue, M):
    ubar = np.concatenate([ue, 2.0 / 3.0 * G / kappa * ue])
    se = np.abs(ubar).max()
    # each of the 48 inputs is truncated by < s_e 2^-7M; |K^INT8| row L1 <= 1130
    return kappa * ds / 256.0 * se * 1130 * 2.0 ** (-7 * M)


@pytest.mark.parametrize("seed", range(6))
def test_tc_int_stages_precision(orc, seed):
    """Table 3 pattern: M=8 agrees with the exact value to FP64 level, M=4 to
    roughly FP32 level, and every M stays inside its truncation bound."""
    rng = np.random.default_rng(100 + seed)
    ds, kappa, G = 2e-3, rng.uniform(1e9, 3e10), rng.uniform(1e8, 1e10)
    ue = rng.uniform(-1, 1, 24) * 10.0 ** rng.uniform(-9, -3)
    exact = np.array([float(v) for v in _exact_ku(ds, kappa, G, ue)])
    fscale = np.abs(exact).max()
    errs = {}
    for M in range(1, 9):
        f = orc.ku_element_tc_int(ds, kappa, G, M, ue)
        err = np.abs(f - exact).max()
        bound = _int_error_bound(ds, kappa, G, ue, M) + 64 * 2.0 ** -52 * fscale
        assert err <= bound, (M, err, bound)
        errs[M] = err / fscale
    assert errs[8] < 1e-14
    assert 1e-12 < errs[4] < 1e-6
    assert errs[2] > errs[4] > errs[8]


def test_tc_int_zero_and_scaling(orc):
    z = orc.ku_element_tc_int(1.0, 2.0, 1.0, 8, np.zeros(24))
    assert (z == 0).all()
    # scaling u by a power of two scales the result exactly (s_e absorbs it)
    rng = np.random.default_rng(9)
    ue = rng.uniform(-1, 1, 24)
    a = orc.ku_element_tc_int(1.0, 2.0, 1.0, 8, ue)
    b = orc.ku_element_tc_int(1.0, 2.0, 1.0, 8, ue * 2.0 ** -20)
    assert np.array_equal(a * 2.0 ** -20, b)


def test_direct_expansion_equivalence():
    """Eqs. intcomp1-3 with a = 2^7, N = M and the hierarchical INT64 -> INT8
    split give the same integer sum (the text after Eq. int8comp2):  emulated
    here on random scaled vectors in exact integers."""
    rng = np.random.default_rng(3)
    for _ in range(50):
        us = rng.uniform(-1, 1)
        M = 8
        # direct: ubar_INT(i) = trunc(a * residual), residual scaled by a each stage
        digits, res = [], Fraction(us)
        for _i in range(M):
            d = int(res * 128)          # trunc toward zero
            digits.append(d)
            res = res * 128 - d
        direct = sum(d * 128 ** (M - 1 - i) for i, d in enumerate(digits))
        hier = int(Fraction(us) * 2 ** 56)
        assert direct == hier
