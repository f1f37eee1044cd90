"""Rayleigh coefficients of the C ABI (host-only call, no GPU): the damping
ratio h(w) = alpha / (2 w) + beta w / 2 of C = alpha M + beta K equals h at
both given frequencies and stays below it between them."""
import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe


@pytest.mark.parametrize("h,f1,f2", [(0.02, 100e3, 125e3), (0.05, 3.0, 10.0), (0.01, 7.0, 7.0)])
def test_rayleigh_ratio_hits_both_frequencies(h, f1, f2):
    alpha, beta = vfe.vfe_rayleigh_coefficients(h, f1, f2)
    ratio = lambda f: alpha / (4 * np.pi * f) + beta * np.pi * f
    assert ratio(f1) == pytest.approx(h, rel=1e-14)
    assert ratio(f2) == pytest.approx(h, rel=1e-14)
    for f in np.linspace(f1, f2, 7)[1:-1]:
        assert ratio(f) <= h * (1 + 1e-14)


@pytest.mark.parametrize("args", [(-0.1, 1.0, 2.0), (0.1, 0.0, 2.0), (0.1, 3.0, 2.0)])
def test_rayleigh_rejects_bad_input(args):
    with pytest.raises(vfe.VfeError) as e:
        vfe.vfe_rayleigh_coefficients(*args)
    assert e.value.code == vfe.VFE_EINVAL
