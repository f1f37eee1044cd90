"""GPU parity of K u (Section 2, Eq. OVFEMstiff / Eq. GE:TC) against the
FP64 oracle, and bit-exactness of the tensor-core integer partial products."""
from fractions import Fraction

import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.closed_forms import OV_ALPHA, element_closed_form
from tests.gpu_common import KU_TOL, PATHS, rel_max

pytestmark = pytest.mark.gpu

SHAPES = [(1, 1, 1), (3, 2, 2), (17, 5, 4), (15, 15, 3), (16, 16, 2), (31, 16, 9),
          (33, 31, 9), (14, 47, 5), (7, 3, 40)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("path", ["tc", "fp64"])
def test_ku_matches_oracle(orc, shape, path):
    mesh = W.random_mesh(sum(shape), shape=shape, void_frac=0.15)
    u = W.random_displacement(mesh, 7)
    ref = orc.ku(0, mesh, u)
    with vfe.Mesh(mesh, path=PATHS[path], source=False, receivers=False) as m:
        f = m.internal_force(u)
    assert rel_max(f, ref) <= KU_TOL


@pytest.mark.parametrize("shape", [(4, 3, 5), (17, 16, 3)])
def test_ku_vfem_fp64(orc, shape):
    mesh = W.random_mesh(50 + sum(shape), shape=shape, void_frac=0.1)
    u = W.random_displacement(mesh, 8)
    ref = orc.ku(1, mesh, u)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_FP64, kind=vfe.VFE_VFEM, source=False,
                  receivers=False) as m:
        f = m.internal_force(u)
    assert rel_max(f, ref) <= KU_TOL


def _exact_int_matrices():
    Kk = element_closed_form(OV_ALPHA, 1, 1, 0, exact=True)
    Kg = element_closed_form(OV_ALPHA, 1, Fraction(-2, 3), 1, exact=True)
    return ([[int(256 * v) for v in row] for row in Kk],
            [[int(384 * v) for v in row] for row in Kg])


@pytest.mark.parametrize("shape", [(3, 2, 2), (17, 5, 4), (33, 31, 9)])
def test_tc_partials_bit_exact(shape):
    """The tensor core's integer partial products equal exact integer
    arithmetic: P = K^kappa q_e and Q = K^G' q_e for the digitised inputs."""
    mesh = W.random_mesh(100 + sum(shape), shape=shape, void_frac=0.1)
    u = W.random_displacement(mesh, 9)
    nx, ny, nz = shape
    ne = nx * ny * nz
    ids = np.arange(ne) if ne <= 300 else np.random.default_rng(1).choice(ne, 300, replace=False)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False) as m:
        out, sh, F = vfe.vfe_debug_tc_partials(m.handle, u, ids)
    q = np.rint(np.ldexp(u, F)).astype(np.int64) >> sh
    Kk, Kg = _exact_int_matrices()
    for row, e in zip(out, ids):
        i, j, k = e % nx, (e // nx) % ny, e // (nx * ny)
        qe = []
        for a in range(8):
            n = W.node_index(shape, i + (a & 1), j + ((a >> 1) & 1), k + (a >> 2))
            qe += [int(q[3 * n + c]) for c in range(3)]
        exp = [sum(Kk[r][s] * qe[s] for s in range(24)) for r in range(24)]
        exp += [sum(Kg[r][s] * qe[s] for s in range(24)) for r in range(24)]
        assert [int(v) for v in row] == exp, e


def test_ku_full_size_sampled(orc):
    """128x128x64 (1.05 M elements) in the launch configuration the step uses:
    sampled nodes against the oracle computed one node at a time, plus the
    rigid-translation property everywhere."""
    mesh = W.config2()
    u = W.random_displacement(mesh, 11)
    nn = len(u) // 3
    sel = np.random.default_rng(2).choice(nn, 2000, replace=False)
    ref = orc.ku_nodes(0, mesh, u, sel)
    for path in ("tc", "fp64"):
        with vfe.Mesh(mesh, path=PATHS[path], source=False, receivers=False) as m:
            f = m.internal_force(u).reshape(-1, 3)
            assert rel_max(f[sel], ref) <= KU_TOL, path
            t = np.zeros(3 * nn); t[2::3] = 1e-3
            ft = m.internal_force(t)
            assert np.abs(ft).max() <= 1e-12 * np.abs(f).max() * 1e3, path


@pytest.mark.parametrize("path", ["tc", "fp64"])
@pytest.mark.parametrize("bit,code", [(1, vfe.VFE_ETIMEOUT), (2, vfe.VFE_ETIMEOUT),
                                      (4, vfe.VFE_ECUDA)])
def test_status_word_is_reported(path, bit, code):
    """A failure flagged on the device (injected from the host here, as a
    kernel flags a bounded wait that gave up) fails the calls that read it."""
    mesh = W.random_mesh(61, shape=(6, 5, 4), void_frac=0.0)
    with vfe.Mesh(mesh, path=PATHS[path], source=False, receivers=False) as m:
        assert vfe.load().vfe_debug_inject_status(m.handle, bit) == vfe.VFE_OK
        with pytest.raises(vfe.VfeError) as e:
            m.internal_force(W.random_displacement(mesh, 1))
        assert e.value.code == code
        m.step(1)
        with pytest.raises(vfe.VfeError) as e:
            m.synchronize()
        assert e.value.code == code
