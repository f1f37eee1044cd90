"""The node-stencil tensor-core kernel (uniform-material node planes).

Where every element around a column of nodes shares one material, the
tensor-core path forms K u per node: the element products of Eq. GE:TC summed
over a node's eight elements are one 27-point integer stencil per material
part.  Checked here

* bit for bit: the kernel's integer partial sums P = S^k q and S^G q, and the
  node's own q, against exact integer stencils built from the hand-derived
  closed form of the element (independent of the library), zero outside the
  mesh;
* K u against the FP64 oracle, on meshes with uniform blocks, material
  interfaces, voids and mesh faces, and against the element kernel alone
  (stencil off).  Without per-node corrections only the uniform runs go to
  the stencil kernel; with them (meshes of 8 Mi elements or more, or
  stencil=2) every column-plane does, each node taking the most frequent
  material around it, and a correction launch after the kernel exchanges
  the material of the node's other elements (another material, void, or
  outside the mesh);
* time steps from a state and from rest (source, receivers) against the
  oracle, and the state after steps with the stencil on and off.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2404_13683_gb300 import vfe
from paper_2404_13683_gb300 import workloads as W
from tests.closed_forms import OV_ALPHA, element_closed_form
from tests.gpu_common import KU_TOL, oracle_source, rel_l2, rel_max

pytestmark = pytest.mark.gpu


def _node_stencils():
    """S^k and S^G' (dict offset -> 3x3 int) of the integer element matrices
    K^kappa = 256 K_e(1, 0) and K^G' = 384 K_e(0, 1) at ds = 1, summed over
    the eight elements around a node."""
    Kk = element_closed_form(OV_ALPHA, 1, 1, 0, exact=True)
    Kg = element_closed_form(OV_ALPHA, 1, Fraction(-2, 3), 1, exact=True)
    Ik = [[int(256 * v) for v in r] for r in Kk]
    Ig = [[int(384 * v) for v in r] for r in Kg]
    out = []
    for I in (Ik, Ig):
        S = {}
        for e in range(8):
            o = (-(e & 1), -((e >> 1) & 1), -((e >> 2) & 1))
            a = -o[0] - 2 * o[1] - 4 * o[2]
            for b in range(8):
                off = (o[0] + (b & 1), o[1] + ((b >> 1) & 1), o[2] + ((b >> 2) & 1))
                blk = S.setdefault(off, np.zeros((3, 3), dtype=np.int64))
                for i in range(3):
                    for j in range(3):
                        blk[i, j] += I[3 * a + i][3 * b + j]
        out.append(S)
    return out


def layered(shape, seed=1, void_top=0, inclusion=True):
    """Horizontal layers (uniform runs) with an optional block inclusion and
    void cells on top (mixed and void runs)."""
    nx, ny, nz = shape
    k = np.arange(nz)[:, None, None] * np.ones((nz, ny, nx), dtype=np.int64)
    mat = np.where(k >= nz // 2, 0, 1)
    if inclusion:
        mat[nz // 3: nz // 3 + 3, ny // 3: ny // 3 + 4, nx // 2: nx // 2 + 5] = 2
    if void_top:
        mat[nz - void_top:] = -1
    table = [[1800.0, 700.0, 2000.0], [2600.0, 1100.0, 2200.0], [1500.0, 500.0, 1900.0]]
    rng = np.random.default_rng(seed)
    src = (nx // 2, ny // 2, nz // 2)
    rec = [(int(rng.integers(0, nx + 1)), int(rng.integers(0, ny + 1)), int(nz // 2 + 1))
           for _ in range(4)]
    return W._mesh(shape, 1.0, mat, table, W._source(src, 60.0), rec, 40,
                   "layered_%dx%dx%d" % shape)


SHAPES = [(47, 40, 12), (33, 31, 20), (64, 33, 9)]


@pytest.mark.parametrize("faces", [False, True])
@pytest.mark.parametrize("shape", SHAPES)
def test_stencil_partials_bit_exact(shape, faces):
    mesh = layered(shape)
    u = W.random_displacement(mesh, 3)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False,
                  stencil=2 if faces else 1) as m:
        out, cov, sh, F = vfe.vfe_debug_stencil_partials(m.handle, u)
    assert cov.sum() > 0, "the mesh has no uniform run"
    q = (np.rint(np.ldexp(u, F)).astype(np.int64) >> sh).reshape(-1, 3)
    Sk, Sg = _node_stencils()
    nx, ny, nz = shape
    idx = np.flatnonzero(cov)
    i, j, k = idx % (nx + 1), (idx // (nx + 1)) % (ny + 1), idx // ((nx + 1) * (ny + 1))
    on_face = (i == 0) | (i == nx) | (j == 0) | (j == ny) | (k == 0) | (k == nz)
    if faces:   # face, edge and corner nodes, and the material interfaces
        assert ((i == 0) | (i == nx)).any() and ((j == 0) | (j == ny)).any()
        assert (((i == 0) | (i == nx)) & ((j == 0) | (j == ny))).any()
        assert (k == 0).any() and (k == nz).any() and (k == nz // 2).any()
        assert ((k == 0) & (i == 0) & (j == 0)).any()
    else:
        assert not on_face.any()
    P = np.zeros((len(idx), 3), dtype=np.int64)
    Q = np.zeros((len(idx), 3), dtype=np.int64)
    for (ox, oy, oz), blk in Sk.items():
        # a neighbour outside the mesh holds zero
        inside = ((i + ox >= 0) & (i + ox <= nx) & (j + oy >= 0) & (j + oy <= ny) &
                  (k + oz >= 0) & (k + oz <= nz))
        nb = np.where(inside, (i + ox) + (nx + 1) * ((j + oy) + (ny + 1) * (k + oz)), 0)
        qn = q[nb] * inside[:, None]
        P += qn @ blk.T
        g = Sg[(ox, oy, oz)] - (1024 * np.eye(3, dtype=np.int64) if (ox, oy, oz) == (0, 0, 0) else 0)
        Q += qn @ g.T
    assert np.array_equal(out[idx, 0:3], P)
    assert np.array_equal(out[idx, 3:6], Q)
    assert np.array_equal(out[idx, 6:9], q[idx])
    assert not out[~cov].any()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("void_top", [0, 3])
def test_stencil_ku_matches_oracle(orc, shape, void_top):
    mesh = layered(shape, void_top=void_top)
    u = W.random_displacement(mesh, 7)
    ref = orc.ku(0, mesh, u)
    res = {}
    for on in (2, True, False):   # per-node corrections, uniform runs only, element kernel only
        with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False, stencil=on) as m:
            res[on] = m.internal_force(u)
        assert rel_max(res[on], ref) <= KU_TOL, on
    assert rel_max(res[True], res[False]) <= KU_TOL
    # nodes with no solid element feel no force
    massless = orc.node_mass(0, mesh) == 0
    assert not res[True].reshape(-1, 3)[massless].any()


@pytest.mark.parametrize("nsteps", [1, 5])
def test_stencil_steps_from_state(orc, nsteps):
    mesh = layered((47, 40, 12), void_top=2)
    mass = orc.node_mass(0, mesh)
    nx, ny, _ = mesh["shape"]
    free = mass > 0
    free[: (nx + 1) * (ny + 1)] = False
    rng = np.random.default_rng(8)
    u = rng.uniform(-1e-3, 1e-3, 3 * len(mass)) * np.repeat(free, 3)
    um = u + rng.uniform(-1e-5, 1e-5, len(u)) * np.repeat(free, 3)
    dt = orc.dt(0, mesh, 0.5)
    _, uo, umo = orc.run(0, mesh, dt, nsteps, u0=u, um1=um, return_state=True)
    for on in (True, False):
        with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False, stencil=on) as m:
            vfe.vfe_set_state(m.handle, u, um)
            m.step(nsteps)
            ug, ugm = vfe.vfe_get_state(m.handle)
        assert rel_max(ug, uo) <= 1e-13, on
        assert rel_max(ugm, umo) <= 1e-13, on


def test_stencil_corrected_nodes_steps_from_state(orc):
    """Every column-plane in the stencil kernel (stencil=2), the nodes at the
    material and void interfaces and the mesh faces corrected after it:
    steps from a state against the oracle."""
    mesh = layered((47, 40, 12), void_top=2)
    mass = orc.node_mass(0, mesh)
    nx, ny, _ = mesh["shape"]
    free = mass > 0
    free[: (nx + 1) * (ny + 1)] = False
    rng = np.random.default_rng(18)
    u = rng.uniform(-1e-3, 1e-3, 3 * len(mass)) * np.repeat(free, 3)
    um = u + rng.uniform(-1e-5, 1e-5, len(u)) * np.repeat(free, 3)
    dt = orc.dt(0, mesh, 0.5)
    _, uo, umo = orc.run(0, mesh, dt, 5, u0=u, um1=um, return_state=True)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False, stencil=2) as m:
        # prologue, stencil kernel, corrections (no plane left to the element kernel)
        assert vfe.vfe_get_launches_per_step(m.handle) == 3
        vfe.vfe_set_state(m.handle, u, um)
        m.step(5)
        ug, ugm = vfe.vfe_get_state(m.handle)
    assert rel_max(ug, uo) <= 1e-13
    assert rel_max(ugm, umo) <= 1e-13


def test_stencil_traces_from_rest(orc):
    """Source and receivers (their planes go to the element kernel), 120 steps."""
    mesh = layered((40, 36, 16), void_top=2)
    dt = orc.dt(0, mesh, 0.5)
    n = 120
    ref = orc.run(0, mesh, dt, n, source=oracle_source(mesh), receivers=W.receiver_nodes(mesh))
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC) as m:
        m.step(n)
        tr = m.traces()
    assert rel_l2(tr, ref) <= 1e-9


BIG = (100, 94, 40)   # several planes per CTA in each kernel


def test_stencil_ku_multi_plane_segments(orc):
    mesh = layered(BIG, void_top=4)
    u = W.random_displacement(mesh, 17)
    ref = orc.ku(0, mesh, u)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False) as m:
        out, cov, sh, F = vfe.vfe_debug_stencil_partials(m.handle, u)
        f = m.internal_force(u)
    assert cov.sum() > 20000
    assert rel_max(f, ref) <= KU_TOL


@pytest.mark.parametrize("nsteps", [1, 2, 6])
def test_stencil_multi_plane_steps_on_off(orc, nsteps):
    mesh = layered(BIG, void_top=4)
    mass = orc.node_mass(0, mesh)
    nx, ny, _ = mesh["shape"]
    free = mass > 0
    free[: (nx + 1) * (ny + 1)] = False
    rng = np.random.default_rng(9)
    u = rng.uniform(-1e-3, 1e-3, 3 * len(mass)) * np.repeat(free, 3)
    um = u + rng.uniform(-1e-5, 1e-5, len(u)) * np.repeat(free, 3)
    dt = orc.dt(0, mesh, 0.5)
    _, uo, _ = orc.run(0, mesh, dt, nsteps, u0=u, um1=um, return_state=True)
    got = {}
    for on in (True, False):
        with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False, stencil=on) as m:
            vfe.vfe_set_state(m.handle, u, um)
            m.step(nsteps)
            got[on], _ = vfe.vfe_get_state(m.handle)
    err_on, err_off = rel_max(got[True], uo), rel_max(got[False], uo)
    assert err_off <= 1e-13
    assert err_on <= 1e-13, (err_on, np.argmax(np.abs(got[True] - uo)) // 3)


# per-node corrections where several materials and voids meet at one node
# (several correction entries per node) and on the dipping-layer generator
def _blocky(shape, seed):
    """Four materials and voids in 3x3x3 blocks: nodes where up to eight
    values meet, voids touching the mesh faces."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    blocks = rng.integers(-1, 4, size=((nz + 2) // 3, (ny + 2) // 3, (nx + 2) // 3))
    mat = blocks.repeat(3, 0).repeat(3, 1).repeat(3, 2)[:nz, :ny, :nx]
    table = [[1800.0, 700.0, 2000.0], [2600.0, 1100.0, 2200.0], [1500.0, 500.0, 1900.0],
             [3100.0, 1500.0, 2500.0]]
    return W._mesh(shape, 1.0, mat, table, W._source((nx // 2, ny // 2, nz // 2), 60.0), [], 40,
                   "blocky_%dx%dx%d" % shape)


CORR_MESHES = [("blocky", lambda: _blocky((37, 34, 14), 5)),
               ("random", lambda: W.random_mesh(6, shape=(33, 31, 9), n_mat=4, void_frac=0.2,
                                                h=1.0)),
               ("dipping", lambda: W.config3(shape=(48, 44, 24)))]


@pytest.mark.parametrize("name,make", CORR_MESHES)
def test_stencil_corrections_ku_matches_oracle(orc, name, make):
    mesh = make()
    u = W.random_displacement(mesh, 27)
    ref = orc.ku(0, mesh, u)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False, stencil=2) as m:
        out, cov, _, _ = vfe.vfe_debug_stencil_partials(m.handle, u)
        f = m.internal_force(u)
    # nearly every node with a solid element is in a stencil run
    solid = orc.node_mass(0, mesh) > 0
    assert cov[solid].mean() > 0.9
    assert rel_max(f, ref) <= KU_TOL
    assert not f.reshape(-1, 3)[~solid].any()


@pytest.mark.parametrize("name,make", CORR_MESHES)
def test_stencil_corrections_steps_match_oracle(orc, name, make):
    mesh = make()
    mass = orc.node_mass(0, mesh)
    nx, ny, _ = mesh["shape"]
    free = mass > 0
    free[: (nx + 1) * (ny + 1)] = False
    rng = np.random.default_rng(28)
    u = rng.uniform(-1e-3, 1e-3, 3 * len(mass)) * np.repeat(free, 3)
    um = u + rng.uniform(-1e-5, 1e-5, len(u)) * np.repeat(free, 3)
    dt = orc.dt(0, mesh, 0.5)
    _, uo, umo = orc.run(0, mesh, dt, 4, u0=u, um1=um, return_state=True)
    for on in (2, False):
        with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False, stencil=on) as m:
            vfe.vfe_set_state(m.handle, u, um)
            m.step(4)
            ug, ugm = vfe.vfe_get_state(m.handle)
        assert rel_max(ug, uo) <= 1e-13, on
        assert rel_max(ugm, umo) <= 1e-13, on


def test_stencil_corrections_traces_from_rest(orc):
    """Dipping layers under a void top with the source and the receivers
    (their planes in the element kernel, the rest in the stencil kernel with
    corrections): 150 steps against the oracle's traces."""
    mesh = W.config3(shape=(48, 44, 24))
    si, sj, sk = mesh["source"]["ijk"]
    # receivers a few nodes from the source, so that the wave reaches them
    mesh["receivers"] = np.array([(si + a, sj + b, sk + c) for a, b, c in
                                  ((4, 0, 0), (-3, 2, 0), (0, -4, 1), (2, 3, -3), (-4, -4, 2),
                                   (5, 1, -2), (0, 0, 5), (-2, 5, -4))], dtype=np.int32)
    dt = orc.dt(0, mesh, 0.5)
    n = 150
    ref = orc.run(0, mesh, dt, n, source=oracle_source(mesh), receivers=W.receiver_nodes(mesh))
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, stencil=2) as m:
        assert vfe.vfe_get_launches_per_step(m.handle) == 4
        m.step(n)
        tr = m.traces()
    assert rel_l2(tr, ref) <= 1e-9


EDGE_SHAPES = [(1, 1, 1), (2, 3, 1), (5, 4, 2), (14, 16, 3), (16, 14, 2), (31, 1, 5), (15, 15, 4)]


@pytest.mark.parametrize("shape", EDGE_SHAPES)
def test_stencil_corrections_edge_meshes(orc, shape):
    """Per-node corrections (stencil=2) on meshes one or two elements thick,
    narrower than a node column (both x faces in one column), single
    elements, and with voids: K u and three steps from a state against the
    oracle."""
    mesh = W.random_mesh(400 + sum(shape), shape=shape, n_mat=3, void_frac=0.25, h=1.0)
    if not (mesh["material_ids"] >= 0).any():
        mesh["material_ids"][0] = 0
    u = W.random_displacement(mesh, 5)
    ref = orc.ku(0, mesh, u)
    mass = orc.node_mass(0, mesh)
    nx, ny, _ = mesh["shape"]
    free = mass > 0
    free[: (nx + 1) * (ny + 1)] = False
    rng = np.random.default_rng(6)
    us = rng.uniform(-1e-3, 1e-3, 3 * len(mass)) * np.repeat(free, 3)
    um = us + rng.uniform(-1e-5, 1e-5, len(us)) * np.repeat(free, 3)
    dt = orc.dt(0, mesh, 0.5)
    _, uo, umo = orc.run(0, mesh, dt, 3, u0=us, um1=um, return_state=True)
    with vfe.Mesh(mesh, path=vfe.VFE_PATH_TC, source=False, receivers=False, stencil=2) as m:
        f = m.internal_force(u)
        vfe.vfe_set_state(m.handle, us, um)
        m.step(3)
        ug, ugm = vfe.vfe_get_state(m.handle)
    assert rel_max(f, ref) <= KU_TOL
    assert rel_max(ug, uo) <= 1e-13
    assert rel_max(ugm, umo) <= 1e-13
