"""CPU tests of the C-ABI library: exports, host preprocessing parity with
the oracle (bit-exact integer connectivity, FP64 coefficients and weights
within rounding), renumbering invariance and error statuses.  No GPU call:
meshes are built with device = -1 (host tables only)."""
import ctypes
import re

import numpy as np
import pytest

import oracle
from conftest import ROOT
from paper_2102_12933_gb300 import fdu, inputs


def test_library_exports_every_declared_symbol():
    header = open(f"{ROOT}/include/fdu.h").read()
    declared = set(re.findall(r"^(?:fdu_status|const char \*)\s*(fdu_\w+)\(", header, re.M))
    assert declared == set(fdu.EXPORTS)
    lib = ctypes.CDLL(fdu.lib_path() if fdu.load() else None)
    for name in declared:
        assert hasattr(lib, name), name
    assert b"sm_103a" in fdu.load().fdu_version()


def _pair(n=40, seed=1001, **kw):
    m, w0 = inputs.vortex_case(n, seed=seed)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=-1, **kw)
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly, degree=kw.get("lsq_degree", 2), levels=kw.get("lsq_levels", 2))
    om.build_weights()
    return m, M, om


@pytest.mark.parametrize("levels,degree", [(2, 2), (1, 1), (2, 3)])
def test_host_tables_match_oracle(levels, degree):
    m, M, om = _pair(n=37, seed=77, lsq_levels=levels, lsq_degree=degree)
    assert np.array_equal(M.edges(), om.edges())
    s1, x1 = M.edge_stencils()
    s2, x2 = om.stencils()
    assert np.array_equal(s1, s2)
    assert np.abs(x1 - x2).max() < 1e-13
    a, b = M.div_stencils(), om.div_stencils()
    for i in (0, 1, 4, 5):  # offsets and ids: bit-exact
        assert np.array_equal(a[i], b[i])
    for i in (2, 3, 6):  # weights: QR vs Jacobi SVD pseudo-inverse
        assert np.abs(a[i] - b[i]).max() <= 1e-11 * (1 + np.abs(b[i]).max())


def test_info_counts():
    m, M, om = _pair(n=40)
    info = M.info()
    assert info["nv"] == 1600 and info["ne"] == 4800 and info["nt"] == 3200 and info["n_real"] == 1600
    assert info["sell_width"] == 32
    assert 12 <= info["J_min"] <= info["J_max"] <= 30


@pytest.mark.parametrize("kind", ["torus", "ghost box"])
def test_host_tables_do_not_depend_on_the_thread_count(kind):
    """Edges, 1D stencils and divergence stencils are built in parallel
    chunks; every thread count gives the same bits.  The meshes have more
    than 1024 vertices so that the tables are built by several threads."""
    if kind == "torus":
        m, _ = inputs.vortex_case(48, seed=21)
        build = lambda t: fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=-1, host_threads=t)
    else:
        m = inputs.box_lattice(40, ghost_layers=5, seed=22)
        build = lambda t: fdu.Mesh(m.xy, m.tri, 0.0, 0.0, device=-1, host_threads=t, ghost_donor=m.ghost_donor)
    ref = build(1)
    for t in (2, 5):
        M = build(t)
        assert np.array_equal(M.edges(), ref.edges())
        for x, y in zip(M.edge_stencils(), ref.edge_stencils()):
            assert np.array_equal(x, y)
        for x, y in zip(M.div_stencils(), ref.div_stencils()):
            assert np.array_equal(x, y)


def test_stencil_error_names_the_same_vertex_for_any_thread_count():
    """An open box whose first ten rows are (Dirichlet) ghosts and whose
    other sides have none: the parallel divergence-stencil build reports the
    lowest vertex whose stencil holds an edge without a 1D stencil, as a
    serial build does (here a vertex several 256-vertex chunks in)."""
    b = inputs.box_lattice(40, ghost_layers=0, seed=23)
    donor = np.full(b.nv, -1, np.int32)
    low = np.arange(b.nv) < 400
    donor[low] = np.nonzero(low)[0]
    msgs = set()
    for t in (1, 3, 8):
        with pytest.raises(fdu.FduError) as e:
            fdu.Mesh(b.xy, b.tri, 0.0, 0.0, device=-1, host_threads=t, ghost_donor=donor)
        assert e.value.status == -3
        msgs.add(str(e.value))
    assert len(msgs) == 1, msgs
    assert re.search(r"vertex (\d+)", msgs.pop()).group(1) != "0"


def test_renumbering_is_invisible():
    """Permuting the caller's vertex ids permutes the outputs and nothing else."""
    m, _ = inputs.vortex_case(24, seed=5)
    pm, perm = inputs.permute_vertices(m, seed=9)
    A = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=-1)
    B = fdu.Mesh(pm.xy, pm.tri, pm.Lx, pm.Ly, device=-1)
    ea = A.edges()
    eb = perm[B.edges()]  # back to the unpermuted ids
    ka = {tuple(sorted(e)) for e in ea.tolist()}
    kb = {tuple(sorted(e)) for e in eb.tolist()}
    assert ka == kb
    C = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=-1, renumber=0)
    for x, y in zip(A.div_stencils(), C.div_stencils()):
        assert np.array_equal(x, y)


def test_error_statuses():
    m, _ = inputs.vortex_case(12, seed=3)
    bad = m.tri.copy()
    bad[0, 0] = m.nv + 5
    with pytest.raises(fdu.FduError) as e:
        fdu.Mesh(m.xy, bad, m.Lx, m.Ly, device=-1)
    assert e.value.status == -2
    flipped = m.tri.copy()
    flipped[3] = flipped[3, ::-1]
    with pytest.raises(fdu.FduError) as e:
        fdu.Mesh(m.xy, flipped, m.Lx, m.Ly, device=-1)
    assert e.value.status == -2
    with pytest.raises(fdu.FduError) as e:
        fdu.Mesh(m.xy, m.tri, 0.0, 0.0, device=-1)  # periodic without lengths
    assert e.value.status == -1
    with pytest.raises(fdu.FduError) as e:
        fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=-1, lsq_degree=9)
    assert e.value.status == -1
    # an open mesh without ghost layers: edges at the boundary have no 1D
    # stencil, yet boundary vertices would need them
    b = inputs.box_lattice(8, ghost_layers=0)
    with pytest.raises(fdu.FduError) as e:
        fdu.Mesh(b.xy, b.tri, 0.0, 0.0, device=-1, ghost_donor=np.full(b.nv, -1, np.int32))
    assert e.value.status == -3
    # one-level stencils cannot carry degree-3 polynomials (18 unknowns > 4N conditions)
    with pytest.raises(fdu.FduError) as e:
        fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=-1, lsq_levels=1, lsq_degree=3)
    assert e.value.status == -4
    # host-only meshes refuse device calls
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=-1)
    with pytest.raises(fdu.FduError) as e:
        M.residual()
    assert e.value.status == -8


def test_degenerate_inputs_fail_cleanly():
    """Empty and minimal inputs return error statuses (no crash, no
    partial object)."""
    tri1 = np.array([[0, 1, 2]], np.int32)
    xy1 = np.array([[0, 0], [1, 0], [0, 1.0]])
    cases = [
        ("no vertices", np.zeros((0, 2)), np.zeros((0, 3), np.int32), 0.0, 0.0, -1),
        ("no triangles", np.random.default_rng(0).random((5, 2)), np.zeros((0, 3), np.int32), 0.0, 0.0, -1),
        ("one triangle, non-periodic without ghost vertices", xy1, tri1, 0.0, 0.0, -1),
        ("one triangle, periodic: no walk finds a forward neighbour", xy1, tri1, 2.0, 2.0, -3),
    ]
    for name, xy, tri, Lx, Ly, status in cases:
        with pytest.raises(fdu.FduError) as e:
            fdu.Mesh(xy, tri, Lx, Ly, device=-1)
        assert e.value.status == status, (name, e.value)
    m, _ = inputs.vortex_case(12, seed=3)
    with pytest.raises(fdu.FduError) as e:
        fdu.Batch([], 10.0, device=-1)
    assert e.value.status == -1 and "at least one mesh" in str(e.value)
    with pytest.raises(fdu.FduError) as e:
        fdu.Batch([(m.xy, m.tri)], 10.0, device=-1)  # batches live on a device
    assert e.value.status == -1


def test_transmissive_box_tables_match_oracle():
    """Four-quadrant Riemann box with 5 ghost layers: real vertices carry
    stencils, ghosts do not; every active edge has a full 1D stencil."""
    m, _ = inputs.riemann_case(21, ghost_layers=5)
    M = fdu.Mesh(m.xy, m.tri, 0.0, 0.0, device=-1, ghost_donor=m.ghost_donor)
    om = oracle.OracleMesh(m.xy, m.tri, 0.0, 0.0, ghost=m.ghost_donor)
    om.build_weights()
    assert M.info()["n_real"] == 21 * 21
    assert np.array_equal(M.edges(), om.edges())
    s1, x1 = M.edge_stencils()
    s2, x2 = om.stencils()
    assert np.array_equal(s1, s2)
    ok = s1[:, 0] >= 0
    assert np.abs(x1[ok] - x2[ok]).max() < 1e-13
    a, b = M.div_stencils(), om.div_stencils()
    for i in (0, 1, 4, 5):
        assert np.array_equal(a[i], b[i])
    for i in (2, 3, 6):
        assert np.abs(a[i] - b[i]).max() <= 1e-11 * (1 + np.abs(b[i]).max())
    ghost = m.ghost_donor >= 0
    assert np.all(np.diff(a[0])[ghost] == 0)  # ghost rows are empty


@pytest.mark.parametrize("degree", [4, 5, 6])
def test_high_degree_weights_match_oracle(degree):
    """Degrees 4-6 (the paper's fifth-order setting is degree 5, Section 2.2.3)."""
    m, M, om = _pair(n=24, seed=91, lsq_degree=degree, lsq_levels=2)
    a, b = M.div_stencils(), om.div_stencils()
    for i in (0, 1, 4, 5):
        assert np.array_equal(a[i], b[i])
    for i in (2, 3, 6):
        assert np.abs(a[i] - b[i]).max() <= 1e-9 * (1 + np.abs(b[i]).max())


@pytest.mark.parametrize("artificial,frac,degree,levels", [(0, 0.5, 2, 2), (1, 0.5, 2, 2), (1, 0.0, 3, 2), (2, 0.5, 2, 1)])
def test_hybrid_host_tables_match_oracle(artificial, frac, degree, levels):
    """Triangles and quadrilaterals with artificial edges (Section 2.2.2):
    edges, 1D stencils and divergence stencils bit-exact, weights within
    rounding."""
    m = inputs.hybrid_lattice(21, L=10.0, jitter=0.2, seed=41, tri_fraction=frac)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=-1, lsq_degree=degree, lsq_levels=levels,
                 artificial_edges=artificial)
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly, degree=degree, levels=levels, artificial=artificial)
    om.build_weights()
    assert np.array_equal(M.edges(), om.edges())
    s1, x1 = M.edge_stencils()
    s2, x2 = om.stencils()
    assert np.array_equal(s1, s2)
    assert np.abs(x1 - x2).max() < 1e-13
    a, b = M.div_stencils(), om.div_stencils()
    for i in (0, 1, 4, 5):
        assert np.array_equal(a[i], b[i])
    for i in (2, 3, 6):
        assert np.abs(a[i] - b[i]).max() <= 1e-11 * (1 + np.abs(b[i]).max())
    assert M.info()["nt"] == m.nt


def test_far_apex_edges_match_oracle_and_rescue_the_fit():
    m = inputs.union_jack_lattice(16, L=10.0)
    cells = (np.arange(0, 3 * m.nt + 1, 3, dtype=np.int64), m.tri.astype(np.int32).ravel())
    with pytest.raises(fdu.FduError, match="RANK_DEFICIENT"):
        fdu.Mesh(m.xy, cells, 10.0, 10.0, device=-1, lsq_degree=3, lsq_levels=1, artificial_edges=0)
    M = fdu.Mesh(m.xy, cells, 10.0, 10.0, device=-1, lsq_degree=3, lsq_levels=1, artificial_edges=2)
    om = oracle.OracleMesh(m.xy, cells, 10.0, 10.0, degree=3, levels=1, artificial=2)
    assert np.array_equal(M.edges(), om.edges())
    assert np.array_equal(M.edge_stencils()[0], om.stencils()[0])


def test_hybrid_mesh_errors():
    m = inputs.hybrid_lattice(8, L=10.0, jitter=0.0, tri_fraction=0.0)
    off, vtx = m.tri
    with pytest.raises(fdu.FduError, match="ARG"):
        fdu.Mesh(m.xy, (off, vtx), 10.0, 10.0, device=-1, artificial_edges=3)
    cw = vtx.copy().reshape(-1, 4)[:, ::-1].ravel()  # clockwise quads
    with pytest.raises(fdu.FduError, match="MESH"):
        fdu.Mesh(m.xy, (off, cw), 10.0, 10.0, device=-1)
    bent = vtx.copy().reshape(-1, 4)
    bent[0] = bent[0][[0, 2, 1, 3]]  # self-intersecting (not convex)
    with pytest.raises(fdu.FduError, match="MESH"):
        fdu.Mesh(m.xy, (off, bent.ravel()), 10.0, 10.0, device=-1)
    five = (np.array([0, 5], np.int64), np.array([0, 1, 2, 3, 4], np.int32))
    with pytest.raises(fdu.FduError, match="MESH"):
        fdu.Mesh(m.xy, five, 10.0, 10.0, device=-1)
    with pytest.raises(ValueError):
        fdu.Mesh(m.xy, np.zeros((1, 3), np.int32), 10.0, 10.0, device=-1, artificial_edges=1)


def test_channel_with_dirichlet_ghosts_matches_oracle():
    """Periodic in y, Dirichlet ghost columns in x (the shock-vortex setup)."""
    m, _ = inputs.shock_vortex_case(40)
    M = fdu.Mesh(m.xy, m.tri, 0.0, 80.0, device=-1, ghost_donor=m.ghost_donor)
    om = oracle.OracleMesh(m.xy, m.tri, 0.0, 80.0, ghost=m.ghost_donor)
    om.build_weights()
    assert M.info()["n_real"] == int(np.sum(m.ghost_donor < 0))
    assert np.array_equal(M.edges(), om.edges())
    assert np.array_equal(M.edge_stencils()[0], om.stencils()[0])
    a, b = M.div_stencils(), om.div_stencils()
    for i in (0, 1, 4, 5):
        assert np.array_equal(a[i], b[i])
    # a ghost whose donor is another ghost is rejected
    bad = m.ghost_donor.copy()
    g = np.nonzero(bad >= 0)[0]
    bad[g[0]] = g[1]
    with pytest.raises(fdu.FduError, match="ARG"):
        fdu.Mesh(m.xy, m.tri, 0.0, 80.0, device=-1, ghost_donor=bad)
