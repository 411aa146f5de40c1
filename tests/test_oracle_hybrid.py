"""Pins of the oracle's hybrid meshes and artificial edges (Section 2.2.2,
Figs. l1-hyb and l1-tria4), against what the geometry fixes:

- quadrilateral lattice with both diagonals of every quad (the dashed edge of
  Fig. l1-hyb): the king's graph, 8 neighbours per vertex, E = 4V, one-level
  stencil of 8 vertices and 20 edges (8 at O, 8 lattice sides and 4 quad
  diagonals between neighbours), 36 conditions;
- "Union Jack" triangulation, where every other vertex has 4 neighbours (Fig.
  l1-tria4): a degree-3 one-level fit needs 18 conditions and a valence-4
  vertex has 4 + 4 edges and 4 neighbours, 16 conditions, so without
  artificial edges the least squares fails; with them each valence-4 vertex
  is joined to exactly the four lattice points at (+-h, +-h) (the figure's
  dashed lines) and nothing is added at valence-8 vertices;
- exactness of the least-squares divergence for polynomial fluxes, free-stream
  preservation and the degree-2 convergence rate on these meshes.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12933_gb300 import inputs


def _min_image(d, L):
    return d - L * np.rint(d / L) if L > 0 else d


def _neighbours(edges, nv):
    nb = [set() for _ in range(nv)]
    for a, b in edges.tolist():
        nb[a].add(b)
        nb[b].add(a)
    return nb


def _cells_of(m):
    """Triangles of a triangle mesh as the CSR cell pair."""
    return (np.arange(0, 3 * m.nt + 1, 3, dtype=np.int64), np.ascontiguousarray(m.tri, dtype=np.int32).ravel())


def test_quad_lattice_with_diagonals_is_the_kings_graph():
    n, L = 12, 1.0
    m = inputs.hybrid_lattice(n, L=L, jitter=0.0, tri_fraction=0.0)
    plain = oracle.OracleMesh(m.xy, m.tri, L, L, degree=1, levels=1, artificial=0)
    assert plain.ne == 2 * m.nv
    om = oracle.OracleMesh(m.xy, m.tri, L, L, degree=2, levels=1, artificial=1)
    assert om.ne == 4 * m.nv
    nb = _neighbours(om.edges(), m.nv)
    h = L / n
    for o in range(m.nv):
        d = _min_image(m.xy[sorted(nb[o])] - m.xy[o], L) / h
        assert sorted(map(tuple, np.rint(d).astype(int).tolist())) == sorted(
            (i, j) for i in (-1, 0, 1) for j in (-1, 0, 1) if (i, j) != (0, 0))
    voff, vid, _, _, eoff, eid, _ = om.div_stencils()
    assert np.all(np.diff(voff) == 8)
    assert np.all(np.diff(eoff) == 20)
    # without the diagonals the one-level stencil is 4 vertices and 4 edges
    voff0, _, _, _, eoff0, _, _ = plain.div_stencils()
    assert np.all(np.diff(voff0) == 4) and np.all(np.diff(eoff0) == 4)


def test_union_jack_far_apex_edges():
    n, L = 12, 10.0
    m = inputs.union_jack_lattice(n, L=L)
    cells = _cells_of(m)
    h = L / n
    base = _neighbours(oracle.OracleMesh(m.xy, cells, L, L, degree=3, levels=1, artificial=0).edges(), m.nv)
    val = np.array([len(s) for s in base])
    assert sorted(set(val.tolist())) == [4, 8]
    # the degree-3 one-level fit fails without artificial edges ...
    with pytest.raises(oracle.OracleError):
        oracle.OracleMesh(m.xy, cells, L, L, degree=3, levels=1, artificial=0).build_weights()
    # ... and with them each valence-4 vertex gains exactly its four corners at (+-h, +-h)
    om = oracle.OracleMesh(m.xy, cells, L, L, degree=3, levels=1, artificial=2)
    nb = _neighbours(om.edges(), m.nv)
    for o in range(m.nv):
        added = sorted(nb[o] - base[o])
        if val[o] == 8:
            assert added == []
        else:
            d = np.rint(_min_image(m.xy[added] - m.xy[o], L) / h).astype(int)
            assert sorted(map(tuple, d.tolist())) == [(-1, -1), (-1, 1), (1, -1), (1, 1)]
    assert om.ne == 3 * m.nv + 2 * int(np.sum(val == 4))
    om.build_weights()
    # on a triangle mesh mode 1 adds nothing (there are no quadrilaterals)
    assert oracle.OracleMesh(m.xy, cells, L, L, degree=2, levels=2, artificial=1).ne == 3 * m.nv


def _lsq_exact(m, L, degree, levels, artificial, seed):
    om = oracle.OracleMesh(m.xy, m.tri, L, L, degree=degree, levels=levels, artificial=artificial)
    om.build_weights()
    voff, vid, wf, wg, eoff, eid, we = om.div_stencils()
    e, nrm = om.edges(), om.normals()
    rng = np.random.default_rng(seed)
    for o in range(0, m.nv, 5):
        cf = rng.standard_normal((degree + 1, degree + 1))
        cg = rng.standard_normal((degree + 1, degree + 1))

        def P(c, x, y):
            return sum(c[i, j] * x ** i * y ** j for i in range(degree + 1) for j in range(degree + 1 - i))

        dv = _min_image(m.xy[vid[voff[o]:voff[o + 1]]] - m.xy[o], L)
        ee = eid[eoff[o]:eoff[o + 1]]
        d0 = _min_image(m.xy[e[ee, 0]] - m.xy[o], L)
        de = _min_image(m.xy[e[ee, 1]] - m.xy[e[ee, 0]], L)
        mid = d0 + 0.5 * de
        f0, g0 = cf[0, 0], cg[0, 0]
        fj, gj = P(cf, dv[:, 0], dv[:, 1]), P(cg, dv[:, 0], dv[:, 1])
        r = nrm[ee, 0] * P(cf, mid[:, 0], mid[:, 1]) + nrm[ee, 1] * P(cg, mid[:, 0], mid[:, 1])
        div = (wf[voff[o]:voff[o + 1]] @ (fj - f0) + wg[voff[o]:voff[o + 1]] @ (gj - g0)
               + we[eoff[o]:eoff[o + 1]] @ (r - nrm[ee, 0] * f0 - nrm[ee, 1] * g0))
        exact = cf[1, 0] + cg[0, 1]
        assert abs(div - exact) < 1e-9 * (1 + abs(exact))


@pytest.mark.parametrize("degree,levels,artificial", [(2, 2, 1), (3, 2, 1), (2, 1, 1), (2, 2, 0)])
def test_lsq_divergence_exact_on_hybrid_mesh(degree, levels, artificial):
    m = inputs.hybrid_lattice(12, L=1.0, jitter=0.2, seed=23, tri_fraction=0.5)
    _lsq_exact(m, 1.0, degree, levels, artificial, seed=degree)


def test_lsq_divergence_exact_with_far_apex_edges():
    m = inputs.union_jack_lattice(12, L=1.0)
    m = inputs.Mesh(xy=m.xy, tri=_cells_of(m), Lx=1.0, Ly=1.0)
    _lsq_exact(m, 1.0, 3, 1, 2, seed=7)


def test_free_stream_preserved_on_hybrid_mesh():
    m = inputs.hybrid_lattice(16, L=10.0, jitter=0.2, seed=8)
    one = np.ones(m.nv)
    w = inputs.primitive_to_conservative(1.3 * one, 0.7 * one, -0.4 * one, 2.1 * one)
    om = oracle.OracleMesh(m.xy, m.tri, 10.0, 10.0, artificial=1)
    assert np.abs(om.residual(w)).max() < 1e-12


def test_vortex_residual_rate_on_quad_lattice():
    """Degree-2 two-level least squares on the quadrilateral lattice with its
    diagonals: the residual error of the vortex (Section 3.1) falls at a rate
    approaching 2 (1.65, 1.90 over n = 20, 40, 80)."""
    errs = []
    for n in (20, 40, 80):
        m = inputs.hybrid_lattice(n, L=10.0, jitter=0.0, tri_fraction=0.0)
        w0 = inputs.isentropic_vortex(m.xy)
        d = 1e-5
        ex = (inputs.isentropic_vortex(m.xy, t=d) - inputs.isentropic_vortex(m.xy, t=-d)) / (2 * d)
        om = oracle.OracleMesh(m.xy, m.tri, 10.0, 10.0, degree=2, artificial=1)
        errs.append(np.mean(np.abs(om.residual(w0)[:, 0] - ex[:, 0])))
    rates = [math.log(errs[i] / errs[i + 1]) / math.log(2) for i in range(2)]
    assert rates[0] > 1.5 and rates[1] > 1.8
