"""GPU parity of precision 48: the FP64 state pipeline with the double-word
edge flux (FP32-pair arithmetic for the increments, FP64 for the state-sized
terms), through the C-ABI, against the FP64 oracle on the same seeded
inputs, at the FP64 path's own tolerance: relative L2 <= 1e-12 per
component for the residual and for state changes over RK steps, and the
same positivity fallbacks edge for edge (a count that must agree exactly).
"""
import numpy as np
import pytest

import oracle
from paper_2102_12933_gb300 import fdu, inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def rel_l2(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def check_residual(om, M, w, sel=None):
    M.set_state(w)
    M.fallback_count(reset=True)
    got = M.residual(48)
    want, nf = om.residual(w, return_fallbacks=True)
    assert M.fallback_count() == nf
    if sel is not None:
        got, want = got[sel], want[sel]
    for k in range(4):
        assert rel_l2(got[:, k], want[:, k]) <= 1e-12, k
    return got


@pytest.mark.parametrize("n,seed", [(40, 1001), (37, 4242)])
def test_vortex_residual(n, seed):
    m, w0 = inputs.vortex_case(n, seed=seed)
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0)
    got = check_residual(om, M, w0)
    # the FP64 path and precision 48 agree to the same level
    M.set_state(w0)
    for k in range(4):
        assert rel_l2(got[:, k], M.residual(64)[:, k]) <= 1e-12


@pytest.mark.parametrize("degree,levels", [(1, 1), (3, 2), (5, 2)])
def test_other_stencils_and_degrees(degree, levels):
    m, w0 = inputs.vortex_case(30, seed=31)
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly, degree=degree, levels=levels)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, lsq_degree=degree, lsq_levels=levels, device=0)
    check_residual(om, M, w0)


def test_rk_steps_and_graph_replay():
    m, w0 = inputs.vortex_case(40, seed=1001)
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0)
    dt = om.max_dt(w0, 0.5)
    w = w0.copy()
    for _ in range(20):
        w = om.rk3_step(w, dt)
    M.set_state(w0)
    M.rk_steps(dt, 20, 48)
    got = M.get_state()
    for k in range(4):
        assert rel_l2(got[:, k] - w0[:, k], w[:, k] - w0[:, k]) <= 1e-12
    # single steps give the graph's bits
    M.set_state(w0)
    for _ in range(20):
        M.rk_step(dt, 48)
    assert np.array_equal(M.get_state(), got)


def test_strong_jump_fallbacks():
    m = inputs.torus_lattice(40, L=2.0, jitter=0.2, seed=12)
    x, y = m.xy[:, 0] - 1.0, m.xy[:, 1] - 1.0
    inside = (np.abs(x) < 0.5) & (np.abs(y) < 0.5)
    z = np.zeros(m.nv)
    w = inputs.primitive_to_conservative(np.where(inside, 1.0, 0.02), z + 0.3, z - 0.2, np.where(inside, 1.0, 1e-4))
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0)
    check_residual(om, M, w)


def test_riemann_transmissive_residual_and_adaptive_steps():
    m, w0 = inputs.riemann_case(41, ghost_layers=5, seed=1003)
    real = m.ghost_donor < 0
    om = oracle.OracleMesh(m.xy, m.tri, 0.0, 0.0, ghost=m.ghost_donor)
    M = fdu.Mesh(m.xy, m.tri, 0.0, 0.0, device=0, ghost_donor=m.ghost_donor)
    check_residual(om, M, w0, sel=real)
    cfl, t_end, nsteps = 0.5, 0.3, 6
    M.set_state(w0)
    done, t = M.advance(cfl, t_end, 48, max_steps=nsteps)
    assert done == nsteps
    w, tt = w0.copy(), 0.0
    for _ in range(nsteps):
        dt = min(om.max_dt(w, cfl), t_end - tt)
        w = om.rk3_step(w, dt)
        tt += dt
    assert abs(t - tt) <= 1e-14 * tt
    got = M.get_state()
    for k in range(4):
        assert rel_l2(got[real, k] - w0[real, k], w[real, k] - w0[real, k]) <= 1e-10
    gi = np.nonzero(~real)[0]
    assert np.array_equal(got[gi], got[m.ghost_donor[gi]])


def test_shock_vortex_dirichlet_steps():
    m, w0 = inputs.shock_vortex_case(40)
    g = m.ghost_donor >= 0
    om = oracle.OracleMesh(m.xy, m.tri, 0.0, 80.0, ghost=m.ghost_donor)
    om.set_positivity(0.1)
    M = fdu.Mesh(m.xy, m.tri, 0.0, 80.0, device=0, ghost_donor=m.ghost_donor, positivity_alpha=0.1)
    check_residual(om, M, w0, sel=~g)
    M.set_state(w0)
    steps, t = M.advance(0.5, 10.0, 48, max_steps=8)
    assert steps == 8
    w, tt = w0.copy(), 0.0
    for _ in range(8):
        dt = min(om.max_dt(w, 0.5), 10.0 - tt)
        w = om.rk3_step(w, dt)
        tt += dt
    got = M.get_state()
    assert np.array_equal(got[g], w0[g])
    for k in range(4):
        assert rel_l2(got[:, k] - w0[:, k], w[:, k] - w0[:, k]) <= 1e-10


def test_hybrid_mesh_residual():
    m = inputs.hybrid_lattice(33, L=10.0, jitter=0.2, seed=51, tri_fraction=0.5)
    w0 = inputs.isentropic_vortex(m.xy)
    om = oracle.OracleMesh(m.xy, m.tri, 10.0, 10.0, artificial=1)
    M = fdu.Mesh(m.xy, m.tri, 10.0, 10.0, device=0, artificial_edges=1)
    check_residual(om, M, w0)


def test_full_size_sampled_parity():
    """250k-vertex vortex mesh in the benchmark's launch configuration: the
    residual on the whole mesh, checked at sampled vertices the oracle
    computes one by one (random ones plus the vortex core)."""
    m, w0 = inputs.vortex_case(500, seed=1002)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0)
    M.set_state(w0)
    got = M.residual(48)
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
    rng = np.random.default_rng(5)
    mask = np.zeros(m.nv, np.uint8)
    mask[rng.choice(m.nv, 1500, replace=False)] = 1
    mask[np.argsort(-np.abs(w0[:, 1] / w0[:, 0] - 1.0))[:500]] = 1
    want = om.residual(w0, mask=mask)
    sel = mask.astype(bool)
    for k in range(4):
        assert rel_l2(got[sel, k], want[sel, k]) <= 1e-12
    full64 = M.residual(64)
    for k in range(4):
        assert rel_l2(got[:, k], full64[:, k]) <= 1e-12


def test_precision_argument_checked():
    m, w0 = inputs.vortex_case(12, seed=3)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0)
    M.set_state(w0)
    with pytest.raises(fdu.FduError):
        M.residual(47)
