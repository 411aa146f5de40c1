"""GPU parity on hybrid triangle / quadrilateral meshes with artificial edges
(Section 2.2.2, Figs. l1-hyb and l1-tria4), through fdu_mesh_create_cells.

The kernels see only edges, 1D stencils and divergence tables, so the
tolerances are those of the triangle meshes: FP64 residual and RK states
<= 1e-12 relative L2 against the oracle, FP32 residual <= 1e-4, and the
residual VJP against central differences of the oracle <= 1e-6.
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


@pytest.fixture(scope="module")
def hybrid():
    # 33 x 33 lattice: 1089 vertices, a ragged last SELL slice
    m = inputs.hybrid_lattice(33, L=10.0, jitter=0.2, seed=51, tri_fraction=0.5)
    w0 = inputs.isentropic_vortex(m.xy)
    om = oracle.OracleMesh(m.xy, m.tri, 10.0, 10.0, artificial=1)
    M = fdu.Mesh(m.xy, m.tri, 10.0, 10.0, device=0, artificial_edges=1)
    return m, w0, om, M


def test_hybrid_residual_f64_matches_oracle(hybrid):
    m, w0, om, M = hybrid
    M.set_state(w0)
    got = M.residual(64)
    want = om.residual(w0)
    for k in range(4):
        assert rel_l2(got[:, k], want[:, k]) <= 1e-12


def test_hybrid_rk_steps_match_oracle(hybrid):
    m, w0, om, M = hybrid
    M.set_state(w0)
    dt = M.max_dt(0.5)
    assert dt == pytest.approx(om.max_dt(w0, 0.5), rel=1e-14)
    M.rk_steps(dt, 5, 64)
    got = M.get_state()
    w = w0.copy()
    for _ in range(5):
        w = om.rk3_step(w, dt)
    for k in range(4):
        assert rel_l2(got[:, k] - w0[:, k], w[:, k] - w0[:, k]) <= 1e-12


def test_hybrid_residual_f32_error(hybrid):
    m, w0, om, M = hybrid
    M.set_state(w0)
    got = M.residual(32)
    want = om.residual(w0)
    for k in range(4):
        assert rel_l2(got[:, k], want[:, k]) <= 1e-4


def test_far_apex_mesh_degree3_one_level_matches_oracle():
    m = inputs.union_jack_lattice(24, L=10.0)
    cells = (np.arange(0, 3 * m.nt + 1, 3, dtype=np.int64), m.tri.astype(np.int32).ravel())
    w0 = inputs.isentropic_vortex(m.xy)
    om = oracle.OracleMesh(m.xy, cells, 10.0, 10.0, degree=3, levels=1, artificial=2)
    M = fdu.Mesh(m.xy, cells, 10.0, 10.0, device=0, lsq_degree=3, lsq_levels=1, artificial_edges=2)
    M.set_state(w0)
    got = M.residual(64)
    want = om.residual(w0)
    for k in range(4):
        assert rel_l2(got[:, k], want[:, k]) <= 1e-12


def test_hybrid_residual_vjp_dot_product(hybrid):
    m, w0, om, M = hybrid
    rng = np.random.default_rng(5)
    x, y = m.xy[:, 0], m.xy[:, 1]
    w = w0.copy()
    for c in range(4):  # smooth perturbation: no smoothness indicator at rounding level
        w[:, c] *= 1.0 + 0.02 * np.sin(2 * np.pi * (x + 1.3 * c) / 10) * np.cos(2 * np.pi * (y - 0.7 * c) / 10)
    d = rng.standard_normal(w.shape) * np.abs(w).mean(0) * 1e-2
    lam = rng.standard_normal(w.shape)
    M.set_state(w)
    adj = float(np.sum(M.residual_vjp(lam) * d))
    fds = [np.sum(lam * (om.residual(w + h * d) - om.residual(w - h * d))) / (2 * h)
           for h in (3e-5, 1e-5, 3e-6, 1e-6)]
    assert min(abs(f - adj) / abs(adj) for f in fds) < 1e-6
