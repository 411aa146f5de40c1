"""The hand-written adjoint against the oracle's exact directional
derivatives: <lam, J d> with J d the oracle's complex-step tangent (exact
to rounding, tests/test_oracle_tangent.py) and <J^T lam, d> from the GPU's
vector-Jacobian products.  Both linearise the same function at the same
state, so the two agree to rounding; the bound is 1e-10 relative, for the
residual, one RK3 step and a checkpointed run of several steps, on a
periodic, a transmissive and a Dirichlet mesh, over several seeded
directions each, with the edge-flux VJP in FP64 and in double words
(precision 48).  (Central differences reach only about 1e-8 here; they
are the check in tests/test_gpu_adjoint.py.)
"""
import numpy as np
import pytest

import oracle
from paper_2102_12933_gb300 import fdu, inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

TOL = 1e-10
DIRECTIONS = 4


def _vortex_smooth(m):
    w = inputs.isentropic_vortex(m.xy)
    x, y = m.xy[:, 0], m.xy[:, 1]
    for c in range(4):
        w[:, c] *= 1.0 + 0.02 * np.sin(2 * np.pi * (x + 1.3 * c) / 10) * np.cos(2 * np.pi * (y - 0.7 * c) / 10)
    return w


def _box_smooth(xy, L):
    x, y = xy[:, 0] / L, xy[:, 1] / L
    tp = 2 * np.pi
    return inputs.primitive_to_conservative(1.0 + 0.2 * np.sin(tp * x + 0.3) * np.cos(tp * y - 0.5),
                                            0.3 + 0.1 * np.cos(tp * y + 1.1), -0.2 + 0.1 * np.sin(tp * x - 0.4),
                                            1.0 + 0.15 * np.cos(tp * (x + y) + 0.7))


@pytest.fixture(scope="module", params=["periodic", "transmissive", "dirichlet"])
def case(request):
    if request.param == "periodic":
        m = inputs.torus_lattice(24, L=10.0, jitter=0.2, seed=77)
        w = _vortex_smooth(m)
        om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
        M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0)
    elif request.param == "transmissive":
        m = inputs.box_lattice(20, ghost_layers=5, jitter=0.1, seed=88)
        w = _box_smooth(m.xy, 1.0)
        om = oracle.OracleMesh(m.xy, m.tri, 0.0, 0.0, ghost=m.ghost_donor)
        M = fdu.Mesh(m.xy, m.tri, 0.0, 0.0, device=0, ghost_donor=m.ghost_donor)
    else:
        m = inputs.channel_lattice(16, ghost_layers=5)
        w = _box_smooth(m.xy, 80.0)
        om = oracle.OracleMesh(m.xy, m.tri, 0.0, 80.0, ghost=m.ghost_donor)
        M = fdu.Mesh(m.xy, m.tri, 0.0, 80.0, device=0, ghost_donor=m.ghost_donor)
    return request.param, m, w, om, M


@pytest.fixture(params=[64, 48], ids=["adjoint64", "adjoint48"])
def aprec(request):
    """Arithmetic of the edge-flux VJP: FP64, or double words (precision 48)."""
    return request.param


def _pairs(w, seed):
    rng = np.random.default_rng(seed)
    for _ in range(DIRECTIONS):
        d = rng.standard_normal(w.shape) * np.abs(w).mean(0) * 1e-2
        lam = rng.standard_normal(w.shape)
        yield d, lam


def _check(adj, tan):
    assert abs(adj - tan) <= TOL * abs(tan), (adj, tan, abs(adj - tan) / abs(tan))


def test_residual_vjp_against_tangents(case, aprec):
    kind, m, w, om, M = case
    M.set_adjoint_precision(aprec)
    M.set_state(w)
    for d, lam in _pairs(w, 21):
        _check(float(np.sum(M.residual_vjp(lam) * d)), float(np.sum(lam * om.residual_jvp(w, d))))


def test_rk_step_vjp_against_tangents(case, aprec):
    kind, m, w, om, M = case
    M.set_adjoint_precision(aprec)
    M.set_state(w)
    dt = M.max_dt(0.5)
    for d, lam in _pairs(w, 22):
        M.set_state(w)
        g = M.rk_step_vjp(dt, lam)
        _, jd = om.rk3_steps_jvp(w, d, dt)
        _check(float(np.sum(g * d)), float(np.sum(lam * jd)))


def test_adjoint_rk_against_tangents(case, aprec):
    kind, m, w, om, M = case
    M.set_adjoint_precision(aprec)
    M.set_state(w)
    dt = 0.5 * M.max_dt(0.5)
    n = 5
    for d, lam in _pairs(w, 23):
        M.set_state(w)
        g = M.adjoint_rk(dt, n, lam, checkpoint_every=2)
        _, jd = om.rk3_steps_jvp(w, d, dt, n=n)
        _check(float(np.sum(g * d)), float(np.sum(lam * jd)))


@pytest.mark.parametrize("aprec", [64, 48], ids=["adjoint64", "adjoint48"])
def test_fifty_step_density_misfit_gradient(aprec):
    """The adjoint workload's shape on the 1600-vertex vortex mesh: gradient
    of J = 1/2 sum (rho(T) - rho_exact(T))^2 after 50 SSP-RK3 steps with a
    checkpoint every 10 steps, against the oracle's tangent of the 50-step
    map.  With eps = 1e-6 (smooth weights).  With the paper's eps = 1e-40
    the unperturbed vortex's near-uniform far field puts smoothness
    indicators at rounding level, where each side's derivative follows its
    own rounding (measured: 1e-5 relative); the smooth-state cases above
    cover eps = 1e-40."""
    mesh, w0 = inputs.vortex_case(40, seed=1005)
    eps = 1e-6
    M = fdu.Mesh(mesh.xy, mesh.tri, mesh.Lx, mesh.Ly, device=0, weno_eps=eps)
    M.set_adjoint_precision(aprec)
    M.set_state(w0)
    dt = M.max_dt(0.5)
    n_steps = 50
    M.rk_steps(dt, n_steps, 64)
    wT = M.get_state()
    lam = np.zeros_like(wT)
    lam[:, 0] = wT[:, 0] - inputs.isentropic_vortex(mesh.xy, t=n_steps * dt)[:, 0]
    M.set_state(w0)
    g = M.adjoint_rk(dt, n_steps, lam, checkpoint_every=10)
    om = oracle.OracleMesh(mesh.xy, mesh.tri, mesh.Lx, mesh.Ly)
    rng = np.random.default_rng(6006)
    for _ in range(2):
        d = rng.standard_normal(w0.shape)
        _, jd = om.rk3_steps_jvp(w0, d, dt, n=n_steps, eps=eps)
        _check(float(np.sum(g * d)), float(np.sum(lam * jd)))
