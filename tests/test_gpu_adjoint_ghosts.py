"""Hand-written adjoint on meshes with ghost layers (the transmissive box of
the Riemann problem and the Dirichlet channel of the shock-vortex problem,
Section 3.2): dot-product tests <lam, J d> = <J^T lam, d>, J d from central
finite differences of the oracle, which takes every state through the ghost
fill (transmissive ghosts copy their donors, Dirichlet ghosts keep theirs).

So the derivative of the residual or of an RK step with respect to a
transmissive ghost row is 0 (the fill overwrites it) and its effect through
the stencils lands on the donor's row; a Dirichlet ghost row is the
derivative with respect to that fixed boundary value.  The states are smooth
and subsonic, with per-component phase shifts, so that no smoothness
indicator sits at the WENO epsilon.  The best of a short ladder of steps is
compared at 1e-6 relative, the gradient target of the periodic tests.
"""
import numpy as np
import pytest

import oracle
from paper_2102_12933_gb300 import fdu, inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def smooth_state(xy, Lx, Ly):
    x, y = xy[:, 0] / Lx, xy[:, 1] / Ly
    tp = 2 * np.pi
    rho = 1.0 + 0.2 * np.sin(tp * x + 0.3) * np.cos(tp * y - 0.5)
    u = 0.3 + 0.1 * np.cos(tp * y + 1.1)
    v = -0.2 + 0.1 * np.sin(tp * x - 0.4)
    p = 1.0 + 0.15 * np.cos(tp * (x + y) + 0.7)
    return inputs.primitive_to_conservative(rho, u, v, p)


def fd_dot(f, w, d, lam, hs=(3e-5, 1e-5, 3e-6, 1e-6, 3e-7)):
    return [np.sum(lam * (f(w + h * d) - f(w - h * d))) / (2 * h) for h in hs]


def best_rel(ref, cands):
    return min(abs(c - ref) / abs(ref) for c in cands)


@pytest.fixture(scope="module", params=["transmissive", "dirichlet"])
def case(request):
    if request.param == "transmissive":
        # 20 x 20 box with 5 ghost layers on every side: 900 vertices
        m = inputs.box_lattice(20, ghost_layers=5, jitter=0.1, seed=88)
        w = smooth_state(m.xy, 1.0, 1.0)
    else:
        # channel [-65, 15] x [-40, 40), h = 5, 5 Dirichlet ghost columns each side
        m = inputs.channel_lattice(16, ghost_layers=5)
        w = smooth_state(m.xy, 80.0, 80.0)
    g = m.ghost_donor
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly, ghost=g)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0, ghost_donor=g)
    return request.param, m, w, om, M


def filled(m, w):
    """w through the ghost fill: each ghost row takes its donor's."""
    out = w.copy()
    gh = m.ghost_donor >= 0
    out[gh] = w[m.ghost_donor[gh]]
    return out


def _dl(w, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal(w.shape) * np.abs(w).mean(0) * 1e-2
    lam = rng.standard_normal(w.shape)
    return d, lam


def _check_ghost_rows(kind, m, grad):
    ghost = m.ghost_donor >= 0
    assert ghost.sum() > 0
    if kind == "transmissive":
        assert np.all(grad[ghost] == 0)
    else:
        # the boundary values reach the real vertices through the stencils
        assert np.abs(grad[ghost]).max() > 0


def test_residual_vjp_with_ghosts(case):
    kind, m, w, om, M = case
    d, lam = _dl(w, 11)
    M.set_state(w)
    g = M.residual_vjp(lam)
    _check_ghost_rows(kind, m, g)
    adj = float(np.sum(g * d))
    assert best_rel(adj, fd_dot(lambda x: om.residual(x), w, d, lam)) < 1e-6


def test_rk_step_vjp_with_ghosts(case):
    kind, m, w, om, M = case
    d, lam = _dl(w, 12)
    M.set_state(w)
    dt = M.max_dt(0.5)
    g = M.rk_step_vjp(dt, lam)
    _check_ghost_rows(kind, m, g)
    # the state is not changed: it is still w after the ghost fill
    np.testing.assert_array_equal(M.get_state(), filled(m, w))
    adj = float(np.sum(g * d))
    assert best_rel(adj, fd_dot(lambda x: om.rk3_step(x, dt), w, d, lam)) < 1e-6
    if kind == "dirichlet":
        # a Dirichlet ghost keeps its value through the step: a cotangent on
        # the ghost rows alone comes back unchanged (to the rounding of the
        # stage weights 1/3 + 3/4 * 2/3 + 1/4 * 2/3 = 1) and reaches no real row
        ghost = m.ghost_donor >= 0
        lam2 = np.where(ghost[:, None], lam, 0.0)
        M.set_state(w)
        g2 = M.rk_step_vjp(dt, lam2)
        assert np.all(g2[~ghost] == 0)
        np.testing.assert_allclose(g2, lam2, rtol=1e-15, atol=0)


@pytest.mark.parametrize("K", [1, 2, 5])
def test_adjoint_rk_with_ghosts(case, K):
    kind, m, w, om, M = case
    d, lam = _dl(w, 13)
    M.set_state(w)
    dt = 0.5 * M.max_dt(0.5)
    n = 4

    def run(x):
        for _ in range(n):
            x = om.rk3_step(x, dt)
        return x

    g = M.adjoint_rk(dt, n, lam, checkpoint_every=K)
    _check_ghost_rows(kind, m, g)
    adj = float(np.sum(g * d))
    assert best_rel(adj, fd_dot(run, w, d, lam)) < 1e-6
    # the mesh holds w again (after the ghost fill)
    np.testing.assert_array_equal(M.get_state(), filled(m, w))


def test_rk_adjoint_refuses_positivity_safeguard():
    m = inputs.channel_lattice(16, ghost_layers=5)
    w = smooth_state(m.xy, 80.0, 80.0)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0, ghost_donor=m.ghost_donor, positivity_alpha=0.1)
    M.set_state(w)
    M.residual_vjp(np.ones_like(w))  # the residual does not use the safeguard
    with pytest.raises(fdu.FduError):
        M.rk_step_vjp(0.01, np.ones_like(w))
    with pytest.raises(fdu.FduError):
        M.adjoint_rk(0.01, 2, np.ones_like(w))
