"""Hand-written adjoint: dot-product tests <lam, J d> = <J^T lam, d> with J d
from central finite differences of the GPU forward and of the oracle.

The state is the vortex plus a smooth perturbation of every component, so
that no smoothness indicator sits near the WENO epsilon (where the weights
are not differentiable and finite differences see a different branch).
Central differences with step h have truncation error O(h^2) and rounding
error O(eps/h); the best of a short ladder of steps is compared at 1e-6
relative (the stated gradient target), the oracle-derived reference likewise.
"""
import numpy as np
import pytest

import oracle
from paper_2102_12933_gb300 import fdu, inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def smooth_state(m):
    w = inputs.isentropic_vortex(m.xy)
    x, y = m.xy[:, 0], m.xy[:, 1]
    for c in range(4):
        w[:, c] *= 1.0 + 0.02 * np.sin(2 * np.pi * (x + 1.3 * c) / 10) * np.cos(2 * np.pi * (y - 0.7 * c) / 10)
    return w


@pytest.fixture(scope="module")
def case():
    m = inputs.torus_lattice(30, L=10.0, jitter=0.2, seed=77)
    w = smooth_state(m)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0)
    return m, w, M


def fd_dot(f, w, d, lam, hs=(3e-5, 1e-5, 3e-6, 1e-6, 3e-7)):
    out = []
    for h in hs:
        out.append(np.sum(lam * (f(w + h * d) - f(w - h * d))) / (2 * h))
    return out


def best_rel(ref, cands):
    return min(abs(c - ref) / abs(ref) for c in cands)


def test_residual_vjp_dot_product_gpu_and_oracle(case):
    m, w, M = case
    rng = np.random.default_rng(1)
    d = rng.standard_normal(w.shape) * np.abs(w).mean(0) * 1e-2
    lam = rng.standard_normal(w.shape)
    M.set_state(w)
    g = M.residual_vjp(lam)
    adj = float(np.sum(g * d))

    def gpu_res(x):
        M.set_state(x)
        return M.residual(64)

    assert best_rel(adj, fd_dot(gpu_res, w, d, lam)) < 1e-6
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
    assert best_rel(adj, fd_dot(lambda x: om.residual(x), w, d, lam)) < 1e-6
    # device buffers give the same numbers
    lt = torch.tensor(lam, device="cuda")
    gt = torch.empty_like(lt)
    M.set_state(w)
    M.residual_vjp(lt, out=gt)
    torch.cuda.synchronize()
    assert np.array_equal(gt.cpu().numpy(), g)


def test_rk_step_vjp_dot_product(case):
    m, w, M = case
    rng = np.random.default_rng(2)
    d = rng.standard_normal(w.shape) * np.abs(w).mean(0) * 1e-2
    lam = rng.standard_normal(w.shape)
    M.set_state(w)
    dt = M.max_dt(0.5)
    g = M.rk_step_vjp(dt, lam)
    assert np.array_equal(M.get_state(), w)  # state unchanged
    adj = float(np.sum(g * d))

    def step(x):
        M.set_state(x)
        M.rk_step(dt, 64)
        return M.get_state()

    assert best_rel(adj, fd_dot(step, w, d, lam)) < 1e-6


def test_adjoint_rk_gradient_of_density_misfit(case):
    """J = 1/2 sum (rho(T) - rho_exact(T))^2 after 20 steps, checkpoint every 10."""
    m, w, M = case
    M.set_state(w)
    dt = M.max_dt(0.5)
    n = 20
    ex = inputs.isentropic_vortex(m.xy, t=n * dt)

    def J_and_lam(x):
        M.set_state(x)
        M.rk_steps(dt, n, 64)
        wt = M.get_state()
        r = wt[:, 0] - ex[:, 0]
        lam = np.zeros_like(wt)
        lam[:, 0] = r
        return 0.5 * float(np.sum(r * r)), lam

    J0, lamT = J_and_lam(w)
    M.set_state(w)
    g = M.adjoint_rk(dt, n, lamT, checkpoint_every=10)
    assert np.array_equal(M.get_state(), w)
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = rng.standard_normal(w.shape) * np.abs(w).mean(0) * 1e-2
        adj = float(np.sum(g * d))
        fds = [(J_and_lam(w + h * d)[0] - J_and_lam(w - h * d)[0]) / (2 * h) for h in (1e-4, 3e-5, 1e-5, 3e-6, 1e-6, 3e-7)]
        assert best_rel(adj, fds) < 1e-6


def test_checkpoint_interval_does_not_change_the_gradient(case):
    m, w, M = case
    M.set_state(w)
    dt = M.max_dt(0.5)
    lam = np.random.default_rng(4).standard_normal(w.shape)
    outs = []
    for k in (1, 3, 5, 10, 12, 20):  # uneven last segments, one segment, interval beyond the run
        M.set_state(w)
        outs.append(M.adjoint_rk(dt, 12, lam, checkpoint_every=k))
        assert np.array_equal(M.get_state(), w)  # the mesh is back at the initial state
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_autograd_functions(case):
    from paper_2102_12933_gb300.autograd import Residual, RKSteps

    m, w, M = case
    w0 = torch.tensor(w, device="cuda", requires_grad=True)
    M.set_state(w)
    dt = M.max_dt(0.5)
    wT = RKSteps.apply(w0, M, dt, 6, 3)
    loss = 0.5 * (wT[:, 0] ** 2).sum()
    loss.backward()
    lam = np.zeros_like(w)
    lam[:, 0] = wT[:, 0].detach().cpu().numpy()
    M.set_state(w)
    ref = M.adjoint_rk(dt, 6, lam, checkpoint_every=3)
    assert np.array_equal(w0.grad.cpu().numpy(), ref)
    w1 = torch.tensor(w, device="cuda", requires_grad=True)
    r = Residual.apply(w1, M)
    (r * r).sum().backward()
    M.set_state(w)
    lam2 = 2 * M.residual(64)
    M.set_state(w)
    assert np.array_equal(w1.grad.cpu().numpy(), M.residual_vjp(lam2))


def test_autograd_functions_precision48(case):
    """precision = 48 runs the forward in precision 48 and the backward with
    the adjoint precision 48 (restored afterwards); the gradients are the
    direct calls' bits, and within 1e-10 of the FP64 ones."""
    from paper_2102_12933_gb300.autograd import Residual, RKSteps

    m, w, M = case
    w0 = torch.tensor(w, device="cuda", requires_grad=True)
    M.set_state(w)
    dt = M.max_dt(0.5)
    wT = RKSteps.apply(w0, M, dt, 6, 3, 48)
    loss = 0.5 * (wT[:, 0] ** 2).sum()
    loss.backward()
    assert M.adjoint_precision == 64
    lam = np.zeros_like(w)
    lam[:, 0] = wT[:, 0].detach().cpu().numpy()
    M.set_adjoint_precision(48)
    M.set_state(w)
    ref = M.adjoint_rk(dt, 6, lam, checkpoint_every=3)
    M.set_adjoint_precision(64)
    assert np.array_equal(w0.grad.cpu().numpy(), ref)
    M.set_state(w)
    ref64 = M.adjoint_rk(dt, 6, lam, checkpoint_every=3)
    assert np.linalg.norm(ref - ref64) <= 1e-10 * np.linalg.norm(ref64)
    w1 = torch.tensor(w, device="cuda", requires_grad=True)
    r = Residual.apply(w1, M, 48)
    (r * r).sum().backward()
    M.set_state(w)
    lam2 = 2 * M.residual(48)
    M.set_adjoint_precision(48)
    M.set_state(w)
    want = M.residual_vjp(lam2)
    M.set_adjoint_precision(64)
    assert np.array_equal(w1.grad.cpu().numpy(), want)
