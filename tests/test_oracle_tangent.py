"""Pins of the oracle's complex-step tangents (the directional derivatives
J d that the GPU adjoint is checked against), against what is fixed
independently of them:

- the real part of the complex evaluation is the oracle's value, bit for bit
  (the complex copy takes the same branches and the imaginary parts are far
  below the rounding of the real parts);
- J d agrees with central differences of the real oracle to their own
  accuracy (truncation O(h^2) plus rounding O(eps/h), best of a ladder);
- J is linear: J(a d1 + b d2) = a J d1 + b J d2 to rounding;
- free stream (Section 2.2.1 is exact for constant fluxes): the residual of
  every uniform state is zero, so at a uniform state J d = 0 for any
  uniform perturbation d;
- the RK3 step's tangent at dt -> 0 tends to the identity plus dt times the
  residual's tangent (Shu-Osher stages with L -> J d), and over several
  steps matches central differences of the stepped oracle;
- ghost layers: a transmissive ghost's tangent is its donor's (the fill
  copies it), and the residual's tangent does not depend on the ghost rows
  of d.  Central differences agree away from the boundary only: the fill
  makes the ghost layers constant along the normal, so sub-stencils inside
  them have beta = eps exactly, where the nonlinear weights are not
  differentiable (a perturbation of size h moves beta to h^2 >> eps = 1e-40)
  and differences see another branch than the derivative.
"""
import numpy as np
import pytest

import oracle
from paper_2102_12933_gb300 import inputs


def _smooth(m, amp=0.02):
    w = inputs.isentropic_vortex(m.xy)
    x, y = m.xy[:, 0], m.xy[:, 1]
    for c in range(4):
        w[:, c] *= 1.0 + amp * np.sin(2 * np.pi * (x + 1.3 * c) / 10) * np.cos(2 * np.pi * (y - 0.7 * c) / 10)
    return w


@pytest.fixture(scope="module")
def case():
    m, _ = inputs.vortex_case(16, seed=1001)
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
    w = _smooth(m)
    rng = np.random.default_rng(3)
    d = rng.standard_normal(w.shape) * np.abs(w).mean(0) * 1e-2
    return m, om, w, d


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_real_part_is_the_oracle(case):
    m, om, w, d = case
    val, _ = om.residual_jvp(w, d, return_value=True)
    assert np.array_equal(val, om.residual(w))
    state, _ = om.rk3_steps_jvp(w, d, 0.01, n=2)
    assert np.array_equal(state, om.rk3_step(om.rk3_step(w, 0.01), 0.01))


def test_tangent_matches_central_differences(case):
    m, om, w, d = case
    jd = om.residual_jvp(w, d)
    errs = [rel((om.residual(w + h * d) - om.residual(w - h * d)) / (2 * h), jd) for h in (1e-5, 1e-6, 1e-7)]
    assert min(errs) < 1e-7


def test_tangent_is_linear(case):
    m, om, w, d = case
    d2 = np.roll(d, 7, axis=0) * 0.5
    lhs = om.residual_jvp(w, 2.0 * d - 3.0 * d2)
    rhs = 2.0 * om.residual_jvp(w, d) - 3.0 * om.residual_jvp(w, d2)
    assert rel(lhs, rhs) < 1e-12


def test_free_stream_tangent_vanishes():
    m, _ = inputs.vortex_case(16, seed=1001)
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
    one = np.ones(m.nv)
    w = inputs.primitive_to_conservative(1.2 * one, 0.4 * one, -0.3 * one, 0.9 * one)
    d = np.tile(np.array([0.3, -0.1, 0.25, 0.7]), (m.nv, 1))
    jd = om.residual_jvp(w, d)
    # the residual's size at a unit gradient is about |d| / h: compare with it
    h = 10.0 / 16
    assert np.abs(jd).max() < 1e-12 * np.abs(d).max() / h


def test_rk3_tangent(case):
    m, om, w, d = case
    dt = 1e-7
    _, jstep = om.rk3_steps_jvp(w, d, dt)
    jres = om.residual_jvp(w, d)
    assert rel((jstep - d) / dt, jres) < 1e-5  # O(dt) from the stages
    dt = 0.5 * om.max_dt(w, 0.5)
    _, j3 = om.rk3_steps_jvp(w, d, dt, n=3)

    def run(x):
        for _ in range(3):
            x = om.rk3_step(x, dt)
        return x

    errs = [rel((run(w + h * d) - run(w - h * d)) / (2 * h), j3) for h in (1e-5, 1e-6, 1e-7)]
    assert min(errs) < 1e-7


def test_ghost_layers():
    n = 30
    m = inputs.box_lattice(n, ghost_layers=5, jitter=0.1, seed=88)
    x, y = m.xy[:, 0], m.xy[:, 1]
    w = inputs.primitive_to_conservative(1 + 0.2 * np.sin(2 * np.pi * x), 0.3 + 0.1 * np.cos(2 * np.pi * y),
                                         -0.2 + 0.1 * np.sin(2 * np.pi * x), 1 + 0.1 * np.cos(2 * np.pi * (x + y)))
    om = oracle.OracleMesh(m.xy, m.tri, 0.0, 0.0, ghost=m.ghost_donor)
    rng = np.random.default_rng(4)
    d = rng.standard_normal(w.shape) * 1e-2
    ghost = m.ghost_donor >= 0
    d2 = d.copy()
    d2[ghost] = rng.standard_normal((int(ghost.sum()), 4))
    jd, jd2 = om.residual_jvp(w, d), om.residual_jvp(w, d2)
    assert np.array_equal(jd, jd2)  # the fill overwrites the ghost rows of d
    # central differences two lattice spacings and more from the boundary
    dist = np.minimum.reduce([x, 1 - x, y, 1 - y])
    inner = (~ghost) & (dist > 2.0 / (n - 1))
    errs = [rel(((om.residual(w + h * d) - om.residual(w - h * d)) / (2 * h))[inner], jd[inner])
            for h in (1e-5, 1e-6, 1e-7)]
    assert min(errs) < 1e-7
    # after a step the ghosts hold their donors' tangents
    _, js = om.rk3_steps_jvp(w, d, 1e-3)
    gi = np.nonzero(ghost)[0]
    assert np.array_equal(js[gi], js[m.ghost_donor[gi]])
