"""Pins of the Dirichlet ghost boundary and the shock-vortex initial data
(Section 3.2), against what the mathematics fixes:

- Rankine-Hugoniot: the stationary shock's two states carry the same
  x-fluxes of mass, momentum and energy, and the upstream Mach number is 1.2;
- the vortex is isentropic (p / rho^gamma = 1/gamma) and decays to the
  upstream state;
- Dirichlet ghosts (their own donor) keep their state exactly through RK
  steps, and a uniform flow in the channel (periodic in y, Dirichlet ghost
  columns in x) is preserved to rounding.
"""
import numpy as np

import oracle
from paper_2102_12933_gb300 import inputs

G = 1.4


def _xflux(w):
    rho, mx, my, E = w.T
    u = mx / rho
    p = (G - 1) * (E - 0.5 * (mx * mx + my * my) / rho)
    return np.stack([mx, mx * u + p, my * u, (E + p) * u], 1)


def test_shock_states_satisfy_rankine_hugoniot():
    xy = np.array([[5.0, 30.0], [-5.0, 30.0]])
    w = inputs.shock_vortex(xy, mach_vortex=0.0)
    f = _xflux(w)
    assert np.allclose(f[0], f[1], rtol=1e-14, atol=1e-14)
    rho, u = w[0, 0], w[0, 1] / w[0, 0]
    p = (G - 1) * (w[0, 3] - 0.5 * w[0, 1] ** 2 / rho)
    assert abs(-u / np.sqrt(G * p / rho) - 1.2) < 1e-14
    assert w[1, 0] > w[0, 0]  # compression across the shock


def test_vortex_is_isentropic_and_decays():
    rng = np.random.default_rng(3)
    xy = np.stack([rng.uniform(0.5, 8, 500), rng.uniform(-4, 4, 500)], 1)
    w = inputs.shock_vortex(xy)
    rho = w[:, 0]
    p = (G - 1) * (w[:, 3] - 0.5 * (w[:, 1] ** 2 + w[:, 2] ** 2) / rho)
    assert np.allclose(p / rho ** G, 1 / G, rtol=1e-13)
    far = inputs.shock_vortex(np.array([[14.0, 30.0]]))[0]
    assert np.allclose(far, inputs.shock_vortex(np.array([[14.0, 30.0]]), mach_vortex=0.0)[0], atol=1e-12)


def test_dirichlet_ghosts_keep_their_state():
    m, w0 = inputs.shock_vortex_case(40)
    g = m.ghost_donor >= 0
    assert np.all(m.ghost_donor[g] == np.nonzero(g)[0])
    om = oracle.OracleMesh(m.xy, m.tri, 0.0, 80.0, ghost=m.ghost_donor)
    w = w0.copy()
    for _ in range(3):
        w = om.rk3_step(w, 0.5 * om.max_dt(w, 0.5))
    assert np.array_equal(w[g], w0[g])
    assert not np.array_equal(w[~g], w0[~g])


def test_uniform_flow_preserved_in_channel():
    m, _ = inputs.shock_vortex_case(40)
    om = oracle.OracleMesh(m.xy, m.tri, 0.0, 80.0, ghost=m.ghost_donor)
    real = m.ghost_donor < 0
    one = np.ones(m.nv)
    w = inputs.primitive_to_conservative(1.3 * one, -0.7 * one, 0.2 * one, 2.1 * one)
    assert np.abs(om.residual(w)[real]).max() < 1e-12
