"""Shock-vortex interaction (Section 3.2) on the GPU against the oracle:
periodic in y, Dirichlet ghost columns in x, the stage positivity safeguard
on (alpha 0.1, identical on both sides).

FP64 after 10 adaptive steps: relative L2 of the state increment <= 1e-10
(the safeguard's halving decisions are taken in the same order on both
sides; rounding differences grow slowly near the shock).  Dirichlet ghosts
keep their state bit for bit; FP32 stays within 1e-5 of FP64.
"""
import numpy as np
import pytest

import oracle
from paper_2102_12933_gb300 import fdu, inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_shock_vortex_steps_match_oracle_and_keep_dirichlet_ghosts():
    m, w0 = inputs.shock_vortex_case(80)
    g = m.ghost_donor >= 0
    om = oracle.OracleMesh(m.xy, m.tri, 0.0, 80.0, ghost=m.ghost_donor)
    om.set_positivity(0.1)
    M = fdu.Mesh(m.xy, m.tri, 0.0, 80.0, device=0, ghost_donor=m.ghost_donor, positivity_alpha=0.1)
    M.set_state(w0)
    t_end = 10.0
    steps, t = M.advance(0.5, t_end, 64, max_steps=10)
    assert steps == 10
    got = M.get_state()
    w, tt = w0.copy(), 0.0
    for _ in range(10):
        dt = min(om.max_dt(w, 0.5), t_end - tt)
        w = om.rk3_step(w, dt)
        tt += dt
    assert t == pytest.approx(tt, rel=1e-12)
    for k in range(4):
        assert rel_l2(got[:, k] - w0[:, k], w[:, k] - w0[:, k]) <= 1e-10
    assert np.array_equal(got[g], w0[g])
    # FP32 residual path with FP64 accumulation, same steps
    M.set_state(w0)
    M.advance(0.5, t_end, 32, max_steps=10)
    got32 = M.get_state()
    assert np.array_equal(got32[g], w0[g])
    for k in (0, 3):
        assert rel_l2(got32[~g, k], got[~g, k]) <= 1e-5
