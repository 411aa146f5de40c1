"""GPU parity at the full sizes of the larger workloads, on outputs the oracle
computes one by one (sampled vertices, the oracle's masked residual):

  - the four-quadrant Riemann problem on the 1000 x 1000 lattice of [0,1]^2
    with five transmissive ghost layers (1.02M vertices), at its
    discontinuous initial state: random vertices plus the vertices along
    the quadrant interfaces, where the positivity fallback and the
    nonlinear weights' switching act;
  - the 64-mesh batch of uneven periodic vortex meshes (3.2M vertices in
    one fdu_mesh), through the residual entry point, at sampled vertices of
    its largest and smallest meshes, its weakest vortex and two others.

Tolerances as in tests/test_gpu_parity.py: FP64 and precision 48 within
1e-12 relative L2 per component, the FP32 path within 1e-4 on the Riemann
mesh.  On the batch the FP32 bound is 1e-4 x max(1, 5 / beta) for a mesh
whose vortex has strength beta: the FP32 error is set by the rounding of the
weighted flux sums (2^-24 x the free-stream flux scale / h, the same for every
vortex), while the residual it is divided by grows with the vortex
strength; 1e-4 is the bound of the beta = 5 meshes.
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


def test_riemann_million_vertex_sampled_parity():
    m, w0 = inputs.riemann_case(1000, ghost_layers=5, seed=1003)
    real = m.ghost_donor < 0
    assert m.nv > 1_000_000
    M = fdu.Mesh(m.xy, m.tri, 0.0, 0.0, device=0, ghost_donor=m.ghost_donor)
    M.set_state(w0)
    got = {p: M.residual(p) for p in (64, 48, 32)}
    M.close()
    rng = np.random.default_rng(33)
    x, y = m.xy[:, 0], m.xy[:, 1]
    mask = np.zeros(m.nv, np.uint8)
    mask[rng.choice(np.flatnonzero(real), 1500, replace=False)] = 1
    near = real & ((np.abs(x - 0.5) < 0.004) | (np.abs(y - 0.5) < 0.004))
    mask[rng.choice(np.flatnonzero(near), min(1500, int(near.sum())), replace=False)] = 1
    om = oracle.OracleMesh(m.xy, m.tri, 0.0, 0.0, ghost=m.ghost_donor)
    want = om.residual(w0, mask=mask)
    sel = mask.astype(bool)
    assert np.abs(want[sel]).max() > 1.0  # the interfaces are in the sample
    for p, tol in ((64, 1e-12), (48, 1e-12), (32, 1e-4)):
        for k in range(4):
            assert rel_l2(got[p][sel, k], want[sel, k]) <= tol, (p, k)
        assert np.array_equal(got[p][~real], np.zeros_like(got[p][~real])), p


def test_batch_of_64_meshes_sampled_parity():
    n_i, beta, centres = inputs.batch_sizes(64, seed=2004)
    cases = [inputs.vortex_case(int(n_i[i]), seed=3000 + i, beta=float(beta[i]), centre=tuple(centres[i]))
             for i in range(len(n_i))]
    B = fdu.Batch([(m.xy, m.tri) for m, _ in cases], L=10.0, device=0)
    assert B.n_meshes == 64 and B.nv > 3_000_000
    B.set_state(np.concatenate([w for _, w in cases]))
    got = {p: B.residual(p) for p in (64, 48, 32)}
    B.close()
    sizes = np.array([m.nv for m, _ in cases])
    # the largest and smallest meshes, the weakest vortex, two others
    pick = sorted({int(np.argmax(sizes)), int(np.argmin(sizes)), int(np.argmin(beta)), 17, 42})
    rng = np.random.default_rng(44)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for i in pick:
        m, w = cases[i]
        mask = np.zeros(m.nv, np.uint8)
        mask[rng.choice(m.nv, min(800, m.nv), replace=False)] = 1
        want = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly).residual(w, mask=mask)
        sel = mask.astype(bool)
        for p, tol in ((64, 1e-12), (48, 1e-12), (32, 1e-4 * max(1.0, 5.0 / float(beta[i])))):
            g = got[p][off[i]:off[i + 1]]
            for k in range(4):
                assert rel_l2(g[sel, k], want[sel, k]) <= tol, (i, p, k)
