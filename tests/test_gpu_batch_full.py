"""The batched persistent stage on its full-size path: four periodic vortex
meshes of 40k-120k vertices (312k vertices, 936k edges), large enough that
every grid-stride loop of the persistent kernel runs many times.  Launch
shapes with one block per SM give each thread the most iterations (at 128
threads a block: about 48 edges and 16 vertices per thread on 152 SMs).

Checked against the FP64 oracle after 2 SSP-RK3 steps at each mesh's own
CFL-0.5 time step, on the first and the largest (last) mesh:
  - FP64 and precision 48: relative L2 of the state increment <= 1e-12 per
    component;
  - FP32 residual path with FP64 accumulation: the increment (a weighted
    sum of FP32 residuals) <= 1e-4 per component, the state's rho and rhoE
    <= 1e-5 relative L2 (the FP32 targets);
and every launch shape gives the same bits (each edge and vertex is computed
independently of the grid-stride assignment).
"""
import numpy as np
import pytest

import oracle
from paper_2102_12933_gb300 import fdu, inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

# (n, seed, vortex strength, centre): 40,000 / 62,500 / 90,000 / 119,716 vertices
SPECS = [(200, 21, 2.5, (4.0, 6.0)), (250, 22, 4.0, (5.5, 3.5)), (300, 23, 1.5, (6.5, 5.0)),
         (346, 24, 5.0, (5.0, 5.0))]
STEPS = 2
CHECKED = (0, 3)  # meshes compared with the oracle


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def big_batch():
    cases = [inputs.vortex_case(n, seed=s, beta=b, centre=c) for n, s, b, c in SPECS]
    B = fdu.Batch([(m.xy, m.tri) for m, _ in cases], L=10.0, device=0)
    w0 = np.concatenate([w for _, w in cases])
    B.set_state(w0)
    dts = B.batch_max_dt(0.5)
    want = {}
    for i in CHECKED:
        m, w = cases[i]
        om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
        assert om.max_dt(w, 0.5) == pytest.approx(dts[i], rel=1e-14)
        wo = w.copy()
        for _ in range(STEPS):
            wo = om.rk3_step(wo, dts[i])
        want[i] = wo
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    yield B, cases, w0, dts, want, sms
    B.close()


def _run(B, w0, dts, prec, threads, blocks_per_sm):
    B.set_launch(threads, blocks_per_sm)
    B.set_state(w0)
    B.set_dt(dts)
    B.batch_rk_steps(STEPS, prec)
    return B.get_state()


def test_grid_stride_loops_run_many_times(big_batch):
    B, cases, w0, dts, want, sms = big_batch
    assert B.nv >= 10 * 128 * sms and B.ne >= 30 * 128 * sms
    assert B.nv >= 5 * 256 * sms


@pytest.mark.parametrize("prec", [64, 48])
def test_full_size_batch_matches_oracle(big_batch, prec):
    B, cases, w0, dts, want, sms = big_batch
    ref = None
    for threads, bps in ((128, 1), (256, 1), (128, 2)):
        got = _run(B, w0, dts, prec, threads, bps)
        if ref is None:
            ref = got
            for i in CHECKED:
                sl = slice(B.offsets[i], B.offsets[i + 1])
                w = cases[i][1]
                for k in range(4):
                    assert rel_l2(got[sl, k] - w[:, k], want[i][:, k] - w[:, k]) <= 1e-12, (prec, i, k)
        else:
            assert np.array_equal(got, ref), (prec, threads, bps)


def test_full_size_batch_f32_error_against_oracle(big_batch):
    B, cases, w0, dts, want, sms = big_batch
    ref = None
    t, b, _ = B.autotune(32)
    for threads, bps in ((128, 1), (256, 1), (t, b)):
        got = _run(B, w0, dts, 32, threads, bps)
        if ref is None:
            ref = got
            for i in CHECKED:
                sl = slice(B.offsets[i], B.offsets[i + 1])
                w = cases[i][1]
                for k in range(4):
                    assert rel_l2(got[sl, k] - w[:, k], want[i][:, k] - w[:, k]) <= 1e-4, (i, k)
                for k in (0, 3):
                    assert rel_l2(got[sl, k], want[i][:, k]) <= 1e-5, (i, k)
        else:
            assert np.array_equal(got, ref), (threads, bps)
