"""Batched meshes: one cooperative persistent launch per RK stage over many
independent periodic vortex meshes of uneven size.

The persistent kernel runs the same per-edge and per-vertex arithmetic as
the standalone kernels, so every mesh of a batch must advance exactly as it
does alone (FP64 and precision 48: relative L2 of the state increment
<= 1e-13; FP32 residual path: <= 1e-6), and one mesh is also checked against
the oracle (<= 1e-12).
The bounded grid barrier's failure path is exercised by a wait that cannot
complete: it must come back as FDU_ERR_TIMEOUT, not as a fault or a hang.
"""
import numpy as np
import pytest

import oracle
from paper_2102_12933_gb300 import fdu, inputs

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

SPECS = [(16, 11, 2.0, (4.0, 5.0)), (23, 12, 5.0, (5.0, 5.5)), (29, 13, 3.0, (6.0, 4.0))]


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def batch():
    cases = []
    for n, seed, beta, centre in SPECS:
        m, w0 = inputs.vortex_case(n, seed=seed, beta=beta, centre=centre)
        cases.append((m, w0))
    B = fdu.Batch([(m.xy, m.tri) for m, _ in cases], L=10.0, device=0)
    w0 = np.concatenate([w for _, w in cases])
    return B, cases, w0


def test_batch_layout(batch):
    B, cases, w0 = batch
    assert B.n_meshes == 3
    assert list(np.diff(B.offsets)) == [m.nv for m, _ in cases]


def test_batch_dt_matches_single_meshes(batch):
    B, cases, w0 = batch
    B.set_state(w0)
    dts = B.batch_max_dt(0.5)
    for (m, w), dt in zip(cases, dts):
        M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0)
        M.set_state(w)
        assert dt == M.max_dt(0.5)


@pytest.mark.parametrize("prec,tol", [(64, 1e-13), (48, 1e-13), (32, 1e-6)])
def test_batch_steps_match_single_meshes(batch, prec, tol):
    B, cases, w0 = batch
    B.set_state(w0)
    dts = B.batch_max_dt(0.5)
    B.set_dt(dts)
    B.batch_rk_steps(4, prec)
    got = B.get_state()
    for i, ((m, w), dt) in enumerate(zip(cases, dts)):
        M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0)
        M.set_state(w)
        for _ in range(4):
            M.rk_step(dt, prec)
        want = M.get_state()
        sl = slice(B.offsets[i], B.offsets[i + 1])
        for k in range(4):
            assert rel_l2(got[sl, k] - w[:, k], want[:, k] - w[:, k]) <= tol


def test_batch_mesh_matches_oracle(batch):
    B, cases, w0 = batch
    B.set_state(w0)
    dts = B.batch_max_dt(0.5)
    B.set_dt(dts)
    B.batch_rk_steps(3, 64)
    got = B.get_state()
    m, w = cases[1]
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
    wo = w.copy()
    for _ in range(3):
        wo = om.rk3_step(wo, dts[1])
    sl = slice(B.offsets[1], B.offsets[2])
    for k in range(4):
        assert rel_l2(got[sl, k] - w[:, k], wo[:, k] - w[:, k]) <= 1e-12


@pytest.mark.parametrize("prec", [32, 48])
def test_autotune_keeps_state_and_picks_admissible_shape(batch, prec):
    B, cases, w0 = batch
    B.set_state(w0)
    B.set_dt(B.batch_max_dt(0.5))
    t, b, ms = B.autotune(prec)
    assert t in (128, 256, 512) and b >= 1 and ms > 0
    assert np.array_equal(B.get_state(), w0)


def test_barrier_timeout_is_reported_not_hung(batch):
    B, cases, w0 = batch
    B.set_state(w0)
    B.set_dt(B.batch_max_dt(0.5))
    assert B.barrier_selftest() == -6  # FDU_ERR_TIMEOUT
    assert np.array_equal(B.get_state(), w0)
    # the batch still steps correctly afterwards
    B.batch_rk_steps(1, 64)
    a = B.get_state()
    B.set_state(w0)
    B.batch_rk_steps(1, 64)
    assert np.array_equal(a, B.get_state())


@pytest.mark.parametrize("prec", [32, 64, 48])
def test_launch_shape_does_not_change_results(batch, prec):
    # every edge and vertex is computed independently of the grid-stride
    # assignment, so any admissible launch shape gives the same bits
    B, cases, w0 = batch
    B.set_state(w0)
    B.set_dt(B.batch_max_dt(0.5))
    ref = None
    shapes = ((128, 1), (256, 1), (512, 1), (128, 2)) if prec != 64 else ((128, 1), (256, 1), (128, 2), (128, 3))
    for t, b in shapes:
        B.set_launch(t, b)
        B.set_state(w0)
        B.batch_rk_steps(2, prec)
        s = B.get_state()
        if ref is None:
            ref = s
        assert np.array_equal(s, ref)


def test_launch_shape_arguments_are_checked(batch):
    B, cases, w0 = batch
    for t, b in ((100, 1), (256, 0), (128, 1000)):
        with pytest.raises(fdu.FduError):
            B.set_launch(t, b)


def test_shape_too_large_for_fp64_is_an_error_not_a_launch(batch):
    # the FP64 stage kernel does not fit 512 threads per block: the step
    # reports FDU_ERR_ARG before any launch and leaves the state untouched
    B, cases, w0 = batch
    B.set_state(w0)
    B.set_dt(B.batch_max_dt(0.5))
    B.set_launch(512, 1)
    with pytest.raises(fdu.FduError):
        B.batch_rk_steps(1, 64)
    assert np.array_equal(B.get_state(), w0)
    B.set_launch(128, 1)
