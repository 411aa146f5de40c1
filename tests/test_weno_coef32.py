"""The FP32 path's NU-WENO5 coefficients, which its edge kernel forms in
registers from each edge's four stencil gaps, against the oracle's FP64
construction (Appendix: sub-stencil interpolants at the edge midpoint, their
smoothness indicators, and the linear weights C_K):

  - value coefficients against the oracle's sub-stencil Lagrange values;
  - each indicator's quadratic form, applied to random point values,
    against the oracle's indicator of the same values;
  - C_0/C_1 and C_2/C_1 of both states against the oracle's linear weights,

on every edge of a jittered periodic lattice and on strongly uneven random
stencils (neighbouring gaps differing by up to 400x).  The bound is 4e-6
relative: the gaps are rounded to FP32 once (2^-24) and every factor of the
closed forms is a sum of positive terms, so a few ulps remain; a wrong
coefficient would be off by O(1).  The argument checks run on the host.
"""
import numpy as np
import pytest

import oracle
from paper_2102_12933_gb300 import fdu, inputs

torch = pytest.importorskip("torch")
needs_gpu = pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")

TOL = 4e-6


def _uneven_stencils(n, seed):
    rng = np.random.default_rng(seed)
    g = np.exp(rng.uniform(np.log(0.05), np.log(20.0), size=(n, 4)))  # L1-L2, L2-L3, R1-R2, R2-R3
    xi = np.zeros((n, 6))
    xi[:, 2], xi[:, 3] = -0.5, 0.5
    xi[:, 1] = -0.5 - g[:, 0]
    xi[:, 0] = xi[:, 1] - g[:, 1]
    xi[:, 4] = 0.5 + g[:, 2]
    xi[:, 5] = xi[:, 4] + g[:, 3]
    return xi


def _check_block(xi, k, rng):
    for i in range(xi.shape[0]):
        x = xi[i]
        xl = x[:5]
        xr = -x[::-1][:5]  # the right state's stencil, mirrored: R3, R2, R1, L1, L2
        Ll, Lr = oracle.substencil_coeffs(xl), oracle.substencil_coeffs(xr)
        want_vals = [Ll[0, 0], Ll[0, 1], Ll[1, 0], Ll[1, 2], Ll[2, 1], Ll[2, 2], Lr[0, 0], Lr[0, 1]]
        got_vals = k[i, [0, 1, 5, 6, 10, 11, 15, 16]]
        np.testing.assert_allclose(got_vals, want_vals, rtol=TOL, atol=0)
        Cl, Cr = oracle.linear_weights(xl), oracle.linear_weights(xr)
        np.testing.assert_allclose(k[i, 20:24], [Cl[0] / Cl[1], Cl[2] / Cl[1], Cr[0] / Cr[1], Cr[2] / Cr[1]],
                                   rtol=TOL, atol=0)
        u = rng.standard_normal(6)  # values at L3, L2, L1, R1, R2, R3
        bl = oracle.smoothness(xl, u[:5])
        br = oracle.smoothness(xr, u[::-1][:5])
        a, b, c, d = u[0] - u[2], u[1] - u[2], u[3] - u[2], u[4] - u[2]
        e, f = u[5] - u[3], u[4] - u[3]
        for m, (p, q), want in ((k[i, 2:5], (a, b), bl[0]), (k[i, 7:10], (b, c), bl[1]),
                                (k[i, 12:15], (c, d), bl[2]), (k[i, 17:20], (e, f), br[0])):
            terms = np.array([m[0] * p * p, m[1] * p * q, m[2] * q * q])
            assert abs(terms.sum() - want) <= TOL * np.abs(terms).sum(), (i, m, want)


@pytest.mark.gpu
@needs_gpu
def test_coefficients_of_a_jittered_lattice():
    m, _ = inputs.vortex_case(60, seed=1002)
    M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=-1)
    _, xi = M.edge_stencils()
    M.close()
    k = fdu.check_weno_coef32(xi)
    assert k.shape == (xi.shape[0], 24) and np.all(np.isfinite(k))
    _check_block(xi, k, np.random.default_rng(71))


@pytest.mark.gpu
@needs_gpu
def test_coefficients_of_uneven_stencils():
    xi = _uneven_stencils(2000, seed=72)
    k = fdu.check_weno_coef32(xi)
    _check_block(xi, k, np.random.default_rng(73))
    # uniform spacing: the classical WENO5 values (3/8, -5/4 | -1/8, 3/8 | 3/4, -1/8),
    # C = (1/16, 10/16, 5/16), so C_0/C_1 = 1/10 and C_2/C_1 = 1/2
    k = fdu.check_weno_coef32(np.array([[-2.5, -1.5, -0.5, 0.5, 1.5, 2.5]]))[0]
    np.testing.assert_allclose(k[[0, 1, 5, 6, 10, 11, 15, 16]], [3 / 8, -5 / 4, -1 / 8, 3 / 8, 3 / 4, -1 / 8,
                                                                 3 / 8, -5 / 4], rtol=1e-6)
    np.testing.assert_allclose(k[20:24], [0.1, 0.5, 0.1, 0.5], rtol=1e-6)


def test_coefficient_check_rejects_bad_coordinates():
    """Checked on the host before any device call."""
    good = np.array([[-2.5, -1.5, -0.5, 0.5, 1.5, 2.5]])
    for bad in (good + np.array([0, 0, 0.1, 0, 0, 0]),       # L1 not at -1/2
                good[:, [1, 0, 2, 3, 4, 5]],                  # L3, L2 swapped
                good + np.array([0, 0, 0, 0, 2.0, 0])):       # R2 beyond R3
        with pytest.raises(fdu.FduError) as e:
            fdu.check_weno_coef32(bad)
        assert e.value.status == -1  # FDU_ERR_ARG
    assert fdu.check_weno_coef32(np.zeros((0, 6))).shape == (0, 24)


def _rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.gpu
@needs_gpu
def test_compact_form_fp32_parity_with_the_oracle():
    """The FP32 path with the compact coefficient form (mesh option f32_coef =
    1) under the FP32 path's bounds against the oracle: residual within 1e-4
    relative L2 per component, density and energy after 20 RK3 steps within
    1e-5; and within FP32 rounding of the default form (the FP64-built block
    streamed in FP32)."""
    m, w0 = inputs.vortex_case(40, seed=1001)
    om = oracle.OracleMesh(m.xy, m.tri, m.Lx, m.Ly)
    Mc = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0, f32_coef=1)
    Md = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0)
    Mc.set_state(w0)
    Md.set_state(w0)
    got, dflt = Mc.residual(32), Md.residual(32)
    want = om.residual(w0)
    for k in range(4):
        assert _rel_l2(got[:, k], want[:, k]) <= 1e-4
        assert _rel_l2(got[:, k], dflt[:, k]) <= 2e-5
    dt = om.max_dt(w0, 0.5)
    Mc.rk_steps(dt, 20, 32)
    wc = Mc.get_state()
    wo = w0.copy()
    for _ in range(20):
        wo = om.rk3_step(wo, dt)
    assert _rel_l2(wc[:, 0], wo[:, 0]) <= 1e-5
    assert _rel_l2(wc[:, 3], wo[:, 3]) <= 1e-5
    Mc.close()
    Md.close()


@pytest.mark.gpu
@needs_gpu
def test_compact_form_batch_matches_single_meshes():
    """The batched persistent stage takes the compact form's branch when the
    batch is built with f32_coef = 1: four FP32 steps of each mesh in the batch
    against the same mesh alone with the same option (the tolerance of the
    batch tests for FP32)."""
    cases = [inputs.vortex_case(n, seed=s) for n, s in ((16, 7101), (23, 7102), (29, 7103))]
    B = fdu.Batch([(m.xy, m.tri) for m, _ in cases], L=10.0, device=0, f32_coef=1)
    w0 = np.concatenate([w for _, w in cases])
    B.set_state(w0)
    dts = B.batch_max_dt(0.5)
    B.set_dt(dts)
    B.batch_rk_steps(4, 32)
    got = B.get_state()
    for i, ((m, w), dt) in enumerate(zip(cases, dts)):
        M = fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=0, f32_coef=1)
        M.set_state(w)
        for _ in range(4):
            M.rk_step(dt, 32)
        want = M.get_state()
        M.close()
        sl = slice(B.offsets[i], B.offsets[i + 1])
        for k in range(4):
            assert _rel_l2(got[sl, k] - w[:, k], want[:, k] - w[:, k]) <= 1e-6
    B.close()


def test_f32_coef_option_is_checked():
    """Checked on the host before any device use."""
    m, _ = inputs.vortex_case(8, seed=7104)
    with pytest.raises(fdu.FduError) as e:
        fdu.Mesh(m.xy, m.tri, m.Lx, m.Ly, device=-1, f32_coef=2)
    assert e.value.status == -1  # FDU_ERR_ARG
