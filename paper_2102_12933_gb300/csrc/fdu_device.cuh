// Device helpers shared by the forward and adjoint kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fdu {
namespace dev {

// ------------------------------------------------------------------ helpers
// A conservative FP64 record (rho, rho u, rho v, rho E), 16-byte aligned.
struct __align__(16) dbl4 {
    double x, y, z, w;
};
__device__ __forceinline__ dbl4 dbl4_make(double x, double y, double z, double w) { return dbl4{x, y, z, w}; }
__device__ __forceinline__ dbl4 ld4(const double *p, int64_t i) {
    const double2 *q = reinterpret_cast<const double2 *>(p + 4 * i);
    const double2 a = __ldg(q), b = __ldg(q + 1);
    return dbl4_make(a.x, a.y, b.x, b.y);
}
// The same record as one 256-bit load, for the library's own buffers (their
// rows are 32-byte aligned) that the kernel only reads.
__device__ __forceinline__ dbl4 ld4v(const double *p, int64_t i) {
    dbl4 r;
    asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];" : "=d"(r.x), "=d"(r.y), "=d"(r.z), "=d"(r.w) : "l"(p + 4 * i));
    return r;
}
__device__ __forceinline__ void st4(double *p, int64_t i, dbl4 v) {
    double2 *q = reinterpret_cast<double2 *>(p + 4 * i);
    q[0] = make_double2(v.x, v.y);
    q[1] = make_double2(v.z, v.w);
}
__device__ __forceinline__ dbl4 sub4(dbl4 a, dbl4 b) {
    return dbl4_make(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ dbl4 add4(dbl4 a, dbl4 b) {
    return dbl4_make(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}
__device__ __forceinline__ dbl4 neg4(dbl4 a) { return dbl4_make(-a.x, -a.y, -a.z, -a.w); }

// x > 0 decided on the integer pipe from the bit pattern (positive doubles
// order as their bits; NaN and -0 give false, as the FP64 comparison does),
// which keeps the comparison off GB300's narrow FP64 pipe.
__device__ __forceinline__ bool pos64(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b <= 0x7FF0000000000000LL;
}

// Reciprocal of a positive normal double from the hardware's approximate
// FP64 reciprocal y (PTX rcp.approx.ftz.f64) and one correction of third
// order in its residual e = 1 - x y: 1/x = y / (1 - e) = y (1 + e + e^2) +
// O(e^3), three FP64 operations.  With the approximation's relative error
// e the truncation is below e^3, far under the rounding level for the
// approximation's accuracy (the tests hold the result to 2 ulp of IEEE
// division).
__device__ __forceinline__ double recip64(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// One Newton-Raphson step from the hardware approximation: relative error
// the square of the approximation's (about 2^-20 on GB300), so near 2^-40,
// ample for quotients whose error is damped by a small
// multiplier (the nonlinear WENO weights: an error d omega moves the
// interpolant by d omega (v_k - v), and v_k - v is O(h^3)).
__device__ __forceinline__ double recip64_fast(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// 1/sqrt(x) of a positive normal double from the hardware's approximate
// FP64 reciprocal square root y (PTX rsqrt.approx.ftz.f64) and one
// correction of third order in its residual e = 1 - x y^2, from the series
// (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + O(e^3):
//   1/sqrt(x) = y + (y e) (1/2 + 3e/8) + O(e^3),
// five FP64 operations (checked against 1/sqrt(x) in extended precision by
// the tests).
__device__ __forceinline__ double rsqrt64(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y * y, 1.0);
    return fma(y * e, fma(0.375, e, 0.5), y);
}

// x / 2 on the integer pipe, without a branch: for a normal x whose half is
// normal the exponent field drops by one (exact); infinities and NaN are
// returned as they are; zero, and the halves below the normal range
// (|x| < 2^-1021), become a zero of x's sign.
__device__ __forceinline__ double half64(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const unsigned ex = ((unsigned)hi >> 20) & 0x7FFu;
    const int h2 = ex > 1u ? (ex < 0x7FFu ? hi - 0x00100000 : hi) : (int)((unsigned)hi & 0x80000000u);
    return __hiloint2double(h2, ex > 1u ? lo : 0);
}

// 2 x on the integer pipe, exact, without a branch: a normal x below the top
// binade gains one in its exponent field; a subnormal x (exponent field 0)
// doubles by shifting its significand; the top binade overflows to
// infinity; infinities and NaN are returned as they are.
__device__ __forceinline__ double twice64(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned long long mag = b & 0x7FFFFFFFFFFFFFFFULL;
    const unsigned ex = (unsigned)(mag >> 52);
    const unsigned long long r = ex == 0u      ? mag << 1
                                 : ex < 0x7FEu ? mag + (1ULL << 52)
                                 : ex == 0x7FEu ? 0x7FF0000000000000ULL
                                                : mag;
    return __longlong_as_double((long long)(r | (b & 0x8000000000000000ULL)));
}

// Per-state quantities reused by the Roe average and the physical flux.
struct Prim64 {
    double r;   // rho^-1/2
    double ir;  // 1/rho
    double p;   // pressure
};
// p = (gamma - 1) (E - (|m|^2 / 2) / rho), the halving on the integer pipe.
__device__ __forceinline__ Prim64 prim64(const dbl4 &w, double gm1) {
    Prim64 q;
    q.r = rsqrt64(w.x);
    q.ir = q.r * q.r;
    q.p = gm1 * fma(-half64(fma(w.z, w.z, w.y * w.y)), q.ir, w.w);
    return q;
}

// Roe average of two states (weights sqrt(rho)) and the eigen-quantities
// of the flux Jacobian along n; hgm1 = (gamma - 1) / 2.
struct Roe64 {
    double u, v, H, c, ic, b1, qn, qt, hq2, nx, ny;
    double b1h, ich;  // b1 / 2 and ic / 2, the factors project64 applies
    double inv;       // 1 / (sum of the sides' sqrt(rho)), kept for the adjoint
};
// Roe average from the two sides' records (same result as roe64).
__device__ __forceinline__ Roe64 roe64_from_records(const dbl4 &qa, const dbl4 &qb, double nx, double ny, double gm1,
                                                    double hgm1) {
    Roe64 R;
    const double inv = recip64(qa.x + qb.x);
    R.inv = inv;
    R.u = (qa.y + qb.y) * inv;
    R.v = (qa.z + qb.z) * inv;
    R.H = (qa.w + qb.w) * inv;
    R.hq2 = half64(R.u * R.u + R.v * R.v);
    const double c2 = gm1 * (R.H - R.hq2);
    R.ic = rsqrt64(c2);
    R.c = c2 * R.ic;
    const double ic2 = R.ic * R.ic;
    R.b1 = gm1 * ic2;
    R.b1h = hgm1 * ic2;  // hgm1 = (gamma - 1) / 2
    R.ich = half64(R.ic);
    R.nx = nx;
    R.ny = ny;
    R.qn = R.u * nx + R.v * ny;
    R.qt = R.v * nx - R.u * ny;
    return R;
}

__device__ __forceinline__ Roe64 roe64(const dbl4 &a, const Prim64 &pa, const dbl4 &b, const Prim64 &pb,
                                      double nx, double ny, double gm1, double hgm1) {
    Roe64 R;
    const double sa = a.x * pa.r, sb = b.x * pb.r;
    const double inv = recip64(sa + sb);
    R.inv = inv;
    // the sides' weights r / (sqrt(rho_a) + sqrt(rho_b)) formed once
    const double ra = pa.r * inv, rb = pb.r * inv;
    R.u = fma(a.y, ra, b.y * rb);
    R.v = fma(a.z, ra, b.z * rb);
    R.H = fma(a.w + pa.p, ra, (b.w + pb.p) * rb);
    R.hq2 = half64(R.u * R.u + R.v * R.v);
    const double c2 = gm1 * (R.H - R.hq2);
    R.ic = rsqrt64(c2);
    R.c = c2 * R.ic;
    const double ic2 = R.ic * R.ic;
    R.b1 = gm1 * ic2;
    R.b1h = hgm1 * ic2;  // hgm1 = (gamma - 1) / 2
    R.ich = half64(R.ic);
    R.nx = nx;
    R.ny = ny;
    R.qn = R.u * nx + R.v * ny;
    R.qt = R.v * nx - R.u * ny;
    return R;
}

// Characteristic components of a conservative difference (left eigenvectors
// of dF_n/dw at the Roe state; fields ordered q_n - c, q_n (entropy), q_n
// (shear), q_n + c).
// phi/2 and psi/2 are formed directly (factors b1/2, ic/2), so the four
// fields cost no separate halving.
__device__ __forceinline__ dbl4 project64(const Roe64 &R, const dbl4 &d) {
    // d.w starts the chain, so the four terms take three fused multiply-adds
    const double phh = R.b1h * fma(-R.v, d.z, fma(-R.u, d.y, fma(R.hq2, d.x, d.w)));
    const double psh = (R.qn * d.x - R.nx * d.y - R.ny * d.z) * R.ich;
    return dbl4_make(phh + psh, fma(-2.0, phh, d.x), R.nx * d.z - R.ny * d.y - R.qt * d.x, phh - psh);
}
// Conservative difference from characteristic components (right eigenvectors).
__device__ __forceinline__ dbl4 unproject64(const Roe64 &R, const dbl4 &c) {
    const double ac = c.x + c.w;  // acoustic pair
    const double rho = ac + c.y;
    const double dd = R.c * (c.w - c.x);
    return dbl4_make(rho, R.u * rho + R.nx * dd - R.ny * c.z, R.v * rho + R.ny * dd + R.nx * c.z,
                        R.H * ac + R.hq2 * c.y + R.qn * dd + R.qt * c.z);
}

// base + the conservative difference of unproject64, with base taken into
// the fused multiply-add chains (three additions fewer than add4 after
// unproject64).
__device__ __forceinline__ dbl4 unproject_add64(const Roe64 &R, const dbl4 &c, const dbl4 &base) {
    const double ac = c.x + c.w;
    const double rho = ac + c.y;
    const double dd = R.c * (c.w - c.x);
    return dbl4_make(base.x + rho, fma(R.u, rho, fma(R.nx, dd, fma(-R.ny, c.z, base.y))),
                     fma(R.v, rho, fma(R.ny, dd, fma(R.nx, c.z, base.z))),
                     fma(R.H, ac, fma(R.hq2, c.y, fma(R.qn, dd, fma(R.qt, c.z, base.w)))));
}

// NU-WENO5 increments of one characteristic field (Appendix), both sides.
// Differences: a = L3-L1, b = L2-L1, c = R1-L1, d = R2-L1 (left centre L1),
// e = R3-R1, f = R2-R1 (right centre R1).  k is the edge's coefficient block
// (fdu_internal.h, 5 values per sub-stencil): sub-stencils S_a..S_d give
// values v (increments) and smoothness indicators beta as quadratic forms
// of their two differences.  The nonlinear weights alpha_k = C_k / (beta_k +
// eps), omega = alpha / sum(alpha) (p = 1) are applied as
// C_k prod_{l != k}(beta_l + eps) over their sum: the same quotient with one
// reciprocal per side; the block stores C_0/C_1, C_2/C_1 (C_1 -> 1).
struct WenoField {
    double va, vb, vc, vd, ba, bb, bc, bd;
};
__device__ __forceinline__ WenoField weno_field64(const double *k, double a, double b, double c, double d, double e,
                                                  double f, double eps) {
    WenoField W;
    const double b2 = b * b, c2 = c * c;
    W.va = fma(k[0], a, k[1] * b);
    W.vb = fma(k[5], b, k[6] * c);
    W.vc = fma(k[10], c, k[11] * d);
    W.vd = fma(k[15], e, k[16] * f);
    // m0 x^2 + m1 x y + m2 y^2 + eps as x (m0 x + m1 y) + m2 y^2 + eps, with
    // y^2 shared between neighbouring sub-stencils: three products per field
    // fewer than the expanded form
    W.ba = fma(a, fma(k[2], a, k[3] * b), fma(k[4], b2, eps));
    W.bb = fma(b, fma(k[7], b, k[8] * c), fma(k[9], c2, eps));
    W.bc = fma(d, fma(k[14], d, k[13] * c), fma(k[12], c2, eps));
    W.bd = fma(e, fma(k[17], e, k[18] * f), fma(k[19], f * f, eps));
    return W;
}

// The form the adjoint differentiates: right increments from R1 (S_c's and
// S_b's values shifted by -c), from a field's values and indicators
// (weno_field64).
__device__ __forceinline__ void weno_combine64(const double *k, const WenoField &W, double c, double &dl,
                                               double &dr) {
    const double bbc = W.bb * W.bc;
    const double l0 = k[20] * bbc, l1 = W.ba * W.bc, l2 = k[21] * (W.ba * W.bb);
    dl = fma(l0, W.va, fma(l1, W.vb, l2 * W.vc)) * recip64_fast(l0 + l1 + l2);
    const double r0 = k[22] * bbc, r1 = W.bd * W.bb, r2 = k[23] * (W.bd * W.bc);
    dr = fma(r0, W.vd, fma(r1, W.vc - c, r2 * (W.vb - c))) * recip64_fast(r0 + r1 + r2);
}

// The forward kernel's form: the right increments are taken from L1 instead
// (S_d's value shifted by +c), so that w_R = L1 + R dr:
// sum r_k (v_k - c) / sum r_k + c = sum r_k v_k' / sum r_k.
__device__ __forceinline__ void weno_pair64_l1(const double *k, double a, double b, double c, double d, double e,
                                               double f, double eps, double &dl, double &dr) {
    const WenoField W = weno_field64(k, a, b, c, d, e, f, eps);
    // left: (C0 bb bc va + ba bc vb + C2 ba bb vc) / (C0 bb bc + ba bc + C2 ba bb)
    // with bc factored from the first two terms; right: (D0 bb bc vd' + bd bb vc
    // + D2 bd bc vb) / (D0 bb bc + bd bb + D2 bd bc) with bb factored from the
    // first two (one product fewer per field than the term-by-term sums); vd' =
    // vd + c is formed with c inside its fused multiply-adds (W.vd is not used)
    const double g = k[20] * W.bb, m = k[21] * (W.ba * W.bb);
    dl = fma(W.bc, fma(g, W.va, W.ba * W.vb), m * W.vc) * recip64_fast(fma(W.bc, g + W.ba, m));
    const double s = k[22] * W.bc, q = k[23] * (W.bd * W.bc);
    const double vdc = fma(k[15], e, fma(k[16], f, c));
    dr = fma(W.bb, fma(s, vdc, W.bd * W.vc), q * W.vb) * recip64_fast(fma(W.bb, s + W.bd, q));
}

}  // namespace dev
}  // namespace fdu
