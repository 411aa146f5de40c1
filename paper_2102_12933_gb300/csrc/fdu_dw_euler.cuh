// Double-word (FP32-pair) Euler helpers shared by the precision-48 edge flux
// and its adjoint (device only): 4-vectors, FP64 loads, the Roe average and
// the characteristic projections of Section 2.3.1.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "fdu_dw.cuh"

namespace fdu {
namespace dwa {

struct dw4 {
    dw x, y, z, w;
};
__device__ __forceinline__ dw4 d4(dw x, dw y, dw z, dw w) { return dw4{x, y, z, w}; }
__device__ __forceinline__ dw4 add4_sl(const dw4 &a, const dw4 &b) {
    return d4(add_sl(a.x, b.x), add_sl(a.y, b.y), add_sl(a.z, b.z), add_sl(a.w, b.w));
}
__device__ __forceinline__ dw4 sub4_sl(const dw4 &a, const dw4 &b) {
    return d4(add_sl(a.x, neg(b.x)), add_sl(a.y, neg(b.y)), add_sl(a.z, neg(b.z)), add_sl(a.w, neg(b.w)));
}

struct d4v {
    double x, y, z, w;
};
__device__ __forceinline__ d4v ldd4(const double *p, int64_t i) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p) + 2 * i);
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 2 * i + 1);
    return d4v{a.x, a.y, b.x, b.y};
}

__device__ __forceinline__ dw4 d2dw4(const d4v &v) { return d4(d2dw(v.x), d2dw(v.y), d2dw(v.z), d2dw(v.w)); }

// ---- Roe average and characteristic projections (double words)
struct RoeW {
    dw u, v, H, c, ic, qn, qt, hq2, b1h, ich, nx, ny;
};
__device__ __forceinline__ RoeW roe_finish(dw u, dw v, dw H, dw nx, dw ny, dw gm1) {
    RoeW R;
    R.u = u;
    R.v = v;
    R.H = H;
    R.hq2 = scale(add_sl(mul_u(u, u), mul_u(v, v)), 0.5f);
    const dw c2 = mul(gm1, sub_sl(H, R.hq2));
    R.ic = rsqrt(c2);
    R.c = mul(c2, R.ic);
    R.b1h = scale(mul(gm1, mul(R.ic, R.ic)), 0.5f);
    R.ich = scale(R.ic, 0.5f);
    R.nx = nx;
    R.ny = ny;
    R.qn = add_sl(mul_u(u, nx), mul_u(v, ny));
    R.qt = sub_sl(mul_u(v, nx), mul_u(u, ny));
    return R;
}
// Roe average from the sides' records (sqrt rho, sqrt rho u, sqrt rho v, sqrt rho H)
__device__ __forceinline__ RoeW roe_records(const dw4 &qa, const dw4 &qb, dw nx, dw ny, dw gm1) {
    const dw inv = recip(add_sl(qa.x, qb.x));
    return roe_finish(mul(add_sl(qa.y, qb.y), inv), mul(add_sl(qa.z, qb.z), inv), mul(add_sl(qa.w, qb.w), inv), nx,
                      ny, gm1);
}
// fields q_n - c, q_n (entropy), q_n (shear), q_n + c
// Sums of increments (here and in the WENO values and weighted sums) take
// the sloppy sum: its absolute error, about u^2 (|x| + |y|), is of the
// order of the increments' own rounding.
__device__ __forceinline__ dw4 project(const RoeW &R, const dw4 &d) {
    const dw phh = mul(R.b1h, add_sl(sub_sl(sub_sl(mul_u(R.hq2, d.x), mul_u(R.u, d.y)), mul_u(R.v, d.z)), d.w));
    const dw psh = mul(sub_sl(sub_sl(mul_u(R.qn, d.x), mul_u(R.nx, d.y)), mul_u(R.ny, d.z)), R.ich);
    return d4(add_sl(phh, psh), sub_sl(d.x, scale(phh, 2.0f)),
              sub_sl(sub_sl(mul_u(R.nx, d.z), mul_u(R.ny, d.y)), mul_u(R.qt, d.x)), sub_sl(phh, psh));
}
__device__ __forceinline__ dw4 unproject(const RoeW &R, const dw4 &c) {
    const dw ac = add_sl(c.x, c.w);
    const dw rho = add_sl(ac, c.y);
    const dw dd = mul(R.c, sub_sl(c.w, c.x));
    return d4(rho, sub_sl(add_sl(mul_u(R.u, rho), mul_u(R.nx, dd)), mul_u(R.ny, c.z)),
              add_sl(add_sl(mul_u(R.v, rho), mul_u(R.ny, dd)), mul_u(R.nx, c.z)),
              add_sl(add_sl(add_sl(mul_u(R.H, ac), mul_u(R.hq2, c.y)), mul_u(R.qn, dd)), mul_u(R.qt, c.z)));
}

}  // namespace dwa
}  // namespace fdu
