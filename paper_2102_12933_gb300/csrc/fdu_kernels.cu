// sm_103a kernels of the unstructured-mesh FDM residual and SSP-RK3 stage.
//
//   edge flux  : per edge, gather the six states of its 1D curvilinear
//                stencil, project differences on the characteristic
//                fields of the Roe average of the edge's end states,
//                interpolate each field to the edge midpoint with
//                non-uniform WENO5 from both sides (Appendix), back-project
//                and evaluate a Roe flux along the edge (Section 2.3.1).
//   divergence : per vertex, a1 + b2 of the least-squares fit, i.e. the
//                weighted sum of vertex fluxes f_j, g_j and edge fluxes r_k
//                (Section 2.2.1), SELL-32 layout (a warp reads 32
//                consecutive ids / weights per entry); optionally fused
//                with the SSP-RK3 stage combination and the vertex fluxes
//                of the new state.
//
// Everything is gather-bound or scalar-ALU-bound: there is no dense
// contraction, so no tensor-core path.
#include <cuda_runtime.h>

#include <cstdint>

#include "fdu_internal.h"
#include "fdu_kernels.cuh"
#include "fdu_device.cuh"
#include "fdu_dw.cuh"
#include "fdu_dw_edge.cuh"

namespace fdu {
namespace {

using namespace dev;

// ------------------------------------------------------------------ FP64 edge flux
__device__ __forceinline__ void edge_flux_f64_body(const EdgeArgs &A, const int64_t e) {
    const double *__restrict__ w = static_cast<const double *>(A.w);
    const double *__restrict__ coef = static_cast<const double *>(A.coef);
    const double gm1 = A.gm1, hgm1 = A.hgm1;
    const int64_t ne = A.ne;
    int32_t s[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = __ldg(A.sten + (int64_t)i * ne + e);
    const dbl4 L1 = ld4v(w, s[2]), R1 = ld4v(w, s[3]);
    const double nx = __ldg(coef + (int64_t)kCoefN * ne + e);
    const double ny = __ldg(coef + (int64_t)(kCoefN + 1) * ne + e);

    // characteristic decomposition at the Roe average of the end states
    // (per-vertex Roe records when the stage kernel provided them)
    const Roe64 C = A.Q ? roe64_from_records(ld4v(A.Q, s[2]), ld4v(A.Q, s[3]), nx, ny, gm1, hgm1)
                        : roe64(L1, prim64(L1, gm1), R1, prim64(R1, gm1), nx, ny, gm1, hgm1);
    const dbl4 cM = project64(C, sub4(R1, L1));               // R1 - L1
    const dbl4 cL2 = project64(C, sub4(ld4v(w, s[1]), L1));    // L2 - L1
    const dbl4 cL3 = project64(C, sub4(ld4v(w, s[0]), L1));    // L3 - L1
    const dbl4 cR2 = project64(C, sub4(ld4v(w, s[4]), R1));    // R2 - R1
    const dbl4 cR3 = project64(C, sub4(ld4v(w, s[5]), R1));    // R3 - R1

    double k[kCoefN];
#pragma unroll
    for (int i = 0; i < kCoefN; ++i) k[i] = __ldg(coef + (int64_t)i * ne + e);
    const dbl4 cR2L = add4(cR2, cM);  // R2 - L1
    dbl4 dl, dr;
    weno_pair64_l1(k, cL3.x, cL2.x, cM.x, cR2L.x, cR3.x, cR2.x, A.eps, dl.x, dr.x);
    weno_pair64_l1(k, cL3.y, cL2.y, cM.y, cR2L.y, cR3.y, cR2.y, A.eps, dl.y, dr.y);
    weno_pair64_l1(k, cL3.z, cL2.z, cM.z, cR2L.z, cR3.z, cR2.z, A.eps, dl.z, dr.z);
    weno_pair64_l1(k, cL3.w, cL2.w, cM.w, cR2L.w, cR3.w, cR2.w, A.eps, dl.w, dr.w);

    // both interpolated states from L1 (R (R1 - L1)_char = R1 - L1)
    dbl4 wl = unproject_add64(C, dl, L1);
    dbl4 wr = unproject_add64(C, dr, L1);
    Prim64 pl, pr;
    bool ok = pos64(wl.x) && pos64(wr.x);
    if (ok) {
        pl = prim64(wl, gm1);
        pr = prim64(wr, gm1);
        ok = pos64(pl.p) && pos64(pr.p);
    }
    if (!ok) {  // positivity fallback: first-order end states
        wl = L1;
        wr = R1;
        pl = prim64(L1, gm1);
        pr = prim64(R1, gm1);
        atomicAdd(A.fallback, 1ull);
    }

    // Roe flux with Harten's entropy fix (delta = 0.1 c), in the one-sided
    // form F_L + R diag((lambda - |lambda|)/2) L (w_R - w_L): equal to
    // (F_L + F_R)/2 - R |Lambda| L (w_R - w_L)/2 because the Roe matrix
    // satisfies F_R - F_L = R Lambda L (w_R - w_L)
    const Roe64 Q = roe64(wl, pl, wr, pr, nx, ny, gm1, hgm1);
    const dbl4 a = project64(Q, sub4(wr, wl));
    // (l - |l|_fixed) / 2 is min(l, 0) where |l| >= delta and, where Harten's
    // |l|_fixed = (l^2 + delta^2) / (2 delta) applies, -(l - delta)^2 / (4 delta).
    // Both tests run on the integer pipe: |l| < delta compares the bit
    // patterns of two non-negative doubles (delta = 0.1 c is positive), and
    // a NaN l is passed through as the FP64 form would.
    const double delta = 0.1 * Q.c, h4d = 2.5 * Q.ic;  // 1 / (4 delta)
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    auto neg = [&](double l) {
        const long long b = __double_as_longlong(l);
        const unsigned long long ab = (unsigned long long)b & 0x7FFFFFFFFFFFFFFFULL;
        if (ab < dbits) {
            const double s = l - delta;
            return -(s * s) * h4d;
        }
        return (b < 0 || ab > 0x7FF0000000000000ULL) ? l : 0.0;
    };
    const double nu = neg(Q.qn), nm = neg(Q.qn - Q.c), np = neg(Q.qn + Q.c);
    const dbl4 D = unproject64(Q, dbl4_make(nm * a.x, nu * a.y, nu * a.z, np * a.w));
    const double qnl = (wl.y * nx + wl.z * ny) * pl.ir;
    dbl4 f;
    f.x = fma(wl.x, qnl, D.x);
    f.y = fma(wl.y, qnl, fma(pl.p, nx, D.y));
    f.z = fma(wl.z, qnl, fma(pl.p, ny, D.z));
    f.w = fma(wl.w + pl.p, qnl, D.w);
    st4(static_cast<double *>(A.r), e, f);
}

// ------------------------------------------------------------------ vertex fluxes
// f, g of a state from its primitives (1/rho, p): the same quantities the
// Roe record needs, so the two share one reciprocal square root.
__device__ __forceinline__ void euler_fg(const dbl4 &w, const Prim64 &P, dbl4 &f, dbl4 &g) {
    const double u = w.y * P.ir, v = w.z * P.ir;
    f = dbl4_make(w.y, fma(w.y, u, P.p), w.z * u, (w.w + P.p) * u);
    g = dbl4_make(w.z, w.y * v, fma(w.z, v, P.p), (w.w + P.p) * v);
}
// Roe-weighted record of a state: (s, s u, s v, s H) with s = sqrt(rho),
// computed with the same operations roe64 applies to each side.
__device__ __forceinline__ dbl4 roe_record64(const dbl4 &w, const Prim64 &P) {
    return dbl4_make(w.x * P.r, w.y * P.r, w.z * P.r, (w.w + P.p) * P.r);
}

__global__ void vertex_flux_f64_kernel(const double *__restrict__ w, double *__restrict__ F, double *__restrict__ Q,
                                       int64_t n, double gm1) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const dbl4 s = ld4(w, v);
    const Prim64 P = prim64(s, gm1);
    dbl4 f, g;
    euler_fg(s, P, f, g);
    st4(F, 2 * v, f);
    st4(F, 2 * v + 1, g);
    if (Q) st4(Q, v, roe_record64(s, P));
}

// Forward-Euler part of an SSP-RK3 stage, fe = ws + theta dt L.  Without
// the safeguard theta = 1.  With it (alpha > 0), theta is the largest of
// 1, 1/2, ..., 2^-20 (else 0) with rho(fe) >= alpha rho(ws) and
// p(fe) >= alpha p(ws), so that the stage combination of w_n and fe stays
// physical (the set of physical states is convex).
__device__ __forceinline__ dbl4 forward_euler(const dbl4 &ws, const dbl4 &L, double dt, double gm1, double alpha,
                                             unsigned long long *limited) {
    dbl4 fe = dbl4_make(fma(dt, L.x, ws.x), fma(dt, L.y, ws.y), fma(dt, L.z, ws.z), fma(dt, L.w, ws.w));
    if (alpha > 0.0) {
        auto pres = [&](const dbl4 &q) { return gm1 * (q.w - 0.5 * (q.y * q.y + q.z * q.z) / q.x); };
        const double ps = pres(ws);
        double th = 1.0;
        bool ok = false;
        for (int k = 0; k <= 20; ++k) {
            fe = dbl4_make(fma(th * dt, L.x, ws.x), fma(th * dt, L.y, ws.y), fma(th * dt, L.z, ws.z),
                           fma(th * dt, L.w, ws.w));
            if (fe.x >= alpha * ws.x && pres(fe) >= alpha * ps) {
                ok = true;
                break;
            }
            th *= 0.5;
        }
        if (!ok) {
            th = 0.0;
            fe = ws;
        }
        if (th < 1.0) atomicAdd(limited, 1ull);
    }
    return fe;
}

// Two adjacent float4 (record j of a [n][2] float4 buffer: FP32 vertex fluxes
// (f, g), or an edge's double-word increments) as one 32-byte load; the
// buffers are 32-byte aligned and read-only in the kernel.
__device__ __forceinline__ void ld_fg32(const float4 *F, int64_t j, float4 &f, float4 &g) {
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(f.x), "=f"(f.y), "=f"(f.z), "=f"(f.w), "=f"(g.x), "=f"(g.y), "=f"(g.z), "=f"(g.w)
        : "l"(F + 2 * j));
}

// ------------------------------------------------------------------ FP64 divergence (+ RK stage)
// Position i of the SELL tables; the vertex it holds is A.perm[i].  With
// DWE (precision 48) the edge entries are double-word increments
// r_k - F_n(L1_k) with double-word weights, summed in double words (terms of
// the size of the increments), and the vertex weights carry the folded
// F_n(L1_k) parts.
// Loads of the FP64 / precision-48 divergence tables: read once per stage,
// so in the stage modes they do not allocate in L1 (which keeps it for the
// flux gathers) and each miss asks L2 for 256 bytes; precision-48 divergence
// 0.1435 -> 0.1385 ms at 250k vertices, the FP64 one (FP64-pipe bound)
// unchanged.
template <int MODE> __device__ __forceinline__ int32_t tld(const int32_t *p) {
    if (MODE == 0) return __ldg(p);
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
template <int MODE> __device__ __forceinline__ double tld(const double *p) {
    if (MODE == 0) return __ldg(p);
    double v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
}
template <int MODE> __device__ __forceinline__ float2 tld(const float2 *p) {
    if (MODE == 0) return __ldg(p);
    float2 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
    return v;
}
template <int MODE, bool DWE = false>
__device__ __forceinline__ void div_f64_body(const DivArgs &A, const int64_t i) {
    const int64_t sl = i / kSell;
    const int lane = (int)(i % kSell);
    const int64_t v = A.perm ? (int64_t)__ldg(A.perm + i) : i;
    const double *__restrict__ F = static_cast<const double *>(A.F);
    const double *__restrict__ r = static_cast<const double *>(A.r);
    const double *__restrict__ wf = static_cast<const double *>(A.wf);
    const double *__restrict__ wg = static_cast<const double *>(A.wg);
    const double *__restrict__ we = static_cast<const double *>(A.we);
    dbl4 acc = dbl4_make(0, 0, 0, 0);
    {
        const int64_t b = __ldg(A.slice_voff + sl) + lane, e = __ldg(A.slice_voff + sl + 1);
#pragma unroll 4
        for (int64_t p = b; p < e; p += kSell) {
            const int32_t j = tld<MODE>(A.vid + p);
            const double a = tld<MODE>(wf + p), c = tld<MODE>(wg + p);
            const dbl4 f = ld4v(F, 2 * (int64_t)j), g = ld4v(F, 2 * (int64_t)j + 1);
            acc.x = fma(a, f.x, fma(c, g.x, acc.x));
            acc.y = fma(a, f.y, fma(c, g.y, acc.y));
            acc.z = fma(a, f.z, fma(c, g.z, acc.z));
            acc.w = fma(a, f.w, fma(c, g.w, acc.w));
        }
    }
    if (DWE) {
        using namespace dwa;
        const float2 *__restrict__ we2 = static_cast<const float2 *>(A.we);
        const float4 *__restrict__ rd = static_cast<const float4 *>(A.r);
        dot2 sx{0.0f, 0.0f}, sy = sx, sz = sx, sw = sx;
        const int64_t b = __ldg(A.slice_eoff + sl) + lane, e = __ldg(A.slice_eoff + sl + 1);
#pragma unroll 4
        for (int64_t p = b; p < e; p += kSell) {
            const int32_t k = tld<MODE>(A.eid + p);
            const float2 wq = tld<MODE>(we2 + p);
            const dw a = dw_make(wq.x, wq.y);
            float4 q0, q1;
            ld_fg32(rd, k, q0, q1);  // the edge's two double-word float4, one 32-byte load
            dot2_add(sx, a, dw_make(q0.x, q0.y));
            dot2_add(sy, a, dw_make(q0.z, q0.w));
            dot2_add(sz, a, dw_make(q1.x, q1.y));
            dot2_add(sw, a, dw_make(q1.z, q1.w));
        }
        const dw rx = dot2_result(sx), ry = dot2_result(sy), rz = dot2_result(sz), rw = dot2_result(sw);
        acc.x += f2d(rx.h) + f2d(rx.l);
        acc.y += f2d(ry.h) + f2d(ry.l);
        acc.z += f2d(rz.h) + f2d(rz.l);
        acc.w += f2d(rw.h) + f2d(rw.l);
    } else {
        const int64_t b = __ldg(A.slice_eoff + sl) + lane, e = __ldg(A.slice_eoff + sl + 1);
#pragma unroll 4
        for (int64_t p = b; p < e; p += kSell) {
            const int32_t k = tld<MODE>(A.eid + p);
            const double a = tld<MODE>(we + p);
            const dbl4 q = ld4v(r, k);
            acc.x = fma(a, q.x, acc.x);
            acc.y = fma(a, q.y, acc.y);
            acc.z = fma(a, q.z, acc.z);
            acc.w = fma(a, q.w, acc.w);
        }
    }
    {
        const double *cfg = static_cast<const double *>(A.cfg);
        const double cf = __ldg(cfg + v), cg = __ldg(cfg + A.n_real + v);
        const dbl4 f = ld4v(F, 2 * v), g = ld4v(F, 2 * v + 1);
        acc.x = fma(cf, f.x, fma(cg, g.x, acc.x));
        acc.y = fma(cf, f.y, fma(cg, g.y, acc.y));
        acc.z = fma(cf, f.z, fma(cg, g.z, acc.z));
        acc.w = fma(cf, f.w, fma(cg, g.w, acc.w));
    }
    const dbl4 L = neg4(acc);  // dw/dt = -(a1 + b2)
    if (MODE == 0) {
        const int64_t row = A.out_map ? (int64_t)__ldg(A.out_map + v) : v;
        st4(A.out, row, L);
        return;
    }
    const double dt = A.comp ? __ldg(A.dt_comp + __ldg(A.comp + v)) : (A.dt_dev ? *A.dt_dev : A.dt);
    const dbl4 ws = ld4v(A.ws, v);
    const dbl4 fe = forward_euler(ws, L, dt, A.gm1, A.pos_alpha, A.limited);
    dbl4 o;
    if (MODE == 1) {
        o = fe;
    } else {
        const dbl4 wn = ld4v(A.wn, v);
        const double cn = MODE == 2 ? 0.75 : 1.0 / 3.0;
        const double cs = MODE == 2 ? 0.25 : 2.0 / 3.0;
        o.x = fma(cn, wn.x, cs * fe.x);
        o.y = fma(cn, wn.y, cs * fe.y);
        o.z = fma(cn, wn.z, cs * fe.z);
        o.w = fma(cn, wn.w, cs * fe.w);
    }
    st4(A.wout, v, o);
    const Prim64 P = prim64(o, A.gm1);
    dbl4 f, g;
    euler_fg(o, P, f, g);
    double *Fo = static_cast<double *>(A.Fout);
    st4(Fo, 2 * v, f);
    st4(Fo, 2 * v + 1, g);
    if (A.Qout) st4(A.Qout, v, roe_record64(o, P));
}

// ================================================================== FP32 path
// The FP32 residual reads an FP32 copy of the state and, per edge, the
// FP64-built NU-WENO5 block rounded to FP32 (104 bytes), or in the compact
// form (mesh option f32_coef = 1) the edge's four stencil gaps and normal
// (24 bytes), from which it forms the coefficients in registers; weights,
// fluxes and sums are FP32.  Reciprocals use the hardware approximation
// (rcp.approx, about one ulp), well inside the FP32 path's error against
// FP64.
__device__ __forceinline__ float rcp32(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// Read-once loads of the streamed edge tables (the FP32 coefficient block or
// gaps): they do not allocate in L1, which keeps its capacity for the state
// gathers (edge kernel 0.031 -> 0.0275 ms at 250k vertices).
__device__ __forceinline__ float4 ld_stream4(const float4 *p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}
__device__ __forceinline__ float4 sub4f(float4 a, float4 b) {
    return make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
}
__device__ __forceinline__ float4 add4f(float4 a, float4 b) {
    return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

struct Prim32 {
    float r, ir, p;
};
__device__ __forceinline__ Prim32 prim32(const float4 &w, float gm1) {
    Prim32 q;
    q.r = rsqrtf(w.x);
    q.ir = q.r * q.r;
    q.p = gm1 * (w.w - 0.5f * (w.y * w.y + w.z * w.z) * q.ir);
    return q;
}
struct Roe32 {
    float u, v, H, c, ic, b1h, ich, qn, qt, hq2, nx, ny;  // b1h = b1 / 2, ich = ic / 2
};
__device__ __forceinline__ Roe32 roe32(const float4 &a, const Prim32 &pa, const float4 &b, const Prim32 &pb, float nx,
                                      float ny, float gm1) {
    Roe32 R;
    const float sa = a.x * pa.r, sb = b.x * pb.r;
    const float inv = rcp32(sa + sb);
    R.u = (a.y * pa.r + b.y * pb.r) * inv;
    R.v = (a.z * pa.r + b.z * pb.r) * inv;
    R.H = ((a.w + pa.p) * pa.r + (b.w + pb.p) * pb.r) * inv;
    R.hq2 = 0.5f * (R.u * R.u + R.v * R.v);
    const float c2 = gm1 * (R.H - R.hq2);
    R.ic = rsqrtf(c2);
    R.c = c2 * R.ic;
    R.b1h = 0.5f * gm1 * R.ic * R.ic;
    R.ich = 0.5f * R.ic;
    R.nx = nx;
    R.ny = ny;
    R.qn = R.u * nx + R.v * ny;
    R.qt = R.v * nx - R.u * ny;
    return R;
}
// pre-halved factors (phi/2, psi/2) and the sum started from d.w
__device__ __forceinline__ float4 project32(const Roe32 &R, const float4 &d) {
    const float phh = R.b1h * fmaf(-R.v, d.z, fmaf(-R.u, d.y, fmaf(R.hq2, d.x, d.w)));
    const float psh = (R.qn * d.x - R.nx * d.y - R.ny * d.z) * R.ich;
    return make_float4(phh + psh, fmaf(-2.0f, phh, d.x), R.nx * d.z - R.ny * d.y - R.qt * d.x, phh - psh);
}
__device__ __forceinline__ float4 unproject32(const Roe32 &R, const float4 &c) {
    const float rho = c.x + c.y + c.w;
    const float dd = R.c * (c.w - c.x);
    return make_float4(rho, R.u * rho + R.nx * dd - R.ny * c.z, R.v * rho + R.ny * dd + R.nx * c.z,
                       R.H * (c.x + c.w) + R.hq2 * c.y + R.qn * dd + R.qt * c.z);
}
// base + unproject32(R, c), with base taken into the fused multiply-adds
__device__ __forceinline__ float4 unproject_add32(const Roe32 &R, const float4 &c, const float4 &base) {
    const float ac = c.x + c.w;
    const float rho = ac + c.y;
    const float dd = R.c * (c.w - c.x);
    return make_float4(base.x + rho, fmaf(R.u, rho, fmaf(R.nx, dd, fmaf(-R.ny, c.z, base.y))),
                       fmaf(R.v, rho, fmaf(R.ny, dd, fmaf(R.nx, c.z, base.z))),
                       fmaf(R.H, ac, fmaf(R.hq2, c.y, fmaf(R.qn, dd, fmaf(R.qt, c.z, base.w)))));
}

// FP32 NU-WENO5 increments of one field, both sides (same sub-stencil
// sharing and block layout as weno_pair64_l1).  Weights alpha_k = C_k /
// (beta_k + eps32), omega = alpha / sum(alpha); the four reciprocals of
// (beta + eps32) serve both sides (a product form would underflow in FP32).
__device__ __forceinline__ void weno_pair32(const float *k, float a, float b, float c, float d, float e, float f,
                                            float eps, float &dl, float &dr) {
    const float b2 = b * b, c2 = c * c;
    const float va = fmaf(k[0], a, k[1] * b), vb = fmaf(k[5], b, k[6] * c);
    const float vc = fmaf(k[10], c, k[11] * d), vd = fmaf(k[15], e, k[16] * f);
    const float ia = rcp32(fmaf(k[2], a * a, fmaf(k[3], a * b, fmaf(k[4], b2, eps))));
    const float ib = rcp32(fmaf(k[7], b2, fmaf(k[8], b * c, fmaf(k[9], c2, eps))));
    const float ic = rcp32(fmaf(k[12], c2, fmaf(k[13], c * d, fmaf(k[14], d * d, eps))));
    const float id = rcp32(fmaf(k[17], e * e, fmaf(k[18], e * f, fmaf(k[19], f * f, eps))));
    // middle linear weights are 1 (the block stores C_0/C_1, C_2/C_1);
    // right increments from L1 (S_d's value shifted by +c), as in the FP64 kernel
    const float l0 = k[20] * ia, l1 = ib, l2 = k[21] * ic;
    dl = fmaf(l0, va, fmaf(l1, vb, l2 * vc)) * rcp32(l0 + l1 + l2);
    const float r0 = k[22] * id, r1 = ic, r2 = k[23] * ib;
    dr = fmaf(r0, vd + c, fmaf(r1, vc, r2 * vb)) * rcp32(r0 + r1 + r2);
}

// NU-WENO5 coefficients of one edge in FP32 (Appendix: the sub-stencil
// interpolants' values at the midpoint, their smoothness indicators, and
// the linear weights that make the combination the degree-4 interpolant,
// Eq. S5), in the order of the coefficient block (fdu_internal.h), from
// the four gaps between consecutive stencil points along the curve, each
// divided by the arc length L1-R1:
//   a = L1-L2, b = L2-L3, c = R1-R2, d = R2-R3,
// so that the left side's points are -(1/2+a+b), -(1/2+a), -1/2, 1/2,
// 1/2+c and the right side's (mirrored) the same with (a, b, c) -> (c, d,
// a).  A sub-stencil's Lagrange basis value at 0 of a point x_j is
// x_a x_b / ((x_j - x_a)(x_j - x_b)) over its other two points, its slope
// -(x_a + x_b) / (...) and its curvature 2 / (...); the smoothness
// indicator (slope)^2 + (13/12)(2 curvature)^2 (unit spacing between L1
// and R1) is kept as the quadratic form of the two differences.  The
// linear weights have the closed forms
//   C_0 = (1/2)(1/2+c) / ((1+a+b)(1+a+b+c)),
//   C_2 = (1/2+a+b)(1/2+a) / ((1+a+b+c)(1+a+c)),   C_1 = 1 - C_0 - C_2
// (ratios of degree-4 and sub-stencil Lagrange values), of which the block
// keeps C_0/C_1 and C_2/C_1.  Every factor is a sum of positive gaps, so
// no step cancels.
constexpr float kT3 = 13.0f / 3.0f;  // (13/12) x 2^2
// outer sub-stencil of a side (points -(1/2+a+b), -(1/2+a), -1/2): values
// of its two outer points' differences and the indicator's form
__device__ __forceinline__ void weno_outer32(float a, float b, float *k) {
    const float ab = a + b;
    const float r0 = rcp32(b * ab), r1 = -rcp32(a * b);
    const float s0 = 1.0f + a, s1 = 1.0f + ab;
    k[0] = 0.5f * (0.5f + a) * r0;
    k[1] = 0.5f * (0.5f + ab) * r1;
    k[2] = r0 * r0 * fmaf(s0, s0, kT3);
    k[3] = 2.0f * r0 * r1 * fmaf(s0, s1, kT3);
    k[4] = r1 * r1 * fmaf(s1, s1, kT3);
}
// C_0/C_1 and C_2/C_1 of a side from its gaps (a, b) and the far side's c
__device__ __forceinline__ void weno_ratios32(float a, float b, float c, float *k) {
    const float p = 1.0f + a + b, r = 1.0f + a + c;
    const float n0r = 0.5f * (0.5f + c) * r, n2p = (0.5f + a + b) * (0.5f + a) * p;
    const float ir = rcp32((p + c) * p * r - n0r - n2p);
    k[0] = n0r * ir;
    k[1] = n2p * ir;
}
__device__ __forceinline__ void weno_coef32(const float4 g, float *k) {
    const float a = g.x, b = g.y, c = g.z, d = g.w;
    weno_outer32(a, b, k);  // S_a
    {                       // S_b: points -(1/2+a), -1/2, 1/2
        const float r2 = rcp32(1.0f + a), r0 = rcp32(a * (1.0f + a));
        k[5] = -0.25f * r0;
        k[6] = 0.5f * (0.5f + a) * r2;
        k[7] = kT3 * r0 * r0;
        k[8] = 2.0f * kT3 * r0 * r2;
        k[9] = fmaf(kT3 * r2, r2, 1.0f);
    }
    {  // S_c: points -1/2, 1/2, 1/2+c
        const float r1 = -rcp32(c), r2 = rcp32(c * (1.0f + c));
        k[10] = -0.5f * (0.5f + c) * r1;
        k[11] = -0.25f * r2;
        k[12] = fmaf(kT3 * r1, r1, 1.0f);
        k[13] = 2.0f * kT3 * r1 * r2;
        k[14] = kT3 * r2 * r2;
    }
    weno_outer32(c, d, k + 15);  // S_d
    weno_ratios32(a, b, c, k + kCoefCL);
    weno_ratios32(c, d, a, k + kCoefCR);
}

// GAPS: the compact coefficient form (the values formed here from the
// edge's stencil gaps); otherwise the FP64-built block rounded to FP32.
template <bool GAPS>
__device__ __forceinline__ void edge_flux_f32_body(const EdgeArgs &A, const int64_t e) {
    const float4 *__restrict__ w = static_cast<const float4 *>(A.w);
    const float *__restrict__ g = static_cast<const float *>(A.coef);
    const float gm1 = A.gm1f;
    const float eps = A.epsf;
    const int64_t ne = A.ne;
    int32_t s[6];
    // the stencil ids are read once as well (the divergence that follows gains
    // more than this kernel loses: 0.055 -> 0.0537 against 0.0275 -> 0.0283 ms)
#pragma unroll
    for (int i = 0; i < 6; ++i)
        asm("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(s[i]) : "l"(A.sten + (int64_t)i * ne + e));
    float k[kCoefN];
    float nx, ny;
    if (GAPS) {
        // the edge's stencil gaps ([ne] float4) and normal ([ne] float2 after them)
        const float2 nq = __ldg(reinterpret_cast<const float2 *>(g + (int64_t)4 * ne) + e);
        nx = nq.x;
        ny = nq.y;
        weno_coef32(ld_stream4(reinterpret_cast<const float4 *>(g) + e), k);
    } else {
        // six float4 of values ([c/4][ne] float4, component c%4), then the
        // normal as one float2 ([ne] float2 after them)
        const float4 *__restrict__ g4 = reinterpret_cast<const float4 *>(g);
#pragma unroll
        for (int i = 0; i < kEdgeCoef32Vec; ++i) {
            const float4 q = ld_stream4(g4 + (int64_t)i * ne + e);
            k[4 * i] = q.x;
            k[4 * i + 1] = q.y;
            k[4 * i + 2] = q.z;
            k[4 * i + 3] = q.w;
        }
        const float2 nq = __ldg(reinterpret_cast<const float2 *>(g + (int64_t)4 * kEdgeCoef32Vec * ne) + e);
        nx = nq.x;
        ny = nq.y;
    }
    const float4 L1 = __ldg(w + s[2]), R1 = __ldg(w + s[3]);
    const Prim32 pL1 = prim32(L1, gm1), pR1 = prim32(R1, gm1);
    const Roe32 C = roe32(L1, pL1, R1, pR1, nx, ny, gm1);
    const float4 cM = project32(C, sub4f(R1, L1));
    const float4 cL2 = project32(C, sub4f(__ldg(w + s[1]), L1));
    const float4 cL3 = project32(C, sub4f(__ldg(w + s[0]), L1));
    const float4 cR2 = project32(C, sub4f(__ldg(w + s[4]), R1));
    const float4 cR3 = project32(C, sub4f(__ldg(w + s[5]), R1));
    const float4 cR2L = add4f(cR2, cM);
    float4 dl, dr;
    weno_pair32(k, cL3.x, cL2.x, cM.x, cR2L.x, cR3.x, cR2.x, eps, dl.x, dr.x);
    weno_pair32(k, cL3.y, cL2.y, cM.y, cR2L.y, cR3.y, cR2.y, eps, dl.y, dr.y);
    weno_pair32(k, cL3.z, cL2.z, cM.z, cR2L.z, cR3.z, cR2.z, eps, dl.z, dr.z);
    weno_pair32(k, cL3.w, cL2.w, cM.w, cR2L.w, cR3.w, cR2.w, eps, dl.w, dr.w);

    float4 wl = unproject_add32(C, dl, L1);
    float4 wr = unproject_add32(C, dr, L1);
    Prim32 pl, pr;
    bool ok = wl.x > 0.f && wr.x > 0.f;
    if (ok) {
        pl = prim32(wl, gm1);
        pr = prim32(wr, gm1);
        ok = pl.p > 0.f && pr.p > 0.f;
    }
    if (!ok) {
        wl = L1;
        wr = R1;
        pl = pL1;
        pr = pR1;
        atomicAdd(A.fallback, 1ull);
    }
    // one-sided Roe flux F_L + R diag((lambda - |lambda|)/2) L (w_R - w_L)
    const Roe32 Q = roe32(wl, pl, wr, pr, nx, ny, gm1);
    const float4 a = project32(Q, sub4f(wr, wl));
    const float delta = 0.1f * Q.c, h2d = 5.0f * Q.ic;
    auto neg = [&](float l) {
        const float m = fabsf(l);
        return 0.5f * (l - (m < delta ? fmaf(l, l, delta * delta) * h2d : m));
    };
    const float nu = neg(Q.qn), nm = neg(Q.qn - Q.c), np = neg(Q.qn + Q.c);
    const float4 D = unproject32(Q, make_float4(nm * a.x, nu * a.y, nu * a.z, np * a.w));
    const float qnl = (wl.y * nx + wl.z * ny) * pl.ir;
    float4 f;
    f.x = fmaf(wl.x, qnl, D.x);
    f.y = fmaf(wl.y, qnl, fmaf(pl.p, nx, D.y));
    f.z = fmaf(wl.z, qnl, fmaf(pl.p, ny, D.z));
    f.w = fmaf(wl.w + pl.p, qnl, D.w);
    static_cast<float4 *>(A.r)[e] = f;
}

__device__ __forceinline__ void euler_fg32(const float4 &w, float gm1, float4 &f, float4 &g) {
    const float ir = rcp32(w.x);
    const float u = w.y * ir, v = w.z * ir;
    const float p = gm1 * (w.w - 0.5f * (w.y * u + w.z * v));
    f = make_float4(w.y, fmaf(w.y, u, p), w.z * u, (w.w + p) * u);
    g = make_float4(w.z, w.y * v, fmaf(w.z, v, p), (w.w + p) * v);
}

__global__ void vertex_flux_f32_kernel(const double *__restrict__ w, float4 *__restrict__ F, float4 *__restrict__ w32,
                                       int64_t n, float gm1) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const dbl4 d = ld4(w, v);
    const float4 s = make_float4((float)d.x, (float)d.y, (float)d.z, (float)d.w);
    w32[v] = s;
    float4 f, g;
    euler_fg32(s, gm1, f, g);
    F[2 * v] = f;
    F[2 * v + 1] = g;
}

template <int MODE>
__device__ __forceinline__ void div_f32_finish(const DivArgs &A, const int64_t v, float4 acc) {
    const float4 *__restrict__ F = static_cast<const float4 *>(A.F);
    {
        const float *cfg = static_cast<const float *>(A.cfg);
        const float cf = __ldg(cfg + v), cg = __ldg(cfg + A.n_real + v);
        const float4 f = __ldg(F + 2 * v), g = __ldg(F + 2 * v + 1);
        acc.x = fmaf(cf, f.x, fmaf(cg, g.x, acc.x));
        acc.y = fmaf(cf, f.y, fmaf(cg, g.y, acc.y));
        acc.z = fmaf(cf, f.z, fmaf(cg, g.z, acc.z));
        acc.w = fmaf(cf, f.w, fmaf(cg, g.w, acc.w));
    }
    const dbl4 L = dbl4_make(-(double)acc.x, -(double)acc.y, -(double)acc.z, -(double)acc.w);
    if (MODE == 0) {
        const int64_t row = A.out_map ? (int64_t)__ldg(A.out_map + v) : v;
        st4(A.out, row, L);
        return;
    }
    // SSP-RK3 combination in FP64
    const double dt = A.comp ? __ldg(A.dt_comp + __ldg(A.comp + v)) : (A.dt_dev ? *A.dt_dev : A.dt);
    const dbl4 ws = ld4(A.ws, v);
    const dbl4 fe = forward_euler(ws, L, dt, A.gm1, A.pos_alpha, A.limited);
    dbl4 o;
    if (MODE == 1) {
        o = fe;
    } else {
        const dbl4 wn = ld4(A.wn, v);
        const double cn = MODE == 2 ? 0.75 : 1.0 / 3.0;
        const double cs = MODE == 2 ? 0.25 : 2.0 / 3.0;
        o.x = fma(cn, wn.x, cs * fe.x);
        o.y = fma(cn, wn.y, cs * fe.y);
        o.z = fma(cn, wn.z, cs * fe.z);
        o.w = fma(cn, wn.w, cs * fe.w);
    }
    st4(A.wout, v, o);
    const float4 s32 = make_float4((float)o.x, (float)o.y, (float)o.z, (float)o.w);
    A.w32out[v] = s32;
    float4 f, g;
    euler_fg32(s32, A.gm1f, f, g);
    float4 *Fo = static_cast<float4 *>(A.Fout);
    Fo[2 * v] = f;
    Fo[2 * v + 1] = g;
}

// Loads of the streamed divergence tables: read once per stage, so they do
// not allocate in L1 (which keeps its capacity for the flux gathers), and
// each miss asks L2 for 256 bytes (the row's 128-byte line and the next).
__device__ __forceinline__ int32_t ld_stream(const int32_t *p) {
    int32_t v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ float ld_stream(const float *p) {
    float v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}
// Table loads of the FP32 divergence: streaming loads in the fused stage
// (modes 1..3: 0.066 -> 0.062 ms at 250k vertices), plain cached loads for
// the residual alone (mode 0, where the streaming form measured slower).
template <int MODE, class T>
__device__ __forceinline__ T ld_table(const T *p) {
    if (MODE != 0) return ld_stream(p);
    return __ldg(p);
}

template <int MODE>
__device__ __forceinline__ void div_f32_body(const DivArgs &A, const int64_t v) {
    const int64_t sl = v / kSell;
    const int lane = (int)(v % kSell);
    const float4 *__restrict__ F = static_cast<const float4 *>(A.F);
    const float4 *__restrict__ r = static_cast<const float4 *>(A.r);
    const float *__restrict__ wf = static_cast<const float *>(A.wf);
    const float *__restrict__ wg = static_cast<const float *>(A.wg);
    const float *__restrict__ we = static_cast<const float *>(A.we);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    {
        const int64_t b = __ldg(A.slice_voff + sl) + lane, e = __ldg(A.slice_voff + sl + 1);
#pragma unroll 4
        for (int64_t p = b; p < e; p += kSell) {
            const int32_t j = ld_table<MODE>(A.vid + p);
            const float a = ld_table<MODE>(wf + p), c = ld_table<MODE>(wg + p);
            float4 f, g;
            ld_fg32(F, j, f, g);
            acc.x = fmaf(a, f.x, fmaf(c, g.x, acc.x));
            acc.y = fmaf(a, f.y, fmaf(c, g.y, acc.y));
            acc.z = fmaf(a, f.z, fmaf(c, g.z, acc.z));
            acc.w = fmaf(a, f.w, fmaf(c, g.w, acc.w));
        }
    }
    {
        const int64_t b = __ldg(A.slice_eoff + sl) + lane, e = __ldg(A.slice_eoff + sl + 1);
#pragma unroll 8
        for (int64_t p = b; p < e; p += kSell) {
            const int32_t k = ld_table<MODE>(A.eid + p);
            const float a = ld_table<MODE>(we + p);
            const float4 q = __ldg(r + k);
            acc.x = fmaf(a, q.x, acc.x);
            acc.y = fmaf(a, q.y, acc.y);
            acc.z = fmaf(a, q.z, acc.z);
            acc.w = fmaf(a, q.w, acc.w);
        }
    }
    div_f32_finish<MODE>(A, v, acc);
}

// ------------------------------------------------------------------ kernels
__global__ void __launch_bounds__(kEdgeBlock) edge_flux_f64_kernel(EdgeArgs A) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= A.ne) return;
    if (A.dt_dev && *A.dt_dev == 0.0) return;  // adaptive run already at t_end
    edge_flux_f64_body(A, e);
}
// compact form: 80 registers, 24 warps per SM; the streamed block: 95 registers
// and 20 warps (at 80 it spills)
template <bool GAPS>
__global__ void __launch_bounds__(kEdgeBlock, GAPS ? 6 : 5) edge_flux_f32_kernel(EdgeArgs A) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= A.ne) return;
    if (A.dt_dev && *A.dt_dev == 0.0) return;  // adaptive run already at t_end
    edge_flux_f32_body<GAPS>(A, e);
}
template <int MODE, bool DWE>
__global__ void __launch_bounds__(kDivBlock) div_f64_kernel(DivArgs A) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= A.n_real) return;
    if (MODE != 0 && A.dt_dev && *A.dt_dev == 0.0) return;  // adaptive run already at t_end
    div_f64_body<MODE, DWE>(A, v);
}
template <int MODE>
__global__ void __launch_bounds__(kDivBlock) div_f32_kernel(DivArgs A) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= A.n_real) return;
    if (MODE != 0 && A.dt_dev && *A.dt_dev == 0.0) return;  // adaptive run already at t_end
    div_f32_body<MODE>(A, v);
}

// Grid-wide barrier for a cooperative launch, with a bounded wait: thread 0
// of each block arrives on *count; the last arrival resets it and advances
// *gen; the others spin on *gen at most `limit` times (with a short sleep).
// Returns false (and sets *err) if the wait ran out.  Once *err is set no
// block arrives any more (a block finding it set at entry, or while it
// waits, gives up), so a count left short by a timed-out barrier is never
// completed by a later barrier of the same call; the host resets count,
// gen and err before the next call.
__device__ bool grid_barrier(unsigned int *count, volatile unsigned int *gen, unsigned int nblocks,
                             unsigned long long limit, int *err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int *verr = err;
        ok = 0;
        if (*verr == 0) {
            ok = 1;
            const unsigned int g = *gen;
            __threadfence();
            const unsigned int arrived = atomicAdd(count, 1u);
            if (arrived == nblocks - 1) {
                *count = 0;
                __threadfence();
                atomicAdd((unsigned int *)gen, 1u);
            } else {
                unsigned long long it = 0;
                while (*gen == g) {
                    if (*verr != 0 || ++it > limit) {
                        ok = 0;
                        atomicExch(err, 1);
                        break;
                    }
                    __nanosleep(64);
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// A persistent launch after a timed-out barrier of the same call does no
// work: its state would rest on a stage that did not complete.  Thread 0
// reads the flag for its block, so the whole block takes the same branch.
__device__ __forceinline__ bool barrier_failed(const int *err) {
    __shared__ int failed;
    if (threadIdx.x == 0) failed = *(const volatile int *)err;
    __syncthreads();
    return failed != 0;
}

// One SSP-RK3 stage over every mesh of a batch in one cooperative launch:
// all edge fluxes, a grid barrier, then every vertex's divergence and stage
// update (grid-stride loops; MODE = stage 1..3).
template <int PREC, int MODE>
__global__ void stage_persistent_kernel(EdgeArgs EA, DivArgs DA, unsigned int *bar_count, unsigned int *bar_gen,
                                        unsigned int nblocks_expected, unsigned long long spin_limit, int *err) {
    if (barrier_failed(err)) return;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t e = t0; e < EA.ne; e += stride) {
        if (PREC == 64) edge_flux_f64_body(EA, e);
        else if (EA.coef_gaps) edge_flux_f32_body<true>(EA, e);
        else edge_flux_f32_body<false>(EA, e);
    }
    __threadfence();
    if (!grid_barrier(bar_count, bar_gen, nblocks_expected, spin_limit, err)) return;
    for (int64_t v = t0; v < DA.n_real; v += stride) {
        if (PREC == 64) div_f64_body<MODE>(DA, v);
        else div_f32_body<MODE>(DA, v);
    }
}

// Precision 48: the same stage with the double-word edge flux (its staging in
// dynamic shared memory, kDwSlots double words per thread) and the folded
// divergence.  At most 512 threads a block, so at most 128 registers.
template <int MODE>
__global__ void __launch_bounds__(512, 1)
    stage_persistent_dw_kernel(EdgeArgs EA, DivArgs DA, unsigned int *bar_count, unsigned int *bar_gen,
                               unsigned int nblocks_expected, unsigned long long spin_limit, int *err) {
    if (barrier_failed(err)) return;
    extern __shared__ float2 dw_stage[];
    const dwa::Stage T{dw_stage + threadIdx.x, (int)blockDim.x};
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t e = t0; e < EA.ne; e += stride) dwa::edge_flux_dw_body(EA, e, T);
    __threadfence();
    if (!grid_barrier(bar_count, bar_gen, nblocks_expected, spin_limit, err)) return;
    for (int64_t v = t0; v < DA.n_real; v += stride) div_f64_body<MODE, true>(DA, v);
}

// ------------------------------------------------------------------ support kernels
// Smallest row index whose state has rho <= 0 (or NaN) or a non-finite
// momentum or energy (set_state's physical check).
__global__ void check_rows_kernel(const double *__restrict__ w, int64_t n, unsigned long long *bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const dbl4 s = ld4(w, i);
    if (!(s.x > 0.0) || !isfinite(s.y) || !isfinite(s.z) || !isfinite(s.w)) atomicMin(bad, (unsigned long long)i);
}

__global__ void permute_rows_kernel(const double *__restrict__ in, double *__restrict__ out,
                                    const int32_t *__restrict__ map, int64_t n, bool gather) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t m = __ldg(map + i);
    if (gather) st4(out, i, ld4(in, m));  // out[i] = in[map[i]]
    else st4(out, m, ld4(in, i));         // out[map[i]] = in[i]
}

// Ghost vertices (internal ids n_real .. n_real+n_ghost-1).  A transmissive
// ghost copies its donor's state and fluxes (reading of the configs'
// transmissive boundary); a Dirichlet ghost (its own donor) takes its fixed
// state and fluxes from wsrc / Fsrc, the buffers of the step's start state
// (a no-op when they are the buffers being filled).  F holds `fq` 16-byte
// words per vertex.
__global__ void ghost_fill_kernel(double *__restrict__ w, const double *wsrc, uint4 *__restrict__ F, const uint4 *Fsrc,
                                  int fq, float4 *__restrict__ w32, const int32_t *__restrict__ donor, int64_t n_real,
                                  int64_t n_ghost) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_ghost) return;
    const int64_t g = n_real + i, d = __ldg(donor + i);
    if (d == g) {
        if (w && wsrc && w != wsrc) st4(w, g, ld4(wsrc, g));
        if (F && Fsrc && F != Fsrc)
            for (int c = 0; c < fq; ++c) F[fq * g + c] = Fsrc[fq * g + c];
        return;
    }
    if (w) st4(w, g, ld4(w, d));
    if (F)
        for (int c = 0; c < fq; ++c) F[fq * g + c] = F[fq * d + c];
    if (w32) w32[g] = w32[d];
}

// min over vertices of h_v / (|u| + c), as the bit pattern of a positive double
__global__ void max_dt_kernel(const double *__restrict__ w, const double *__restrict__ hmin, int64_t n, double gamma,
                              unsigned long long *slot, const int32_t *__restrict__ comp) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double t = INFINITY;
    if (v < n) {
        const dbl4 s = ld4(w, v);
        const double ir = 1.0 / s.x;
        const double u = s.y * ir, vv = s.z * ir;
        const double p = (gamma - 1.0) * (s.w - 0.5 * (s.y * u + s.z * vv));
        const double c = sqrt(gamma * p * ir);
        t = hmin[v] / (sqrt(u * u + vv * vv) + c);
        if (!(t > 0)) t = 0;  // non-physical state: report dt = 0
    }
    if (comp) {  // one slot per component
        if (v < n) atomicMin(slot + __ldg(comp + v), (unsigned long long)__double_as_longlong(t));
        return;
    }
    for (int o = 16; o > 0; o >>= 1) t = fmin(t, __shfl_xor_sync(0xffffffffu, t, o));
    if ((threadIdx.x & 31) == 0) atomicMin(slot, (unsigned long long)__double_as_longlong(t));
}

// FMA-throughput probe: 8 independent chains x = x*a + b per thread.
template <class T>
__global__ void fma_probe_kernel(T *out, int iters, T a, T b) {
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = x[k] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dt_finalize_kernel(unsigned long long *slot, double *tstate, double cfl, double t_end,
                                   unsigned long long *nsteps) {
    const double bound = __longlong_as_double((long long)*slot);
    const double t = tstate[0];
    double dt = cfl * bound;
    const double rem = t_end - t;
    if (!(bound > 0.0) || !(bound < INFINITY)) {
        dt = 0.0;
        tstate[2] = 1.0;  // non-physical state
    } else if (rem <= 1e-12 * fabs(t_end)) {
        dt = 0.0;
    } else if (rem < dt) {
        dt = rem;
    }
    tstate[1] = dt;
    tstate[0] = dt > 0.0 ? (rem < cfl * bound ? t_end : t + dt) : t;
    if (dt > 0.0) *nsteps += 1;
    *slot = 0x7FF0000000000000ull;
}

// which: 0 recip64, 1 rsqrt64, 2 half64, 3 twice64
__global__ void recip_check_kernel(const double *x, double *y, int64_t n, int which) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    y[i] = which == 0 ? recip64(v) : which == 1 ? rsqrt64(v) : which == 2 ? half64(v) : twice64(v);
}

// the FP32 edge kernel's coefficient block of n edges from their gaps
__global__ void weno_coef32_check_kernel(const float4 *g, float *k, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float c[kCoefN];
    weno_coef32(g[i], c);
#pragma unroll
    for (int j = 0; j < kCoefN; ++j) k[(int64_t)kCoefN * i + j] = c[j];
}

inline unsigned blocks(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void launch_vertex_flux_f64(const double *w, double *F, int64_t n, double gamma, cudaStream_t s, double *Q) {
    if (n > 0) vertex_flux_f64_kernel<<<blocks(n, 256), 256, 0, s>>>(w, F, Q, n, gamma - 1.0);
}
void launch_vertex_flux_f32(const double *w, float4 *F, float4 *w32, int64_t n, double gamma, cudaStream_t s) {
    if (n > 0) vertex_flux_f32_kernel<<<blocks(n, 256), 256, 0, s>>>(w, F, w32, n, (float)(gamma - 1.0));
}
void launch_edge_flux_f64(const EdgeArgs &a, cudaStream_t s) {
    if (a.ne > 0) edge_flux_f64_kernel<<<blocks(a.ne, kEdgeBlock), kEdgeBlock, 0, s>>>(a);
}
void launch_edge_flux_f32(const EdgeArgs &a, cudaStream_t s) {
    if (a.ne <= 0) return;
    if (a.coef_gaps) edge_flux_f32_kernel<true><<<blocks(a.ne, kEdgeBlock), kEdgeBlock, 0, s>>>(a);
    else edge_flux_f32_kernel<false><<<blocks(a.ne, kEdgeBlock), kEdgeBlock, 0, s>>>(a);
}
template <bool DWE>
void launch_div_f64_t(const DivArgs &a, int mode, cudaStream_t s) {
    const unsigned g = blocks(a.n_real, kDivBlock);
    switch (mode) {
        case 0: div_f64_kernel<0, DWE><<<g, kDivBlock, 0, s>>>(a); break;
        case 1: div_f64_kernel<1, DWE><<<g, kDivBlock, 0, s>>>(a); break;
        case 2: div_f64_kernel<2, DWE><<<g, kDivBlock, 0, s>>>(a); break;
        default: div_f64_kernel<3, DWE><<<g, kDivBlock, 0, s>>>(a); break;
    }
}
void launch_div_f64(const DivArgs &a, int mode, cudaStream_t s) {
    if (a.n_real <= 0) return;
    if (a.dw_edges) launch_div_f64_t<true>(a, mode, s);
    else launch_div_f64_t<false>(a, mode, s);
}
void launch_div_f32(const DivArgs &a, int mode, cudaStream_t s) {
    if (a.n_real <= 0) return;
    const unsigned g = blocks(a.n_real, kDivBlock);
    switch (mode) {
        case 0: div_f32_kernel<0><<<g, kDivBlock, 0, s>>>(a); break;
        case 1: div_f32_kernel<1><<<g, kDivBlock, 0, s>>>(a); break;
        case 2: div_f32_kernel<2><<<g, kDivBlock, 0, s>>>(a); break;
        default: div_f32_kernel<3><<<g, kDivBlock, 0, s>>>(a); break;
    }
}
void launch_check_rows(const double *w, int64_t n, unsigned long long *bad, cudaStream_t s) {
    if (n > 0) check_rows_kernel<<<blocks(n, 256), 256, 0, s>>>(w, n, bad);
}
void launch_permute_rows(const double *in, double *out, const int32_t *map, int64_t n, bool gather, cudaStream_t s) {
    if (n > 0) permute_rows_kernel<<<blocks(n, 256), 256, 0, s>>>(in, out, map, n, gather);
}
void launch_ghost_fill(double *w, const double *wsrc, void *F, const void *Fsrc, int fq, float4 *w32,
                       const int32_t *donor, int64_t n_real, int64_t n_ghost, cudaStream_t s) {
    if (n_ghost > 0)
        ghost_fill_kernel<<<blocks(n_ghost, 256), 256, 0, s>>>(w, wsrc, static_cast<uint4 *>(F),
                                                               static_cast<const uint4 *>(Fsrc), fq, w32, donor, n_real,
                                                               n_ghost);
}
void launch_max_dt(const double *w, const double *hmin, int64_t n, double gamma, unsigned long long *slot,
                   cudaStream_t s, const int32_t *comp) {
    if (n > 0) max_dt_kernel<<<blocks(n, 256), 256, 0, s>>>(w, hmin, n, gamma, slot, comp);
}

namespace {
template <int PREC, int MODE>
cudaError_t coop(const EdgeArgs &ea, const DivArgs &da, unsigned int *c, unsigned int *g, unsigned int ne,
                 unsigned long long lim, int *err, int threads, int nb, cudaStream_t s) {
    EdgeArgs a = ea;
    DivArgs d = da;
    void *args[] = {&a, &d, &c, &g, &ne, &lim, &err};
    return cudaLaunchCooperativeKernel((const void *)stage_persistent_kernel<PREC, MODE>, dim3(nb), dim3(threads),
                                       args, 0, s);
}
}  // namespace

namespace {
size_t dw_stage_bytes(int threads) { return (size_t)dwa::kDwSlots * sizeof(float2) * threads; }
template <int MODE>
cudaError_t coop48(const EdgeArgs &ea, const DivArgs &da, unsigned int *c, unsigned int *g, unsigned int ne,
                   unsigned long long lim, int *err, int threads, int nb, cudaStream_t s) {
    EdgeArgs a = ea;
    DivArgs d = da;
    void *args[] = {&a, &d, &c, &g, &ne, &lim, &err};
    const size_t bytes = dw_stage_bytes(threads);
    cudaError_t e = cudaFuncSetAttribute((const void *)stage_persistent_dw_kernel<MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel((const void *)stage_persistent_dw_kernel<MODE>, dim3(nb), dim3(threads), args,
                                       bytes, s);
}
}  // namespace

cudaError_t launch_stage_persistent(int prec, int mode, const EdgeArgs &ea, const DivArgs &da, unsigned int *bar_count,
                                    unsigned int *bar_gen, unsigned int nblocks_expected,
                                    unsigned long long spin_limit, int *err, int threads, int nb, cudaStream_t s) {
    const unsigned int ne = nblocks_expected;
    if (prec == 48) {
        if (mode == 1) return coop48<1>(ea, da, bar_count, bar_gen, ne, spin_limit, err, threads, nb, s);
        if (mode == 2) return coop48<2>(ea, da, bar_count, bar_gen, ne, spin_limit, err, threads, nb, s);
        return coop48<3>(ea, da, bar_count, bar_gen, ne, spin_limit, err, threads, nb, s);
    }
    if (prec == 64) {
        if (mode == 1) return coop<64, 1>(ea, da, bar_count, bar_gen, ne, spin_limit, err, threads, nb, s);
        if (mode == 2) return coop<64, 2>(ea, da, bar_count, bar_gen, ne, spin_limit, err, threads, nb, s);
        return coop<64, 3>(ea, da, bar_count, bar_gen, ne, spin_limit, err, threads, nb, s);
    }
    if (mode == 1) return coop<32, 1>(ea, da, bar_count, bar_gen, ne, spin_limit, err, threads, nb, s);
    if (mode == 2) return coop<32, 2>(ea, da, bar_count, bar_gen, ne, spin_limit, err, threads, nb, s);
    return coop<32, 3>(ea, da, bar_count, bar_gen, ne, spin_limit, err, threads, nb, s);
}

int persistent_blocks_per_sm(int prec, int threads) {
    int n = 0;
    // the three stage modes share their register footprint; mode 3 stands for all
    if (prec == 48) {
        const size_t bytes = dw_stage_bytes(threads);
        for (auto k : {stage_persistent_dw_kernel<1>, stage_persistent_dw_kernel<2>, stage_persistent_dw_kernel<3>})
            if (cudaFuncSetAttribute((const void *)k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
                cudaSuccess)
                return 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_persistent_dw_kernel<3>, threads, bytes);
    } else if (prec == 64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_persistent_kernel<64, 3>, threads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, stage_persistent_kernel<32, 3>, threads, 0);
    return n;
}

double fma_probe_tflops(int precision, int sms, void *scratch, cudaStream_t s) {
    const int nb = sms * 8, nt = 256;
    const int iters = precision == 64 ? 2048 : 65536;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (int rep = 0; rep < 2; ++rep) {  // first launch warms up
        cudaEventRecord(a, s);
        if (precision == 64)
            fma_probe_kernel<double><<<nb, nt, 0, s>>>(static_cast<double *>(scratch), iters, 0.999999, 1e-7);
        else
            fma_probe_kernel<float><<<nb, nt, 0, s>>>(static_cast<float *>(scratch), iters, 0.999999f, 1e-7f);
        cudaEventRecord(b, s);
    }
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return 2.0 * 8.0 * iters * (double)nb * nt / (ms * 1e-3) / 1e12;
}

void launch_recip_check(const double *x, double *y, int64_t n, int which, cudaStream_t s) {
    if (n > 0) recip_check_kernel<<<blocks(n, 256), 256, 0, s>>>(x, y, n, which);
}

void launch_weno_coef32_check(const float4 *g, float *k, int64_t n, cudaStream_t s) {
    if (n > 0) weno_coef32_check_kernel<<<blocks(n, 256), 256, 0, s>>>(g, k, n);
}

void launch_dt_finalize(unsigned long long *slot, double *tstate, double cfl, double t_end,
                        unsigned long long *nsteps, cudaStream_t s) {
    dt_finalize_kernel<<<1, 1, 0, s>>>(slot, tstate, cfl, t_end, nsteps);
}

}  // namespace fdu
