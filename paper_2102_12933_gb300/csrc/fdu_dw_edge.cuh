// The precision-48 edge flux (device only): NU-WENO5 of one field in
// double words and the edge-flux body, shared by the standalone kernel
// (fdu_dw.cu) and the batched persistent stage (fdu_kernels.cu).  See
// fdu_dw.cu for the arithmetic's design.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "fdu_dw.cuh"
#include "fdu_dw_euler.cuh"
#include "fdu_internal.h"
#include "fdu_kernels.cuh"

namespace fdu {
namespace dwa {

// ---- NU-WENO5 increments of one field, both sides (the block layout and
// sub-stencil sharing of weno_pair64_l1; right increments from L1)
__device__ __forceinline__ int bexp(float x) { return (int)((__float_as_uint(x) >> 23) & 0xffu); }

__device__ __forceinline__ void weno_pair_dw(const dw *k, dw a, dw b, dw c, dw d, dw e, dw f, dw eps_m, int eps_e,
                                             dw &dl, dw &dr) {
    const dw va = add_sl(mul_u(k[0], a), mul_u(k[1], b));
    const dw vb = add_sl(mul_u(k[5], b), mul_u(k[6], c));
    const dw vc = add_sl(mul_u(k[10], c), mul_u(k[11], d));
    const dw vd = add_sl(mul_u(k[15], e), mul_u(k[16], f));
    const dw vdc = add_sl(vd, c);  // S_d's value from L1
    // common power-of-two scale of the six differences: max |.| in [1/2, 1)
    const float mx = fmaxf(fmaxf(fmaxf(fabsf(a.h), fabsf(b.h)), fmaxf(fabsf(c.h), fabsf(d.h))),
                           fmaxf(fabsf(e.h), fabsf(f.h)));
    const int be = bexp(mx);
    const int K = be == 0 ? 0 : be - 126;                  // mx in [2^(K-1), 2^K)
    const float lam = __uint_as_float((unsigned)(127 - K) << 23);  // 2^-K (K in [-125, 128])
    a = scale(a, lam);
    b = scale(b, lam);
    c = scale(c, lam);
    d = scale(d, lam);
    e = scale(e, lam);
    f = scale(f, lam);
    // eps 2^(-2K) = eps_m 2^(eps_e - 2K) (zero below the float range)
    const int e2 = min(eps_e - 2 * K, 100) + 127;  // beyond 2^100 the weights are the linear ones anyway
    const dw eps = e2 >= 1 ? scale(eps_m, __uint_as_float((unsigned)e2 << 23)) : dw_make(0.0f, 0.0f);
    const dw b2 = mul_u(b, b), c2 = mul_u(c, c);
    auto beta = [&](dw m0, dw m1, dw m2, dw xx, dw xy, dw yy) {
        dw s = add_sl(add_sl(add_sl(mul_u(m0, xx), mul_u(m1, xy)), mul_u(m2, yy)), eps);
        if (s.h < 0x1p-100f) s = dw_make(0x1p-100f, 0.0f);
        return s;
    };
    const dw ra = recip(beta(k[2], k[3], k[4], mul_u(a, a), mul_u(a, b), b2));
    const dw rb = recip(beta(k[7], k[8], k[9], b2, mul_u(b, c), c2));
    const dw rc = recip(beta(k[12], k[13], k[14], c2, mul_u(c, d), mul_u(d, d)));
    const dw rd = recip(beta(k[17], k[18], k[19], mul_u(e, e), mul_u(e, f), mul_u(f, f)));
    // alpha_k = C_k / (beta_k + eps); the block stores C_0/C_1, C_2/C_1 (C_1 -> 1)
    const dw l0 = mul(k[20], ra), l2 = mul(k[21], rc);
    dl = mul(add_sl(add_sl(mul_u(l0, va), mul_u(rb, vb)), mul_u(l2, vc)), recip(add_sl(add_sl(l0, rb), l2)));
    const dw r0 = mul(k[22], rd), r2 = mul(k[23], rb);
    dr = mul(add_sl(add_sl(mul_u(r0, vdc), mul_u(rc, vc)), mul_u(r2, vb)), recip(add_sl(add_sl(r0, rc), r2)));
}

// ---- the edge flux
// Per-thread staging in shared memory, slot j of thread t at [j][t]: the
// five differences (slots 0-19, projected in place) and the WENO
// increments (20-27).  The projections and the four fields run as loops
// over the staged values, so their code is issued from the instruction
// cache once per loop instead of being unrolled five and four times.
constexpr int kDwSlots = 28;
// slot j of a thread at S[j * stride] (stride = the threads of the block)
struct Stage {
    float2 *S;
    int stride;
};
__device__ __forceinline__ void st_dw(const Stage &T, int j, dw v) { T.S[j * T.stride] = make_float2(v.h, v.l); }
__device__ __forceinline__ dw ld_dw(const Stage &T, int j) {
    const float2 q = T.S[j * T.stride];
    return dw_make(q.x, q.y);
}
__device__ __forceinline__ void st_dw4(const Stage &S, int j, const dw4 &v) {
    st_dw(S, j, v.x);
    st_dw(S, j + 1, v.y);
    st_dw(S, j + 2, v.z);
    st_dw(S, j + 3, v.w);
}
__device__ __forceinline__ dw4 ld_dw4(const Stage &S, int j) {
    return d4(ld_dw(S, j), ld_dw(S, j + 1), ld_dw(S, j + 2), ld_dw(S, j + 3));
}

__device__ __forceinline__ void edge_flux_dw_body(const EdgeArgs &A, const int64_t e, const Stage &S) {
    const double *__restrict__ w = static_cast<const double *>(A.w);
    const int64_t ne = A.ne;
    const dw gm1 = dw_make(A.dw_gm1[0], A.dw_gm1[1]);
    int32_t s[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = __ldg(A.sten + (int64_t)i * ne + e);
    const float2 nq = __ldg(A.coefdw + (int64_t)kCoefN * ne + e), mq = __ldg(A.coefdw + (int64_t)(kCoefN + 1) * ne + e);
    const dw nx = dw_make(nq.x, nq.y), ny = dw_make(mq.x, mq.y);
    const d4v L1 = ldd4(w, s[2]);
    dw4 b;  // L1 in double words
    {
        // FP64 differences, then double words: R1-L1, L2-L1, L3-L1, R2-R1, R3-R1
        auto diff = [](const d4v &p, const d4v &q) { return d2dw4(d4v{p.x - q.x, p.y - q.y, p.z - q.z, p.w - q.w}); };
        const d4v R1 = ldd4(w, s[3]);
        st_dw4(S, 0, diff(R1, L1));
        st_dw4(S, 4, diff(ldd4(w, s[1]), L1));
        st_dw4(S, 8, diff(ldd4(w, s[0]), L1));
        st_dw4(S, 12, diff(ldd4(w, s[4]), R1));
        st_dw4(S, 16, diff(ldd4(w, s[5]), R1));
        b = d2dw4(L1);
    }
    const RoeW C = roe_records(d2dw4(ldd4(A.Q, s[2])), d2dw4(ldd4(A.Q, s[3])), nx, ny, gm1);
#pragma unroll 1
    for (int j = 0; j < 20; j += 4) st_dw4(S, j, project(C, ld_dw4(S, j)));

    {
        dw k[kCoefN];
#pragma unroll
        for (int i = 0; i < kCoefN; ++i) {
            const float2 q = __ldg(A.coefdw + (int64_t)i * ne + e);
            k[i] = dw_make(q.x, q.y);
        }
        const dw eps_m = dw_make(A.dw_eps[0], A.dw_eps[1]);
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {
            const dw c = ld_dw(S, i), f = ld_dw(S, 12 + i);
            dw dl, dr;
            weno_pair_dw(k, ld_dw(S, 8 + i), ld_dw(S, 4 + i), c, add_sl(f, c), ld_dw(S, 16 + i), f, eps_m, A.dw_eps_e,
                         dl, dr);
            st_dw(S, 20 + i, dl);
            st_dw(S, 24 + i, dr);
        }
    }

    // increments of both interpolated states from L1
    dw4 il = unproject(C, ld_dw4(S, 20)), ir = unproject(C, ld_dw4(S, 24));

    // primitives of L1
    const dw ib = recip(b.x);
    const dw ub = mul(b.y, ib), vb = mul(b.z, ib);
    const dw qnb = add_sl(mul_u(ub, nx), mul_u(vb, ny));
    const dw mu = add_sl(mul_u(b.y, ub), mul_u(b.z, vb));  // |m|^2 / rho
    const dw pb = mul(gm1, sub_sl(b.w, scale(mu, 0.5f)));

    // a side's state from its increment: rho', 1/sqrt(rho'), the normal
    // velocity increment and the pressure increment
    struct Side {
        dw rho, r, ir, dq, dp, p;
    };
    auto side = [&](const dw4 &dd, Side &Sd) {
        Sd.rho = add_sl(b.x, dd.x);
        if (!(Sd.rho.h > 0.0f)) return false;
        Sd.r = rsqrt(Sd.rho);
        Sd.ir = mul(Sd.r, Sd.r);
        Sd.dq = mul(sub_sl(add_sl(mul_u(dd.y, nx), mul_u(dd.z, ny)), mul_u(qnb, dd.x)), Sd.ir);
        // K' - K = ((2m + dm).dm - (|m|^2/rho) drho) / (2 rho')
        const dw t = sub_sl(add_sl(mul_u(add_sl(scale(b.y, 2.0f), dd.y), dd.y),
                                   mul_u(add_sl(scale(b.z, 2.0f), dd.z), dd.z)),
                            mul_u(mu, dd.x));
        Sd.dp = mul(gm1, sub_sl(dd.w, scale(mul(t, Sd.ir), 0.5f)));
        Sd.p = add_sl(pb, Sd.dp);
        return Sd.p.h > 0.0f;
    };
    Side SL, SR;
    bool ok = side(il, SL);
    ok = ok && side(ir, SR);
    if (!ok) {  // positivity fallback: first-order end states
        const d4v R1 = ldd4(w, s[3]);
        il = d4(dw_make(0.0f), dw_make(0.0f), dw_make(0.0f), dw_make(0.0f));
        ir = d2dw4(d4v{R1.x - L1.x, R1.y - L1.y, R1.z - L1.z, R1.w - L1.w});
        side(il, SL);
        side(ir, SR);
        atomicAdd(A.fallback, 1ull);
    }

    // flux increment F_n(w_L) - F_n(L1)
    const dw qnl = add_sl(qnb, SL.dq);
    dw4 out;
    out.x = add_sl(mul_u(il.y, nx), mul_u(il.z, ny));
    out.y = add_sl(add_sl(mul_u(il.y, qnl), mul_u(b.y, SL.dq)), mul_u(SL.dp, nx));
    out.z = add_sl(add_sl(mul_u(il.z, qnl), mul_u(b.z, SL.dq)), mul_u(SL.dp, ny));
    out.w = add_sl(mul_u(add_sl(il.w, SL.dp), qnl), mul_u(add_sl(b.w, pb), SL.dq));

    // Roe dissipation at the Roe average of (w_L, w_R)
    {
        const dw4 wl = add4_sl(b, il), wr = add4_sl(b, ir);
        const dw sa = mul_u(SL.rho, SL.r), sb = mul_u(SR.rho, SR.r);
        const dw inv = recip(add_sl(sa, sb));
        const RoeW Q = roe_finish(mul(add_sl(mul_u(wl.y, SL.r), mul_u(wr.y, SR.r)), inv),
                                  mul(add_sl(mul_u(wl.z, SL.r), mul_u(wr.z, SR.r)), inv),
                                  mul(add_sl(mul_u(add_sl(wl.w, SL.p), SL.r), mul_u(add_sl(wr.w, SR.p), SR.r)), inv),
                                  nx, ny, gm1);
        const dw4 a = project(Q, sub4_sl(ir, il));
        const dw delta = mul(Q.c, dw_make(A.dw_tenth[0], A.dw_tenth[1]));
        const dw h2d = mul(Q.ic, 5.0f);  // 1 / (2 delta)
        auto negp = [&](dw l) {  // (l - |l|_fixed) / 2
            const dw m = dabs(l);
            if (m.h < delta.h || (m.h == delta.h && m.l < delta.l))
                return scale(sub_sl(l, mul(add_sl(mul_u(l, l), mul_u(delta, delta)), h2d)), 0.5f);
            return l.h < 0.0f ? l : dw_make(0.0f);
        };
        const dw nu = negp(Q.qn), nm = negp(sub_sl(Q.qn, Q.c)), np = negp(add_sl(Q.qn, Q.c));
        const dw4 D = unproject(Q, d4(mul(nm, a.x), mul(nu, a.y), mul(nu, a.z), mul(np, a.w)));
        out = add4_sl(out, D);
    }

    // the increment r - F_n(L1); the divergence adds F_n(L1) through its
    // folded vertex weights
    float4 *r = static_cast<float4 *>(A.r);
    r[2 * e] = make_float4(out.x.h, out.x.l, out.y.h, out.y.l);
    r[2 * e + 1] = make_float4(out.z.h, out.z.l, out.w.h, out.w.l);
}

}  // namespace dwa
}  // namespace fdu
