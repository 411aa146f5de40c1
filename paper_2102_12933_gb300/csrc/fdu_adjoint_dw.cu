// Edge-flux VJP of precision 48: the FP64 edge VJP (fdu_adjoint.cu) with its
// arithmetic in double words (FP32 pairs, about 48 significant bits), which
// GB300 issues at 64 times its FP64 rate.  It differentiates the same function
// (the symmetric Roe form and the R1-based right state, Section 2.3.1 and the
// Appendix) and takes the same branches (positivity fallback, entropy-fix band,
// sign of lambda); cotangents are sums of products of increments and
// Jacobian entries, for which the double-word rounding (about 1e-13 relative)
// is far inside the gradient's use.
//
// The nonlinear weights use the range-safe form of the forward kernel: per
// field the differences are scaled by lambda = 2^-K (max |difference| in
// [1/2, 1)) and beta' = lambda^2 (beta + eps), bounded below by 2^-100;
// omega = alpha / sum(alpha), alpha_k = C_k / beta'_k, and
//   d(dl)/d(beta'_k) = -omega_k (v_k - dl) / beta'_k,
//   d(beta'_k)/d(x)  = lambda (2 m0 x' + m1 y')  (x' = lambda x),
// zero where the bound holds beta' (a sub-stencil whose differences are
// below 2^-50 of the field's largest).
#include <cuda_runtime.h>

#include <cstdint>

#include "fdu_adjoint.cuh"
#include "fdu_dw.cuh"
#include "fdu_dw_euler.cuh"
#include "fdu_internal.h"
#include "fdu_kernels.cuh"

namespace fdu {
namespace {

using namespace dwa;

constexpr int kVjpBlock = 64;
constexpr int kVjpSlots = 64;
// per-thread shared-memory slots (float2 double words), slot j of thread t at [j][t]
constexpr int kSlotC = 0;     // characteristic projections of R1-L1, L2-L1, L3-L1, R2-R1, R3-R1 (5 x 4)
constexpr int kSlotW = 20;    // per field: va vb vc vd B'a B'b B'c B'd (4 x 8); reverse: the six cotangents
constexpr int kSlotS = 52;    // per field: (lambda, clamp bits)
constexpr int kSlotLR = 56;   // per field: dl, dr

__device__ __forceinline__ void st_s(float2 *S, int j, dw v) { S[j * kVjpBlock] = make_float2(v.h, v.l); }
__device__ __forceinline__ dw ld_s(const float2 *S, int j) {
    const float2 q = S[j * kVjpBlock];
    return dw_make(q.x, q.y);
}
__device__ __forceinline__ void st_s4(float2 *S, int j, const dw4 &v) {
    st_s(S, j, v.x);
    st_s(S, j + 1, v.y);
    st_s(S, j + 2, v.z);
    st_s(S, j + 3, v.w);
}
__device__ __forceinline__ dw4 ld_s4(const float2 *S, int j) {
    return d4(ld_s(S, j), ld_s(S, j + 1), ld_s(S, j + 2), ld_s(S, j + 3));
}
__device__ __forceinline__ dw4 zero4() { return d4(dw_make(0.0f), dw_make(0.0f), dw_make(0.0f), dw_make(0.0f)); }
__device__ __forceinline__ void acc(dw &a, dw b) { a = add_sl(a, b); }
__device__ __forceinline__ void acc4(dw4 &a, const dw4 &b) { a = add4_sl(a, b); }
__device__ __forceinline__ dw mulsum(dw a, dw b, dw c, dw d) { return add_sl(mul_u(a, b), mul_u(c, d)); }
__device__ __forceinline__ double to64(dw x) { return f2d(x.h) + f2d(x.l); }

// ---- forward pieces not in the edge-flux kernel's increment form
struct PrimW {
    dw r, ir, p;  // rho^-1/2, 1/rho, p
};
struct PrimWBar {
    dw r = dw_make(0.0f), ir = dw_make(0.0f), p = dw_make(0.0f);
};
__device__ __forceinline__ PrimW prim_w(const dw4 &w, dw gm1) {
    PrimW P;
    P.r = rsqrt(w.x);
    P.ir = mul(P.r, P.r);
    P.p = mul(gm1, sub_sl(w.w, scale(mul(add_sl(mul_u(w.y, w.y), mul_u(w.z, w.z)), P.ir), 0.5f)));
    return P;
}
// symmetric Roe average of two states (the roe64 of the FP64 kernels)
__device__ __forceinline__ RoeW roe_w(const dw4 &a, const PrimW &pa, const dw4 &b, const PrimW &pb, dw nx, dw ny,
                                      dw gm1) {
    const dw inv = recip(add_sl(mul_u(a.x, pa.r), mul_u(b.x, pb.r)));
    return roe_finish(mul(mulsum(a.y, pa.r, b.y, pb.r), inv), mul(mulsum(a.z, pa.r, b.z, pb.r), inv),
                      mul(mulsum(add_sl(a.w, pa.p), pa.r, add_sl(b.w, pb.p), pb.r), inv), nx, ny, gm1);
}

struct RoeWBar {
    dw u = dw_make(0.0f), v = dw_make(0.0f), H = dw_make(0.0f), c = dw_make(0.0f), ic = dw_make(0.0f),
       b1 = dw_make(0.0f), qn = dw_make(0.0f), qt = dw_make(0.0f), hq2 = dw_make(0.0f);
};

// ---- reverse pieces (the FP64 helpers of fdu_adjoint.cu, term for term)
__device__ __forceinline__ void prim_vjp_w(const dw4 &w, const PrimW &P, const PrimWBar &B, dw gm1, dw4 &wb) {
    const dw ke2 = add_sl(mul_u(w.y, w.y), mul_u(w.z, w.z));
    const dw pg = mul(B.p, gm1);
    const dw irb = sub_sl(B.ir, scale(mul(pg, ke2), 0.5f));
    const dw rb = add_sl(B.r, scale(mul(irb, P.r), 2.0f));
    acc(wb.x, neg(scale(mul(rb, mul(P.r, P.ir)), 0.5f)));
    acc(wb.y, neg(mul(pg, mul(w.y, P.ir))));
    acc(wb.z, neg(mul(pg, mul(w.z, P.ir))));
    acc(wb.w, pg);
}

__device__ __forceinline__ void roe_vjp_w(const dw4 &a, const PrimW &pa, const dw4 &b, const PrimW &pb,
                                          const RoeW &R, const RoeWBar &Rb, dw gm1, dw4 &ab, PrimWBar &pab, dw4 &bb,
                                          PrimWBar &pbb) {
    dw ub = add_sl(Rb.u, sub_sl(mul_u(Rb.qn, R.nx), mul_u(Rb.qt, R.ny)));
    dw vb = add_sl(Rb.v, add_sl(mul_u(Rb.qn, R.ny), mul_u(Rb.qt, R.nx)));
    const dw ic2 = mul(R.ic, R.ic);
    const dw icb = add_sl(Rb.ic, scale(mul(mul(Rb.b1, gm1), R.ic), 2.0f));
    const dw c2b = scale(sub_sl(mul_u(Rb.c, R.ic), mul_u(icb, mul(ic2, R.ic))), 0.5f);
    const dw c2g = mul(c2b, gm1);
    const dw Hb = add_sl(Rb.H, c2g);
    const dw hq2b = sub_sl(Rb.hq2, c2g);
    ub = add_sl(ub, mul(hq2b, R.u));
    vb = add_sl(vb, mul(hq2b, R.v));
    const dw inv = recip(add_sl(mul_u(a.x, pa.r), mul_u(b.x, pb.r)));
    const dw U = mulsum(a.y, pa.r, b.y, pb.r);
    const dw V = mulsum(a.z, pa.r, b.z, pb.r);
    const dw Ea = add_sl(a.w, pa.p), Eb = add_sl(b.w, pb.p);
    const dw Hn = mulsum(Ea, pa.r, Eb, pb.r);
    const dw invb = add_sl(mulsum(ub, U, vb, V), mul_u(Hb, Hn));
    const dw Ub = mul(ub, inv), Vb = mul(vb, inv), Hnb = mul(Hb, inv);
    const dw sbar = neg(mul(invb, mul(inv, inv)));
    acc(ab.x, mul(sbar, pa.r));
    acc(pab.r, mul(sbar, a.x));
    acc(bb.x, mul(sbar, pb.r));
    acc(pbb.r, mul(sbar, b.x));
    acc(ab.y, mul(Ub, pa.r));
    acc(pab.r, mul(Ub, a.y));
    acc(bb.y, mul(Ub, pb.r));
    acc(pbb.r, mul(Ub, b.y));
    acc(ab.z, mul(Vb, pa.r));
    acc(pab.r, mul(Vb, a.z));
    acc(bb.z, mul(Vb, pb.r));
    acc(pbb.r, mul(Vb, b.z));
    const dw ha = mul(Hnb, pa.r), hb = mul(Hnb, pb.r);
    acc(ab.w, ha);
    acc(pab.p, ha);
    acc(pab.r, mul(Hnb, Ea));
    acc(bb.w, hb);
    acc(pbb.p, hb);
    acc(pbb.r, mul(Hnb, Eb));
}

// c = project(R, d): d's and R's cotangents (R.b1 = 2 R.b1h, R.ic = 2 R.ich)
__device__ __forceinline__ void project_vjp_w(const RoeW &R, const dw4 &d, const dw4 &cb, dw4 &db, RoeWBar &Rb) {
    const dw b1 = scale(R.b1h, 2.0f);
    const dw phib = sub_sl(scale(add_sl(cb.x, cb.w), 0.5f), cb.y);
    const dw psib = scale(sub_sl(cb.x, cb.w), 0.5f);
    acc(db.x, sub_sl(cb.y, mul_u(R.qt, cb.z)));
    acc(db.y, neg(mul(R.ny, cb.z)));
    acc(db.z, mul(R.nx, cb.z));
    acc(Rb.qt, neg(mul(d.x, cb.z)));
    const dw inner_phi = add_sl(sub_sl(sub_sl(mul_u(R.hq2, d.x), mul_u(R.u, d.y)), mul_u(R.v, d.z)), d.w);
    acc(Rb.b1, mul(phib, inner_phi));
    const dw t = mul(phib, b1);
    acc(Rb.hq2, mul(t, d.x));
    acc(Rb.u, neg(mul(t, d.y)));
    acc(Rb.v, neg(mul(t, d.z)));
    acc(db.x, mul(t, R.hq2));
    acc(db.y, neg(mul(t, R.u)));
    acc(db.z, neg(mul(t, R.v)));
    acc(db.w, t);
    const dw inner_psi = sub_sl(sub_sl(mul_u(R.qn, d.x), mul_u(R.nx, d.y)), mul_u(R.ny, d.z));
    acc(Rb.ic, mul(psib, inner_psi));
    const dw s = mul(psib, R.ic);
    acc(Rb.qn, mul(s, d.x));
    acc(db.x, mul(s, R.qn));
    acc(db.y, neg(mul(s, R.nx)));
    acc(db.z, neg(mul(s, R.ny)));
}

// d = unproject(R, c): c's and R's cotangents
__device__ __forceinline__ void unproject_vjp_w(const RoeW &R, const dw4 &c, const dw4 &dbar, dw4 &cb, RoeWBar &Rb) {
    const dw acw = add_sl(c.x, c.w);
    const dw rho = add_sl(acw, c.y);
    const dw cwx = sub_sl(c.w, c.x);
    const dw dd = mul(R.c, cwx);
    const dw rhob = add_sl(dbar.x, mulsum(R.u, dbar.y, R.v, dbar.z));
    const dw ddb = add_sl(mulsum(R.nx, dbar.y, R.ny, dbar.z), mul_u(R.qn, dbar.w));
    acc(Rb.u, mul(rho, dbar.y));
    acc(Rb.v, mul(rho, dbar.z));
    acc(Rb.H, mul(acw, dbar.w));
    acc(Rb.hq2, mul(c.y, dbar.w));
    acc(Rb.qn, mul(dd, dbar.w));
    acc(Rb.qt, mul(c.z, dbar.w));
    acc(Rb.c, mul(cwx, ddb));
    const dw hw = mul(R.H, dbar.w), cd = mul(R.c, ddb);
    acc(cb.x, sub_sl(add_sl(rhob, hw), cd));
    acc(cb.y, add_sl(rhob, mul(R.hq2, dbar.w)));
    acc(cb.z, add_sl(sub_sl(mul_u(R.nx, dbar.z), mul_u(R.ny, dbar.y)), mul_u(R.qt, dbar.w)));
    acc(cb.w, add_sl(add_sl(rhob, hw), cd));
}

// F_n(w) with the primitives of prim_w; reverse into w and P
__device__ __forceinline__ void fluxn_vjp_w(const dw4 &w, const PrimW &P, dw nx, dw ny, const dw4 &fb, dw4 &wb,
                                            PrimWBar &Pb) {
    const dw mn = mulsum(w.y, nx, w.z, ny);
    const dw q = mul(mn, P.ir);
    const dw Ep = add_sl(w.w, P.p);
    const dw qb = add_sl(mulsum(fb.x, w.x, fb.y, w.y), mulsum(fb.z, w.z, fb.w, Ep));
    acc(wb.x, mul(fb.x, q));
    acc(wb.y, mul(fb.y, q));
    acc(wb.z, mul(fb.z, q));
    acc(wb.w, mul(fb.w, q));
    acc(Pb.p, add_sl(mulsum(fb.y, nx, fb.z, ny), mul_u(fb.w, q)));
    const dw mnb = mul(qb, P.ir);
    acc(Pb.ir, mul(qb, mn));
    acc(wb.y, mul(mnb, nx));
    acc(wb.z, mul(mnb, ny));
}

// ---- NU-WENO5 of one field, forward (values, scaled indicators, dl, dr)
// and reverse (cotangents of the six differences a..f)
__device__ __forceinline__ int bexp(float x) { return (int)((__float_as_uint(x) >> 23) & 0xffu); }

struct WScale {
    float lam;  // 2^-K
    int K;
};
__device__ __forceinline__ WScale field_scale(dw a, dw b, dw c, dw d, dw e, dw f) {
    const float mx = fmaxf(fmaxf(fmaxf(fabsf(a.h), fabsf(b.h)), fmaxf(fabsf(c.h), fabsf(d.h))),
                           fmaxf(fabsf(e.h), fabsf(f.h)));
    const int be = bexp(mx);
    WScale s;
    s.K = be == 0 ? 0 : be - 126;
    s.lam = __uint_as_float((unsigned)(127 - s.K) << 23);
    return s;
}

// k: the 24 WENO coefficients of the edge (double words, global memory)
__device__ __forceinline__ dw kc(const float2 *kp, int64_t ne, int i) {
    const float2 q = __ldg(kp + (int64_t)i * ne);
    return dw_make(q.x, q.y);
}

__device__ __forceinline__ void weno_fwd_w(const float2 *kp, int64_t ne, dw a, dw b, dw c, dw d, dw e, dw f,
                                           dw eps_m, int eps_e, float2 *S, int fi) {
    const dw va = add_sl(mul_u(kc(kp, ne, 0), a), mul_u(kc(kp, ne, 1), b));
    const dw vb = add_sl(mul_u(kc(kp, ne, 5), b), mul_u(kc(kp, ne, 6), c));
    const dw vc = add_sl(mul_u(kc(kp, ne, 10), c), mul_u(kc(kp, ne, 11), d));
    const dw vd = add_sl(mul_u(kc(kp, ne, 15), e), mul_u(kc(kp, ne, 16), f));
    const WScale sc = field_scale(a, b, c, d, e, f);
    a = scale(a, sc.lam);
    b = scale(b, sc.lam);
    const dw cs = scale(c, sc.lam);
    d = scale(d, sc.lam);
    e = scale(e, sc.lam);
    f = scale(f, sc.lam);
    const int e2 = min(eps_e - 2 * sc.K, 100) + 127;
    const dw eps = e2 >= 1 ? scale(eps_m, __uint_as_float((unsigned)e2 << 23)) : dw_make(0.0f, 0.0f);
    int clamp = 0;
    auto beta = [&](int bit, dw m0, dw m1, dw m2, dw x, dw y) {
        dw s = add_sl(add_sl(add_sl(mul_u(m0, mul_u(x, x)), mul_u(m1, mul_u(x, y))), mul_u(m2, mul_u(y, y))), eps);
        if (s.h < 0x1p-100f) {
            s = dw_make(0x1p-100f, 0.0f);
            clamp |= bit;
        }
        return s;
    };
    const dw Ba = beta(1, kc(kp, ne, 2), kc(kp, ne, 3), kc(kp, ne, 4), a, b);
    const dw Bb = beta(2, kc(kp, ne, 7), kc(kp, ne, 8), kc(kp, ne, 9), b, cs);
    const dw Bc = beta(4, kc(kp, ne, 12), kc(kp, ne, 13), kc(kp, ne, 14), cs, d);
    const dw Bd = beta(8, kc(kp, ne, 17), kc(kp, ne, 18), kc(kp, ne, 19), e, f);
    const dw ra = recip(Ba), rb = recip(Bb), rc = recip(Bc), rd = recip(Bd);
    const dw l0 = mul(kc(kp, ne, 20), ra), l2 = mul(kc(kp, ne, 21), rc);
    const dw dl = mul(add_sl(add_sl(mul_u(l0, va), mul_u(rb, vb)), mul_u(l2, vc)), recip(add_sl(add_sl(l0, rb), l2)));
    const dw r0 = mul(kc(kp, ne, 22), rd), r2 = mul(kc(kp, ne, 23), rb);
    const dw dr = mul(add_sl(add_sl(mul_u(r0, vd), mul_u(rc, sub_sl(vc, c))), mul_u(r2, sub_sl(vb, c))),
                      recip(add_sl(add_sl(r0, rc), r2)));
    const int w0 = kSlotW + 8 * fi;
    st_s(S, w0 + 0, va);
    st_s(S, w0 + 1, vb);
    st_s(S, w0 + 2, vc);
    st_s(S, w0 + 3, vd);
    st_s(S, w0 + 4, Ba);
    st_s(S, w0 + 5, Bb);
    st_s(S, w0 + 6, Bc);
    st_s(S, w0 + 7, Bd);
    S[(kSlotS + fi) * kVjpBlock] = make_float2(sc.lam, __int_as_float(clamp));
    st_s(S, kSlotLR + 2 * fi, dl);
    st_s(S, kSlotLR + 2 * fi + 1, dr);
}

// Reverse of one field: from (dlb, drb) to the cotangents of a..f, written
// over the field's forward slots as (a, b, c, d, e, f).
__device__ __forceinline__ void weno_rev_w(const float2 *kp, int64_t ne, dw a, dw b, dw c, dw d, dw e, dw f, dw dlb,
                                           dw drb, float2 *S, int fi) {
    const int w0 = kSlotW + 8 * fi;
    const dw va = ld_s(S, w0), vb = ld_s(S, w0 + 1), vc = ld_s(S, w0 + 2), vd = ld_s(S, w0 + 3);
    const dw Ba = ld_s(S, w0 + 4), Bb = ld_s(S, w0 + 5), Bc = ld_s(S, w0 + 6), Bd = ld_s(S, w0 + 7);
    const float2 sq = S[(kSlotS + fi) * kVjpBlock];
    const float lam = sq.x;
    const int clamp = __float_as_int(sq.y);
    const dw dl = ld_s(S, kSlotLR + 2 * fi), dr = ld_s(S, kSlotLR + 2 * fi + 1);
    const dw ra = recip(Ba), rb = recip(Bb), rc = recip(Bc), rd = recip(Bd);
    const dw l0 = mul(kc(kp, ne, 20), ra), l2 = mul(kc(kp, ne, 21), rc);
    const dw iSL = recip(add_sl(add_sl(l0, rb), l2));
    const dw oa = mul(l0, iSL), ob = mul(rb, iSL), oc = mul(l2, iSL);
    const dw r0 = mul(kc(kp, ne, 22), rd), r2 = mul(kc(kp, ne, 23), rb);
    const dw iSR = recip(add_sl(add_sl(r0, rc), r2));
    const dw pd = mul(r0, iSR), pc = mul(rc, iSR), pb = mul(r2, iSR);
    const dw vcr = sub_sl(vc, c), vbr = sub_sl(vb, c);
    const dw vab = mul(dlb, oa);
    const dw vbb = mulsum(dlb, ob, drb, pb);
    const dw vcb = mulsum(dlb, oc, drb, pc);
    const dw vdb = mul(drb, pd);
    const dw cdir = neg(mul(drb, add_sl(pc, pb)));
    // cotangents of the scaled indicators: -omega_k (v_k - d) / B'_k per side
    auto bbar = [&](dw g, dw o, dw v, dw dd, dw rB) { return neg(mul(mul(g, o), mul(sub_sl(v, dd), rB))); };
    const dw z = dw_make(0.0f);
    const dw Bab = (clamp & 1) ? z : bbar(dlb, oa, va, dl, ra);
    const dw Bbb = (clamp & 2) ? z : add_sl(bbar(dlb, ob, vb, dl, rb), bbar(drb, pb, vbr, dr, rb));
    const dw Bcb = (clamp & 4) ? z : add_sl(bbar(dlb, oc, vc, dl, rc), bbar(drb, pc, vcr, dr, rc));
    const dw Bdb = (clamp & 8) ? z : bbar(drb, pd, vd, dr, rd);
    // d beta'/dx = lambda (2 m0 x' + m1 y'), x' = lambda x
    const dw as = scale(a, lam), bs = scale(b, lam), cs = scale(c, lam), ds = scale(d, lam), es = scale(e, lam),
             fs = scale(f, lam);
    auto g1 = [&](dw B, int i0, int i1, dw x, dw y) {  // B lambda (2 k[i0] x + k[i1] y)
        return scale(mul(B, add_sl(scale(mul_u(kc(kp, ne, i0), x), 2.0f), mul_u(kc(kp, ne, i1), y))), lam);
    };
    auto g2 = [&](dw B, int i1, int i2, dw x, dw y) {  // B lambda (k[i1] x + 2 k[i2] y)
        return scale(mul(B, add_sl(mul_u(kc(kp, ne, i1), x), scale(mul_u(kc(kp, ne, i2), y), 2.0f))), lam);
    };
    const dw ab = add_sl(mul(kc(kp, ne, 0), vab), g1(Bab, 2, 3, as, bs));
    const dw bb = add_sl(add_sl(mul(kc(kp, ne, 1), vab), g2(Bab, 3, 4, as, bs)),
                         add_sl(mul(kc(kp, ne, 5), vbb), g1(Bbb, 7, 8, bs, cs)));
    const dw cb = add_sl(add_sl(cdir, add_sl(mul(kc(kp, ne, 6), vbb), g2(Bbb, 8, 9, bs, cs))),
                         add_sl(mul(kc(kp, ne, 10), vcb), g1(Bcb, 12, 13, cs, ds)));
    const dw db = add_sl(mul(kc(kp, ne, 11), vcb), g2(Bcb, 13, 14, cs, ds));
    const dw eb = add_sl(mul(kc(kp, ne, 15), vdb), g1(Bdb, 17, 18, es, fs));
    const dw fb = add_sl(mul(kc(kp, ne, 16), vdb), g2(Bdb, 18, 19, es, fs));
    st_s(S, w0 + 0, ab);
    st_s(S, w0 + 1, bb);
    st_s(S, w0 + 2, cb);
    st_s(S, w0 + 3, db);
    st_s(S, w0 + 4, eb);
    st_s(S, w0 + 5, fb);
}

__device__ __forceinline__ dw comp(const dw4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

__global__ void __launch_bounds__(kVjpBlock, 6) edge_flux_vjp_dw_kernel(AdjEdgeArgs A) {  // 168 registers, 12 warps per SM
    __shared__ float2 stage[kVjpSlots * kVjpBlock];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= A.ne) return;
    float2 *S = stage + threadIdx.x;
    const double *__restrict__ w = A.w;
    const int64_t ne = A.ne;
    const float2 *kp = A.coefdw + e;
    const dw gm1 = dw_make(A.dw_gm1[0], A.dw_gm1[1]);
    const dw eps_m = dw_make(A.dw_eps[0], A.dw_eps[1]);
    int32_t s[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = __ldg(A.sten + (int64_t)i * ne + e);
    const dw nx = kc(kp, ne, kCoefN), ny = kc(kp, ne, kCoefN + 1);

    // ---------------- forward
    const dw4 L1 = d2dw4(ldd4(w, s[2])), R1 = d2dw4(ldd4(w, s[3]));
    // difference j (R1-L1, L2-L1, L3-L1, R2-R1, R3-R1) in FP64, then double
    // words; taken again in the reverse sweep instead of being kept
    auto diff_j = [&](int j) {
        const int32_t p = j == 0 ? s[3] : j == 1 ? s[1] : j == 2 ? s[0] : j == 3 ? s[4] : s[5];
        const int32_t q = j == 0 || j == 1 || j == 2 ? s[2] : s[3];
        const d4v a = ldd4(w, p), b = ldd4(w, q);
        return d2dw4(d4v{a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w});
    };
    const PrimW pL1 = prim_w(L1, gm1), pR1 = prim_w(R1, gm1);
    const RoeW C = roe_w(L1, pL1, R1, pR1, nx, ny, gm1);
#pragma unroll 1
    for (int j = 0; j < 5; ++j) st_s4(S, kSlotC + 4 * j, project(C, diff_j(j)));
    // fields: a = L3-L1, b = L2-L1, c = R1-L1, d = R2-L1, e = R3-R1, f = R2-R1 (characteristic)
#pragma unroll 1
    for (int i = 0; i < 4; ++i) {
        const dw c = ld_s(S, kSlotC + i), f = ld_s(S, kSlotC + 12 + i);
        weno_fwd_w(kp, ne, ld_s(S, kSlotC + 8 + i), ld_s(S, kSlotC + 4 + i), c, add_sl(f, c), ld_s(S, kSlotC + 16 + i), f,
                   eps_m, A.dw_eps_e, S, i);
    }
    dw4 dl, dr;
    dl = d4(ld_s(S, kSlotLR), ld_s(S, kSlotLR + 2), ld_s(S, kSlotLR + 4), ld_s(S, kSlotLR + 6));
    dr = d4(ld_s(S, kSlotLR + 1), ld_s(S, kSlotLR + 3), ld_s(S, kSlotLR + 5), ld_s(S, kSlotLR + 7));
    dw4 wl = add4_sl(L1, unproject(C, dl));
    dw4 wr = add4_sl(R1, unproject(C, dr));
    PrimW pl, pr;
    bool ok = wl.x.h > 0.0f && wr.x.h > 0.0f;
    if (ok) {
        pl = prim_w(wl, gm1);
        pr = prim_w(wr, gm1);
        ok = pl.p.h > 0.0f && pr.p.h > 0.0f;
    }
    if (!ok) {
        wl = L1;
        wr = R1;
        pl = pL1;
        pr = pR1;
    }
    const RoeW Q = roe_w(wl, pl, wr, pr, nx, ny, gm1);
    const dw4 dwv = sub4_sl(wr, wl);
    const dw4 a = project(Q, dwv);
    const dw delta = mul(Q.c, dw_make(A.dw_tenth[0], A.dw_tenth[1]));
    const dw h2d = mul(Q.ic, 5.0f);
    const dw l_u = Q.qn, l_m = sub_sl(Q.qn, Q.c), l_p = add_sl(Q.qn, Q.c);
    auto inband = [&](dw l) {
        const dw m = dabs(l);
        return m.h < delta.h || (m.h == delta.h && m.l < delta.l);
    };
    auto fixv = [&](dw l) { return inband(l) ? mul(add_sl(mul_u(l, l), mul_u(delta, delta)), h2d) : dabs(l); };
    const dw lu = fixv(l_u), lm = fixv(l_m), lp = fixv(l_p);
    const dw4 sv = d4(mul(lm, a.x), mul(lu, a.y), mul(lu, a.z), mul(lp, a.w));

    // ---------------- reverse
    const d4v lam64 = ldd4(A.lam_r, e);
    const dw4 lam = d2dw4(lam64);
    const dw4 Db = d4(scale(lam.x, -0.5f), scale(lam.y, -0.5f), scale(lam.z, -0.5f), scale(lam.w, -0.5f));
    const dw4 Fb = d4(scale(lam.x, 0.5f), scale(lam.y, 0.5f), scale(lam.z, 0.5f), scale(lam.w, 0.5f));
    dw4 wlb = zero4(), wrb = zero4();
    PrimWBar plb, prb;
    fluxn_vjp_w(wl, pl, nx, ny, Fb, wlb, plb);
    fluxn_vjp_w(wr, pr, nx, ny, Fb, wrb, prb);
    RoeWBar Qb;
    dw4 svb = zero4();
    unproject_vjp_w(Q, sv, Db, svb, Qb);
    const dw4 ab = d4(mul(lm, svb.x), mul(lu, svb.y), mul(lu, svb.z), mul(lp, svb.w));
    const dw lmb = mul(a.x, svb.x), lub = mulsum(a.y, svb.y, a.z, svb.z), lpb = mul(a.w, svb.w);
    // entropy fix: |l| or (l^2 + delta^2) / (2 delta), delta = 0.1 c
    dw deltab = dw_make(0.0f);
    const dw idelta = recip(delta);
    auto fix_vjp = [&](dw l, dw fb, dw &lb) {
        if (inband(l)) {
            acc(lb, mul(fb, mul(l, idelta)));
            const dw q = mul(l, idelta);
            acc(deltab, scale(mul(fb, sub_sl(dw_make(1.0f), mul_u(q, q))), 0.5f));
        } else {
            acc(lb, l.h >= 0.0f ? fb : neg(fb));
        }
    };
    dw lub_ = dw_make(0.0f), lmb_ = lub_, lpb_ = lub_;
    fix_vjp(l_u, lub, lub_);
    fix_vjp(l_m, lmb, lmb_);
    fix_vjp(l_p, lpb, lpb_);
    acc(Qb.qn, add_sl(add_sl(lub_, lmb_), lpb_));
    acc(Qb.c, add_sl(sub_sl(lpb_, lmb_), mul(deltab, dw_make(A.dw_tenth[0], A.dw_tenth[1]))));
    dw4 dwb = zero4();
    project_vjp_w(Q, dwv, ab, dwb, Qb);
    acc4(wrb, dwb);
    wlb = sub4_sl(wlb, dwb);
    roe_vjp_w(wl, pl, wr, pr, Q, Qb, gm1, wlb, plb, wrb, prb);
    prim_vjp_w(wl, pl, plb, gm1, wlb);
    prim_vjp_w(wr, pr, prb, gm1, wrb);

    dw4 G0 = zero4(), G1 = zero4(), GL1 = wlb, GR1 = wrb, G4 = zero4(), G5 = zero4();
    if (ok) {
        RoeWBar Cb;
        dw4 dlb = zero4(), drb = zero4();
        unproject_vjp_w(C, dl, wlb, dlb, Cb);
        unproject_vjp_w(C, dr, wrb, drb, Cb);
#pragma unroll 1
        for (int i = 0; i < 4; ++i) {
            const dw c = ld_s(S, kSlotC + i), f = ld_s(S, kSlotC + 12 + i);
            weno_rev_w(kp, ne, ld_s(S, kSlotC + 8 + i), ld_s(S, kSlotC + 4 + i), c, add_sl(f, c),
                       ld_s(S, kSlotC + 16 + i), f, comp(dlb, i), comp(drb, i), S, i);
        }
        // cotangent of each difference's projection, gathered from the four
        // fields' slots (a, b, c, d, e, f) = (L3, L2, M, R2L, R3, R2); d = R2L
        // feeds both M and R2
#pragma unroll 1
        for (int j = 0; j < 5; ++j) {
            dw cbv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int w0 = kSlotW + 8 * i;
                dw v;
                if (j == 0) v = add_sl(ld_s(S, w0 + 2), ld_s(S, w0 + 3));       // M
                else if (j == 1) v = ld_s(S, w0 + 1);                           // L2
                else if (j == 2) v = ld_s(S, w0 + 0);                           // L3
                else if (j == 3) v = add_sl(ld_s(S, w0 + 5), ld_s(S, w0 + 3));  // R2
                else v = ld_s(S, w0 + 4);                                       // R3
                cbv[i] = v;
            }
            dw4 db = zero4();
            project_vjp_w(C, diff_j(j), d4(cbv[0], cbv[1], cbv[2], cbv[3]), db, Cb);
            if (j == 0) {
                acc4(GR1, db);
                GL1 = sub4_sl(GL1, db);
            } else if (j == 1) {
                acc4(G1, db);
                GL1 = sub4_sl(GL1, db);
            } else if (j == 2) {
                acc4(G0, db);
                GL1 = sub4_sl(GL1, db);
            } else if (j == 3) {
                acc4(G4, db);
                GR1 = sub4_sl(GR1, db);
            } else {
                acc4(G5, db);
                GR1 = sub4_sl(GR1, db);
            }
        }
        PrimWBar pL1b, pR1b;
        roe_vjp_w(L1, pL1, R1, pR1, C, Cb, gm1, GL1, pL1b, GR1, pR1b);
        prim_vjp_w(L1, pL1, pL1b, gm1, GL1);
        prim_vjp_w(R1, pR1, pR1b, gm1, GR1);
    }
    double *G = A.G;  // [6][ne][4]
    auto put = [&](int slot, const dw4 &g) {
        double2 *q = reinterpret_cast<double2 *>(G + 4 * ((int64_t)slot * ne + e));
        q[0] = make_double2(to64(g.x), to64(g.y));
        q[1] = make_double2(to64(g.z), to64(g.w));
    };
    put(0, G0);
    put(1, G1);
    put(2, GL1);
    put(3, GR1);
    put(4, G4);
    put(5, G5);
}

}  // namespace

void launch_edge_flux_vjp_dw(const AdjEdgeArgs &a, cudaStream_t s) {
    if (a.ne > 0)
        edge_flux_vjp_dw_kernel<<<(unsigned)((a.ne + kVjpBlock - 1) / kVjpBlock), kVjpBlock, 0, s>>>(a);
}

}  // namespace fdu
