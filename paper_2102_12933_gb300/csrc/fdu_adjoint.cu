// Hand-written adjoint (vector-Jacobian products) of the FP64 residual.
//
// The residual of vertex v is L_v = -( sum_j wf_vj f(w_j) + wg_vj g(w_j)
// + sum_k we_vk r_k + cf_v f(w_v) + cg_v g(w_v) ) (Section 2.2.1, folded
// centre weights), with r_k the edge flux of Section 2.3.1.  Given a
// cotangent lam of L, its VJP is assembled from
//   lam_r[k]   = -sum_v we_vk lam_v                 (edge transpose)
//   lam_f[j]   = -sum_v wf_vj lam_v - cf_j lam_j     (vertex transpose)
//   grad[j]    = (df/dw)^T lam_f[j] + (dg/dw)^T lam_g[j]
//   G[k][slot] = (dr_k/dW_slot)^T lam_r[k]          (edge-flux VJP, recomputing
//                                                    the forward per edge)
//   grad[u]   += sum over (k, slot) with sten[slot][k] = u of G[k][slot]
// All sums are gathers over transposed tables: no atomics, deterministic.
// The piecewise choices of the forward pass (positivity fallback, entropy
// fix band, |lambda|) take the same branch in the reverse pass.
#include <cuda_runtime.h>

#include <cstdint>

#include "fdu_adjoint.cuh"
#include "fdu_device.cuh"
#include "fdu_internal.h"
#include "fdu_kernels.cuh"

namespace fdu {
namespace {
using namespace dev;

// Cotangent accumulators start at -0.0, the additive identity of IEEE
// arithmetic (-0 + x = x for every x, while +0 + -0 = +0), so the compiler
// drops the first addition into each instead of issuing it on the FP64 pipe.
constexpr double kNZ = -0.0;
__device__ __forceinline__ dbl4 nz4() { return dbl4_make(kNZ, kNZ, kNZ, kNZ); }

struct Prim64Bar {
    double r = kNZ, ir = kNZ, p = kNZ;
};
// Cotangents of a Roe64.  The projections' parts through b1h and ich are
// kept as the raw sums sphi = sum phh_bar (c.x + c.w) and spsi = sum psh_bar
// (c.x - c.w) of the projected values c (c.x + c.w = 2 phh, c.x - c.w = 2 psh),
// which roe64_vjp turns into the cotangent of ic: with b1h = hgm1 ic^2 and
// ich = ic / 2, sum phh_bar phh / b1h * d b1h / d ic = c sphi and sum psh_bar
// psh / ich * d ich / d ic = c spsi / 2.
struct Roe64Bar {
    double u = kNZ, v = kNZ, H = kNZ, c = kNZ, qn = kNZ, qt = kNZ, hq2 = kNZ, sphi = kNZ, spsi = kNZ;
};

__device__ __forceinline__ void add_to(dbl4 &a, const dbl4 &b) {
    a.x += b.x;
    a.y += b.y;
    a.z += b.z;
    a.w += b.w;
}

// w -> (r = rho^-1/2, ir = 1/rho = r^2, p = (gamma - 1) E - (gamma - 1)/2 |m|^2 ir)
__device__ __forceinline__ void prim64_vjp(const dbl4 &w, const Prim64 &P, const Prim64Bar &B, double gm1, dbl4 &wb) {
    // the factors 1/2 and 2 are applied to the exponent field (half64, twice64)
    const double pg = B.p * gm1;
    const double irb = fma(-half64(pg), fma(w.y, w.y, w.z * w.z), B.ir);
    const double rb = fma(twice64(P.r), irb, B.r);
    wb.x = fma(rb, -(half64(P.ir) * P.r), wb.x);  // d r / d rho = -r^3 / 2
    const double t = pg * P.ir;
    wb.y = fma(-t, w.y, wb.y);
    wb.z = fma(-t, w.z, wb.z);
    wb.w += pg;
}

// Roe average (a, b) -> R of roe64 (b1h = hgm1 ic^2, ich = ic / 2, c = c2 ic
// with ic = c2^-1/2); accumulates into the primitives' cotangents and the
// states' direct cotangents.  R.u = U inv, R.v = V inv, R.H = Hn inv with
// inv = 1 / (sa + sb), so the cotangent of inv, ub U + vb V + Hb Hn, times
// -inv^2 is -(ub u + vb v + Hb H) inv: the sums U, V, Hn and the reciprocal
// are not formed again.
__device__ __forceinline__ void roe64_vjp(const dbl4 &a, const Prim64 &pa, const dbl4 &b, const Prim64 &pb,
                                          const Roe64 &R, const Roe64Bar &Rb, double gm1, dbl4 &ab, Prim64Bar &pab,
                                          dbl4 &bb, Prim64Bar &pbb) {
    double ub = Rb.u + Rb.qn * R.nx - Rb.qt * R.ny;
    double vb = Rb.v + Rb.qn * R.ny + Rb.qt * R.nx;
    const double icb = R.c * fma(0.5, Rb.spsi, Rb.sphi);
    const double c2b = R.ich * fma(-icb, R.ic * R.ic, Rb.c);  // ich = ic / 2
    const double Hb = Rb.H + c2b * gm1;
    const double hq2b = Rb.hq2 - c2b * gm1;
    ub += hq2b * R.u;
    vb += hq2b * R.v;
    const double inv = R.inv;
    const double Ub = ub * inv, Vb = vb * inv, Hnb = Hb * inv;
    const double sbar = -(ub * R.u + vb * R.v + Hb * R.H) * inv;
    ab.x += sbar * pa.r;
    bb.x += sbar * pb.r;
    ab.y += Ub * pa.r;
    bb.y += Ub * pb.r;
    ab.z += Vb * pa.r;
    bb.z += Vb * pb.r;
    ab.w += Hnb * pa.r;
    pab.p += Hnb * pa.r;
    bb.w += Hnb * pb.r;
    pbb.p += Hnb * pb.r;
    pab.r += sbar * a.x + Ub * a.y + Vb * a.z + Hnb * (a.w + pa.p);
    pbb.r += sbar * b.x + Ub * b.y + Vb * b.z + Hnb * (b.w + pb.p);
}

// c = project64(R, d) = (phh + psh, d.x - 2 phh, nx d.z - ny d.y - qt d.x,
// phh - psh) with phh = b1h (hq2 d.x - u d.y - v d.z + d.w) and psh = ich
// (qn d.x - nx d.y - ny d.z): accumulates d's and R's cotangents, given the
// forward's c (for the parts through b1h and ich, Roe64Bar)
__device__ __forceinline__ void project64_vjp(const Roe64 &R, const dbl4 &d, const dbl4 &c, const dbl4 &cb, dbl4 &db,
                                              Roe64Bar &Rb) {
    const double phhb = fma(-2.0, cb.y, cb.x + cb.w);
    const double pshb = cb.x - cb.w;
    db.x += cb.y - R.qt * cb.z;
    db.y += -R.ny * cb.z;
    db.z += R.nx * cb.z;
    Rb.qt += -d.x * cb.z;
    Rb.sphi = fma(phhb, c.x + c.w, Rb.sphi);
    const double t = phhb * R.b1h;
    Rb.hq2 += t * d.x;
    Rb.u += -t * d.y;
    Rb.v += -t * d.z;
    db.x += t * R.hq2;
    db.y += -t * R.u;
    db.z += -t * R.v;
    db.w += t;
    Rb.spsi = fma(pshb, c.x - c.w, Rb.spsi);
    const double u = pshb * R.ich;
    Rb.qn += u * d.x;
    db.x += u * R.qn;
    db.y += -u * R.nx;
    db.z += -u * R.ny;
}

// d = unproject64(R, c): accumulates c's and R's cotangents
__device__ __forceinline__ void unproject64_vjp(const Roe64 &R, const dbl4 &c, const dbl4 &dbar, dbl4 &cb,
                                                Roe64Bar &Rb) {
    const double rho = c.x + c.y + c.w;
    const double dd = R.c * (c.w - c.x);
    const double rhob = dbar.x + R.u * dbar.y + R.v * dbar.z;
    const double ddb = R.nx * dbar.y + R.ny * dbar.z + R.qn * dbar.w;
    Rb.u += rho * dbar.y;
    Rb.v += rho * dbar.z;
    Rb.H += (c.x + c.w) * dbar.w;
    Rb.hq2 += c.y * dbar.w;
    Rb.qn += dd * dbar.w;
    Rb.qt += c.z * dbar.w;
    Rb.c += (c.w - c.x) * ddb;
    cb.x += rhob + R.H * dbar.w - R.c * ddb;
    cb.y += rhob + R.hq2 * dbar.w;
    cb.z += -R.ny * dbar.y + R.nx * dbar.z + R.qt * dbar.w;
    cb.w += rhob + R.H * dbar.w + R.c * ddb;
}

// weno_field64 (the same arithmetic) with the inner Horner terms of the four
// indicators: h_a = m0 a + m1 b of S_a and likewise h_b, h_c (of d and c),
// h_d; the reverse sweep takes the indicators' slopes as h + m0 x.
struct WenoHorner {
    double ha, hb, hc, hd;
};
__device__ __forceinline__ WenoField weno_field64_h(const double *k, double a, double b, double c, double d, double e,
                                                   double f, double eps, WenoHorner &H) {
    WenoField W;
    const double b2 = b * b, c2 = c * c;
    W.va = fma(k[0], a, k[1] * b);
    W.vb = fma(k[5], b, k[6] * c);
    W.vc = fma(k[10], c, k[11] * d);
    W.vd = fma(k[15], e, k[16] * f);
    H.ha = fma(k[2], a, k[3] * b);
    H.hb = fma(k[7], b, k[8] * c);
    H.hc = fma(k[14], d, k[13] * c);
    H.hd = fma(k[17], e, k[18] * f);
    W.ba = fma(a, H.ha, fma(k[4], b2, eps));
    W.bb = fma(b, H.hb, fma(k[9], c2, eps));
    W.bc = fma(d, H.hc, fma(k[12], c2, eps));
    W.bd = fma(e, H.hd, fma(k[19], f * f, eps));
    return W;
}

// The R1-based combination of one field's values and indicators (the form
// the reverse sweep differentiates; dl, dr as weno_combine64), keeping the
// products and reciprocals the reverse sweep needs.
struct WenoKeep {
    double l0, l1, l2, iDL, dl, r0, r1, r2, iDR, dr, vcr, vbr;  // vcr = vc - c, vbr = vb - c
};
__device__ __forceinline__ void weno_combine64_keep(const double *k, const WenoField &W, double c, WenoKeep &K) {
    const double bbc = W.bb * W.bc;
    K.l0 = k[20] * bbc;
    K.l1 = W.ba * W.bc;
    K.l2 = k[21] * (W.ba * W.bb);
    K.iDL = recip64_fast(K.l0 + K.l1 + K.l2);
    K.dl = fma(K.l0, W.va, fma(K.l1, W.vb, K.l2 * W.vc)) * K.iDL;
    K.r0 = k[22] * bbc;
    K.r1 = W.bd * W.bb;
    K.r2 = k[23] * (W.bd * W.bc);
    K.iDR = recip64_fast(K.r0 + K.r1 + K.r2);
    K.vcr = W.vc - c;
    K.vbr = W.vb - c;
    K.dr = fma(K.r0, W.vd, fma(K.r1, K.vcr, K.r2 * K.vbr)) * K.iDR;
}

// Reverse of the combination for one field: from (dlb, drb) to the
// cotangents of the six differences (a..f), given the field's values and
// indicators W and the kept products K of the forward pass.
__device__ __forceinline__ void weno_pair64_vjp(const double *k, const WenoField &W, const WenoKeep &K,
                                                const WenoHorner &H, double a, double b, double c, double d, double e,
                                                double f, double dlb, double drb, double &ab, double &bb_, double &cb,
                                                double &db, double &eb, double &fb) {
    const double C0 = k[20], C2 = k[21], D0 = k[22], D2 = k[23];  // C_1 = 1 on both sides
    const double vcr = K.vcr, vbr = K.vbr;
    const double NLb = dlb * K.iDL, DLb = -NLb * K.dl;
    const double NRb = drb * K.iDR, DRb = -NRb * K.dr;
    const double l0b = NLb * W.va + DLb, l1b = NLb * W.vb + DLb, l2b = NLb * W.vc + DLb;
    const double r0b = NRb * W.vd + DRb, r1b = NRb * vcr + DRb, r2b = NRb * vbr + DRb;
    const double vab = NLb * K.l0;
    const double vbb = NLb * K.l1 + NRb * K.r2;
    const double vcb = NLb * K.l2 + NRb * K.r1;
    const double vdb = NRb * K.r0;
    const double cdir = -NRb * (K.r1 + K.r2);
    // l0 = C0 bb bc, l1 = ba bc, l2 = C2 ba bb; r0 = D0 bb bc, r1 = bd bb, r2 = D2 bd bc
    const double t0 = l0b * C0, t2 = l2b * C2, u0 = r0b * D0, u2 = r2b * D2;
    const double bab = fma(l1b, W.bc, t2 * W.bb);
    const double bbb = fma(t0, W.bc, fma(t2, W.ba, fma(u0, W.bc, r1b * W.bd)));
    const double bcb = fma(t0, W.bb, fma(l1b, W.ba, fma(u0, W.bb, u2 * W.bd)));
    const double bdb = fma(r1b, W.bb, u2 * W.bc);
    // beta = m0 x^2 + m1 x y + m2 y^2: d/dx = 2 m0 x + m1 y = h + m0 x with the
    // forward's h = m0 x + m1 y, d/dy = m1 x + 2 m2 y
    ab = k[0] * vab + bab * fma(k[2], a, H.ha);
    bb_ = k[1] * vab + bab * (k[3] * a + 2.0 * k[4] * b) + k[5] * vbb + bbb * fma(k[7], b, H.hb);
    cb = cdir + k[6] * vbb + bbb * (k[8] * b + 2.0 * k[9] * c) + k[10] * vcb + bcb * (2.0 * k[12] * c + k[13] * d);
    db = k[11] * vcb + bcb * fma(k[14], d, H.hc);
    eb = k[15] * vdb + bdb * fma(k[17], e, H.hd);
    fb = k[16] * vdb + bdb * (k[18] * e + 2.0 * k[19] * f);
}

// F_n(w) = (rho q, m_x q + p n_x, m_y q + p n_y, (E + p) q), q = m.n / rho,
// written with the primitives of prim64; reverse into w and P.
__device__ __forceinline__ void fluxn_vjp(const dbl4 &w, const Prim64 &P, double nx, double ny, const dbl4 &fb, dbl4 &wb,
                                          Prim64Bar &Pb) {
    const double mn = w.y * nx + w.z * ny;
    const double q = mn * P.ir;
    // f.x = rho q = mn (rho * ir = 1 in exact arithmetic; the forward uses rho * q)
    double qb = fb.x * w.x + fb.y * w.y + fb.z * w.z + fb.w * (w.w + P.p);
    wb.x += fb.x * q;
    wb.y += fb.y * q;
    wb.z += fb.z * q;
    wb.w += fb.w * q;
    Pb.p += fb.y * nx + fb.z * ny + fb.w * q;
    const double mnb = qb * P.ir;
    Pb.ir += qb * mn;
    wb.y += mnb * nx;
    wb.z += mnb * ny;
}

// (df/dw)^T fb + (dg/dw)^T gb at state w
__device__ __forceinline__ dbl4 vertex_flux_vjp(const dbl4 &w, double gm1, const dbl4 &fb, const dbl4 &gb) {
    const double ir = recip64(w.x);  // within 2 ulp of 1 / rho, without the FP64 division sequence
    const double u = w.y * ir, v = w.z * ir;
    const double p = gm1 * (w.w - half64(w.y * u + w.z * v));
    dbl4 wb = nz4();
    double ub = kNZ, vb = kNZ, pb = kNZ;
    // f = (m_x, m_x u + p, m_y u, (E + p) u)
    wb.y += fb.x + fb.y * u;
    ub += fb.y * w.y + fb.z * w.z + fb.w * (w.w + p);
    pb += fb.y + fb.w * u;
    wb.z += fb.z * u;
    wb.w += fb.w * u;
    // g = (m_y, m_x v, m_y v + p, (E + p) v)
    wb.z += gb.x + gb.z * v;
    wb.y += gb.y * v;
    vb += gb.y * w.y + gb.z * w.z + gb.w * (w.w + p);
    pb += gb.z + gb.w * v;
    wb.w += gb.w * v;
    // p = gm1 (E - |m|^2 / (2 rho))
    wb.x += pb * gm1 * half64(u * u + v * v);
    wb.y += -pb * gm1 * u;
    wb.z += -pb * gm1 * v;
    wb.w += pb * gm1;
    // u = m_x / rho, v = m_y / rho
    wb.x += -(ub * u + vb * v) * ir;
    wb.y += ub * ir;
    wb.z += vb * ir;
    return wb;
}

// Edge-flux VJP: recompute edge e's forward pass at state w, then reverse
// from lam (cotangent of r_e) to the six stencil states; G[slot][e].  The
// flux is reversed in the one-sided Roe form F_n(w_L) + R diag(nu) L (w_R -
// w_L), nu = (lambda - |lambda|_fixed) / 2, which equals the symmetric form
// (F_L + F_R)/2 - R |Lambda|_fixed L (w_R - w_L)/2 by Roe's property, so only
// the left physical flux is differentiated.
constexpr int kVjpBlock = 64;
__global__ void __launch_bounds__(kVjpBlock) edge_flux_vjp_kernel(AdjEdgeArgs A) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= A.ne) return;
    const double *__restrict__ w = A.w;
    const double *__restrict__ coef = A.coef;
    const double gm1 = A.gm1, hgm1 = 0.5 * A.gm1;
    const int64_t ne = A.ne;
    int32_t s[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = __ldg(A.sten + (int64_t)i * ne + e);
    const dbl4 W0 = ld4v(w, s[0]), W1 = ld4v(w, s[1]), L1 = ld4v(w, s[2]), R1 = ld4v(w, s[3]), W4 = ld4v(w, s[4]),
               W5 = ld4v(w, s[5]);
    const double nx = __ldg(coef + (int64_t)kCoefN * ne + e), ny = __ldg(coef + (int64_t)(kCoefN + 1) * ne + e);
    const dbl4 lam = ld4v(A.lam_r, e);

    // ---------------- forward
    const Prim64 pL1 = prim64(L1, gm1), pR1 = prim64(R1, gm1);
    const Roe64 C = roe64(L1, pL1, R1, pR1, nx, ny, gm1, hgm1);
    const dbl4 dM = sub4(R1, L1), dL2 = sub4(W1, L1), dL3 = sub4(W0, L1), dR2 = sub4(W4, R1), dR3 = sub4(W5, R1);
    const dbl4 cM = project64(C, dM), cL2 = project64(C, dL2), cL3 = project64(C, dL3), cR2 = project64(C, dR2),
               cR3 = project64(C, dR3);
    const dbl4 cR2L = add4(cR2, cM);
    double k[kCoefN];
#pragma unroll
    for (int i = 0; i < kCoefN; ++i) k[i] = __ldg(coef + (int64_t)i * ne + e);
    // each field's sub-stencil values and indicators and the combination's
    // products, kept in shared memory (thread-private column) for the
    // reverse sweep
    __shared__ double wsm[4 * 22][kVjpBlock];
    const int t = threadIdx.x;
    auto keep = [&](int fi, const WenoField &W, const WenoKeep &K, const WenoHorner &H) {
        double *q = &wsm[fi * 22][t];
        const double v[22] = {W.va, W.vb, W.vc, W.vd, W.ba, W.bb, W.bc, W.bd, K.l0, K.l1, K.l2,
                              K.iDL, K.vcr, K.r0, K.r1, K.r2, K.iDR, K.vbr, H.ha, H.hb, H.hc, H.hd};
#pragma unroll
        for (int i = 0; i < 22; ++i) q[i * kVjpBlock] = v[i];
    };
    // dl, dr of the field stay in registers (the dbl4 dl, dr below)
    auto kept = [&](int fi, double dlf, double drf, WenoField &W, WenoKeep &K, WenoHorner &H) {
        const double *q = &wsm[fi * 22][t];
        W.va = q[0 * kVjpBlock]; W.vb = q[1 * kVjpBlock]; W.vc = q[2 * kVjpBlock]; W.vd = q[3 * kVjpBlock];
        W.ba = q[4 * kVjpBlock]; W.bb = q[5 * kVjpBlock]; W.bc = q[6 * kVjpBlock]; W.bd = q[7 * kVjpBlock];
        K.l0 = q[8 * kVjpBlock]; K.l1 = q[9 * kVjpBlock]; K.l2 = q[10 * kVjpBlock]; K.iDL = q[11 * kVjpBlock];
        K.vcr = q[12 * kVjpBlock]; K.r0 = q[13 * kVjpBlock]; K.r1 = q[14 * kVjpBlock]; K.r2 = q[15 * kVjpBlock];
        K.iDR = q[16 * kVjpBlock]; K.vbr = q[17 * kVjpBlock];
        K.dl = dlf;
        K.dr = drf;
        H.ha = q[18 * kVjpBlock]; H.hb = q[19 * kVjpBlock]; H.hc = q[20 * kVjpBlock]; H.hd = q[21 * kVjpBlock];
    };
    dbl4 dl, dr;
    {
        WenoKeep K;
        WenoHorner H;
        WenoField W = weno_field64_h(k, cL3.x, cL2.x, cM.x, cR2L.x, cR3.x, cR2.x, A.eps, H);
        weno_combine64_keep(k, W, cM.x, K);
        keep(0, W, K, H);
        dl.x = K.dl;
        dr.x = K.dr;
        W = weno_field64_h(k, cL3.y, cL2.y, cM.y, cR2L.y, cR3.y, cR2.y, A.eps, H);
        weno_combine64_keep(k, W, cM.y, K);
        keep(1, W, K, H);
        dl.y = K.dl;
        dr.y = K.dr;
        W = weno_field64_h(k, cL3.z, cL2.z, cM.z, cR2L.z, cR3.z, cR2.z, A.eps, H);
        weno_combine64_keep(k, W, cM.z, K);
        keep(2, W, K, H);
        dl.z = K.dl;
        dr.z = K.dr;
        W = weno_field64_h(k, cL3.w, cL2.w, cM.w, cR2L.w, cR3.w, cR2.w, A.eps, H);
        weno_combine64_keep(k, W, cM.w, K);
        keep(3, W, K, H);
        dl.w = K.dl;
        dr.w = K.dr;
    }
    dbl4 wl = unproject_add64(C, dl, L1);
    dbl4 wr = unproject_add64(C, dr, R1);
    Prim64 pl, pr;
    bool ok = pos64(wl.x) && pos64(wr.x);
    if (ok) {
        pl = prim64(wl, gm1);
        pr = prim64(wr, gm1);
        ok = pos64(pl.p) && pos64(pr.p);
    }
    if (!ok) {
        wl = L1;
        wr = R1;
        pl = pL1;
        pr = pR1;
    }
    const Roe64 Q = roe64(wl, pl, wr, pr, nx, ny, gm1, hgm1);
    const dbl4 dw = sub4(wr, wl);
    const dbl4 a = project64(Q, dw);
    // nu = (l - |l|_fixed) / 2: -(l - delta)^2 / (4 delta) inside Harten's
    // band |l| < delta = 0.1 c (decided on the integer pipe, as the forward
    // kernel does), min(l, 0) outside; with the derivatives d nu / d l and
    // d nu / d delta = (l^2 - delta^2) / (4 delta^2) (0 outside the band)
    const double delta = 0.1 * Q.c, h4d = 2.5 * Q.ic;  // 1 / (4 delta)
    const unsigned long long dbits = (unsigned long long)__double_as_longlong(delta);
    auto wave = [&](double l, double &nu, double &dnu_l, double &dnu_d) {
        const long long b = __double_as_longlong(l);
        const unsigned long long ab_ = (unsigned long long)b & 0x7FFFFFFFFFFFFFFFULL;
        if (ab_ < dbits) {
            const double sd = l - delta;
            nu = -(sd * sd) * h4d;
            dnu_l = -2.0 * sd * h4d;
            dnu_d = sd * (l + delta) * (10.0 * Q.ic) * h4d;
        } else {
            const bool neg = b < 0 || ab_ > 0x7FF0000000000000ULL;
            nu = neg ? l : 0.0;
            dnu_l = neg ? 1.0 : 0.0;
            dnu_d = 0.0;
        }
    };
    double nu_u, nu_m, nu_p, gu, gm, gp, hu, hm, hp;
    wave(Q.qn, nu_u, gu, hu);
    wave(Q.qn - Q.c, nu_m, gm, hm);
    wave(Q.qn + Q.c, nu_p, gp, hp);
    const dbl4 sv = dbl4_make(nu_m * a.x, nu_u * a.y, nu_u * a.z, nu_p * a.w);

    // ---------------- reverse
    dbl4 wlb = nz4(), wrb = nz4();
    Prim64Bar plb, prb;
    fluxn_vjp(wl, pl, nx, ny, lam, wlb, plb);
    Roe64Bar Qb;
    dbl4 svb = nz4();
    unproject64_vjp(Q, sv, lam, svb, Qb);
    const dbl4 ab = dbl4_make(nu_m * svb.x, nu_u * svb.y, nu_u * svb.z, nu_p * svb.w);
    const double nmb = a.x * svb.x, nub = a.y * svb.y + a.z * svb.z, npb = a.w * svb.w;
    const double lub = nub * gu, lmb = nmb * gm, lpb = npb * gp;
    const double deltab = nub * hu + nmb * hm + npb * hp;
    Qb.qn += lub + lmb + lpb;
    Qb.c += lpb - lmb + 0.1 * deltab;
    dbl4 dwb = nz4();
    project64_vjp(Q, dw, a, ab, dwb, Qb);
    add_to(wrb, dwb);
    wlb = sub4(wlb, dwb);
    roe64_vjp(wl, pl, wr, pr, Q, Qb, gm1, wlb, plb, wrb, prb);
    prim64_vjp(wl, pl, plb, gm1, wlb);
    prim64_vjp(wr, pr, prb, gm1, wrb);

    dbl4 G0 = nz4(), G1 = G0, GL1 = wlb, GR1 = wrb, G4 = G0, G5 = G0;
    if (ok) {
        Roe64Bar Cb;
        dbl4 dlb = nz4(), drb = nz4();
        unproject64_vjp(C, dl, wlb, dlb, Cb);
        unproject64_vjp(C, dr, wrb, drb, Cb);
        dbl4 cL3b, cL2b, cMb, cR2Lb, cR3b, cR2b;
        WenoField W;
        WenoKeep K;
        WenoHorner H;
        kept(0, dl.x, dr.x, W, K, H);
        weno_pair64_vjp(k, W, K, H, cL3.x, cL2.x, cM.x, cR2L.x, cR3.x, cR2.x, dlb.x, drb.x, cL3b.x, cL2b.x, cMb.x,
                        cR2Lb.x, cR3b.x, cR2b.x);
        kept(1, dl.y, dr.y, W, K, H);
        weno_pair64_vjp(k, W, K, H, cL3.y, cL2.y, cM.y, cR2L.y, cR3.y, cR2.y, dlb.y, drb.y, cL3b.y, cL2b.y, cMb.y,
                        cR2Lb.y, cR3b.y, cR2b.y);
        kept(2, dl.z, dr.z, W, K, H);
        weno_pair64_vjp(k, W, K, H, cL3.z, cL2.z, cM.z, cR2L.z, cR3.z, cR2.z, dlb.z, drb.z, cL3b.z, cL2b.z, cMb.z,
                        cR2Lb.z, cR3b.z, cR2b.z);
        kept(3, dl.w, dr.w, W, K, H);
        weno_pair64_vjp(k, W, K, H, cL3.w, cL2.w, cM.w, cR2L.w, cR3.w, cR2.w, dlb.w, drb.w, cL3b.w, cL2b.w, cMb.w,
                        cR2Lb.w, cR3b.w, cR2b.w);
        add_to(cR2b, cR2Lb);
        add_to(cMb, cR2Lb);
        dbl4 dMb = nz4(), dL2b = dMb, dL3b = dMb, dR2b = dMb, dR3b = dMb;
        project64_vjp(C, dM, cM, cMb, dMb, Cb);
        project64_vjp(C, dL2, cL2, cL2b, dL2b, Cb);
        project64_vjp(C, dL3, cL3, cL3b, dL3b, Cb);
        project64_vjp(C, dR2, cR2, cR2b, dR2b, Cb);
        project64_vjp(C, dR3, cR3, cR3b, dR3b, Cb);
        add_to(GR1, dMb);
        GL1 = sub4(GL1, dMb);
        add_to(G1, dL2b);
        GL1 = sub4(GL1, dL2b);
        add_to(G0, dL3b);
        GL1 = sub4(GL1, dL3b);
        add_to(G4, dR2b);
        GR1 = sub4(GR1, dR2b);
        add_to(G5, dR3b);
        GR1 = sub4(GR1, dR3b);
        Prim64Bar pL1b, pR1b;
        roe64_vjp(L1, pL1, R1, pR1, C, Cb, gm1, GL1, pL1b, GR1, pR1b);
        prim64_vjp(L1, pL1, pL1b, gm1, GL1);
        prim64_vjp(R1, pR1, pR1b, gm1, GR1);
    }
    double *G = A.G;  // [6][ne][4]
    st4(G, 0 * ne + e, G0);
    st4(G, 1 * ne + e, G1);
    st4(G, 2 * ne + e, GL1);
    st4(G, 3 * ne + e, GR1);
    st4(G, 4 * ne + e, G4);
    st4(G, 5 * ne + e, G5);
}

// lam_r[k] = -sum_v we_vk lam_v (the table holds -we).  Thread i serves edge
// perm[i]; its list is lane i % 32 of SELL-32 slice i / 32 (entry j at
// off[slice] + 32 j + lane, padding with weight 0).
__global__ void adj_edge_lambda_kernel(const int64_t *__restrict__ off, const int32_t *__restrict__ vid,
                                       const double *__restrict__ wt, const int32_t *__restrict__ perm,
                                       const double *__restrict__ lam, double *__restrict__ lam_r, int64_t ne) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ne) return;
    const int64_t k = __ldg(perm + i);
    const int64_t sl = i / kSell;
    dbl4 acc = dbl4_make(0, 0, 0, 0);
    const int64_t end = __ldg(off + sl + 1);
#pragma unroll 4
    for (int64_t p = __ldg(off + sl) + i % kSell; p < end; p += kSell) {
        const double a = __ldg(wt + p);
        const dbl4 l = ld4v(lam, __ldg(vid + p));
        acc.x = fma(a, l.x, acc.x);
        acc.y = fma(a, l.y, acc.y);
        acc.z = fma(a, l.z, acc.z);
        acc.w = fma(a, l.w, acc.w);
    }
    st4(lam_r, k, acc);
}

// grad[j] = (df/dw)^T lam_f + (dg/dw)^T lam_g with lam_f = -sum_v wf_vj lam_v
// (the table holds -wf, -wg; the centre weights are included as the entry
// v = j), then + sum of the edge-flux slot cotangents G[slot][k] over the
// stencil slots that hold j.  Thread i serves vertex perm[i]; both lists are
// SELL-32 like the edge transpose's (padding: weight 0 on j itself, and the
// zero record of G).
__global__ void adj_vertex_kernel(AdjVertexArgs A) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= A.nv) return;
    const int64_t j = __ldg(A.perm + i);
    const int64_t sl = i / kSell;
    const int lane = (int)(i % kSell);
    dbl4 lf = dbl4_make(0, 0, 0, 0), lg = lf;
    {
        const int64_t end = __ldg(A.voff + sl + 1);
#pragma unroll 4
        for (int64_t p = __ldg(A.voff + sl) + lane; p < end; p += kSell) {
            const double a = __ldg(A.wf + p), b = __ldg(A.wg + p);
            const dbl4 l = ld4v(A.lam, __ldg(A.vid + p));
            lf.x = fma(a, l.x, lf.x);
            lf.y = fma(a, l.y, lf.y);
            lf.z = fma(a, l.z, lf.z);
            lf.w = fma(a, l.w, lf.w);
            lg.x = fma(b, l.x, lg.x);
            lg.y = fma(b, l.y, lg.y);
            lg.z = fma(b, l.z, lg.z);
            lg.w = fma(b, l.w, lg.w);
        }
    }
    dbl4 g = vertex_flux_vjp(ld4v(A.w, j), A.gm1, lf, lg);
    {
        const int64_t end = __ldg(A.soff + sl + 1);
#pragma unroll 4
        for (int64_t p = __ldg(A.soff + sl) + lane; p < end; p += kSell) add_to(g, ld4v(A.G, __ldg(A.slot + p)));
    }
    st4(A.grad, j, g);
}

// out = a * x + b * y (+ c * z), elementwise over n records of 4
__global__ void axpby_kernel(double *__restrict__ out, double a, const double *__restrict__ x, double b,
                             const double *__restrict__ y, double c, const double *__restrict__ z, int64_t n4) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n4) return;
    double v = a * x[i];
    if (y) v = fma(b, y[i], v);
    if (z) v = fma(c, z[i], v);
    out[i] = v;
}

// Transpose of the transmissive ghost fill (ghost rows copy their donor's):
// each donor adds its ghosts' cotangents, in ascending ghost order, and the
// ghost rows become 0.  One thread per donor, so the sums are deterministic.
__global__ void ghost_fold_kernel(double *__restrict__ x, const int32_t *__restrict__ donor,
                                  const int64_t *__restrict__ off, const int32_t *__restrict__ ghost, int64_t nd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nd) return;
    const int64_t d = __ldg(donor + i);
    dbl4 acc = ld4(x, d);
    for (int64_t p = __ldg(off + i); p < __ldg(off + i + 1); ++p) {
        const int64_t g = __ldg(ghost + p);
        add_to(acc, ld4(x, g));
        st4(x, g, dbl4_make(0, 0, 0, 0));
    }
    st4(x, d, acc);
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

void launch_ghost_fold(double *x, const int32_t *donor, const int64_t *off, const int32_t *ghost, int64_t nd,
                       cudaStream_t s) {
    if (nd > 0) ghost_fold_kernel<<<nblk(nd, 128), 128, 0, s>>>(x, donor, off, ghost, nd);
}

void launch_residual_vjp(const AdjEdgeArgs &ea, const AdjTables &t, const AdjVertexArgs &va, cudaStream_t s) {
    if (ea.ne > 0) {
        adj_edge_lambda_kernel<<<nblk(ea.ne, 256), 256, 0, s>>>(t.eoff, t.evid, t.ewt, t.eperm, va.lam, ea.lam_r_mut,
                                                               ea.ne);
        if (ea.prec == 48) launch_edge_flux_vjp_dw(ea, s);
        else edge_flux_vjp_kernel<<<nblk(ea.ne, kVjpBlock), kVjpBlock, 0, s>>>(ea);
    }
    if (va.nv > 0) adj_vertex_kernel<<<nblk(va.nv, 256), 256, 0, s>>>(va);
}

void launch_axpby(double *out, double a, const double *x, double b, const double *y, double c, const double *z,
                  int64_t n4, cudaStream_t s) {
    if (n4 > 0) axpby_kernel<<<nblk(n4, 256), 256, 0, s>>>(out, a, x, b, y, c, z, n4);
}

}  // namespace fdu
