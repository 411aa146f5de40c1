// Argument blocks and launchers of the adjoint kernels (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fdu {

// Edge-flux VJP inputs (internal ids, active edges, FP64).
struct AdjEdgeArgs {
    const int32_t *sten;  // [6][ne]
    const double *coef;   // [kEdgeCoef][ne]
    const double *w;      // [nv][4] state the residual is linearised at
    const double *lam_r;  // [ne][4] cotangent of the edge fluxes (read by the VJP kernel)
    double *lam_r_mut;    // the same buffer, written by the transpose gather
    double *G;            // [6][ne][4] cotangents of the stencil states, per slot, then one zero record
    int64_t ne;
    double gm1, eps;
    // precision 48 (double-word edge VJP, fdu_adjoint_dw.cu)
    int prec;              // 64 or 48
    const float2 *coefdw;  // [kEdgeCoef][ne] double-word coefficient block
    float dw_gm1[2], dw_tenth[2], dw_eps[2];
    int dw_eps_e;          // WENO epsilon = dw_eps * 2^dw_eps_e
};

// Edge transpose: for each active edge, the vertices whose divergence
// stencil holds it and the weights w_k, in SELL-32 form over the threads:
// thread i serves edge eperm[i], its entry j sits at eoff[i / 32] + 32 j +
// i % 32, and a slice's lists are padded to its longest with weight 0.
struct AdjTables {
    const int64_t *eoff;  // [ceil(ne / 32) + 1] slice offsets
    const int32_t *evid;
    const double *ewt;    // -w_k: the residual's minus sign carried by the weights
    const int32_t *eperm; // [ne] edge of each thread (list-length order inside windows of 256)
};

// Per-vertex part: vertex transpose (wf, wg of every stencil that holds the
// vertex, centre weights as the vertex's own entry) and stencil incidence,
// both in SELL-32 form over the threads like AdjTables (padding: weight 0 on
// the vertex itself; slot 6 ne, the zero record of G).
struct AdjVertexArgs {
    int64_t nv;
    const int64_t *voff;  // [ceil(nv / 32) + 1] slice offsets
    const int32_t *vid;
    const double *wf, *wg;  // -wf, -wg (and minus the centre weights at v = j)
    const double *lam;    // [nv][4] cotangent of the residual
    const double *w;      // [nv][4] state
    double gm1;
    const int64_t *soff;  // [ceil(nv / 32) + 1] slice offsets of the stencil incidence
    const int64_t *slot;  // index slot * ne + k into G
    const double *G;
    double *grad;         // [nv][4] output
    const int32_t *perm;  // [nv] vertex of each thread (list-length order inside windows of 256)
};

// The double-word edge-flux VJP (precision 48) of the same edge flux.
void launch_edge_flux_vjp_dw(const AdjEdgeArgs &a, cudaStream_t s);
// grad = (dL/dw)^T lam at state w: transpose gathers, edge-flux VJP (FP64, or
// double words when ea.prec == 48), per-vertex flux Jacobians; three launches on s.
void launch_residual_vjp(const AdjEdgeArgs &ea, const AdjTables &t, const AdjVertexArgs &va, cudaStream_t s);
// x <- (transmissive ghost fill)^T x: donor[i] += sum of x over its ghosts
// ghost[off[i] .. off[i+1]-1], which are then zeroed (nd donors, internal ids)
void launch_ghost_fold(double *x, const int32_t *donor, const int64_t *off, const int32_t *ghost, int64_t nd,
                       cudaStream_t s);
// out = a x + b y + c z over n4 doubles (y, z may be null)
void launch_axpby(double *out, double a, const double *x, double b, const double *y, double c, const double *z,
                  int64_t n4, cudaStream_t s);

}  // namespace fdu
