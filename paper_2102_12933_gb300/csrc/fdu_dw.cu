// Edge flux with FP64-level accuracy in double-word FP32 arithmetic.
//
// The same function as edge_flux_f64 (Section 2.3.1 and the Appendix:
// characteristic NU-WENO5 from both sides, Roe flux with Harten's entropy
// fix), arranged so that everything of the size of the state runs in FP64
// and everything of the size of an increment runs in double words (FP32
// pairs, about 48 significant bits), which GB300 executes on its FP32
// pipes at 64 times the FP64 instruction rate.
//
//   FP64 : the five stencil differences R1-L1, L2-L1, L3-L1, R2-R1, R3-R1
//          (exact or correctly rounded); the normal flux F_n(L1) of the
//          edge's left vertex, which the divergence adds through its folded
//          FP64 vertex weights (div_f64_body<MODE, true>).
//   DW   : characteristic projection at the Roe average of (L1, R1), the
//          WENO increments, the flux increment F_n(w_L) - F_n(L1) in a
//          cancellation-free form, and the Roe dissipation
//          D = R diag((lambda - |lambda|_fix)/2) L (w_R - w_L); the kernel
//          writes r - F_n(L1) = [F_n(w_L) - F_n(L1)] + D as double words.
// An error of relative size 2^-46 in an increment of size h |grad w| gives
// an error of that size times h in the flux, which the least-squares
// divergence (weights of size 1/h) does not amplify beyond the FP64 path's
// own rounding.  The NU-WENO5 and edge-flux bodies are in fdu_dw_edge.cuh
// (shared with the batched persistent stage).
//
// FP32 has a narrower exponent range than FP64.  The smoothness indicators
// are formed from the differences of each field scaled by a power of two
// (max |difference| in [1/2, 1)), with epsilon scaled by its square, so the
// nonlinear weights (invariant under a common scale of beta + epsilon) are
// unchanged; beta + epsilon is bounded below by 2^-100, which moves only
// weights between sub-stencils whose differences are below 2^-50 of the
// field's largest, whose values then differ by less than that.  The weights
// are formed as alpha_k = C_k / (beta_k + eps), omega = alpha / sum(alpha):
// the same quotient as the FP64 kernel's product form.
#include <cuda_runtime.h>

#include <cstdint>

#include "fdu_dw.cuh"
#include "fdu_dw_euler.cuh"
#include "fdu_dw_edge.cuh"
#include "fdu_internal.h"
#include "fdu_kernels.cuh"

namespace fdu {
namespace {

using namespace dwa;

__global__ void __launch_bounds__(kEdgeBlock, 4) edge_flux_dw_kernel(EdgeArgs A) {
    __shared__ float2 stage[kDwSlots * kEdgeBlock];
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= A.ne) return;
    if (A.dt_dev && *A.dt_dev == 0.0) return;
    edge_flux_dw_body(A, e, Stage{stage + threadIdx.x, kEdgeBlock});
}

// Accuracy check of the double-word primitives: inputs and outputs as
// doubles (inputs split by d2dw, outputs recombined exactly by f2d).
__global__ void dw_check_kernel(int op, const double *__restrict__ x, const double *__restrict__ y,
                                double *__restrict__ z, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    auto out = [&](dw r) { z[i] = f2d(r.h) + f2d(r.l); };
    if (op == 7) {  // compensated dot product of 8 consecutive pairs
        if (i >= n / 8) return;
        dot2 A{0.0f, 0.0f};
        for (int j = 0; j < 8; ++j) dot2_add(A, d2dw(x[8 * i + j]), d2dw(y[8 * i + j]));
        out(dot2_result(A));
        return;
    }
    if (i >= n) return;
    const dw a = d2dw(x[i]), b = d2dw(y[i]);
    switch (op) {
        case 0: out(a); break;
        case 1: out(add(a, b)); break;
        case 2: out(add_sl(a, b)); break;
        case 3: out(mul(a, b)); break;
        case 4: out(mul_u(a, b)); break;
        case 5: out(recip(a)); break;
        default: out(rsqrt(a)); break;
    }
}

}  // namespace

void launch_dw_check(int op, const double *x, const double *y, double *z, int64_t n, cudaStream_t s) {
    if (n > 0) dw_check_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(op, x, y, z, n);
}

void launch_edge_flux_dw(const EdgeArgs &a, cudaStream_t s) {
    if (a.ne > 0) edge_flux_dw_kernel<<<(unsigned)((a.ne + kEdgeBlock - 1) / kEdgeBlock), kEdgeBlock, 0, s>>>(a);
}

}  // namespace fdu
