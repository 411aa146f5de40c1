// Device-side argument blocks and launchers of libfdu (internal).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace fdu {

constexpr int kSell = 32;        // SELL slice width of the divergence tables (one warp)
constexpr int kEdgeBlock = 128;  // threads per block, edge-flux kernels
constexpr int kDivBlock = 128;   // threads per block, divergence kernels

// Edge-flux inputs (internal ids, SoA over the active edges).
struct EdgeArgs {
    const int32_t *sten;  // [6][ne]  L3 L2 L1 R1 R2 R3
    const void *coef;     // FP64: [kEdgeCoef][ne]; FP32: [6][ne] float4 of values 0..23, or (coef_gaps) [ne]
                          // float4 of stencil gaps; then [ne] float2 (n_x, n_y)
    bool coef_gaps;       // FP32: the block is the compact gaps form (values formed in the kernel)
    const void *w;        // FP64: [nv][4] double; FP32: [nv] float4
    void *r;              // FP64: [ne][4] double; FP32: [ne] float4
    int64_t ne;
    double gm1, eps;      // gamma - 1 and the WENO epsilon (FP64 path)
    double hgm1;          // (gamma - 1) / 2
    float gm1f, epsf;     // the same for the FP32 path
    unsigned long long *fallback;  // edges that fell back to first order (device counter)
    const double *dt_dev; // adaptive stepping: a zero time step here skips the launch
    const double *Q;      // FP64: per-vertex Roe records of the stage state (nullptr = compute per edge)
    // double-word edge flux (precision 48; Q is required there): r receives
    // the increment r_k - F_n(L1_k) as double words, [ne] x two float4
    // (h0, l0, h1, l1), (h2, l2, h3, l3)
    const float2 *coefdw; // [kEdgeCoef][ne] (hi, lo) of the coefficient block
    float dw_gm1[2];      // gamma - 1 as a double word
    float dw_tenth[2];    // 0.1 as a double word
    float dw_eps[2];      // WENO epsilon = dw_eps * 2^dw_eps_e, dw_eps in [1, 2)
    int dw_eps_e;
};

// Divergence (+ optional SSP-RK3 stage) inputs.
struct DivArgs {
    int64_t n_real;              // vertices with a residual (internal ids 0..n_real-1)
    const int64_t *slice_voff;   // [nslice+1] start of each slice's vertex entries
    const int64_t *slice_eoff;   // [nslice+1]
    const int32_t *perm;         // [n_real] vertex at each SELL position (nullptr = position i is vertex i)
    const int32_t *vid;          // vertex entries (SELL: entry j of lane l at off + 32 j + l)
    const void *wf, *wg;         // weights of f_j and g_j
    const int32_t *eid;          // edge entries
    const void *we;              // weights of r_k (double words when dw_edges)
    const void *cfg;             // [2][n_real] centre weights: -(sum wf + sum we nx), -(sum wg + sum we ny)
    const void *F;               // vertex fluxes of the stage state: FP64 [nv][8] (f0..3, g0..3); FP32 [nv][2] float4 pairs
    const void *r;               // edge fluxes (dw_edges: the precision-48 edge increments)
    bool dw_edges;               // precision 48: folded vertex weights, double-word edge part
    // residual output (mode 0)
    double *out;                 // [nv][4] FP64
    const int32_t *out_map;      // internal -> output row (nullptr = internal order)
    // RK stage (modes 1..3)
    const double *wn;            // [nv][4] state at the start of the step
    const double *ws;            // [nv][4] stage input state
    double *wout;                // [nv][4] stage output state (may alias ws)
    void *Fout;                  // vertex fluxes of wout (same layout as F)
    double *Qout;                // FP64: Roe records of wout (nullable)
    float4 *w32out;              // FP32 copy of wout (FP32 residual path), or nullptr
    double dt;
    const double *dt_dev;        // if non-null, dt is read here
    double gm1;                  // gamma - 1
    float gm1f;
    const int32_t *comp;         // batched meshes: component of each internal vertex (nullptr = one mesh)
    const double *dt_comp;       // batched meshes: time step of each component
    double pos_alpha;            // stage positivity safeguard (0 = off)
    unsigned long long *limited; // vertices whose stage update the safeguard scaled
};

// F[v] = (f, g) of w[v]; Q (optional) = Roe records (sqrt rho, sqrt rho u, sqrt rho v, sqrt rho H)
void launch_vertex_flux_f64(const double *w, double *F, int64_t n, double gamma, cudaStream_t s, double *Q = nullptr);
void launch_vertex_flux_f32(const double *w, float4 *F, float4 *w32, int64_t n, double gamma, cudaStream_t s);
void launch_edge_flux_f64(const EdgeArgs &a, cudaStream_t s);
void launch_edge_flux_f32(const EdgeArgs &a, cudaStream_t s);
void launch_edge_flux_dw(const EdgeArgs &a, cudaStream_t s);
// z = double-word primitive `op` of x (and y), device pointers (accuracy check)
void launch_dw_check(int op, const double *x, const double *y, double *z, int64_t n, cudaStream_t s);
void launch_div_f64(const DivArgs &a, int mode, cudaStream_t s);
void launch_div_f32(const DivArgs &a, int mode, cudaStream_t s);
// *bad = min(*bad, first row of w[n][4] with rho <= 0 or a non-finite value)
void launch_check_rows(const double *w, int64_t n, unsigned long long *bad, cudaStream_t s);
void launch_permute_rows(const double *in, double *out, const int32_t *map, int64_t n, bool gather, cudaStream_t s);
void launch_ghost_fill(double *w, const double *wsrc, void *F, const void *Fsrc, int fq, float4 *w32,
                       const int32_t *donor, int64_t n_real, int64_t n_ghost, cudaStream_t s);
// FMA throughput (TFLOP/s) of `precision` 64 or 32 with sms*8 blocks of 256
// threads; scratch holds sms*8*256 elements of that precision.
double fma_probe_tflops(int precision, int sms, void *scratch, cudaStream_t s);
// y[i] = the kernels' FP64 reciprocal (which = 0) or reciprocal square root
// (which = 1) of x[i] (device pointers; accuracy check)
void launch_recip_check(const double *x, double *y, int64_t n, int which, cudaStream_t s);
// k[24 i + j] = value j of the FP32 edge kernel's NU-WENO5 block formed from gaps g[i]
void launch_weno_coef32_check(const float4 *g, float *k, int64_t n, cudaStream_t s);
// Adaptive step: dt = min(cfl * bound, t_end - t) from the reduced bound in
// *slot (bit pattern of a positive double); tstate = (t, dt, nonphysical);
// the slot is reset to +inf for the next reduction; *nsteps counts steps
// with dt > 0.
void launch_dt_finalize(unsigned long long *slot, double *tstate, double cfl, double t_end,
                        unsigned long long *nsteps, cudaStream_t s);
void launch_max_dt(const double *w, const double *hmin, int64_t n, double gamma, unsigned long long *slot,
                   cudaStream_t s, const int32_t *comp = nullptr);

// One SSP-RK3 stage (mode 1..3) of a batch as one cooperative launch of
// `blocks` x `threads` (edge fluxes, bounded grid barrier, divergence +
// stage).  The barrier expects `nblocks_expected` arrivals (= blocks in
// normal use) and gives up after `spin_limit` polls, setting *err.
cudaError_t launch_stage_persistent(int prec, int mode, const EdgeArgs &ea, const DivArgs &da, unsigned int *bar_count,
                                    unsigned int *bar_gen, unsigned int nblocks_expected,
                                    unsigned long long spin_limit, int *err, int threads, int blocks, cudaStream_t s);
// Co-resident blocks per SM of the persistent stage kernel at `threads`.
int persistent_blocks_per_sm(int prec, int threads);

}  // namespace fdu
