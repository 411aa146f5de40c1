// Internal host-side structures of libfdu (not part of the C-ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "fdu.h"

namespace fdu {

// Per-side coefficient block of the difference-form NU-WENO5 (21 values):
//   value  A[k][2] : u~_k - u_c   = A[k][0]*d_a + A[k][1]*d_b
//   slope  P[k][2] : dx u~_k'(0)  (same differences)
//   curv   Q[k][2] : sqrt(13/12) dx^2 u~_k''
//   linear C[3]
// where the differences for sub-stencil k are taken against the shared
// point x_i and use the slots (k=0: x_{i-2}, x_{i-1}), (k=1: x_{i-1},
// x_{i+1}), (k=2: x_{i+1}, x_{i+2}).
constexpr int kSideCoef = 21;

// Edge coefficient block (kEdgeCoef values).  The left state uses the
// sub-stencils S_a = {L3,L2,L1}, S_b = {L2,L1,R1}, S_c = {L1,R1,R2}; the
// right (mirrored) state uses S_d = {R1,R2,R3}, S_c, S_b: S_b and S_c are
// the same quadratics over the same middle interval on both sides, so their
// values and smoothness indicators are computed once.  Each 5-block holds,
// for two differences (x, y), the value coefficients (2) and the smoothness
// indicator as a quadratic form m0 x^2 + m1 x y + m2 y^2 (3):
//   [0..4]   S_a of (L3-L1, L2-L1)      [5..9]   S_b of (L2-L1, R1-L1)
//   [10..14] S_c of (R1-L1, R2-L1)      [15..19] S_d of (R3-R1, R2-R1)
//   [20..21] C_0/C_1, C_2/C_1 of the left state   [22..23] the same of the right state
//   [24..25] n_x, n_y
constexpr int kSubCoef = 5;
constexpr int kCoefCL = 20;
constexpr int kCoefCR = 22;
constexpr int kCoefN = 24;
constexpr int kEdgeCoef = 26;
// FP32 path, default form: the FP64-built block rounded to FP32, values
// 0..23 as six float4 per edge ([6][ne] float4, value c at block c / 4,
// component c % 4), then (n_x, n_y) as one float2 per edge ([ne] float2
// after them): 104 bytes per edge.
constexpr int kEdgeCoef32 = 26;
constexpr int kEdgeCoef32Vec = 6;  // float4 blocks before the normals
// FP32 path, compact form (mesh option f32_coef = 1): the edge's four stencil
// gaps as one float4 per edge ([ne] float4: L1-L2, L2-L3, R1-R2, R2-R3 along
// the curve, each divided by the arc length L1-R1, differenced in FP64),
// then the float2 normals: 24 bytes per edge.  The FP32 edge flux forms
// values 0..23 from the gaps in FP32.
constexpr int kEdgeCoef32Gaps = 6;

struct HostTables {
    int64_t nv = 0, nt = 0, ne = 0, n_real = 0;
    int64_t ne_active = 0;         // edges used by some divergence stencil (internal ids 0..ne_active-1)
    double Lx = 0, Ly = 0, gamma = 1.4;
    int degree = 2, levels = 2;
    std::vector<double> xy;        // [nv][2]
    std::vector<int32_t> ghost;    // [nv] donor or -1 (empty = no ghosts)
    // original-id structures
    std::vector<int32_t> edge;     // [ne][2] v0 < v1, sorted
    std::vector<double> nrm;       // [ne][2]
    std::vector<int64_t> adj_off;  // [nv+1]
    std::vector<int32_t> adj;      // neighbour ids ascending
    std::vector<int32_t> adj_edge; // edge id per adjacency entry
    std::vector<int32_t> sten;     // [ne][6] (-1 when the edge has no stencil)
    std::vector<double> xi;        // [ne][6]
    std::vector<double> coef;      // [ne][kEdgeCoef] FP64 (edges without stencil: zeros)
    std::vector<int64_t> voff, eoff; // [nv+1]
    std::vector<int32_t> vid, eid;
    std::vector<double> wf, wg, we;
    std::vector<double> hmin;      // [nv] shortest edge at each vertex
    // renumbering: internal order -> original and back.  Internal vertex
    // order puts real vertices first (0..n_real-1), ghosts after; internal
    // edge order puts active edges first.
    std::vector<int32_t> v_new2old, v_old2new, e_new2old, e_old2new;
};

// Build every host table.  Returns FDU_OK or an error code with `err` set.
// `comp` (optional, [nv]) groups vertices into independent meshes of a
// batch: the renumbering keeps each component contiguous.
int build_host_tables(const double *xy, int64_t nv, const int32_t *tri, int64_t nt, const fdu_mesh_opts &o,
                      HostTables &T, std::string &err, const int32_t *comp = nullptr);

// Cells of 3 or 4 vertices (counter-clockwise, convex) as CSR.
struct CellList {
    const int64_t *off;  // [n+1]
    const int32_t *vtx;
    int64_t n;
};
// The same from cells; `artificial` = 0: cell sides only; 1: plus both
// diagonals of every quad; 2: plus far-apex edges at vertices short of
// least-squares conditions.
int build_host_tables(const double *xy, int64_t nv, const CellList &cells, int artificial, const fdu_mesh_opts &o,
                      HostTables &T, std::string &err, const int32_t *comp = nullptr);

// Per-side coefficient block from five normalised coordinates (exposed for tests through the C-ABI builder).
void side_coefficients(const double x[5], double out[kSideCoef]);

}  // namespace fdu
