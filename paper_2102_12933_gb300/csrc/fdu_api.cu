// C-ABI of libfdu (declared in include/fdu.h): mesh object, device table
// packing, stage sequencing and CUDA-graph replay of SSP-RK3 steps.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <tuple>
#include <string>
#include <numeric>
#include <vector>

#include "fdu.h"
#include "fdu_internal.h"
#include "fdu_kernels.cuh"
#include "fdu_adjoint.cuh"

using namespace fdu;

namespace {

thread_local std::string g_err;

fdu_status set_err(fdu_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define CK_LAUNCH()                                                                              \
    do {                                                                                         \
        cudaError_t e_ = cudaGetLastError();                                                     \
        if (e_ != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
};

}  // namespace

struct fdu_mesh {
    HostTables T;
    fdu_mesh_opts opts{};
    int device = -1;
    int64_t nv = 0, n_real = 0, n_ghost = 0, ne_act = 0, nslice = 0;
    int64_t vert_nnz_sell = 0, edge_nnz_sell = 0, vert_nnz_sell64 = 0, edge_nnz_sell64 = 0;
    int64_t device_bytes = 0, table_bytes_f64 = 0, table_bytes_f32 = 0;
    std::vector<void *> allocs;
    // tables
    int32_t *sten = nullptr;          // [6][ne_act]
    double *coef64 = nullptr;         // [32][ne_act]
    float *coef32 = nullptr;          // FP32 block: [6][ne_act] float4, or (f32_coef = 1) [ne_act] float4 of gaps; then [ne_act] float2 (n_x, n_y)
    // precision 48 (built on first use): double-word coefficient block
    // [kEdgeCoef][ne_act]; FP64 divergence tables with the left vertex flux
    // of each edge folded into the vertex weights; edge weights as double words
    float2 *coefdw = nullptr;
    double *swf48 = nullptr, *swg48 = nullptr, *cfg48 = nullptr;
    float2 *swe48 = nullptr;
    std::vector<int32_t> order64;     // vertex at each position of the FP64 SELL layout
    int64_t *slice_voff = nullptr, *slice_eoff = nullptr;       // FP32 layout (natural order)
    int64_t *slice_voff64 = nullptr, *slice_eoff64 = nullptr;   // FP64 layout (stencil-size order in windows)
    int32_t *svid64 = nullptr, *seid64 = nullptr, *perm64 = nullptr;
    int32_t *svid = nullptr, *seid = nullptr;
    double *swf64 = nullptr, *swg64 = nullptr, *swe64 = nullptr, *cfg64 = nullptr;
    float *swf32 = nullptr, *swg32 = nullptr, *swe32 = nullptr, *cfg32 = nullptr;
    int32_t *new2old = nullptr;       // [nv] internal -> original vertex
    int32_t *donor = nullptr;         // [n_ghost] internal donor of each ghost
    double *hmin = nullptr;           // [n_real]
    // state
    double *wn = nullptr, *ws = nullptr, *scratch = nullptr;  // [nv][4]
    double *F64[3] = {nullptr, nullptr, nullptr};           // [nv][8]; F64[0] = fluxes of wn
    double *Q64[3] = {nullptr, nullptr, nullptr};           // [nv][4] Roe records, rotating with F64
    float4 *F32[3] = {nullptr, nullptr, nullptr};           // [nv][2]
    float4 *w32 = nullptr;                                  // [nv]
    double *r64 = nullptr;                                  // [ne_act][4]
    float4 *r32 = nullptr;                                  // [ne_act]
    unsigned long long *counters = nullptr;  // [0] fallbacks, [1] dt slot, [2] adaptive slot, [3] adaptive steps,
                                             // [4] stage updates scaled by the positivity safeguard,
                                             // [5] first non-physical row of a state being set
    double *tstate = nullptr;                // adaptive stepping: (t, dt, nonphysical flag)
    bool f64_valid = false, f32_valid = false;              // F64[0] / (w32, F32[0]) describe wn
    cudaStream_t own_stream = nullptr;
    std::map<std::pair<int, double>, cudaGraphExec_t> graphs;
    std::map<std::tuple<int, double, double>, cudaGraphExec_t> adaptive_graphs;
    // batched meshes (fdu_batch_create): components, per-component dt, persistent launches
    int32_t n_comp = 0;
    std::vector<int64_t> comp_voff;   // original-vertex offset of each component
    int32_t *comp = nullptr;          // [n_real] component of each internal vertex
    double *dt_comp = nullptr;        // [n_comp]
    unsigned long long *comp_slots = nullptr;  // [n_comp] dt reductions
    unsigned int *bar = nullptr;      // grid barrier: count, generation
    int *bar_err = nullptr;           // grid barrier timed out
    int pl_threads = 256, pl_blocks = 0;  // persistent launch shape (blocks in total)
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> batch_graphs;
    // adjoint workspace (built on first use)
    bool adj_ready = false;
    int adj_prec = 64;                // adjoint precision: 64, or 48 (double-word VJP, precision-48 steps)
    int64_t *adj_eoff = nullptr, *adj_voff = nullptr, *adj_soff = nullptr, *adj_slot = nullptr;
    int32_t *adj_evid = nullptr, *adj_vvid = nullptr;
    int32_t *adj_eperm = nullptr, *adj_vperm = nullptr;  // thread -> edge / vertex of the transpose kernels
    double *adj_ewt = nullptr, *adj_wf = nullptr, *adj_wg = nullptr;
    double *adj_lam_r = nullptr, *adj_G = nullptr;
    double *adj_S1 = nullptr, *adj_buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    // transpose of the transmissive ghost fill: donors with their ghosts (CSR, internal ids)
    int64_t adj_nfold = 0;
    int32_t *adj_fold_donor = nullptr, *adj_fold_ghost = nullptr;
    int64_t *adj_fold_off = nullptr;
    std::vector<double *> adj_states;  // checkpoints and recomputed step states
    // kernel timing: event pairs per kind (0 edge64, 1 div64, 2 edge32, 3 div32, 4 edge48, 5 div at precision 48)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev[6];
    size_t prof_used[6] = {0, 0, 0, 0, 0, 0};

    template <class T>
    fdu_status alloc(T *&p, size_t count) {
        p = nullptr;
        if (count == 0) count = 1;
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, count * sizeof(T));
        if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        allocs.push_back(q);
        device_bytes += (int64_t)(count * sizeof(T));
        p = static_cast<T *>(q);
        return FDU_OK;
    }
    template <class T>
    fdu_status upload(T *&p, const std::vector<T> &h) {
        fdu_status st = alloc(p, h.size());
        if (st) return st;
        if (!h.empty()) CK(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
        return FDU_OK;
    }
    cudaStream_t stream(void *s) const { return s ? static_cast<cudaStream_t>(s) : own_stream; }
    void release() {
        if (device >= 0) {
            cudaSetDevice(device);
            cudaDeviceSynchronize();
            for (auto &kv : graphs) cudaGraphExecDestroy(kv.second);
            graphs.clear();
            for (auto &kv : adaptive_graphs) cudaGraphExecDestroy(kv.second);
            adaptive_graphs.clear();
            for (auto &kv : batch_graphs) cudaGraphExecDestroy(kv.second);
            batch_graphs.clear();
            for (auto &v : prof_ev)
                for (cudaEvent_t e : v) cudaEventDestroy(e);
            for (void *p : allocs) cudaFree(p);
            allocs.clear();
            adj_states.clear();
            if (own_stream) cudaStreamDestroy(own_stream);
            own_stream = nullptr;
        }
    }
};

namespace {

fdu_status need_device(const fdu_mesh *m) {
    if (!m) return set_err(FDU_ERR_ARG, "null mesh");
    if (m->device < 0) return set_err(FDU_ERR_NODEVICE, "mesh was built with device = -1 (host tables only)");
    cudaError_t e = cudaSetDevice(m->device);
    if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("cudaSetDevice: ") + cudaGetErrorString(e));
    return FDU_OK;
}

// Divergence tables, SELL-32 over internal real vertices: position i of a
// slice order holds vertex order[i]; entry j of lane l at off + 32 j + l.
// The weights come from wf, wg, we (indexed like the host tables' entries).
struct Sell {
    std::vector<int64_t> svo, seo;
    std::vector<int32_t> vid, eid;
    std::vector<double> wf, wg, we;
};
void sell_tables(const fdu_mesh *m, const std::vector<int32_t> &order, const double *wf, const double *wg,
                 const double *we, Sell &S) {
    const HostTables &T = m->T;
    const int64_t nr = m->n_real;
    S.svo.assign(m->nslice + 1, 0);
    S.seo.assign(m->nslice + 1, 0);
    for (int64_t sl = 0; sl < m->nslice; ++sl) {
        int64_t mj = 0, mk = 0;
        for (int64_t i = sl * kSell; i < std::min(nr, (sl + 1) * kSell); ++i) {
            const int64_t o = T.v_new2old[order[i]];
            mj = std::max(mj, T.voff[o + 1] - T.voff[o]);
            mk = std::max(mk, T.eoff[o + 1] - T.eoff[o]);
        }
        S.svo[sl + 1] = S.svo[sl] + mj * kSell;
        S.seo[sl + 1] = S.seo[sl] + mk * kSell;
    }
    S.vid.assign(S.svo[m->nslice], 0);
    S.eid.assign(S.seo[m->nslice], 0);
    S.wf.assign(S.svo[m->nslice], 0.0);
    S.wg.assign(S.svo[m->nslice], 0.0);
    S.we.assign(S.seo[m->nslice], 0.0);
    for (int64_t i = 0; i < nr; ++i) {
        const int32_t v = order[i];
        const int64_t o = T.v_new2old[v], sl = i / kSell, lane = i % kSell;
        const int64_t J = T.voff[o + 1] - T.voff[o], K = T.eoff[o + 1] - T.eoff[o];
        const int64_t mj = (S.svo[sl + 1] - S.svo[sl]) / kSell, mk = (S.seo[sl + 1] - S.seo[sl]) / kSell;
        for (int64_t j = 0; j < mj; ++j) {
            const int64_t p = S.svo[sl] + j * kSell + lane;
            if (j < J) {
                const int64_t q = T.voff[o] + j;
                S.vid[p] = T.v_old2new[T.vid[q]];
                S.wf[p] = wf[q];
                S.wg[p] = wg[q];
            } else {
                S.vid[p] = v;  // padding: weight 0 on the vertex itself
            }
        }
        for (int64_t k = 0; k < mk; ++k) {
            const int64_t p = S.seo[sl] + k * kSell + lane;
            if (k < K) {
                const int64_t q = T.eoff[o] + k;
                S.eid[p] = T.e_old2new[T.eid[q]];
                S.we[p] = we[q];
            } else {
                S.eid[p] = K > 0 ? T.e_old2new[T.eid[T.eoff[o]]] : 0;
            }
        }
    }
}

// The FP32 edge form's four gaps from an edge's stencil coordinates (L1 at
// -1/2, R1 at 1/2): L1-L2, L2-L3, R1-R2, R2-R3 as positive lengths,
// differenced in FP64 and rounded once.
void stencil_gaps(const double xi[6], float g[4]) {
    const double d[4] = {-0.5 - xi[1], xi[1] - xi[0], xi[4] - 0.5, xi[5] - xi[4]};
    for (int c = 0; c < 4; ++c) g[c] = (float)d[c];
}

// Pack host tables into device layouts.
fdu_status upload_tables(fdu_mesh *m) {
    const HostTables &T = m->T;
    const int64_t ne = m->ne_act, nv = m->nv, nr = m->n_real;
    fdu_status st;
    // 1D stencils and coefficient blocks, SoA over internal active edges
    std::vector<int32_t> sten(6 * ne);
    std::vector<double> coef((size_t)kEdgeCoef * ne);
    const bool gaps32 = m->opts.f32_coef == 1;
    std::vector<float> coef32((size_t)(gaps32 ? kEdgeCoef32Gaps : kEdgeCoef32) * ne, 0.0f);
    for (int64_t e = 0; e < ne; ++e) {
        const int64_t o = T.e_new2old[e];
        for (int i = 0; i < 6; ++i) sten[i * ne + e] = T.v_old2new[T.sten[6 * o + i]];
        for (int c = 0; c < kEdgeCoef; ++c) coef[(size_t)c * ne + e] = T.coef[(size_t)kEdgeCoef * o + c];
        if (gaps32) {
            // compact FP32 form: the gaps between consecutive stencil coordinates
            // (the coordinates put L1 at -1/2 and R1 at 1/2), differenced in FP64,
            // as one float4 [ne][4], then the normal as float2 [ne][2]
            stencil_gaps(&T.xi[6 * (size_t)o], &coef32[4 * (size_t)e]);
            for (int c = 0; c < 2; ++c)
                coef32[4 * (size_t)ne + 2 * e + c] = (float)T.coef[(size_t)kEdgeCoef * o + kCoefN + c];
        } else {
            // default FP32 form: the FP64 block rounded to FP32, values 0..23 as
            // float4 vectors [c/4][ne][c%4], then the normal as float2 [ne][2]
            for (int c = 0; c < kEdgeCoef; ++c) {
                const float v = (float)T.coef[(size_t)kEdgeCoef * o + c];
                if (c < 4 * kEdgeCoef32Vec)
                    coef32[((size_t)(c / 4) * ne + e) * 4 + c % 4] = v;
                else
                    coef32[(size_t)4 * kEdgeCoef32Vec * ne + 2 * e + (c - 4 * kEdgeCoef32Vec)] = v;
            }
        }
    }
    if ((st = m->upload(m->sten, sten))) return st;
    if ((st = m->upload(m->coef64, coef))) return st;
    if ((st = m->upload(m->coef32, coef32))) return st;
    // divergence tables, SELL-32 over internal real vertices (sell_tables)
    m->nslice = (nr + kSell - 1) / kSell;
    // centre weights per vertex
    std::vector<double> cfg(2 * std::max<int64_t>(nr, 1), 0.0);
    for (int64_t v = 0; v < nr; ++v) {
        const int64_t o = T.v_new2old[v];
        double sf = 0, sg = 0, sx = 0, sy = 0;
        for (int64_t q = T.voff[o]; q < T.voff[o + 1]; ++q) {
            sf += T.wf[q];
            sg += T.wg[q];
        }
        for (int64_t q = T.eoff[o]; q < T.eoff[o + 1]; ++q) {
            const int32_t e = T.eid[q];
            sx += T.we[q] * T.nrm[2 * e];
            sy += T.we[q] * T.nrm[2 * e + 1];
        }
        cfg[v] = -(sf + sx);
        cfg[nr + v] = -(sg + sy);
    }
    // FP32: natural (Hilbert) order, which keeps the flux gathers of a warp
    // local; FP64: inside windows of 256 positions the vertices are sorted
    // by decreasing stencil size, so a slice's lanes have nearly equal entry
    // counts and little padding (the FP64 loops are bound by the FP64 pipe,
    // which padding entries occupy like real ones)
    std::vector<int32_t> natural(std::max<int64_t>(nr, 1)), sorted;
    std::iota(natural.begin(), natural.end(), 0);
    sorted = natural;
    for (int64_t w0 = 0; w0 < nr; w0 += 256) {
        const int64_t w1 = std::min<int64_t>(nr, w0 + 256);
        std::stable_sort(sorted.begin() + w0, sorted.begin() + w1, [&](int32_t x, int32_t y) {
            const int64_t ox = T.v_new2old[x], oy = T.v_new2old[y];
            const int64_t jx = T.voff[ox + 1] - T.voff[ox], jy = T.voff[oy + 1] - T.voff[oy];
            if (jx != jy) return jx > jy;
            return T.eoff[ox + 1] - T.eoff[ox] > T.eoff[oy + 1] - T.eoff[oy];
        });
    }
    Sell S32, S64;
    sell_tables(m, natural, T.wf.data(), T.wg.data(), T.we.data(), S32);
    sell_tables(m, sorted, T.wf.data(), T.wg.data(), T.we.data(), S64);
    m->order64 = sorted;
    m->vert_nnz_sell = S32.svo[m->nslice];
    m->edge_nnz_sell = S32.seo[m->nslice];
    m->vert_nnz_sell64 = S64.svo[m->nslice];
    m->edge_nnz_sell64 = S64.seo[m->nslice];
    if ((st = m->upload(m->slice_voff, S32.svo))) return st;
    if ((st = m->upload(m->slice_eoff, S32.seo))) return st;
    if ((st = m->upload(m->svid, S32.vid))) return st;
    if ((st = m->upload(m->seid, S32.eid))) return st;
    auto to32 = [](const std::vector<double> &a) { return std::vector<float>(a.begin(), a.end()); };
    if ((st = m->upload(m->swf32, to32(S32.wf)))) return st;
    if ((st = m->upload(m->swg32, to32(S32.wg)))) return st;
    if ((st = m->upload(m->swe32, to32(S32.we)))) return st;
    if ((st = m->upload(m->cfg32, to32(cfg)))) return st;
    if ((st = m->upload(m->slice_voff64, S64.svo))) return st;
    if ((st = m->upload(m->slice_eoff64, S64.seo))) return st;
    if ((st = m->upload(m->svid64, S64.vid))) return st;
    if ((st = m->upload(m->seid64, S64.eid))) return st;
    if ((st = m->upload(m->swf64, S64.wf))) return st;
    if ((st = m->upload(m->swg64, S64.wg))) return st;
    if ((st = m->upload(m->swe64, S64.we))) return st;
    if ((st = m->upload(m->cfg64, cfg))) return st;
    if ((st = m->upload(m->perm64, sorted))) return st;
    if ((st = m->upload(m->new2old, T.v_new2old))) return st;
    std::vector<int32_t> donor(std::max<int64_t>(m->n_ghost, 1), 0);
    for (int64_t i = 0; i < m->n_ghost; ++i) donor[i] = T.v_old2new[T.ghost[T.v_new2old[nr + i]]];
    if ((st = m->upload(m->donor, donor))) return st;
    std::vector<double> hm(std::max<int64_t>(nr, 1), 0.0);
    for (int64_t v = 0; v < nr; ++v) hm[v] = T.hmin[T.v_new2old[v]];
    if ((st = m->upload(m->hmin, hm))) return st;
    m->table_bytes_f64 = (int64_t)(sten.size() * 4 + coef.size() * 8 + (S64.svo.size() + S64.seo.size()) * 8 +
                                   S64.vid.size() * 4 + S64.eid.size() * 4 + sorted.size() * 4 +
                                   (S64.wf.size() + S64.wg.size() + S64.we.size() + cfg.size()) * 8);
    m->table_bytes_f32 = (int64_t)(sten.size() * 4 + coef32.size() * 4 + (S32.svo.size() + S32.seo.size()) * 8 +
                                   S32.vid.size() * 4 + S32.eid.size() * 4 +
                                   (S32.wf.size() + S32.wg.size() + S32.we.size() + cfg.size()) * 4);
    // state and work buffers
    if ((st = m->alloc(m->wn, 4 * nv))) return st;
    if ((st = m->alloc(m->ws, 4 * nv))) return st;
    if ((st = m->alloc(m->scratch, 4 * nv))) return st;
    for (int i = 0; i < 3; ++i) {
        if ((st = m->alloc(m->F64[i], 8 * nv))) return st;
        if ((st = m->alloc(m->Q64[i], 4 * nv))) return st;
        if ((st = m->alloc(m->F32[i], 2 * nv))) return st;
    }
    if ((st = m->alloc(m->w32, nv))) return st;
    if ((st = m->alloc(m->r64, 4 * ne))) return st;
    if ((st = m->alloc(m->r32, ne))) return st;
    if ((st = m->alloc(m->counters, 6))) return st;
    CK(cudaMemset(m->counters, 0, 6 * sizeof(unsigned long long)));
    {
        const unsigned long long inf_bits = 0x7FF0000000000000ull;
        CK(cudaMemcpy(m->counters + 2, &inf_bits, sizeof inf_bits, cudaMemcpyHostToDevice));
    }
    if ((st = m->alloc(m->tstate, 4))) return st;
    CK(cudaMemset(m->tstate, 0, 4 * sizeof(double)));
    CK(cudaMemset(m->wn, 0, 4 * nv * sizeof(double)));
    return FDU_OK;
}

// Precision 48: the FP64 state pipeline (FP64 divergence and stage) with
// the double-word edge flux.
inline bool fp64_state(int prec) { return prec != 32; }
inline int prof_kind(int prec) { return prec == 64 ? 0 : prec == 32 ? 2 : 4; }

// Precision 64, 32 or 48.  The first use of 48 builds its tables:
//  - the double-word edge coefficient block (hi = the FP32 rounding of each
//    FP64 coefficient, lo = the FP32 rounding of the remainder);
//  - divergence tables in the FP64 SELL layout where the edge flux, which
//    the precision-48 edge kernel leaves as the increment
//    r_k - F_n(L1_k) = r_k - (n_x f + n_y g)(L1_k), has its left-vertex part
//    folded into the weights of that vertex's fluxes:
//      sum_k w_k r_k = sum_k w_k (n_x,k f_L1k + n_y,k g_L1k) + sum_k w_k (r_k - F_n(L1_k)),
//    the first sum going into w_f, w_g (or the centre weights when L1_k is
//    the vertex itself) and the second taken in double words.
//    Both ends of every stencil edge are in the vertex's own stencil, so
//    the folding adds no entries; a mesh where that fails is refused.
fdu_status check_precision(fdu_mesh *m, int prec) {
    if (prec != 64 && prec != 32 && prec != 48) return set_err(FDU_ERR_ARG, "precision must be 64, 48 or 32");
    if (prec != 48 || m->coefdw) return FDU_OK;
    const HostTables &T = m->T;
    const int64_t ne = m->ne_act, nr = m->n_real;
    fdu_status st;
    auto split = [](double x) {
        const float h = (float)x;
        return make_float2(h, (float)(x - (double)h));
    };
    std::vector<double> wf(T.wf), wg(T.wg), cfg(2 * std::max<int64_t>(nr, 1), 0.0);
    for (int64_t v = 0; v < nr; ++v) {
        const int64_t o = T.v_new2old[v];
        double sf = 0, sg = 0, sx = 0, sy = 0;
        for (int64_t q = T.voff[o]; q < T.voff[o + 1]; ++q) {
            sf += T.wf[q];
            sg += T.wg[q];
        }
        for (int64_t q = T.eoff[o]; q < T.eoff[o + 1]; ++q) {
            const int32_t e = T.eid[q];
            sx += T.we[q] * T.nrm[2 * e];
            sy += T.we[q] * T.nrm[2 * e + 1];
        }
        double cf = -(sf + sx), cg = -(sg + sy);
        for (int64_t q = T.eoff[o]; q < T.eoff[o + 1]; ++q) {
            const int32_t e = T.eid[q];
            const int32_t L = T.sten[6 * (int64_t)e + 2];
            const double ax = T.we[q] * T.nrm[2 * e], ay = T.we[q] * T.nrm[2 * e + 1];
            if (L == o) {
                cf += ax;
                cg += ay;
                continue;
            }
            int64_t j = T.voff[o];
            while (j < T.voff[o + 1] && T.vid[j] != L) ++j;
            if (j == T.voff[o + 1])
                return set_err(FDU_ERR_MESH, "precision 48: an edge's left vertex is outside the vertex's stencil");
            wf[j] += ax;
            wg[j] += ay;
        }
        cfg[v] = cf;
        cfg[nr + v] = cg;
    }
    Sell S;
    sell_tables(m, m->order64, wf.data(), wg.data(), T.we.data(), S);
    std::vector<float2> we2(S.we.size());
    for (size_t i = 0; i < we2.size(); ++i) we2[i] = split(S.we[i]);
    std::vector<float2> k((size_t)kEdgeCoef * ne);
    for (int64_t e = 0; e < ne; ++e) {
        const int64_t o = T.e_new2old[e];
        for (int c = 0; c < kEdgeCoef; ++c) k[(size_t)c * ne + e] = split(T.coef[(size_t)kEdgeCoef * o + c]);
    }
    if ((st = m->upload(m->swf48, S.wf))) return st;
    if ((st = m->upload(m->swg48, S.wg))) return st;
    if ((st = m->upload(m->cfg48, cfg))) return st;
    if ((st = m->upload(m->swe48, we2))) return st;
    return m->upload(m->coefdw, k);
}

// Double-word constants of the precision-48 edge flux.
void dw_split(double x, float out[2]) {
    out[0] = (float)x;
    out[1] = (float)(x - (double)out[0]);
}

EdgeArgs edge_args(fdu_mesh *m, int prec, const void *w) {
    EdgeArgs a{};
    a.sten = m->sten;
    a.coef = fp64_state(prec) ? (const void *)m->coef64 : (const void *)m->coef32;
    a.coef_gaps = !fp64_state(prec) && m->opts.f32_coef == 1;
    a.w = w;
    a.r = fp64_state(prec) ? (void *)m->r64 : (void *)m->r32;
    if (prec == 48) {
        a.coefdw = m->coefdw;
        dw_split(m->opts.gamma - 1.0, a.dw_gm1);
        dw_split(0.1, a.dw_tenth);
        int ee = 0;
        const double mant = std::frexp(m->opts.weno_eps, &ee);  // eps = mant 2^ee, mant in [1/2, 1)
        dw_split(2.0 * mant, a.dw_eps);
        a.dw_eps_e = ee - 1;
    }
    a.ne = m->ne_act;
    a.gm1 = m->opts.gamma - 1.0;
    a.hgm1 = 0.5 * a.gm1;
    a.eps = m->opts.weno_eps;
    a.gm1f = (float)(m->opts.gamma - 1.0);
    a.epsf = (float)m->opts.weno_eps32;
    a.fallback = m->counters;
    a.dt_dev = nullptr;
    a.Q = nullptr;
    return a;
}

DivArgs div_args(fdu_mesh *m, int prec, int fin) {
    DivArgs a{};
    a.n_real = m->n_real;
    a.slice_voff = m->slice_voff;
    a.slice_eoff = m->slice_eoff;
    a.vid = m->svid;
    a.eid = m->seid;
    if (fp64_state(prec)) {
        a.slice_voff = m->slice_voff64;
        a.slice_eoff = m->slice_eoff64;
        a.vid = m->svid64;
        a.eid = m->seid64;
        a.perm = m->perm64;
        a.wf = m->swf64; a.wg = m->swg64; a.we = m->swe64; a.cfg = m->cfg64;
        a.F = m->F64[fin]; a.r = m->r64;
        if (prec == 48) {  // folded vertex weights, double-word edge increments (in r64's storage)
            a.wf = m->swf48; a.wg = m->swg48; a.we = m->swe48; a.cfg = m->cfg48;
            a.dw_edges = true;
        }
    } else {
        a.wf = m->swf32; a.wg = m->swg32; a.we = m->swe32; a.cfg = m->cfg32;
        a.F = m->F32[fin]; a.r = m->r32;
    }
    a.gm1 = m->opts.gamma - 1.0;
    a.gm1f = (float)(m->opts.gamma - 1.0);
    a.pos_alpha = m->opts.positivity_alpha;
    a.limited = m->counters + 4;
    return a;
}

// Event pair around one launch of kernel kind k (nullptr when not profiling).
cudaEvent_t *prof_pair(fdu_mesh *m, int kind, bool allowed) {
    if (!m->prof_on || !allowed) return nullptr;
    std::vector<cudaEvent_t> &v = m->prof_ev[kind];
    const size_t i = m->prof_used[kind]++;
    while (v.size() < 2 * (i + 1)) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        v.push_back(e);
    }
    return &v[2 * i];
}

template <class F>
void timed(fdu_mesh *m, int kind, bool allowed, cudaStream_t s, F &&launch) {
    cudaEvent_t *p = prof_pair(m, kind, allowed);
    if (p) cudaEventRecord(p[0], s);
    launch();
    if (p) cudaEventRecord(p[1], s);
}

// Make F64[0] (or w32 and F32[0]) describe the current state wn.
void ensure_fluxes(fdu_mesh *m, int prec, cudaStream_t s) {
    if (fp64_state(prec) && !m->f64_valid) {
        launch_vertex_flux_f64(m->wn, m->F64[0], m->nv, m->opts.gamma, s, m->Q64[0]);
        m->f64_valid = true;
    }
    if (prec == 32 && !m->f32_valid) {
        launch_vertex_flux_f32(m->wn, m->F32[0], m->w32, m->nv, m->opts.gamma, s);
        m->f32_valid = true;
    }
}

// One SSP-RK3 step: three (edge flux, divergence + stage) pairs.  Stage i
// reads fluxes F[i-1] and writes F[i mod 3], so F[0] holds the fluxes of
// the new state at the end and a captured step can be replayed as is.
void enqueue_stages(fdu_mesh *m, int prec, double dt, const double *dt_dev, cudaStream_t s, bool prof, int first,
                    int last) {
    const bool f64 = fp64_state(prec);
    const int fq = f64 ? 4 : 2;  // 16-byte words of vertex fluxes per vertex
    const int kd = prof_kind(prec);
    for (int stage = first; stage <= last; ++stage) {
        const double *win = stage == 1 ? m->wn : m->ws;
        timed(m, kd, prof, s, [&] {
            EdgeArgs ea = edge_args(m, prec, f64 ? (const void *)win : (const void *)m->w32);
            ea.dt_dev = dt_dev;
            if (f64) ea.Q = m->Q64[stage - 1];
            if (prec == 64) launch_edge_flux_f64(ea, s);
            else if (prec == 48) launch_edge_flux_dw(ea, s);
            else launch_edge_flux_f32(ea, s);
        });
        DivArgs a = div_args(m, prec, stage - 1);
        a.wn = m->wn;
        a.ws = win;
        a.wout = stage == 3 ? m->wn : m->ws;
        a.Fout = f64 ? (void *)m->F64[stage % 3] : (void *)m->F32[stage % 3];
        a.Qout = f64 ? m->Q64[stage % 3] : nullptr;
        a.w32out = prec == 32 ? m->w32 : nullptr;
        a.dt = dt;
        a.dt_dev = dt_dev;
        timed(m, kd + 1, prof, s, [&] {
            if (f64) launch_div_f64(a, stage, s);
            else launch_div_f32(a, stage, s);
        });
        if (m->n_ghost > 0) {
            // Dirichlet ghosts take their fixed values from the step's start buffers (wn, F[0], Q[0])
            const void *F0 = f64 ? (const void *)m->F64[0] : (const void *)m->F32[0];
            launch_ghost_fill(a.wout, m->wn, a.Fout, F0, fq, prec == 32 ? m->w32 : nullptr, m->donor, m->n_real,
                              m->n_ghost, s);
            if (a.Qout) launch_ghost_fill(nullptr, nullptr, a.Qout, m->Q64[0], 2, nullptr, m->donor, m->n_real, m->n_ghost, s);
        }
    }
}

void enqueue_step(fdu_mesh *m, int prec, double dt, const double *dt_dev, cudaStream_t s, bool prof) {
    enqueue_stages(m, prec, dt, dt_dev, s, prof, 1, 3);
}

// ---------------------------------------------------------------- adjoint
fdu_status adjoint_setup(fdu_mesh *m) {
    if (m->adj_ready) return FDU_OK;
    const HostTables &T = m->T;
    const int64_t nv = m->nv, ne = m->ne_act;
    // edge transpose and vertex transpose (with centre weights), internal ids
    std::vector<int64_t> ecnt(ne + 1, 0), vcnt(nv + 1, 0), scnt(nv + 1, 0);
    for (int64_t v = 0; v < m->n_real; ++v) {
        const int64_t o = T.v_new2old[v];
        for (int64_t q = T.eoff[o]; q < T.eoff[o + 1]; ++q) ecnt[T.e_old2new[T.eid[q]] + 1]++;
        for (int64_t q = T.voff[o]; q < T.voff[o + 1]; ++q) vcnt[T.v_old2new[T.vid[q]] + 1]++;
        vcnt[v + 1]++;
    }
    for (int64_t k = 0; k < ne; ++k)
        for (int i = 0; i < 6; ++i) scnt[T.v_old2new[T.sten[6 * (int64_t)T.e_new2old[k] + i]] + 1]++;
    for (int64_t k = 0; k < ne; ++k) ecnt[k + 1] += ecnt[k];
    for (int64_t v = 0; v < nv; ++v) {
        vcnt[v + 1] += vcnt[v];
        scnt[v + 1] += scnt[v];
    }
    std::vector<int32_t> evid(ecnt[ne]), vvid(vcnt[nv]);
    std::vector<double> ewt(ecnt[ne]), wf(vcnt[nv]), wg(vcnt[nv]);
    std::vector<int64_t> slot(scnt[nv]);
    std::vector<int64_t> ef(ecnt.begin(), ecnt.end() - 1), vf(vcnt.begin(), vcnt.end() - 1), sf(scnt.begin(), scnt.end() - 1);
    for (int64_t v = 0; v < m->n_real; ++v) {
        const int64_t o = T.v_new2old[v];
        double sf_ = 0, sg_ = 0, sx = 0, sy = 0;
        for (int64_t q = T.eoff[o]; q < T.eoff[o + 1]; ++q) {
            const int32_t e = T.eid[q];
            const int64_t p = ef[T.e_old2new[e]]++;
            evid[p] = (int32_t)v;
            ewt[p] = -T.we[q];  // the residual is minus the divergence: the sign rides on the weights
            sx += T.we[q] * T.nrm[2 * e];
            sy += T.we[q] * T.nrm[2 * e + 1];
        }
        for (int64_t q = T.voff[o]; q < T.voff[o + 1]; ++q) {
            const int64_t p = vf[T.v_old2new[T.vid[q]]]++;
            vvid[p] = (int32_t)v;
            wf[p] = -T.wf[q];
            wg[p] = -T.wg[q];
            sf_ += T.wf[q];
            sg_ += T.wg[q];
        }
        const int64_t p = vf[v]++;  // centre weights, as in the forward's folded form
        vvid[p] = (int32_t)v;
        wf[p] = sf_ + sx;  // minus the centre weights -(sum wf + sum we nx), likewise g
        wg[p] = sg_ + sy;
    }
    for (int64_t k = 0; k < ne; ++k)
        for (int i = 0; i < 6; ++i) slot[sf[T.v_old2new[T.sten[6 * (int64_t)T.e_new2old[k] + i]]]++] = i * ne + k;
    fdu_status st;
    // the transpose kernels give one thread a list (edges: the stencils that
    // hold the edge; vertices: the stencils and stencil slots that hold the
    // vertex); inside windows of 256 consecutive ids the threads are ordered
    // by list length, so the lanes of a warp walk lists of about one length
    auto window_order = [](int64_t n, const std::function<int64_t(int64_t)> &len) {
        std::vector<int32_t> perm(std::max<int64_t>(n, 1));
        std::iota(perm.begin(), perm.begin() + n, 0);
        for (int64_t w0 = 0; w0 < n; w0 += 256)
            std::stable_sort(perm.begin() + w0, perm.begin() + std::min<int64_t>(n, w0 + 256),
                             [&](int32_t a, int32_t b) { return len(a) > len(b); });
        return perm;
    };
    const std::vector<int32_t> eperm = window_order(ne, [&](int64_t k) { return ecnt[k + 1] - ecnt[k]; });
    const std::vector<int32_t> vperm = window_order(nv, [&](int64_t v) {
        return (vcnt[v + 1] - vcnt[v]) * 8 + (scnt[v + 1] - scnt[v]) * 4;  // FP64 work of each list
    });
    // The lists in SELL-32 form, in thread order: slice s holds the lists of
    // threads 32 s .. 32 s + 31, entry j of lane l at off[s] + 32 j + l, every
    // list of a slice padded to the slice's longest (a warp's table loads are
    // then contiguous).  sell_fill calls put(dst, thread item, entry index, or
    // -1 for padding).
    auto sell_offsets = [](int64_t n, const std::vector<int32_t> &perm, const std::vector<int64_t> &csr) {
        const int64_t ns = (n + kSell - 1) / kSell;
        std::vector<int64_t> off(ns + 1, 0);
        for (int64_t sl = 0; sl < ns; ++sl) {
            int64_t mx = 0;
            for (int64_t i = sl * kSell; i < std::min(n, (sl + 1) * kSell); ++i)
                mx = std::max(mx, csr[perm[i] + 1] - csr[perm[i]]);
            off[sl + 1] = off[sl] + mx * kSell;
        }
        return off;
    };
    auto sell_fill = [](int64_t n, const std::vector<int32_t> &perm, const std::vector<int64_t> &csr,
                        const std::vector<int64_t> &off, const std::function<void(int64_t, int32_t, int64_t)> &put) {
        for (int64_t sl = 0; sl + 1 < (int64_t)off.size(); ++sl) {
            const int64_t len = (off[sl + 1] - off[sl]) / kSell;
            for (int64_t lane = 0; lane < kSell; ++lane) {
                const int64_t i = sl * kSell + lane;
                const int32_t item = i < n ? perm[i] : 0;
                const int64_t cnt = i < n ? csr[item + 1] - csr[item] : 0;
                for (int64_t j = 0; j < len; ++j) put(off[sl] + j * kSell + lane, item, j < cnt ? csr[item] + j : -1);
            }
        }
    };
    {
        const std::vector<int64_t> off = sell_offsets(ne, eperm, ecnt);
        std::vector<int32_t> sid(off.back(), 0);
        std::vector<double> swt(off.back(), 0.0);
        sell_fill(ne, eperm, ecnt, off, [&](int64_t d, int32_t, int64_t q) {
            if (q < 0) return;  // padding: weight 0 on vertex 0
            sid[d] = evid[q];
            swt[d] = ewt[q];
        });
        if ((st = m->upload(m->adj_eoff, off))) return st;
        if ((st = m->upload(m->adj_evid, sid))) return st;
        if ((st = m->upload(m->adj_ewt, swt))) return st;
    }
    {
        const std::vector<int64_t> off = sell_offsets(nv, vperm, vcnt), soff = sell_offsets(nv, vperm, scnt);
        std::vector<int32_t> sid(off.back(), 0);
        std::vector<double> swf(off.back(), 0.0), swg(off.back(), 0.0);
        std::vector<int64_t> sslot(soff.back(), 6 * ne);  // padding: the zero record after the 6 ne slot records
        sell_fill(nv, vperm, vcnt, off, [&](int64_t d, int32_t v, int64_t q) {
            sid[d] = q >= 0 ? vvid[q] : v;  // padding: weight 0 on the vertex itself
            if (q < 0) return;
            swf[d] = wf[q];
            swg[d] = wg[q];
        });
        sell_fill(nv, vperm, scnt, soff, [&](int64_t d, int32_t, int64_t q) {
            if (q >= 0) sslot[d] = slot[q];
        });
        if ((st = m->upload(m->adj_voff, off))) return st;
        if ((st = m->upload(m->adj_vvid, sid))) return st;
        if ((st = m->upload(m->adj_wf, swf))) return st;
        if ((st = m->upload(m->adj_wg, swg))) return st;
        if ((st = m->upload(m->adj_soff, soff))) return st;
        if ((st = m->upload(m->adj_slot, sslot))) return st;
    }
    if ((st = m->upload(m->adj_eperm, eperm))) return st;
    if ((st = m->upload(m->adj_vperm, vperm))) return st;
    if ((st = m->alloc(m->adj_lam_r, 4 * ne))) return st;
    // 6 ne slot records and one zero record that padded slot entries point at
    // (the edge-flux VJP writes only the first 6 ne)
    if ((st = m->alloc(m->adj_G, 6 * 4 * ne + 4))) return st;
    CK(cudaMemset(m->adj_G, 0, (6 * 4 * ne + 4) * sizeof(double)));
    if ((st = m->alloc(m->adj_S1, 4 * nv))) return st;
    for (int i = 0; i < 5; ++i)
        if ((st = m->alloc(m->adj_buf[i], 4 * nv))) return st;
    // transmissive ghosts grouped by donor (a Dirichlet ghost is its own
    // donor: its state is an input of its own, nothing to fold)
    {
        std::vector<std::pair<int32_t, int32_t>> dg;  // (donor, ghost), internal ids
        for (int64_t g = m->n_real; g < nv; ++g) {
            const int32_t o = T.v_new2old[g], od = T.ghost[o];
            if (od >= 0 && od != o) dg.push_back({T.v_old2new[od], (int32_t)g});
        }
        std::sort(dg.begin(), dg.end());
        std::vector<int32_t> donor, ghost;
        std::vector<int64_t> off{0};
        for (size_t i = 0; i < dg.size(); ++i) {
            if (donor.empty() || donor.back() != dg[i].first) {
                if (!donor.empty()) off.push_back((int64_t)ghost.size());
                donor.push_back(dg[i].first);
            }
            ghost.push_back(dg[i].second);
        }
        if (!donor.empty()) off.push_back((int64_t)ghost.size());
        m->adj_nfold = (int64_t)donor.size();
        if (m->adj_nfold > 0) {
            if ((st = m->upload(m->adj_fold_donor, donor))) return st;
            if ((st = m->upload(m->adj_fold_off, off))) return st;
            if ((st = m->upload(m->adj_fold_ghost, ghost))) return st;
        }
    }
    m->adj_ready = true;
    return FDU_OK;
}

// x <- (ghost fill)^T x (no-op without transmissive ghosts)
void fold_ghosts(fdu_mesh *m, double *x, cudaStream_t s) {
    launch_ghost_fold(x, m->adj_fold_donor, m->adj_fold_off, m->adj_fold_ghost, m->adj_nfold, s);
}

// out = (dL/dw)^T lam at state w (all internal order)
void enqueue_residual_vjp(fdu_mesh *m, const double *w, const double *lam, double *out, cudaStream_t s) {
    AdjEdgeArgs ea{};
    ea.sten = m->sten;
    ea.coef = m->coef64;
    ea.w = w;
    ea.lam_r = m->adj_lam_r;
    ea.lam_r_mut = m->adj_lam_r;
    ea.G = m->adj_G;
    ea.ne = m->ne_act;
    ea.gm1 = m->opts.gamma - 1.0;
    ea.eps = m->opts.weno_eps;
    ea.prec = m->adj_prec;
    if (m->adj_prec == 48) {
        const EdgeArgs e48 = edge_args(m, 48, w);
        ea.coefdw = e48.coefdw;
        for (int i = 0; i < 2; ++i) {
            ea.dw_gm1[i] = e48.dw_gm1[i];
            ea.dw_tenth[i] = e48.dw_tenth[i];
            ea.dw_eps[i] = e48.dw_eps[i];
        }
        ea.dw_eps_e = e48.dw_eps_e;
    }
    AdjTables t{m->adj_eoff, m->adj_evid, m->adj_ewt, m->adj_eperm};
    AdjVertexArgs va{};
    va.nv = m->nv;
    va.voff = m->adj_voff;
    va.vid = m->adj_vvid;
    va.wf = m->adj_wf;
    va.wg = m->adj_wg;
    va.lam = lam;
    va.w = w;
    va.gm1 = m->opts.gamma - 1.0;
    va.soff = m->adj_soff;
    va.slot = m->adj_slot;
    va.G = m->adj_G;
    va.grad = out;
    va.perm = m->adj_vperm;
    launch_residual_vjp(ea, t, va, s);
}

// lam_prev = (dw'/dw)^T lam_next for one SSP-RK3 step from the state wn
// (internal order; wn is not changed, ws and the stage flux buffers are, and
// lam_next is folded in place).
void enqueue_rk_step_vjp(fdu_mesh *m, double dt, double *lam_next, double *lam_prev, cudaStream_t s,
                         const double *S0 = nullptr, const double *S1 = nullptr, const double *S2 = nullptr) {
    const int64_t n4 = 4 * m->nv;
    double *t = m->adj_buf[2], *ls2 = m->adj_buf[3], *ls1 = m->adj_buf[4];
    if (!S0) {  // recompute the stage states from wn
        ensure_fluxes(m, m->adj_prec, s);
        enqueue_stages(m, m->adj_prec, dt, nullptr, s, false, 1, 1);
        cudaMemcpyAsync(m->adj_S1, m->ws, n4 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        enqueue_stages(m, m->adj_prec, dt, nullptr, s, false, 2, 2);  // ws = S2
        S0 = m->wn;
        S1 = m->adj_S1;
        S2 = m->ws;
    }
    // Each stage output is P(.), P the ghost fill (transmissive ghosts copy
    // their donors; Dirichlet ghosts keep their value, which the stage
    // combination of ghost rows with zero residual reproduces), so each
    // stage's cotangent goes through P^T (fold_ghosts, in place) first.
    // w' = P(1/3 S0 + 2/3 (S2 + dt L(S2)))
    fold_ghosts(m, lam_next, s);
    enqueue_residual_vjp(m, S2, lam_next, t, s);
    launch_axpby(ls2, 2.0 / 3.0, lam_next, 2.0 / 3.0 * dt, t, 0.0, nullptr, n4, s);
    // S2 = P(3/4 S0 + 1/4 (S1 + dt L(S1)))
    fold_ghosts(m, ls2, s);
    enqueue_residual_vjp(m, S1, ls2, t, s);
    launch_axpby(ls1, 0.25, ls2, 0.25 * dt, t, 0.0, nullptr, n4, s);
    // S1 = P(S0 + dt L(S0))
    fold_ghosts(m, ls1, s);
    enqueue_residual_vjp(m, S0, ls1, t, s);
    launch_axpby(lam_prev, 1.0 / 3.0, lam_next, 0.75, ls2, 1.0, ls1, n4, s);
    launch_axpby(lam_prev, 1.0, lam_prev, dt, t, 0.0, nullptr, n4, s);
    // S0 = P(w): the caller's ghost rows are overwritten by the fill
    fold_ghosts(m, lam_prev, s);
}

// One SSP-RK3 step of a batch: three cooperative persistent launches.
cudaError_t enqueue_step_persistent(fdu_mesh *m, int prec, cudaStream_t s, unsigned int expected,
                                    unsigned long long spin_limit) {
    for (int stage = 1; stage <= 3; ++stage) {
        const double *win = stage == 1 ? m->wn : m->ws;
        const bool f64 = fp64_state(prec);
        EdgeArgs ea = edge_args(m, prec, f64 ? (const void *)win : (const void *)m->w32);
        DivArgs a = div_args(m, prec, stage - 1);
        a.wn = m->wn;
        a.ws = win;
        a.wout = stage == 3 ? m->wn : m->ws;
        a.Fout = f64 ? (void *)m->F64[stage % 3] : (void *)m->F32[stage % 3];
        a.Qout = f64 ? m->Q64[stage % 3] : nullptr;
        if (f64) ea.Q = m->Q64[stage - 1];
        a.w32out = prec == 32 ? m->w32 : nullptr;
        a.comp = m->comp;
        a.dt_comp = m->dt_comp;
        cudaError_t e = launch_stage_persistent(prec, stage, ea, a, m->bar, m->bar + 1, expected, spin_limit,
                                                m->bar_err, m->pl_threads, m->pl_blocks, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One adaptive step: reduce the time-step bound on the device, finalise
// dt = min(cfl * bound, t_end - t) into tstate, then the three stages read
// dt from there (and skip their work once t_end is reached).
void enqueue_adaptive_step(fdu_mesh *m, int prec, double cfl, double t_end, cudaStream_t s) {
    launch_max_dt(m->wn, m->hmin, m->n_real, m->opts.gamma, m->counters + 2, s);
    launch_dt_finalize(m->counters + 2, m->tstate, cfl, t_end, m->counters + 3, s);
    enqueue_step(m, prec, 0.0, m->tstate + 1, s, false);
}

}  // namespace

// ====================================================================== no-allocation residual
// Scratch of fdu_residual_noalloc: the caller's state in internal order
// [FDU_NOALLOC_MAX_VERTICES][4], vertex fluxes [..][8] and edge fluxes
// [FDU_NOALLOC_MAX_EDGES][4], all FP64, in one array that every GPU loading
// the library holds until the process exits.
namespace {
constexpr int64_t kNoallocDoubles = 4 * (int64_t)FDU_NOALLOC_MAX_VERTICES + 8 * (int64_t)FDU_NOALLOC_MAX_VERTICES +
                                    4 * (int64_t)FDU_NOALLOC_MAX_EDGES;
static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

// Device address of the scratch array on the current device.  Looked up on
// every call: the lookup reads the loaded module's symbol table and
// allocates nothing, and it follows a context that was reset and created
// again (a cached address would then be stale).
fdu_status noalloc_scratch(double **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess)
        return set_err(FDU_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    *out = static_cast<double *>(p);
    return FDU_OK;
}
}  // namespace

// ====================================================================== C-ABI
extern "C" {

const char *fdu_version(void) { return "fdu 0.1 (sm_103a)"; }
const char *fdu_last_error(void) { return g_err.c_str(); }

fdu_status fdu_default_opts(fdu_mesh_opts *o) {
    if (!o) return set_err(FDU_ERR_ARG, "null opts");
    std::memset(o, 0, sizeof *o);
    o->Lx = 0;
    o->Ly = 0;
    o->weno_eps = 1e-40;
    o->weno_eps32 = 1e-30;
    o->gamma = 1.4;
    o->lsq_degree = 2;
    o->lsq_levels = 2;
    o->bc = FDU_BC_PERIODIC;
    o->renumber = 1;
    o->device = 0;
    o->host_threads = 0;
    o->ghost_donor = nullptr;
    o->positivity_alpha = 0.0;
    o->f32_coef = 0;
    return FDU_OK;
}

static fdu_status mesh_create(const double *xy, int64_t nv, const CellList &cells, int artificial,
                              const fdu_mesh_opts *opts, fdu_mesh **out) {
    if (out) *out = nullptr;
    if (!xy || !cells.off || !cells.vtx || !opts || !out) return set_err(FDU_ERR_ARG, "null argument");
    if (nv < 3 || cells.n < 1 || nv > INT32_MAX / 2) return set_err(FDU_ERR_ARG, "bad vertex or cell count");
    if (artificial < 0 || artificial > 2) return set_err(FDU_ERR_ARG, "artificial_edges must be 0, 1 or 2");
    if (opts->lsq_degree < 1 || opts->lsq_degree > 6 || opts->lsq_levels < 1 || opts->lsq_levels > 2)
        return set_err(FDU_ERR_ARG, "lsq_degree must be 1..6 and lsq_levels 1..2");
    if (!(opts->positivity_alpha >= 0.0 && opts->positivity_alpha < 1.0))
        return set_err(FDU_ERR_ARG, "positivity_alpha must be in [0, 1)");
    if (opts->f32_coef != 0 && opts->f32_coef != 1) return set_err(FDU_ERR_ARG, "f32_coef must be 0 or 1");
    if (!(opts->gamma > 1.0) || !(opts->weno_eps > 0) || !(opts->weno_eps32 > 0))
        return set_err(FDU_ERR_ARG, "gamma must be > 1 and the WENO epsilons > 0");
    if (opts->bc == FDU_BC_PERIODIC && !(opts->Lx > 0 && opts->Ly > 0))
        return set_err(FDU_ERR_ARG, "periodic meshes need Lx > 0 and Ly > 0");
    if (opts->bc == FDU_BC_TRANSMISSIVE && !opts->ghost_donor)
        return set_err(FDU_ERR_ARG, "transmissive meshes need ghost_donor");
    fdu_mesh *m = new (std::nothrow) fdu_mesh();
    if (!m) return set_err(FDU_ERR_ARG, "out of host memory");
    m->opts = *opts;
    m->opts.ghost_donor = nullptr;
    std::string err;
    int st = build_host_tables(xy, nv, cells, artificial, *opts, m->T, err);
    if (st != FDU_OK) {
        delete m;
        return set_err(st, err);
    }
    m->nv = nv;
    m->n_real = m->T.n_real;
    m->n_ghost = nv - m->T.n_real;
    m->ne_act = m->T.ne_active;
    m->device = opts->device;
    if (m->device >= 0) {
        cudaError_t e = cudaSetDevice(m->device);
        if (e == cudaSuccess) e = cudaStreamCreate(&m->own_stream);
        if (e != cudaSuccess) {
            delete m;
            return set_err(FDU_ERR_CUDA, std::string("device setup: ") + cudaGetErrorString(e));
        }
        st = upload_tables(m);
        if (st != FDU_OK) {
            std::string keep = g_err;
            m->release();
            delete m;
            return set_err(st, keep);
        }
    }
    *out = m;
    return FDU_OK;
}

fdu_status fdu_mesh_create(const double *xy, int64_t nv, const int32_t *tri, int64_t nt, const fdu_mesh_opts *opts,
                           fdu_mesh **out) {
    if (out) *out = nullptr;
    if (!tri) return set_err(FDU_ERR_ARG, "null argument");
    if (nt < 1) return set_err(FDU_ERR_ARG, "bad vertex or triangle count");
    std::vector<int64_t> off(nt + 1);
    for (int64_t t = 0; t <= nt; ++t) off[t] = 3 * t;
    return mesh_create(xy, nv, CellList{off.data(), tri, nt}, 0, opts, out);
}

fdu_status fdu_mesh_create_cells(const double *xy, int64_t nv, const int64_t *cell_off, const int32_t *cell_vtx,
                                 int64_t ncells, int artificial_edges, const fdu_mesh_opts *opts, fdu_mesh **out) {
    if (out) *out = nullptr;
    if (!cell_off || !cell_vtx || ncells < 1) return set_err(FDU_ERR_ARG, "null argument or no cells");
    if (cell_off[0] != 0) return set_err(FDU_ERR_ARG, "cell_off[0] must be 0");
    for (int64_t c = 0; c < ncells; ++c)
        if (cell_off[c + 1] < cell_off[c]) return set_err(FDU_ERR_ARG, "cell_off must be non-decreasing");
    return mesh_create(xy, nv, CellList{cell_off, cell_vtx, ncells}, artificial_edges, opts, out);
}

fdu_status fdu_mesh_destroy(fdu_mesh *m) {
    if (!m) return FDU_OK;
    m->release();
    delete m;
    return FDU_OK;
}

fdu_status fdu_mesh_info_get(const fdu_mesh *m, fdu_mesh_info *out) {
    if (!m || !out) return set_err(FDU_ERR_ARG, "null argument");
    std::memset(out, 0, sizeof *out);
    const HostTables &T = m->T;
    out->nv = T.nv;
    out->ne = T.ne;
    out->nt = T.nt;
    out->n_real = T.n_real;
    out->div_vert_nnz = (int64_t)T.vid.size();
    out->div_edge_nnz = (int64_t)T.eid.size();
    int32_t jmin = INT32_MAX, jmax = 0, kmin = INT32_MAX, kmax = 0;
    for (int64_t v = 0; v < T.nv; ++v) {
        if (!T.ghost.empty() && T.ghost[v] >= 0) continue;
        const int32_t J = (int32_t)(T.voff[v + 1] - T.voff[v]), K = (int32_t)(T.eoff[v + 1] - T.eoff[v]);
        jmin = std::min(jmin, J); jmax = std::max(jmax, J);
        kmin = std::min(kmin, K); kmax = std::max(kmax, K);
    }
    out->J_min = jmin; out->J_max = jmax; out->K_min = kmin; out->K_max = kmax;
    out->device_bytes = m->device_bytes;
    out->table_bytes_f64 = m->table_bytes_f64;
    out->table_bytes_f32 = m->table_bytes_f32;
    out->sell_width = kSell;
    out->sell_vert_nnz = m->vert_nnz_sell;
    out->sell_edge_nnz = m->edge_nnz_sell;
    out->sell_vert_nnz64 = m->vert_nnz_sell64;
    out->sell_edge_nnz64 = m->edge_nnz_sell64;
    return FDU_OK;
}

fdu_status fdu_get_edges(const fdu_mesh *m, int32_t *e) {
    if (!m || !e) return set_err(FDU_ERR_ARG, "null argument");
    std::memcpy(e, m->T.edge.data(), m->T.edge.size() * sizeof(int32_t));
    return FDU_OK;
}

fdu_status fdu_get_edge_stencils(const fdu_mesh *m, int32_t *s, double *xi) {
    if (!m) return set_err(FDU_ERR_ARG, "null mesh");
    if (s) std::memcpy(s, m->T.sten.data(), m->T.sten.size() * sizeof(int32_t));
    if (xi) std::memcpy(xi, m->T.xi.data(), m->T.xi.size() * sizeof(double));
    return FDU_OK;
}

fdu_status fdu_get_div_sizes(const fdu_mesh *m, int64_t *vn, int64_t *en) {
    if (!m || !vn || !en) return set_err(FDU_ERR_ARG, "null argument");
    *vn = (int64_t)m->T.vid.size();
    *en = (int64_t)m->T.eid.size();
    return FDU_OK;
}

fdu_status fdu_get_div_stencils(const fdu_mesh *m, int64_t *voff, int32_t *vid, double *wf, double *wg, int64_t *eoff,
                                int32_t *eid, double *we) {
    if (!m || !voff || !vid || !eoff || !eid) return set_err(FDU_ERR_ARG, "null argument");
    const HostTables &T = m->T;
    std::memcpy(voff, T.voff.data(), T.voff.size() * sizeof(int64_t));
    std::memcpy(eoff, T.eoff.data(), T.eoff.size() * sizeof(int64_t));
    std::memcpy(vid, T.vid.data(), T.vid.size() * sizeof(int32_t));
    std::memcpy(eid, T.eid.data(), T.eid.size() * sizeof(int32_t));
    if (wf) std::memcpy(wf, T.wf.data(), T.wf.size() * sizeof(double));
    if (wg) std::memcpy(wg, T.wg.data(), T.wg.size() * sizeof(double));
    if (we) std::memcpy(we, T.we.data(), T.we.size() * sizeof(double));
    return FDU_OK;
}

fdu_status fdu_set_state(fdu_mesh *m, const double *w, int on_device, void *stream) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!w) return set_err(FDU_ERR_ARG, "null state");
    cudaStream_t s = m->stream(stream);
    if (on_device) {
        launch_permute_rows(w, m->wn, m->new2old, m->nv, true, s);
        CK_LAUNCH();
    } else {
        // one copy of the caller's rows (a DMA when they are pinned), checked
        // and permuted to the internal order on the device; on a non-physical
        // row the state is left as it was
        const unsigned long long none = ~0ull;
        unsigned long long bad = none;
        CK(cudaMemcpyAsync(m->counters + 5, &none, sizeof none, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(m->scratch, w, 4 * m->nv * sizeof(double), cudaMemcpyHostToDevice, s));
        launch_check_rows(m->scratch, m->nv, m->counters + 5, s);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(&bad, m->counters + 5, sizeof bad, cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (bad != none)
            return set_err(FDU_ERR_NONPHYSICAL, "state row " + std::to_string(bad) + " has rho <= 0 or a non-finite value");
        launch_permute_rows(m->scratch, m->wn, m->new2old, m->nv, true, s);
        CK_LAUNCH();
    }
    if (m->n_ghost > 0) {
        launch_ghost_fill(m->wn, nullptr, nullptr, nullptr, 0, nullptr, m->donor, m->n_real, m->n_ghost, s);
        CK_LAUNCH();
    }
    m->f64_valid = m->f32_valid = false;
    CK(cudaMemsetAsync(m->tstate, 0, 3 * sizeof(double), s));
    CK(cudaMemsetAsync(m->counters + 3, 0, sizeof(unsigned long long), s));
    return FDU_OK;
}

fdu_status fdu_get_state(const fdu_mesh *mc, double *w, int on_device, void *stream) {
    fdu_mesh *m = const_cast<fdu_mesh *>(mc);
    fdu_status st = need_device(m);
    if (st) return st;
    if (!w) return set_err(FDU_ERR_ARG, "null state");
    cudaStream_t s = m->stream(stream);
    if (on_device) {
        launch_permute_rows(m->wn, w, m->new2old, m->nv, false, s);
        CK_LAUNCH();
    } else {
        launch_permute_rows(m->wn, m->scratch, m->new2old, m->nv, false, s);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(w, m->scratch, 4 * m->nv * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return FDU_OK;
}

fdu_status fdu_residual(fdu_mesh *m, int precision, double *dwdt, int on_device, void *stream) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!dwdt) return set_err(FDU_ERR_ARG, "null output");
    if ((st = check_precision(m, precision))) return st;
    cudaStream_t s = m->stream(stream);
    ensure_fluxes(m, precision, s);
    double *out = on_device ? dwdt : m->scratch;
    if (m->n_ghost > 0) CK(cudaMemsetAsync(out, 0, 4 * m->nv * sizeof(double), s));
    const int kd = prof_kind(precision);
    const bool f64 = fp64_state(precision);
    timed(m, kd, true, s, [&] {
        EdgeArgs ea = edge_args(m, precision, f64 ? (const void *)m->wn : (const void *)m->w32);
        ea.Q = f64 ? m->Q64[0] : nullptr;
        if (precision == 64) launch_edge_flux_f64(ea, s);
        else if (precision == 48) launch_edge_flux_dw(ea, s);
        else launch_edge_flux_f32(ea, s);
    });
    DivArgs a = div_args(m, precision, 0);
    a.out = out;
    a.out_map = m->new2old;
    timed(m, kd + 1, true, s, [&] {
        if (f64) launch_div_f64(a, 0, s);
        else launch_div_f32(a, 0, s);
    });
    CK_LAUNCH();
    if (!on_device) {
        CK(cudaMemcpyAsync(dwdt, m->scratch, 4 * m->nv * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return FDU_OK;
}

fdu_status fdu_max_dt(fdu_mesh *m, double cfl, double *dt, void *stream) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!dt || !(cfl > 0)) return set_err(FDU_ERR_ARG, "need cfl > 0 and an output pointer");
    cudaStream_t s = m->stream(stream);
    const unsigned long long inf_bits = 0x7FF0000000000000ull;
    CK(cudaMemcpyAsync(m->counters + 1, &inf_bits, sizeof inf_bits, cudaMemcpyHostToDevice, s));
    launch_max_dt(m->wn, m->hmin, m->n_real, m->opts.gamma, m->counters + 1, s);
    CK_LAUNCH();
    unsigned long long bits = 0;
    CK(cudaMemcpyAsync(&bits, m->counters + 1, sizeof bits, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double v;
    std::memcpy(&v, &bits, sizeof v);
    if (!(v > 0) || !std::isfinite(v)) return set_err(FDU_ERR_NONPHYSICAL, "non-physical state in the time-step bound");
    *dt = cfl * v;
    return FDU_OK;
}

fdu_status fdu_rk_step(fdu_mesh *m, double dt, int precision, void *stream) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!(dt > 0) || !std::isfinite(dt)) return set_err(FDU_ERR_ARG, "dt must be positive and finite");
    if ((st = check_precision(m, precision))) return st;
    cudaStream_t s = m->stream(stream);
    ensure_fluxes(m, precision, s);
    enqueue_step(m, precision, dt, nullptr, s, true);
    CK_LAUNCH();
    if (fp64_state(precision)) m->f32_valid = false;
    else m->f64_valid = false;
    return FDU_OK;
}

fdu_status fdu_rk_steps(fdu_mesh *m, double dt, int precision, int n_steps, void *stream) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!(dt > 0) || !std::isfinite(dt) || n_steps < 0) return set_err(FDU_ERR_ARG, "need dt > 0 and n_steps >= 0");
    if ((st = check_precision(m, precision))) return st;
    if (n_steps == 0) return FDU_OK;
    cudaStream_t s = m->stream(stream);
    ensure_fluxes(m, precision, s);
    CK_LAUNCH();
    auto key = std::make_pair(precision, dt);
    auto it = m->graphs.find(key);
    if (it == m->graphs.end()) {
        // capture on a blocking side stream (the legacy stream cannot be captured)
        cudaStream_t cs = m->own_stream;
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, s));
        CK(cudaStreamWaitEvent(cs, ev, 0));
        CK(cudaEventDestroy(ev));
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        enqueue_step(m, precision, dt, nullptr, cs, false);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t ge;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        it = m->graphs.emplace(key, ge).first;
    }
    for (int i = 0; i < n_steps; ++i) CK(cudaGraphLaunch(it->second, s));
    if (fp64_state(precision)) m->f32_valid = false;
    else m->f64_valid = false;
    return FDU_OK;
}

fdu_status fdu_advance(fdu_mesh *m, double cfl, double t_end, int precision, int64_t max_steps, int64_t *steps_done,
                       double *t_out, void *stream) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!(cfl > 0) || !std::isfinite(t_end) || max_steps < 0)
        return set_err(FDU_ERR_ARG, "need cfl > 0, a finite t_end and max_steps >= 0");
    if ((st = check_precision(m, precision))) return st;
    cudaStream_t s = m->stream(stream);
    ensure_fluxes(m, precision, s);
    CK_LAUNCH();
    const int batch = 8;
    auto key = std::make_tuple(precision, cfl, t_end);
    auto it = m->adaptive_graphs.find(key);
    if (it == m->adaptive_graphs.end()) {
        cudaStream_t cs = m->own_stream;
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, s));
        CK(cudaStreamWaitEvent(cs, ev, 0));
        CK(cudaEventDestroy(ev));
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        for (int i = 0; i < batch; ++i) enqueue_adaptive_step(m, precision, cfl, t_end, cs);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t ge;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        it = m->adaptive_graphs.emplace(key, ge).first;
    }
    double host[3] = {0, 0, 0};
    unsigned long long n0 = 0, n1 = 0;
    CK(cudaMemcpyAsync(&n0, m->counters + 3, sizeof n0, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(host, m->tstate, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    n1 = n0;
    while (host[0] < t_end && (int64_t)(n1 - n0) < max_steps && host[2] == 0.0) {
        const int64_t left = max_steps - (int64_t)(n1 - n0);
        if (left >= batch) {
            CK(cudaGraphLaunch(it->second, s));
        } else {
            for (int64_t i = 0; i < left; ++i) enqueue_adaptive_step(m, precision, cfl, t_end, s);
            CK_LAUNCH();
        }
        CK(cudaMemcpyAsync(&n1, m->counters + 3, sizeof n1, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(host, m->tstate, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (host[1] == 0.0 && host[0] < t_end && host[2] == 0.0) break;  // no progress
    }
    if (fp64_state(precision)) m->f32_valid = false;
    else m->f64_valid = false;
    if (steps_done) *steps_done = (int64_t)(n1 - n0);
    if (t_out) *t_out = host[0];
    if (host[2] != 0.0) return set_err(FDU_ERR_NONPHYSICAL, "non-physical state in the adaptive time step");
    return FDU_OK;
}

static fdu_status read_counter(fdu_mesh *m, int idx, int64_t *count, int reset, void *stream) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!count) return set_err(FDU_ERR_ARG, "null output");
    cudaStream_t s = m->stream(stream);
    unsigned long long c = 0;
    CK(cudaMemcpyAsync(&c, m->counters + idx, sizeof c, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (reset) CK(cudaMemsetAsync(m->counters + idx, 0, sizeof c, s));
    *count = (int64_t)c;
    return FDU_OK;
}

fdu_status fdu_fallback_count(fdu_mesh *m, int64_t *count, int reset, void *stream) {
    return read_counter(m, 0, count, reset, stream);
}

fdu_status fdu_limited_count(fdu_mesh *m, int64_t *count, int reset, void *stream) {
    return read_counter(m, 4, count, reset, stream);
}

fdu_status fdu_batch_create(int32_t n_meshes, const double *const *xy, const int64_t *nv, const int32_t *const *tri,
                            const int64_t *nt, const fdu_mesh_opts *opts, fdu_mesh **out) {
    if (out) *out = nullptr;
    if (n_meshes < 1) return set_err(FDU_ERR_ARG, "a batch needs at least one mesh");
    if (!xy || !nv || !tri || !nt || !opts || !out) return set_err(FDU_ERR_ARG, "null argument");
    if (opts->ghost_donor || opts->bc != FDU_BC_PERIODIC)
        return set_err(FDU_ERR_ARG, "batches hold periodic meshes (without ghost vertices)");
    if (opts->device < 0) return set_err(FDU_ERR_ARG, "batches need a device");
    if (opts->f32_coef != 0 && opts->f32_coef != 1) return set_err(FDU_ERR_ARG, "f32_coef must be 0 or 1");
    int64_t V = 0, T = 0;
    for (int i = 0; i < n_meshes; ++i) {
        if (!xy[i] || !tri[i] || nv[i] < 3 || nt[i] < 1) return set_err(FDU_ERR_ARG, "bad mesh " + std::to_string(i));
        V += nv[i];
        T += nt[i];
    }
    if (V > INT32_MAX / 2) return set_err(FDU_ERR_ARG, "batch too large");
    std::vector<double> uxy(2 * V);
    std::vector<int32_t> utri(3 * T), comp(V);
    std::vector<int64_t> voff(n_meshes + 1, 0);
    int64_t tv = 0, tt = 0;
    for (int i = 0; i < n_meshes; ++i) {
        voff[i] = tv;
        std::memcpy(&uxy[2 * tv], xy[i], 2 * nv[i] * sizeof(double));
        for (int64_t k = 0; k < 3 * nt[i]; ++k) {
            const int32_t q = tri[i][k];
            if (q < 0 || q >= nv[i]) return set_err(FDU_ERR_MESH, "mesh " + std::to_string(i) + ": bad vertex id");
            utri[3 * tt + k] = (int32_t)(q + tv);
        }
        for (int64_t k = 0; k < nv[i]; ++k) comp[tv + k] = i;
        tv += nv[i];
        tt += nt[i];
    }
    voff[n_meshes] = tv;
    fdu_mesh *m = new (std::nothrow) fdu_mesh();
    if (!m) return set_err(FDU_ERR_ARG, "out of host memory");
    m->opts = *opts;
    std::string err;
    int st = build_host_tables(uxy.data(), V, utri.data(), T, *opts, m->T, err, comp.data());
    if (st != FDU_OK) {
        delete m;
        return set_err(st, err);
    }
    m->nv = V;
    m->n_real = m->T.n_real;
    m->n_ghost = 0;
    m->ne_act = m->T.ne_active;
    m->device = opts->device;
    m->n_comp = n_meshes;
    m->comp_voff = voff;
    cudaError_t e = cudaSetDevice(m->device);
    if (e == cudaSuccess) e = cudaStreamCreate(&m->own_stream);
    if (e != cudaSuccess) {
        delete m;
        return set_err(FDU_ERR_CUDA, std::string("device setup: ") + cudaGetErrorString(e));
    }
    st = upload_tables(m);
    if (st == FDU_OK) {
        std::vector<int32_t> ci(m->n_real);
        for (int64_t v = 0; v < m->n_real; ++v) ci[v] = comp[m->T.v_new2old[v]];
        st = m->upload(m->comp, ci);
    }
    if (st == FDU_OK) st = m->alloc(m->dt_comp, n_meshes);
    if (st == FDU_OK) st = m->alloc(m->comp_slots, n_meshes);
    if (st == FDU_OK) st = m->alloc(m->bar, 2);
    if (st == FDU_OK) st = m->alloc(m->bar_err, 1);
    if (st == FDU_OK) {
        cudaMemset(m->dt_comp, 0, n_meshes * sizeof(double));
        cudaMemset(m->bar, 0, 2 * sizeof(unsigned int));
        cudaMemset(m->bar_err, 0, sizeof(int));
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device);
        m->pl_threads = 256;
        m->pl_blocks = sms * std::max(1, persistent_blocks_per_sm(32, 256));
        if (cudaGetLastError() != cudaSuccess) st = set_err(FDU_ERR_CUDA, "batch setup");
    }
    if (st != FDU_OK) {
        std::string keep = g_err;
        m->release();
        delete m;
        return set_err(st, keep);
    }
    *out = m;
    return FDU_OK;
}

fdu_status fdu_batch_info(const fdu_mesh *m, int32_t *n_meshes, int64_t *vertex_offsets) {
    if (!m || !n_meshes) return set_err(FDU_ERR_ARG, "null argument");
    *n_meshes = m->n_comp;
    if (vertex_offsets) std::memcpy(vertex_offsets, m->comp_voff.data(), m->comp_voff.size() * sizeof(int64_t));
    return FDU_OK;
}

static fdu_status need_batch(fdu_mesh *m) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (m->n_comp < 1) return set_err(FDU_ERR_ARG, "not a batch (use fdu_batch_create)");
    return FDU_OK;
}

fdu_status fdu_batch_max_dt(fdu_mesh *m, double cfl, double *dt, void *stream) {
    fdu_status st = need_batch(m);
    if (st) return st;
    if (!dt || !(cfl > 0)) return set_err(FDU_ERR_ARG, "need cfl > 0 and an output array");
    cudaStream_t s = m->stream(stream);
    std::vector<unsigned long long> bits(m->n_comp, 0x7FF0000000000000ull);
    CK(cudaMemcpyAsync(m->comp_slots, bits.data(), bits.size() * sizeof(bits[0]), cudaMemcpyHostToDevice, s));
    launch_max_dt(m->wn, m->hmin, m->n_real, m->opts.gamma, m->comp_slots, s, m->comp);
    CK_LAUNCH();
    CK(cudaMemcpyAsync(bits.data(), m->comp_slots, bits.size() * sizeof(bits[0]), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int i = 0; i < m->n_comp; ++i) {
        double v;
        std::memcpy(&v, &bits[i], sizeof v);
        if (!(v > 0) || !std::isfinite(v))
            return set_err(FDU_ERR_NONPHYSICAL, "non-physical state in mesh " + std::to_string(i));
        dt[i] = cfl * v;
    }
    return FDU_OK;
}

fdu_status fdu_batch_set_dt(fdu_mesh *m, const double *dt, void *stream) {
    fdu_status st = need_batch(m);
    if (st) return st;
    if (!dt) return set_err(FDU_ERR_ARG, "null dt");
    for (int i = 0; i < m->n_comp; ++i)
        if (!(dt[i] > 0) || !std::isfinite(dt[i])) return set_err(FDU_ERR_ARG, "dt must be positive and finite");
    cudaStream_t s = m->stream(stream);
    CK(cudaMemcpyAsync(m->dt_comp, dt, m->n_comp * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    return FDU_OK;
}

fdu_status fdu_batch_set_launch(fdu_mesh *m, int threads, int blocks_per_sm) {
    fdu_status st = need_batch(m);
    if (st) return st;
    if (threads != 128 && threads != 256 && threads != 512) return set_err(FDU_ERR_ARG, "threads must be 128, 256, 512");
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    const int occ = std::max(persistent_blocks_per_sm(64, threads), persistent_blocks_per_sm(32, threads));
    if (blocks_per_sm < 1 || blocks_per_sm > occ)
        return set_err(FDU_ERR_ARG, "blocks_per_sm must be 1.." + std::to_string(occ) + " at " +
                                        std::to_string(threads) + " threads");
    m->pl_threads = threads;
    m->pl_blocks = sms * blocks_per_sm;
    return FDU_OK;
}

static fdu_status check_barrier(fdu_mesh *m, cudaStream_t s) {
    int e = 0;
    CK(cudaMemcpyAsync(&e, m->bar_err, sizeof e, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (e) {
        CK(cudaMemsetAsync(m->bar, 0, 2 * sizeof(unsigned int), s));
        CK(cudaMemsetAsync(m->bar_err, 0, sizeof(int), s));
        CK(cudaStreamSynchronize(s));
        return set_err(FDU_ERR_TIMEOUT, "a grid barrier of the persistent stage kernel timed out");
    }
    return FDU_OK;
}

constexpr unsigned long long kSpinLimit = 1ull << 24;

fdu_status fdu_batch_rk_steps(fdu_mesh *m, int precision, int n_steps, void *stream) {
    fdu_status st = need_batch(m);
    if (st) return st;
    if (n_steps < 0) return set_err(FDU_ERR_ARG, "bad n_steps");
    if ((st = check_precision(m, precision))) return st;
    if (n_steps == 0) return FDU_OK;
    cudaStream_t s = m->stream(stream);
    const int occ = persistent_blocks_per_sm(precision, m->pl_threads);
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    if (occ < 1) return set_err(FDU_ERR_ARG, "the persistent kernel does not fit " + std::to_string(m->pl_threads) +
                                                 " threads per block at this precision");
    if (m->pl_blocks > occ * sms) m->pl_blocks = occ * sms;  // FP64 kernel holds more registers
    ensure_fluxes(m, precision, s);
    CK_LAUNCH();
    auto key = std::make_tuple(precision, m->pl_threads, m->pl_blocks);
    auto it = m->batch_graphs.find(key);
    if (it == m->batch_graphs.end()) {
        cudaStream_t cs = m->own_stream;
        cudaEvent_t ev;
        CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CK(cudaEventRecord(ev, s));
        CK(cudaStreamWaitEvent(cs, ev, 0));
        CK(cudaEventDestroy(ev));
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaError_t le = enqueue_step_persistent(m, precision, cs, (unsigned)m->pl_blocks, kSpinLimit);
        cudaError_t e = cudaStreamEndCapture(cs, &g);
        if (le != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("persistent launch: ") + cudaGetErrorString(le));
        if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        cudaGraphExec_t ge;
        e = cudaGraphInstantiate(&ge, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        it = m->batch_graphs.emplace(key, ge).first;
    }
    for (int i = 0; i < n_steps; ++i) CK(cudaGraphLaunch(it->second, s));
    if (fp64_state(precision)) m->f32_valid = false;
    else m->f64_valid = false;
    return check_barrier(m, s);
}

fdu_status fdu_batch_autotune(fdu_mesh *m, int precision, int *threads, int *blocks_per_sm, double *ms_per_step) {
    fdu_status st = need_batch(m);
    if (st) return st;
    if ((st = check_precision(m, precision))) return st;
    cudaStream_t s = m->own_stream;
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    // keep the caller's state: tuning steps run on a copy that is put back afterwards
    CK(cudaMemcpyAsync(m->scratch, m->wn, 4 * m->nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    double best = INFINITY;
    int bt = m->pl_threads, bb = m->pl_blocks / std::max(sms, 1);
    for (int t : {128, 256, 512}) {
        const int occ = persistent_blocks_per_sm(precision, t);
        for (int k = 1; k <= occ; ++k) {
            m->pl_threads = t;
            m->pl_blocks = k * sms;
            CK(cudaMemcpyAsync(m->wn, m->scratch, 4 * m->nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
            m->f64_valid = m->f32_valid = false;
            ensure_fluxes(m, precision, s);
            cudaError_t e = enqueue_step_persistent(m, precision, s, (unsigned)m->pl_blocks, kSpinLimit);
            if (e == cudaSuccess) e = cudaEventRecord(a, s);
            for (int r = 0; r < 3 && e == cudaSuccess; ++r)
                e = enqueue_step_persistent(m, precision, s, (unsigned)m->pl_blocks, kSpinLimit);
            if (e == cudaSuccess) e = cudaEventRecord(b, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            if (e != cudaSuccess) continue;  // launch shape not admissible: skip it
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            if (ms / 3.0 < best) {
                best = ms / 3.0;
                bt = t;
                bb = k;
            }
        }
    }
    cudaGetLastError();
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    m->pl_threads = bt;
    m->pl_blocks = bb * sms;
    CK(cudaMemcpyAsync(m->wn, m->scratch, 4 * m->nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaStreamSynchronize(s));
    m->f64_valid = m->f32_valid = false;
    st = check_barrier(m, s);
    if (st) return st;
    if (threads) *threads = bt;
    if (blocks_per_sm) *blocks_per_sm = bb;
    if (ms_per_step) *ms_per_step = best;
    return FDU_OK;
}

fdu_status fdu_batch_barrier_selftest(fdu_mesh *m, int *status) {
    fdu_status st = need_batch(m);
    if (st) return st;
    if (!status) return set_err(FDU_ERR_ARG, "null status");
    cudaStream_t s = m->own_stream;
    // stage 1 with one arrival more than the grid has: the barrier cannot
    // complete, every block gives up after a short bounded wait, and the
    // stage's update phase is skipped (the state is not touched)
    ensure_fluxes(m, 32, s);
    EdgeArgs ea = edge_args(m, 32, m->w32);
    DivArgs a = div_args(m, 32, 0);
    a.wn = m->wn;
    a.ws = m->wn;
    a.wout = m->ws;
    a.Fout = m->F32[1];
    a.w32out = m->w32;
    a.comp = m->comp;
    a.dt_comp = m->dt_comp;
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, m->device));
    const int nb = std::min(m->pl_blocks, persistent_blocks_per_sm(32, m->pl_threads) * sms);
    CK(launch_stage_persistent(32, 1, ea, a, m->bar, m->bar + 1, (unsigned)nb + 1, 20000, m->bar_err, m->pl_threads,
                               nb, s));
    // an ordinary step enqueued behind the failed launch, before the error is
    // read: each of its launches finds the flag set and returns at entry (it
    // neither arrives on the count the failed barrier left nor writes the state)
    const int keep_blocks = m->pl_blocks;
    m->pl_blocks = nb;
    CK(enqueue_step_persistent(m, 32, s, (unsigned)nb, kSpinLimit));
    m->pl_blocks = keep_blocks;
    m->f32_valid = false;  // w32 may hold nothing else than the state, but be conservative
    *status = check_barrier(m, s);
    return FDU_OK;
}

fdu_status fdu_residual_noalloc(const fdu_mesh *mc, const double *w, double *dwdt, void *stream) {
    fdu_mesh *m = const_cast<fdu_mesh *>(mc);
    fdu_status st = need_device(m);
    if (st) return st;
    if (!w || !dwdt) return set_err(FDU_ERR_ARG, "null state or output");
    if (m->nv > FDU_NOALLOC_MAX_VERTICES || m->ne_act > FDU_NOALLOC_MAX_EDGES)
        return set_err(FDU_ERR_ARG, "mesh has " + std::to_string(m->nv) + " vertices and " +
                                        std::to_string(m->ne_act) + " edges; fdu_residual_noalloc supports at most " +
                                        std::to_string(FDU_NOALLOC_MAX_VERTICES) + " and " +
                                        std::to_string(FDU_NOALLOC_MAX_EDGES));
    double *base = nullptr;
    st = noalloc_scratch(&base);  // need_device made the mesh's device current
    if (st) return st;
    double *wi = base;                                       // [MAX_V][4]
    double *F = base + 4 * (int64_t)FDU_NOALLOC_MAX_VERTICES;  // [MAX_V][8]
    double *r = F + 8 * (int64_t)FDU_NOALLOC_MAX_VERTICES;     // [MAX_E][4]
    // a null stream is the legacy default stream (not the mesh's own), so
    // serial calls with a null stream stay ordered across meshes
    cudaStream_t s = stream ? static_cast<cudaStream_t>(stream) : cudaStreamLegacy;
    // every scratch word read below is written first in this call; only the
    // ghost rows of the output must start at zero
    if (m->n_ghost > 0) CK(cudaMemsetAsync(dwdt, 0, 4 * m->nv * sizeof(double), s));
    launch_permute_rows(w, wi, m->new2old, m->nv, true, s);
    if (m->n_ghost > 0) launch_ghost_fill(wi, nullptr, nullptr, nullptr, 0, nullptr, m->donor, m->n_real, m->n_ghost, s);
    launch_vertex_flux_f64(wi, F, m->nv, m->opts.gamma, s);
    EdgeArgs ea = edge_args(m, 64, wi);
    ea.r = r;
    launch_edge_flux_f64(ea, s);
    DivArgs a = div_args(m, 64, 0);
    a.F = F;
    a.r = r;
    a.out = dwdt;
    a.out_map = m->new2old;
    launch_div_f64(a, 0, s);
    CK_LAUNCH();
    return FDU_OK;
}

static fdu_status to_internal(fdu_mesh *m, const double *x, int on_device, double *dst, cudaStream_t s) {
    if (on_device) {
        launch_permute_rows(x, dst, m->new2old, m->nv, true, s);
        CK_LAUNCH();
    } else {
        std::vector<double> h(4 * m->nv);
        for (int64_t i = 0; i < m->nv; ++i) std::memcpy(&h[4 * i], x + 4 * (int64_t)m->T.v_new2old[i], 32);
        CK(cudaMemcpyAsync(dst, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        CK(cudaStreamSynchronize(s));
    }
    return FDU_OK;
}

static fdu_status from_internal(fdu_mesh *m, const double *src, double *y, int on_device, cudaStream_t s) {
    if (on_device) {
        launch_permute_rows(src, y, m->new2old, m->nv, false, s);
        CK_LAUNCH();
    } else {
        launch_permute_rows(src, m->scratch, m->new2old, m->nv, false, s);
        CK_LAUNCH();
        CK(cudaMemcpyAsync(y, m->scratch, 4 * m->nv * sizeof(double), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
    }
    return FDU_OK;
}

fdu_status fdu_residual_vjp(fdu_mesh *m, const double *lam, double *grad, int on_device, void *stream) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!lam || !grad) return set_err(FDU_ERR_ARG, "null argument");
    if ((st = adjoint_setup(m))) return st;
    cudaStream_t s = m->stream(stream);
    if ((st = to_internal(m, lam, on_device, m->adj_buf[0], s))) return st;
    enqueue_residual_vjp(m, m->wn, m->adj_buf[0], m->adj_buf[1], s);
    fold_ghosts(m, m->adj_buf[1], s);  // the residual is taken at P(w)
    CK_LAUNCH();
    return from_internal(m, m->adj_buf[1], grad, on_device, s);
}

fdu_status fdu_rk_step_vjp(fdu_mesh *m, double dt, const double *lam_next, double *lam_prev, int on_device,
                           void *stream) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!lam_next || !lam_prev || !(dt > 0)) return set_err(FDU_ERR_ARG, "null argument or dt <= 0");
    if (m->opts.positivity_alpha > 0)
        return set_err(FDU_ERR_ARG, "the RK adjoint does not differentiate the stage positivity safeguard");
    if ((st = adjoint_setup(m))) return st;
    cudaStream_t s = m->stream(stream);
    if ((st = to_internal(m, lam_next, on_device, m->adj_buf[0], s))) return st;
    enqueue_rk_step_vjp(m, dt, m->adj_buf[0], m->adj_buf[1], s);
    CK_LAUNCH();
    m->f32_valid = false;
    return from_internal(m, m->adj_buf[1], lam_prev, on_device, s);
}

fdu_status fdu_adjoint_rk(fdu_mesh *m, double dt, int n_steps, int checkpoint_every, const double *lam_final,
                          double *grad, int on_device, void *stream) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!lam_final || !grad || !(dt > 0) || n_steps < 1 || checkpoint_every < 1)
        return set_err(FDU_ERR_ARG, "need dt > 0, n_steps >= 1, checkpoint_every >= 1 and both arrays");
    if (m->opts.positivity_alpha > 0)
        return set_err(FDU_ERR_ARG, "the RK adjoint does not differentiate the stage positivity safeguard");
    if ((st = adjoint_setup(m))) return st;
    cudaStream_t s = m->stream(stream);
    const int K = checkpoint_every, nseg = (n_steps + K - 1) / K;
    const size_t bytes = 4 * m->nv * sizeof(double);
    while ((int)m->adj_states.size() < nseg + 3 * K) {
        double *p = nullptr;
        if ((st = m->alloc(p, 4 * m->nv))) return st;
        m->adj_states.push_back(p);
    }
    double *const *ck = m->adj_states.data();          // checkpoints [nseg]
    double *const *stp = m->adj_states.data() + nseg;  // stage states of one segment [K][3]
    // steps i0..i1-1 from the current state, keeping every stage input of
    // the segment (the last step's third stage is not needed)
    auto segment_states = [&](int i0, int i1) -> cudaError_t {
        for (int i = i0; i < i1; ++i) {
            double *const *S = stp + 3 * (i - i0);
            cudaError_t e = cudaMemcpyAsync(S[0], m->wn, bytes, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return e;
            ensure_fluxes(m, m->adj_prec, s);
            enqueue_stages(m, m->adj_prec, dt, nullptr, s, false, 1, 1);
            if ((e = cudaMemcpyAsync(S[1], m->ws, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
            enqueue_stages(m, m->adj_prec, dt, nullptr, s, false, 2, 2);
            if ((e = cudaMemcpyAsync(S[2], m->ws, bytes, cudaMemcpyDeviceToDevice, s)) != cudaSuccess) return e;
            if (i + 1 < i1) enqueue_stages(m, m->adj_prec, dt, nullptr, s, false, 3, 3);
        }
        return cudaSuccess;
    };
    // forward pass from the current state w0, keeping a checkpoint every K
    // steps; the last segment keeps its stage inputs at once, so the reverse
    // pass recomputes only the segments before it
    const int last0 = (nseg - 1) * K;
    ensure_fluxes(m, m->adj_prec, s);
    for (int i = 0; i < last0; ++i) {
        if (i % K == 0) CK(cudaMemcpyAsync(ck[i / K], m->wn, bytes, cudaMemcpyDeviceToDevice, s));
        enqueue_step(m, m->adj_prec, dt, nullptr, s, false);
    }
    CK(cudaMemcpyAsync(ck[nseg - 1], m->wn, bytes, cudaMemcpyDeviceToDevice, s));
    CK(segment_states(last0, n_steps));
    CK_LAUNCH();
    // reverse pass, segment by segment
    double *lam = m->adj_buf[0], *lam_prev = m->adj_buf[1];
    if ((st = to_internal(m, lam_final, on_device, lam, s))) return st;
    for (int seg = nseg - 1; seg >= 0; --seg) {
        const int i0 = seg * K, i1 = std::min(n_steps, i0 + K);
        if (seg < nseg - 1) {  // recompute the segment from its checkpoint
            CK(cudaMemcpyAsync(m->wn, ck[seg], bytes, cudaMemcpyDeviceToDevice, s));
            m->f64_valid = false;
            CK(segment_states(i0, i1));
        }
        for (int i = i1 - 1; i >= i0; --i) {
            double *const *S = stp + 3 * (i - i0);
            enqueue_rk_step_vjp(m, dt, lam, lam_prev, s, S[0], S[1], S[2]);
            std::swap(lam, lam_prev);
        }
        CK(cudaMemcpyAsync(m->wn, stp[0], bytes, cudaMemcpyDeviceToDevice, s));
        m->f64_valid = false;
        CK_LAUNCH();
    }
    // the mesh state is w0 again (the first step state of the first segment)
    m->f64_valid = false;
    m->f32_valid = false;
    return from_internal(m, lam, grad, on_device, s);
}

static fdu_status check_special(int device, const double *x, double *y, int64_t n, int which) {
    if (!x || !y || n < 0) return set_err(FDU_ERR_ARG, "bad arguments");
    if (n == 0) return FDU_OK;
    CK(cudaSetDevice(device));
    double *d = nullptr;
    CK(cudaMalloc(&d, 2 * n * sizeof(double)));
    cudaError_t e = cudaMemcpy(d, x, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_recip_check(d, d + n, n, which, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(y, d + n, n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("accuracy check: ") + cudaGetErrorString(e));
    return FDU_OK;
}

fdu_status fdu_check_recip64(int device, const double *x, double *y, int64_t n) {
    return check_special(device, x, y, n, 0);
}

fdu_status fdu_check_rsqrt64(int device, const double *x, double *y, int64_t n) {
    return check_special(device, x, y, n, 1);
}

fdu_status fdu_check_scale2(int device, const double *x, double *y, int64_t n, int up) {
    return check_special(device, x, y, n, up ? 3 : 2);
}

fdu_status fdu_check_weno_coef32(int device, const double *xi, double *k, int64_t n) {
    if (!xi || !k || n < 0) return set_err(FDU_ERR_ARG, "bad arguments");
    std::vector<float> g(4 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        const double *x = xi + 6 * i;
        if (x[2] != -0.5 || x[3] != 0.5 || !(x[0] < x[1] && x[1] < x[2] && x[3] < x[4] && x[4] < x[5]))
            return set_err(FDU_ERR_ARG, "stencil coordinates of row " + std::to_string(i) +
                                            " are not increasing with L1 = -1/2 and R1 = 1/2");
        stencil_gaps(x, &g[4 * (size_t)i]);
    }
    if (n == 0) return FDU_OK;
    CK(cudaSetDevice(device));
    void *d = nullptr;
    CK(cudaMalloc(&d, (size_t)n * (4 + kCoefN) * sizeof(float)));
    float4 *dg = static_cast<float4 *>(d);
    float *dk = reinterpret_cast<float *>(dg + n);
    std::vector<float> kf((size_t)kCoefN * n);
    cudaError_t e = cudaMemcpy(dg, g.data(), g.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_weno_coef32_check(dg, dk, n, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(kf.data(), dk, kf.size() * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("coefficient check: ") + cudaGetErrorString(e));
    for (size_t i = 0; i < kf.size(); ++i) k[i] = kf[i];
    return FDU_OK;
}

fdu_status fdu_set_adjoint_precision(fdu_mesh *m, int precision) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (precision != 64 && precision != 48) return set_err(FDU_ERR_ARG, "adjoint precision must be 64 or 48");
    if (precision == 48 && (st = check_precision(m, 48))) return st;
    m->adj_prec = precision;
    return FDU_OK;
}

fdu_status fdu_check_dw(int device, int op, const double *x, const double *y, double *z, int64_t n) {
    if (!x || !y || !z || n < 0 || op < 0 || op > 7 || (op == 7 && n % 8 != 0))
        return set_err(FDU_ERR_ARG, "bad arguments");
    if (n == 0) return FDU_OK;
    CK(cudaSetDevice(device));
    double *d = nullptr;
    CK(cudaMalloc(&d, 3 * n * sizeof(double)));
    cudaError_t e = cudaMemcpy(d, x, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + n, y, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_dw_check(op, d, d + n, d + 2 * n, n, nullptr);
        e = cudaGetLastError();
    }
    const int64_t nz = op == 7 ? n / 8 : n;
    if (e == cudaSuccess) e = cudaMemcpy(z, d + 2 * n, nz * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("double-word check: ") + cudaGetErrorString(e));
    return FDU_OK;
}

fdu_status fdu_probe_fma(int device, int precision, double *tflops) {
    if (!tflops || (precision != 64 && precision != 32)) return set_err(FDU_ERR_ARG, "bad precision or output");
    CK(cudaSetDevice(device));
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    void *buf = nullptr;
    CK(cudaMalloc(&buf, (size_t)sms * 8 * 256 * 8));
    const double t = fma_probe_tflops(precision, sms, buf, nullptr);
    cudaError_t e = cudaGetLastError();
    cudaDeviceSynchronize();
    cudaFree(buf);
    if (e != cudaSuccess) return set_err(FDU_ERR_CUDA, std::string("fma probe: ") + cudaGetErrorString(e));
    *tflops = t;
    return FDU_OK;
}

fdu_status fdu_profile(fdu_mesh *m, int enable) {
    fdu_status st = need_device(m);
    if (st) return st;
    m->prof_on = enable != 0;
    return FDU_OK;
}

fdu_status fdu_profile_read(fdu_mesh *m, int kernel, int precision, double *total_ms, int64_t *launches, int reset) {
    fdu_status st = need_device(m);
    if (st) return st;
    if (!total_ms || !launches || (kernel != FDU_KERNEL_EDGE && kernel != FDU_KERNEL_DIV) ||
        (precision != 64 && precision != 32 && precision != 48))
        return set_err(FDU_ERR_ARG, "bad kernel kind, precision or output pointer");
    const int kind = prof_kind(precision) + kernel;
    double tot = 0;
    const size_t n = m->prof_used[kind];
    for (size_t i = 0; i < n; ++i) {
        cudaEvent_t a = m->prof_ev[kind][2 * i], b = m->prof_ev[kind][2 * i + 1];
        CK(cudaEventSynchronize(b));
        float ms = 0;
        CK(cudaEventElapsedTime(&ms, a, b));
        tot += ms;
    }
    *total_ms = tot;
    *launches = (int64_t)n;
    if (reset) m->prof_used[kind] = 0;
    return FDU_OK;
}

}  // extern "C"
