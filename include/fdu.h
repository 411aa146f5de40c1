/*
 * fdu.h -- C-ABI of the GB300 (sm_103a) residual and SSP-RK3 stage of the
 * unstructured-mesh finite difference method for the 2D Euler equations
 * (Zhen, Qu & Cai, arXiv 2102.12933).
 *
 * The calls follow the paper's statement of the problem: build the mesh
 * and its stencils from vertices and triangles, set the state, evaluate
 * the spatial residual dw/dt = -(df/dx + dg/dy) (Section 2.1, Eq. 1;
 * Section 2.2.1), and advance one third-order TVD Runge-Kutta step
 * (Section 3).
 *
 * Conventions common to every call
 *   - Every call returns an fdu_status: FDU_OK (0) or a negative error
 *     code.  No call aborts or exits.  fdu_last_error() returns a message
 *     for the calling thread's last error.
 *   - The library owns every object it creates; inputs are copied.
 *     Outputs go to caller-owned buffers of the stated size.
 *   - Vertex and edge ids in and out are ORIGINAL ids: vertex ids index
 *     the caller's xy array; edge ids index the edge list of
 *     fdu_get_edges (the unique cell sides and artificial edges (v0, v1),
 *     v0 < v1, sorted by (v0, v1)).  Any internal renumbering stays
 *     internal.
 *   - States are conservative records w[nv][4] = (rho, rho u, rho v,
 *     rho E), row-major FP64, with E = e + (u^2 + v^2)/2 and
 *     p = (gamma - 1) rho e (Section 2.1).
 *   - A pointer flagged `on_device = 1` is a raw CUDA device pointer on
 *     the mesh's device (for example torch.Tensor.data_ptr()); with
 *     `on_device = 0` it is host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls that take a stream are asynchronous on it unless
 *     they return a host value or write host memory.
 *   - Not thread-safe per mesh: serialise calls on one fdu_mesh.
 */
#ifndef FDU_H
#define FDU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int fdu_status;
#define FDU_OK 0
#define FDU_ERR_ARG (-1)            /* bad argument (null pointer, size, option) */
#define FDU_ERR_MESH (-2)           /* bad mesh: bad ids, degenerate, inverted or non-convex cell */
#define FDU_ERR_STENCIL (-3)        /* a 1D stencil walk found no forward neighbour */
#define FDU_ERR_RANK_DEFICIENT (-4) /* least-squares system with too few conditions or rank loss */
#define FDU_ERR_CUDA (-5)           /* a CUDA runtime call failed (message has the CUDA error) */
#define FDU_ERR_TIMEOUT (-6)        /* a bounded device wait ran out */
#define FDU_ERR_NONPHYSICAL (-7)    /* NaN, rho <= 0 or p <= 0 in a state */
#define FDU_ERR_NODEVICE (-8)       /* the call needs device tables but the mesh is host-only */

#define FDU_BC_PERIODIC 0
#define FDU_BC_TRANSMISSIVE 1

/* Options of fdu_mesh_create.  fdu_default_opts() fills the paper's
 * settings: NU-WENO5 with eps = 1e-40 and p = 1 (Appendix), two-level
 * divergence stencils (Section 3), gamma = 1.4 (Section 2.1). */
typedef struct fdu_mesh_opts {
    double Lx, Ly;      /* periodic lengths in x and y; 0 = not periodic */
    double weno_eps;    /* epsilon of the nonlinear weights (FP64 path) */
    double weno_eps32;  /* epsilon of the FP32 path (1e-40 is subnormal in FP32) */
    double gamma;       /* ratio of specific heats */
    int lsq_degree;     /* degree p of the least-squares polynomials, 1..6 */
    int lsq_levels;     /* divergence stencil: 1 = one-level, 2 = two-level */
    int bc;             /* FDU_BC_PERIODIC (Lx, Ly > 0, no ghosts) or FDU_BC_TRANSMISSIVE (ghost layers,
                           transmissive or Dirichlet per ghost; Lx or Ly may still be > 0 for a direction
                           that is periodic) */
    int renumber;       /* 1 = locality (Hilbert) renumbering of vertices and edges */
    int device;         /* CUDA device ordinal; -1 = host tables only (no GPU use) */
    int host_threads;   /* threads for host preprocessing; 0 = all cores */
    const int32_t *ghost_donor; /* ghost layers: [nv] -1 for a real vertex; for a ghost vertex the id of a real
                                   vertex whose state and fluxes it copies before every stage (transmissive), or
                                   its own id (Dirichlet: it keeps the state it was given); NULL = none */
    double positivity_alpha;    /* stage positivity safeguard: 0 = off (the paper's method); in (0,1): the
                                   forward-Euler part ws + theta dt L of each vertex's RK stage uses the
                                   largest theta in {1, 1/2, ..., 2^-20, 0} keeping rho and p at least alpha
                                   times the stage input's (the paper has no such safeguard) */
    int f32_coef;               /* NU-WENO5 coefficients of the FP32 path: 0 = the block built in FP64 on the host,
                                   rounded to FP32 and streamed (104 bytes per edge; the default); 1 = formed in
                                   FP32 by the FP32 edge kernel from the edge's four stencil gaps (24 bytes per
                                   edge with the normal; the gaps are built in FP64 on the host) */
} fdu_mesh_opts;

typedef struct fdu_mesh fdu_mesh;

typedef struct fdu_mesh_info {
    int64_t nv, ne, nt;      /* vertices, edges, cells (triangles for fdu_mesh_create) */
    int64_t n_real;          /* vertices that carry a residual (non-ghost) */
    int64_t div_vert_nnz;    /* vertex entries over all divergence stencils */
    int64_t div_edge_nnz;    /* edge entries over all divergence stencils */
    int32_t J_min, J_max, K_min, K_max; /* stencil sizes (vertex, edge entries) */
    int64_t device_bytes;    /* device memory held by the mesh */
    int64_t table_bytes_f64; /* bytes of the FP64 residual's read-only tables */
    int64_t table_bytes_f32; /* bytes of the FP32 residual's read-only tables */
    int32_t sell_width;      /* SELL slice width of the divergence tables */
    int32_t pad0;
    int64_t sell_vert_nnz;   /* vertex entries stored in the FP32 SELL tables (natural vertex order), padding
                                included (0 for host-only meshes) */
    int64_t sell_edge_nnz;   /* edge entries stored in the FP32 SELL tables, padding included */
    int64_t sell_vert_nnz64; /* the same for the FP64 SELL tables, whose slices take the vertices of each window
                                of 256 by decreasing stencil size */
    int64_t sell_edge_nnz64;
} fdu_mesh_info;

/* Library version string and thread-local last error message. */
const char *fdu_version(void);
const char *fdu_last_error(void);

/* Fill *opts with the defaults listed above (periodic lengths 0, device 0). */
fdu_status fdu_default_opts(fdu_mesh_opts *opts);

/* Build the mesh (Section 2.2.2, Section 2.3.1, Appendix, Section 2.2.1):
 * unique edges; per edge the six-vertex 1D curvilinear stencil and its
 * normalised arc-length coordinates; the non-uniform WENO5 coefficient
 * tables; per vertex the divergence stencil and its least-squares weights
 * (the a1 and b2 rows of the pseudo-inverse); all in FP64 on the host,
 * then uploaded to the device unless opts->device = -1.
 *   xy[nv][2] FP64 vertex coordinates; tri[nt][3] int32 vertex ids.
 * Errors: FDU_ERR_ARG, FDU_ERR_MESH, FDU_ERR_STENCIL,
 * FDU_ERR_RANK_DEFICIENT, FDU_ERR_CUDA.  On error *out is NULL. */
fdu_status fdu_mesh_create(const double *xy, int64_t nv, const int32_t *tri, int64_t nt, const fdu_mesh_opts *opts,
                           fdu_mesh **out);

/* The same from a hybrid mesh of triangles and quadrilaterals (Section
 * 2.2.2, Figs. l1-hyb and l1-tria4): cell c has the vertices
 * cell_vtx[cell_off[c] .. cell_off[c+1]-1] (3 or 4 of them, counter-
 * clockwise, convex), cell_off[0] = 0.  The edges are the cell sides plus,
 * by `artificial_edges`:
 *   0  none;
 *   1  both diagonals of every quadrilateral (the dashed edge of Fig. l1-hyb);
 *   2  as 1, and at every vertex O whose one-level stencil gives fewer than
 *      p(p+3) least-squares conditions (2 per neighbour, 1 per edge at O or
 *      between two neighbours; p = lsq_degree) an edge from O to the far
 *      apex of each triangle across the side of O's triangles opposite O,
 *      when that apex is not yet a neighbour (the dashed edges of Fig.
 *      l1-tria4).
 * Artificial edges are ordinary edges afterwards: they get 1D stencils and
 * fluxes and enter the divergence stencils.  Errors as fdu_mesh_create;
 * FDU_ERR_MESH for a cell of another size, a repeated vertex or a clockwise
 * or non-convex cell. */
fdu_status fdu_mesh_create_cells(const double *xy, int64_t nv, const int64_t *cell_off, const int32_t *cell_vtx,
                                 int64_t ncells, int artificial_edges, const fdu_mesh_opts *opts, fdu_mesh **out);

/* Free the mesh and its device memory (synchronises the device first). */
fdu_status fdu_mesh_destroy(fdu_mesh *mesh);

/* Sizes and stencil statistics. */
fdu_status fdu_mesh_info_get(const fdu_mesh *mesh, fdu_mesh_info *out);

/* Edge list e[ne][2] (original ids, v0 < v1, sorted). */
fdu_status fdu_get_edges(const fdu_mesh *mesh, int32_t *e);

/* Per edge (original edge order): the 1D stencil s[ne][6] = (L3, L2, L1 =
 * v0, R1 = v1, R2, R3) in original vertex ids and its normalised
 * coordinates xi[ne][6] (arc length from the edge midpoint divided by the
 * edge length, so xi[.][2] = -1/2 and xi[.][3] = 1/2).  Either pointer
 * may be NULL. */
fdu_status fdu_get_edge_stencils(const fdu_mesh *mesh, int32_t *s, double *xi);

/* Sizes of the divergence-stencil CSR. */
fdu_status fdu_get_div_sizes(const fdu_mesh *mesh, int64_t *vert_nnz, int64_t *edge_nnz);

/* Divergence stencils as CSR over original vertex ids, entries sorted by
 * original id: vertex part voff[nv+1], vid[vert_nnz], weights wf, wg
 * (multiplying f_j - f_O and g_j - g_O); edge part eoff[nv+1],
 * eid[edge_nnz], weight we (multiplying r_k - n_k . (f_O, g_O)).
 * Ghost vertices have empty rows.  Weight pointers may be NULL. */
fdu_status fdu_get_div_stencils(const fdu_mesh *mesh, int64_t *voff, int32_t *vid, double *wf, double *wg,
                                int64_t *eoff, int32_t *eid, double *we);

/* Copy a state w[nv][4] into / out of the mesh (original vertex order).
 * fdu_set_state from host memory (on_device = 0) copies the rows once (a
 * DMA transfer when they are pinned), checks them on the device and
 * synchronises `stream`: FDU_ERR_NONPHYSICAL names the first row with
 * rho <= 0 or a non-finite value, and the mesh keeps its previous state.
 * From device memory the rows are taken as they are, without the check.
 * Both reset the mesh time of fdu_advance to 0. */
fdu_status fdu_set_state(fdu_mesh *mesh, const double *w, int on_device, void *stream);
fdu_status fdu_get_state(const fdu_mesh *mesh, double *w, int on_device, void *stream);

/* Spatial residual dwdt[nv][4] = -(a1 + b2) per component of the current
 * state (Section 2.2.1), with edge fluxes from characteristic NU-WENO5
 * and a Roe flux (Section 2.3.1, Appendix).  precision = 64 computes in
 * FP64; precision = 32 reads FP32 copies of the state and tables and
 * computes in FP32; precision = 48 is the FP64 computation with the edge
 * flux's increments (characteristic projection, WENO, flux increment and
 * Roe dissipation) in double-word FP32 arithmetic (FP32 pairs, about 48
 * significant bits) and its state-sized terms (stencil differences, the
 * vertex flux at the edge's left end, the final sum) in FP64: the same
 * function to the FP64 path's tolerance, faster on parts whose FP64 rate
 * is a small fraction of their FP32 rate.  Its first use builds a
 * double-word copy of the edge coefficient block (192 bytes per edge).
 * Ghost vertices get 0.  With on_device = 0 the call synchronises `stream`
 * before returning.  The RK calls below accept the same three values. */
fdu_status fdu_residual(fdu_mesh *mesh, int precision, double *dwdt, int on_device, void *stream);

/* dt = cfl * min over real vertices of h_v / (|u_v| + c_v), h_v the
 * shortest edge at v, of the current state.  Synchronises `stream`. */
fdu_status fdu_max_dt(fdu_mesh *mesh, double cfl, double *dt, void *stream);

/* One SSP-RK3 step of the current state in place (Shu & Osher):
 * w1 = w + dt L(w); w2 = 3/4 w + 1/4 (w1 + dt L(w1));
 * w <- 1/3 w + 2/3 (w2 + dt L(w2)).  The state and the stage combination
 * stay FP64 for every precision; `precision` selects the residual.
 * dt > 0 is required. */
fdu_status fdu_rk_step(fdu_mesh *mesh, double dt, int precision, void *stream);

/* n_steps SSP-RK3 steps, captured once into a CUDA graph per (precision,
 * dt) and replayed. */
fdu_status fdu_rk_steps(fdu_mesh *mesh, double dt, int precision, int n_steps, void *stream);

/* Advance the current state with SSP-RK3 steps whose time step is computed
 * on the device before every step: dt = min(cfl * min_v h_v / (|u_v| +
 * c_v), t_end - t) (the CFL bound of fdu_max_dt), until the mesh time t
 * reaches t_end or max_steps steps were taken.  The mesh time starts at 0
 * at fdu_set_state.  Steps run as captured CUDA graphs of 8 steps; steps
 * past t_end do no work.  *steps_done (may be NULL) gets the steps taken by
 * this call and *t_out (may be NULL) the time reached.  Synchronises
 * `stream` once per 8 steps.  FDU_ERR_NONPHYSICAL if the bound is not
 * positive and finite. */
fdu_status fdu_advance(fdu_mesh *mesh, double cfl, double t_end, int precision, int64_t max_steps, int64_t *steps_done,
                       double *t_out, void *stream);

/* Vertex stage updates the positivity safeguard scaled (theta < 1), counted
 * since the last reset (reset = 1 zeroes it).  Synchronises `stream`. */
fdu_status fdu_limited_count(fdu_mesh *mesh, int64_t *count, int reset, void *stream);

/* ---- Batches: many independent periodic meshes advanced together ----
 * A batch is one fdu_mesh holding the disjoint union of n_meshes meshes
 * (same opts, in particular the same periodic lengths): mesh i's vertices
 * are rows vertex_offsets[i] .. vertex_offsets[i+1]-1 of every state array,
 * so fdu_set_state / fdu_get_state / fdu_residual work on the batch as on
 * one mesh.  fdu_batch_rk_steps advances every mesh with its own time step
 * in ONE cooperative persistent launch per RK stage (edge fluxes of all
 * meshes, a bounded grid barrier, then every vertex's divergence and stage
 * update), captured once into a CUDA graph per (precision, launch shape).
 * xy[i], tri[i], nv[i], nt[i] describe mesh i as for fdu_mesh_create.
 * Errors: FDU_ERR_ARG for n_meshes < 1, a null array, a mesh with fewer
 * than 3 vertices or no triangle, ghost vertices or non-periodic options,
 * or opts->device < 0 (batches live on a device); FDU_ERR_MESH and the
 * preprocessing errors of fdu_mesh_create for a bad member mesh. */
fdu_status fdu_batch_create(int32_t n_meshes, const double *const *xy, const int64_t *nv, const int32_t *const *tri,
                            const int64_t *nt, const fdu_mesh_opts *opts, fdu_mesh **out);
/* Number of meshes and vertex_offsets[n_meshes+1] (may be NULL). */
fdu_status fdu_batch_info(const fdu_mesh *batch, int32_t *n_meshes, int64_t *vertex_offsets);
/* dt[i] = cfl * (the bound of fdu_max_dt over mesh i) for the current state. */
fdu_status fdu_batch_max_dt(fdu_mesh *batch, double cfl, double *dt, void *stream);
/* Per-mesh time steps used by fdu_batch_rk_steps (host array [n_meshes]). */
fdu_status fdu_batch_set_dt(fdu_mesh *batch, const double *dt, void *stream);
/* n_steps SSP-RK3 steps of every mesh (FP64 state accumulation; the
 * residual at `precision`, 64, 48 or 32 as for fdu_residual; precision 48
 * runs a kernel of its own with its double-word staging in dynamic shared
 * memory).  FDU_ERR_TIMEOUT if a grid barrier's bounded wait ran out.  The
 * batch's state is then undefined: blocks that were still waiting may have
 * given up while the others went on with their part of that stage.  Every
 * later launch of the call finds the error flag set and returns without
 * work or arrival, so no later barrier can release on the count the failed
 * one left; the library resets the barrier before returning.  Set the
 * state again (fdu_set_state) before the next step. */
fdu_status fdu_batch_rk_steps(fdu_mesh *batch, int precision, int n_steps, void *stream);
/* Persistent launch shape: threads per block (128, 256 or 512) and
 * co-resident blocks per SM (1 .. the larger of the FP32 and FP64 stage
 * kernels' occupancy limits; a launch at a precision whose kernel fits fewer
 * blocks per SM uses its own limit).  FDU_ERR_ARG outside these ranges. */
fdu_status fdu_batch_set_launch(fdu_mesh *batch, int threads, int blocks_per_sm);
/* Autotuner: times one RK3 step of the batch for every admissible launch
 * shape (threads 128/256/512 x blocks per SM 1..occupancy) on a copy of the
 * current state, keeps the fastest, restores the state and returns the
 * choice and its time (any output pointer may be NULL). */
fdu_status fdu_batch_autotune(fdu_mesh *batch, int precision, int *threads, int *blocks_per_sm, double *ms_per_step);
/* Failure-path check of the bounded grid barrier: launches one persistent
 * stage whose barrier waits for one block more than the grid holds, so
 * every block's bounded wait runs out, then one ordinary RK3 step (three
 * persistent launches) before the error is read: those launches must find
 * the flag set and do nothing.  *status gets the resulting status
 * (FDU_ERR_TIMEOUT expected) and the state is left unchanged.  No GPU fault
 * or hang is involved: the wait is bounded and the kernel returns. */
fdu_status fdu_batch_barrier_selftest(fdu_mesh *batch, int *status);

/* ---- Adjoint (hand-written vector-Jacobian products, FP64, all single meshes) ----
 * Derivatives of the residual and the RK step as defined above, taking the
 * same branch as the forward pass at the piecewise choices (positivity
 * fallback, entropy-fix band, |lambda|); the WENO weights are
 * differentiable wherever beta_k + eps > 0.  Arrays are [nv][4] in original
 * vertex order, device (on_device = 1) or host pointers.
 * Ghost layers: the state is taken through the ghost fill first, so the
 * rows of a transmissive ghost carry nothing (its cotangent is added to its
 * donor's row) and the rows of a Dirichlet ghost are the derivative with
 * respect to its fixed value.  fdu_rk_step_vjp and fdu_adjoint_rk return
 * FDU_ERR_ARG when the stage positivity safeguard is on (positivity_alpha
 * > 0): the safeguard is not differentiated. */
/* Precision of the adjoint calls below: 64 (FP64, the default) or 48.  With
 * 48 the edge-flux VJP runs in double-word FP32 (the same derivative to about
 * 1e-13, on the FP32 pipes) and the steps that fdu_rk_step_vjp and
 * fdu_adjoint_rk take or recompute are precision-48 steps (the trajectory of
 * fdu_rk_step(..., 48)).  The first use of 48 builds its tables. */
fdu_status fdu_set_adjoint_precision(fdu_mesh *mesh, int precision);
/* grad = (dL/dw)^T lam at the current state. */
fdu_status fdu_residual_vjp(fdu_mesh *mesh, const double *lam, double *grad, int on_device, void *stream);
/* lam_prev = (dw_{n+1}/dw_n)^T lam_next for one SSP-RK3 step of size dt from
 * the current state (the state is not changed). */
fdu_status fdu_rk_step_vjp(fdu_mesh *mesh, double dt, const double *lam_next, double *lam_prev, int on_device,
                           void *stream);
/* Gradient with respect to the current state w0 of a function of the state
 * after n_steps SSP-RK3 steps of size dt, given lam_final = its gradient
 * with respect to that final state: grad = (dw_T/dw0)^T lam_final.  The
 * forward pass keeps a checkpoint every `checkpoint_every` = K steps and
 * the stage states of the last segment; the reverse pass recomputes the
 * stage states of each earlier segment from its checkpoint.  Device memory:
 * ceil(n_steps / K) + 3 K states of nv x 4 doubles (K >= n_steps: one
 * segment, nothing recomputed).  The gradient does not depend on K.  The
 * mesh state is w0 again afterwards. */
fdu_status fdu_adjoint_rk(fdu_mesh *mesh, double dt, int n_steps, int checkpoint_every, const double *lam_final,
                          double *grad, int on_device, void *stream);

/* Edges whose interpolated density or pressure was not positive and that
 * fell back to the first-order end states, counted since the last reset
 * (reset = 1 zeroes the counter after reading).  Synchronises `stream`. */
fdu_status fdu_fallback_count(fdu_mesh *mesh, int64_t *count, int reset, void *stream);

/* Kernel timing for measurement.  With enable = 1, every later
 * fdu_residual / fdu_rk_step records a CUDA event pair around each
 * edge-flux and divergence launch on the call's stream (CUDA-graph replays
 * of fdu_rk_steps are not instrumented).  fdu_profile_read synchronises the
 * recorded events and returns the summed device time (ms) and the launch
 * count of one kernel kind: FDU_KERNEL_EDGE or FDU_KERNEL_DIV at
 * precision 64, 48 or 32; reset = 1 clears that kind's record. */
#define FDU_KERNEL_EDGE 0
#define FDU_KERNEL_DIV 1
fdu_status fdu_profile(fdu_mesh *mesh, int enable);
fdu_status fdu_profile_read(fdu_mesh *mesh, int kernel, int precision, double *total_ms, int64_t *launches,
                            int reset);

/* FP64 residual that allocates no device memory, for callers that cannot
 * call cudaMalloc when they evaluate the residual: for example code that
 * runs under a host framework which has handed all device memory to its own
 * pool and forbids further allocations, or a time-critical loop that cannot
 * afford the implicit device synchronisation cudaMalloc may cause.  The
 * paper has no counterpart; it is the fdu_residual arithmetic (precision
 * 64) with its scratch (the state in internal order, vertex fluxes and
 * edge fluxes) in one fixed array inside the library instead of the mesh's
 * own buffers.  The mesh itself must already exist (fdu_mesh_create
 * allocates).
 *   w[nv][4]     device pointer, the state in original vertex order (input)
 *   dwdt[nv][4]  device pointer, the residual in original vertex order
 *                (output; ghost rows set to 0)
 * Limit: nv <= FDU_NOALLOC_MAX_VERTICES and active edges <=
 * FDU_NOALLOC_MAX_EDGES, otherwise FDU_ERR_ARG.  The array takes
 * 12.6 MB on every GPU that loads the library, for the life of the
 * process.  Each call looks up the array's device address with the mesh's
 * device current (a lookup in the already loaded module, no allocation),
 * so a context torn down and created again is followed.  A null stream is
 * the legacy default stream (cudaStreamLegacy), not the mesh's own stream,
 * so calls a caller issues one after the other from one thread with a
 * null stream are ordered even when they are for different meshes.  Every
 * call uses the same array, which keeps the last call's contents: calls
 * whose work overlaps on the GPU (on different non-null streams, or from
 * different threads) race on it and must be serialised by the caller.
 * The mesh's fallback counter still counts. */
#define FDU_NOALLOC_MAX_VERTICES 65536
#define FDU_NOALLOC_MAX_EDGES 196608
fdu_status fdu_residual_noalloc(const fdu_mesh *mesh, const double *w, double *dwdt, void *stream);

/* Accuracy check of the kernels' FP64 reciprocal (no counterpart in the
 * paper): y[i] = the reciprocal the WENO weights and Roe averages use, for
 * host arrays x[n] of positive normal doubles (Newton-Raphson refinement of
 * the hardware approximation); the tests compare it with IEEE division. */
fdu_status fdu_check_recip64(int device, const double *x, double *y, int64_t n);
/* The same for the kernels' FP64 reciprocal square root (sound speeds and
 * Roe weights): y[i] = 1/sqrt(x[i]) by Newton-Raphson refinement of the
 * hardware approximation, for host arrays of positive normal doubles. */
fdu_status fdu_check_rsqrt64(int device, const double *x, double *y, int64_t n);
/* The kernels' exact scalings by 2 and 1/2 on the integer pipe (no
 * counterpart in the paper): y[i] = 2 x[i] (up != 0) or x[i] / 2 (up == 0)
 * for host arrays of doubles.  Doubling is exact for every input (the top
 * binade overflows to infinity; infinities and NaN are unchanged); halving
 * is exact where the half is a normal double, leaves infinities and NaN
 * unchanged, and gives a zero of x's sign where the half is below the
 * normal range (|x| < 2^-1021). */
fdu_status fdu_check_scale2(int device, const double *x, double *y, int64_t n, int up);
/* Accuracy check of the FP32 path's NU-WENO5 coefficients (Appendix, Eqs.
 * u0-u2, the smoothness indicators and the linear weights C_K; no
 * counterpart in the paper as an entry point).  xi: host [n][6] stencil
 * coordinates of n edges as fdu_get_edge_stencils returns them (L3, L2, L1,
 * R1, R2, R3 along the curve, L1 = -1/2, R1 = 1/2, strictly increasing);
 * k: host [n][24] output, the coefficient block the FP32 edge kernel forms
 * in FP32 from the edge's four gaps, widened to double: per sub-stencil
 * S_a (L3, L2 against L1), S_b (L2, R1 against L1), S_c (R1, R2 against L1)
 * and S_d (R3, R2 against R1) its two value coefficients and the quadratic
 * form (m0, m1, m2) of its smoothness indicator in the same two
 * differences; then C_0/C_1 and C_2/C_1 of the left and of the right state.
 * FDU_ERR_ARG for null pointers, n < 0 or coordinates out of order. */
fdu_status fdu_check_weno_coef32(int device, const double *xi, double *k, int64_t n);
/* Accuracy check of the double-word primitives of precision 48 (no
 * counterpart in the paper).  Host arrays x[n], y[n]; each value is split
 * into a double word as the precision-48 kernels split FP64 inputs, `op`
 * is applied and the double-word result is returned exactly as a double:
 * 0 the split of x, 1 x + y (accurate sum), 2 x + y (sloppy sum), 3 x * y,
 * 4 x * y before renormalisation, 5 1/x, 6 1/sqrt(x) (x > 0 normal), 7 the
 * compensated dot product of each 8 consecutive pairs (n a multiple of 8;
 * z[n/8]).  FDU_ERR_ARG for a bad op or size. */
fdu_status fdu_check_dw(int device, int op, const double *x, const double *y, double *z, int64_t n);

/* Measurement helper with no counterpart in the paper: the FMA throughput
 * (TFLOP/s, FMA = 2 flops) of `device` at precision 64 or 32, from a short
 * kernel of independent FMA chains on every SM.  It is the ALU ceiling
 * that the FP64 residual is compared against.  Synchronises the device. */
fdu_status fdu_probe_fma(int device, int precision, double *tflops);

#ifdef __cplusplus
}
#endif
#endif /* FDU_H */
