/*
 * fdu_oracle.c -- plain, slow, single-threaded FP64 reference of the
 * unstructured-mesh finite difference method of Zhen, Qu & Cai
 * ("A Novel Finite Difference Method for Euler Equations in 2D
 * Unstructured Meshes", arXiv 2102.12933).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this file's library.  It shares no
 * code, header, table or helper with the CUDA path.
 *
 * What it computes, in the paper's order:
 *   - Euler state, fluxes and equation of state (Section 2.1, Eq. 1);
 *   - the edge list and, per edge, the 1D curvilinear stencil of six
 *     vertices (Section 2.3.1, Fig. weno1d-tri) with its arc-length
 *     coordinate along Catmull-Rom curves (Section 2.3.1, Fig. curve_sten);
 *   - fifth-order non-uniform WENO interpolation of characteristic variables
 *     to the edge midpoint (Appendix, Eqs. u0-u2, C_K, smoothness
 *     indicators and nonlinear weights), then a Riemann flux projected on
 *     the edge direction (Section 2.3.1);
 *   - one- and two-level divergence stencils (Section 2.2.2) and the
 *     least-squares flux divergence by the SVD pseudo-inverse
 *     (Section 2.2.1, Eqs. ef, eg, eLinearSystem and the a1+b2 weights);
 *   - third-order TVD Runge-Kutta (Section 3, Shu & Osher);
 *   - directional derivatives of the residual and of RK steps by the
 *     complex step (the state arithmetic of fdu_oracle_state.h compiled a
 *     second time for double complex), the reference for the adjoint.
 *
 * Readings where the paper is silent (stencil-walk rule, curve tangents,
 * arc-length quadrature, Riemann solver, characteristic average, positivity
 * fallback, time step) are marked "Reading:" below.
 *
 * Parity status: every function here is pinned by the CPU tests
 * (polynomial reproduction, closed forms, exactness, convergence rates,
 * the paper's stencil figure and counts).  The stencil-walk rule, the
 * Catmull-Rom parametrisation, the Roe solver and the Roe average used
 * for characteristics are readings: the tests pin their properties, not
 * printed values.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OM_OK 0
#define OM_ERR_ARG -1
#define OM_ERR_MESH -2
#define OM_ERR_STENCIL -3
#define OM_ERR_RANK -4
#define OM_ERR_NONPHYSICAL -7
#define OM_ERR_NOMEM -8

static char om_err[512];
static int fail(int code, const char *msg) {
    snprintf(om_err, sizeof om_err, "%s", msg);
    return code;
}
const char *om_last_error(void) { return om_err; }

/* ------------------------------------------------------------------ */
/* Mesh                                                               */
/* ------------------------------------------------------------------ */
typedef struct om_mesh {
    int64_t nv, nt, ne;
    double Lx, Ly, gamma;
    int degree, levels;
    double *xy;       /* [nv][2] */
    int32_t *edge;    /* [ne][2], v0 < v1, sorted lexicographically */
    double *nrm;      /* [ne][2] unit(x_v1 - x_v0) */
    double *mid;      /* [ne][2] midpoint, x_v0 + d/2 */
    int64_t *adj_off; /* [nv+1] */
    int32_t *adj;     /* neighbour ids, ascending per vertex */
    int32_t *adj_e;   /* edge id of (v, adj) */
    int32_t *sten;    /* [ne][6]  L3 L2 L1 R1 R2 R3 */
    double *xi;       /* [ne][6]  normalised curve coordinates */
    int32_t *ghost;   /* [nv] donor id of ghost vertices (itself: Dirichlet), -1 for real ones (NULL = none) */
    /* divergence stencils (CSR over vertices) */
    int64_t *dv_off;
    int32_t *dv_id;
    int64_t *de_off;
    int32_t *de_id;
    /* LSQ weights, aligned with dv_id / de_id */
    double *wf, *wg, *we;
    uint8_t *has_w;   /* [nv] weights computed for this vertex */
    double pos_alpha; /* positivity safeguard of the stage update (0 = off) */
    int64_t pos_limited; /* vertices whose stage update was scaled */
} om_mesh;

static void disp(const om_mesh *m, int64_t a, int64_t b, double d[2]) {
    d[0] = m->xy[2 * b] - m->xy[2 * a];
    d[1] = m->xy[2 * b + 1] - m->xy[2 * a + 1];
    if (m->Lx > 0) d[0] -= m->Lx * rint(d[0] / m->Lx);
    if (m->Ly > 0) d[1] -= m->Ly * rint(d[1] / m->Ly);
}

static int cmp_pair(const void *p, const void *q) {
    const int32_t *a = (const int32_t *)p, *b = (const int32_t *)q;
    if (a[0] != b[0]) return a[0] < b[0] ? -1 : 1;
    if (a[1] != b[1]) return a[1] < b[1] ? -1 : 1;
    return 0;
}
static int cmp_i32(const void *p, const void *q) {
    int32_t a = *(const int32_t *)p, b = *(const int32_t *)q;
    return a < b ? -1 : (a > b ? 1 : 0);
}

/* edge id of the undirected pair (a, b), or -1 */
static int64_t find_edge(const om_mesh *m, int32_t a, int32_t b) {
    for (int64_t k = m->adj_off[a]; k < m->adj_off[a + 1]; ++k)
        if (m->adj[k] == b) return m->adj_e[k];
    return -1;
}
static int is_adjacent(const om_mesh *m, int32_t a, int32_t b) { return find_edge(m, a, b) >= 0; }

/* ------------------------------------------------------------------ */
/* 1D curvilinear stencil (Section 2.3.1, Fig. weno1d-tri)            */
/* Reading: from the current vertex c, reached along direction d,     */
/* take the unused neighbour q with the largest cosine                */
/* d.(x_q - x_c)/(|d||x_q - x_c|); cosines within 1e-12 of the best   */
/* so far do not replace it (neighbours scanned in ascending id, so   */
/* near-ties go to the smaller id).  The cosine must be positive.     */
/* ------------------------------------------------------------------ */
static int walk_step(const om_mesh *m, int32_t prev, int32_t cur, const int32_t *used, int nused, int32_t *next) {
    double d[2], e[2];
    disp(m, prev, cur, d);
    double dn = sqrt(d[0] * d[0] + d[1] * d[1]);
    int32_t best = -1;
    double sbest = 0;
    for (int64_t k = m->adj_off[cur]; k < m->adj_off[cur + 1]; ++k) {
        int32_t q = m->adj[k];
        int skip = 0;
        for (int u = 0; u < nused; ++u) skip |= (used[u] == q);
        if (skip) continue;
        disp(m, cur, q, e);
        double en = sqrt(e[0] * e[0] + e[1] * e[1]);
        double s = (d[0] * e[0] + d[1] * e[1]) / (dn * en);
        if (best < 0 || s > sbest + 1e-12) {
            best = q;
            sbest = s;
        }
    }
    if (best < 0 || !(sbest > 0)) return OM_ERR_STENCIL;
    *next = best;
    return OM_OK;
}

int om_walk_edge(const om_mesh *m, int64_t k, int32_t s[6]) {
    int32_t v0 = m->edge[2 * k], v1 = m->edge[2 * k + 1];
    int32_t used[6] = {v0, v1};
    int n = 2;
    int32_t r2, r3, l2, l3;
    /* right side first (from v1, away from v0), then left (from v0, away from v1) */
    if (walk_step(m, v0, v1, used, n, &r2)) return OM_ERR_STENCIL;
    used[n++] = r2;
    if (walk_step(m, v1, r2, used, n, &r3)) return OM_ERR_STENCIL;
    used[n++] = r3;
    if (walk_step(m, v1, v0, used, n, &l2)) return OM_ERR_STENCIL;
    used[n++] = l2;
    if (walk_step(m, v0, l2, used, n, &l3)) return OM_ERR_STENCIL;
    s[0] = l3; s[1] = l2; s[2] = v0; s[3] = v1; s[4] = r2; s[5] = r3;
    return OM_OK;
}

/* ------------------------------------------------------------------ */
/* Curve coordinate (Section 2.3.1, Fig. curve_sten).                 */
/* Reading: each side is two cubic Hermite segments.  Tangent at the  */
/* middle-edge end: the middle edge direction (pointing away from the */
/* edge) scaled by the first segment's chord; at the inner vertex the */
/* Catmull-Rom tangent (P2 - P0)/2; at the far end the last chord.    */
/* Arc length: 16-point Gauss-Legendre on each segment.  The 1D       */
/* coordinate is arc length from the edge midpoint, divided by the    */
/* middle edge length.                                                */
/* ------------------------------------------------------------------ */
static double gl_t[16], gl_w[16];
static int gl_ready = 0;

/* Gauss-Legendre nodes on [0,1] by Newton iteration on P_16 */
static void gl_init(void) {
    const int n = 16;
    for (int i = 0; i < n; ++i) {
        double x = cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        {
            double p0 = 1, p1 = x;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (x * p1 - p0) / (x * x - 1);
        }
        gl_t[i] = 0.5 * (1 - x);
        gl_w[i] = 1.0 / ((1 - x * x) * dp * dp); /* 2/((1-x^2)P'^2) on [-1,1], halved */
    }
    gl_ready = 1;
}

/* arc length of the cubic Hermite segment P0 -> P1 with tangents m0, m1 */
static double hermite_length(const double P0[2], const double P1[2], const double m0[2], const double m1[2]) {
    if (!gl_ready) gl_init();
    double s = 0;
    for (int g = 0; g < 16; ++g) {
        double t = gl_t[g];
        double h00 = 6 * t * t - 6 * t, h10 = 3 * t * t - 4 * t + 1, h01 = -6 * t * t + 6 * t, h11 = 3 * t * t - 2 * t;
        double dx = h00 * P0[0] + h10 * m0[0] + h01 * P1[0] + h11 * m1[0];
        double dy = h00 * P0[1] + h10 * m0[1] + h01 * P1[1] + h11 * m1[1];
        s += gl_w[g] * sqrt(dx * dx + dy * dy);
    }
    return s;
}

/* lengths along one side: A = middle-edge end, B, C = next two vertices,
 * O = the other end of the middle edge.  Returns s(A,B), s(B,C). */
static void side_lengths(const double O[2], const double A[2], const double B[2], const double C[2], double *sAB,
                         double *sBC) {
    double dir[2] = {A[0] - O[0], A[1] - O[1]};
    double dl = sqrt(dir[0] * dir[0] + dir[1] * dir[1]);
    double cab = sqrt((B[0] - A[0]) * (B[0] - A[0]) + (B[1] - A[1]) * (B[1] - A[1]));
    double mA[2] = {dir[0] / dl * cab, dir[1] / dl * cab};
    double mB[2] = {0.5 * (C[0] - A[0]), 0.5 * (C[1] - A[1])};
    double mC[2] = {C[0] - B[0], C[1] - B[1]};
    *sAB = hermite_length(A, B, mA, mB);
    *sBC = hermite_length(B, C, mB, mC);
}

/* P[6][2] = L3 L2 L1 R1 R2 R3 as unwrapped points -> xi[6] */
int om_curve_coords(const double *P, double *xi) {
    const double *L3 = P, *L2 = P + 2, *L1 = P + 4, *R1 = P + 6, *R2 = P + 8, *R3 = P + 10;
    double ell = sqrt((R1[0] - L1[0]) * (R1[0] - L1[0]) + (R1[1] - L1[1]) * (R1[1] - L1[1]));
    if (!(ell > 0)) return fail(OM_ERR_MESH, "zero-length middle edge");
    double sR1, sR2, sL1, sL2;
    side_lengths(L1, R1, R2, R3, &sR1, &sR2);
    side_lengths(R1, L1, L2, L3, &sL1, &sL2);
    xi[2] = -0.5;
    xi[3] = 0.5;
    xi[1] = -0.5 - sL1 / ell;
    xi[0] = xi[1] - sL2 / ell;
    xi[4] = 0.5 + sR1 / ell;
    xi[5] = xi[4] + sR2 / ell;
    return OM_OK;
}

static int stencil_points(const om_mesh *m, const int32_t s[6], double P[12]) {
    double d[2];
    /* unwrap along the stencil, L1 at the origin */
    P[4] = 0; P[5] = 0;
    disp(m, s[2], s[1], d); P[2] = d[0]; P[3] = d[1];
    disp(m, s[1], s[0], d); P[0] = P[2] + d[0]; P[1] = P[3] + d[1];
    disp(m, s[2], s[3], d); P[6] = d[0]; P[7] = d[1];
    disp(m, s[3], s[4], d); P[8] = P[6] + d[0]; P[9] = P[7] + d[1];
    disp(m, s[4], s[5], d); P[10] = P[8] + d[0]; P[11] = P[9] + d[1];
    return OM_OK;
}

/* ------------------------------------------------------------------ */
/* Non-uniform WENO5 (Appendix)                                        */
/* x[5] = x_{i-2}..x_{i+2} with (x_i + x_{i+1})/2 = 0; u[5] the values */
/* ------------------------------------------------------------------ */
/* Eqs. u0-u2: the three sub-stencil interpolants evaluated at 0 */
void om_substencil_coeffs(const double *x, double *lag /*[9]*/) {
    double xm2 = x[0], xm1 = x[1], x0 = x[2], xp1 = x[3], xp2 = x[4];
    double d0 = (xm1 - xm2) * (x0 - xm2) * (x0 - xm1);
    lag[0] = xm1 * x0 * (x0 - xm1) / d0;
    lag[1] = -xm2 * x0 * (x0 - xm2) / d0;
    lag[2] = xm2 * xm1 * (xm1 - xm2) / d0;
    double d1 = (x0 - xm1) * (xp1 - xm1) * (xp1 - x0);
    lag[3] = x0 * xp1 * (xp1 - x0) / d1;
    lag[4] = -xm1 * xp1 * (xp1 - xm1) / d1;
    lag[5] = x0 * xm1 * (x0 - xm1) / d1;
    double d2 = (xp1 - x0) * (xp2 - x0) * (xp2 - xp1);
    lag[6] = xp1 * xp2 * (xp2 - xp1) / d2;
    lag[7] = -x0 * xp2 * (xp2 - x0) / d2;
    lag[8] = xp1 * x0 * (xp1 - x0) / d2;
}

/* Eq. C_K: linear (optimal) weights */
void om_linear_weights(const double *x, double *C /*[3]*/) {
    double xm2 = x[0], xm1 = x[1], xp1 = x[3], xp2 = x[4];
    C[0] = xp1 * xp2 / ((xp1 - xm2) * (xp2 - xm2));
    C[1] = -xm2 * (-xm2 - xm1 + xp1 + xp2) * xp2 / ((xp1 - xm2) * (xp2 - xm2) * (xp2 - xm1));
    C[2] = xm2 * xm1 / ((xp2 - xm2) * (xp2 - xm1));
}

/* Eq. S5: the degree-4 interpolant over all five points, evaluated at 0,
 * as a plain Lagrange product (used by the tests only). */
void om_s5_coeffs(const double *x, double *l /*[5]*/) {
    for (int k = 0; k < 5; ++k) {
        double num = 1, den = 1;
        for (int m = 0; m < 5; ++m) {
            if (m == k) continue;
            num *= (0 - x[m]);
            den *= (x[k] - x[m]);
        }
        l[k] = num / den;
    }
}

/* ------------------------------------------------------------------ */
/* State-dependent arithmetic (fdu_oracle_state.h), instantiated twice.  */
/* REAL = double: the oracle.  REAL = double complex: complex-step       */
/* tangents (Squire & Trapp, SIAM Review 40(1), 1998): for a function F  */
/* analytic in the state, F(w + i h d) = F(w) + i h J d + O(h^2), so     */
/* Im F(w + i h d) / h is the directional derivative J d with no         */
/* subtraction, exact to rounding for h = 1e-30.  The complex copy takes */
/* every branch (positivity fallback, entropy-fix band, pivot choice) on */
/* real parts and uses the analytic |x| = sign(Re x) x, so its real part */
/* is the oracle's value and its derivative is that of the same branch.  */
/* ------------------------------------------------------------------ */
int om_build_weights(om_mesh *m, const uint8_t *mask);
#define OM_CAT2(a, b) a##b
#define OM_CAT(a, b) OM_CAT2(a, b)
#define OMS(name) OM_CAT(name, OM_SUFFIX)

#define OM_SUFFIX
#define REAL double
#define RE(x) (x)
#define SQRT(x) sqrt(x)
#define ABSV(x) fabs(x)
#define MAGR(x) fabs(x)
#include "fdu_oracle_state.h"
#undef OM_SUFFIX
#undef REAL
#undef RE
#undef SQRT
#undef ABSV
#undef MAGR

#define OM_SUFFIX _cs
#define REAL double complex
#define RE(x) creal(x)
#define SQRT(x) csqrt(x)
#define ABSV(x) (creal(x) < 0 ? -(x) : (x))
#define MAGR(x) fabs(creal(x))
#include "fdu_oracle_state.h"
#undef OM_SUFFIX
#undef REAL
#undef RE
#undef SQRT
#undef ABSV
#undef MAGR

/* exported for the tests: R (row-major 4x4) and its inverse */
int om_eigvec(const double *a, const double *b, const double *n, double gamma, double *Rout, double *Lout, double *lam) {
    double R[4][4], L[4][4];
    int st = roe_eigen(a, b, n, gamma, R, lam, NULL);
    if (st) return fail(st, "non-physical state in eigenvectors");
    if (inverse4(R, L)) return fail(OM_ERR_NONPHYSICAL, "singular eigenvector matrix");
    memcpy(Rout, R, sizeof R);
    memcpy(Lout, L, sizeof L);
    return OM_OK;
}

/* ------------------------------------------------------------------ */
/* Divergence stencils (Section 2.2.2)                                 */
/* one-level(O): N(O), the edges at O and the edges between members of  */
/* N(O).  two-level(O): union of one-level(j), j in N(O), minus O.      */
/* ------------------------------------------------------------------ */
typedef struct { int32_t *a; int64_t n, cap; } ivec;
static int ivec_push(ivec *v, int32_t x) {
    if (v->n == v->cap) {
        int64_t c = v->cap ? 2 * v->cap : 64;
        int32_t *p = (int32_t *)realloc(v->a, c * sizeof(int32_t));
        if (!p) return -1;
        v->a = p;
        v->cap = c;
    }
    v->a[v->n++] = x;
    return 0;
}
static void ivec_sort_unique(ivec *v) {
    if (!v->n) return;
    qsort(v->a, v->n, sizeof(int32_t), cmp_i32);
    int64_t o = 1;
    for (int64_t i = 1; i < v->n; ++i)
        if (v->a[i] != v->a[o - 1]) v->a[o++] = v->a[i];
    v->n = o;
}

static void one_level(const om_mesh *m, int32_t c, ivec *V, ivec *E) {
    for (int64_t k = m->adj_off[c]; k < m->adj_off[c + 1]; ++k) {
        int32_t a = m->adj[k];
        ivec_push(V, a);
        ivec_push(E, m->adj_e[k]);
        /* ring edges: a-b with both a, b neighbours of c */
        for (int64_t q = m->adj_off[a]; q < m->adj_off[a + 1]; ++q) {
            int32_t b = m->adj[q];
            if (b != c && is_adjacent(m, c, b)) ivec_push(E, m->adj_e[q]);
        }
    }
}

static int build_div_stencils(om_mesh *m) {
    ivec V = {0}, E = {0};
    int64_t nvtot = 0, netot = 0;
    int64_t *voff = (int64_t *)calloc(m->nv + 1, sizeof(int64_t));
    int64_t *eoff = (int64_t *)calloc(m->nv + 1, sizeof(int64_t));
    ivec allV = {0}, allE = {0};
    for (int32_t o = 0; o < m->nv; ++o) {
        V.n = 0;
        E.n = 0;
        if (m->ghost && m->ghost[o] >= 0) {
            voff[o + 1] = nvtot;
            eoff[o + 1] = netot;
            continue;
        }
        if (m->levels == 1) {
            one_level(m, o, &V, &E);
        } else {
            for (int64_t k = m->adj_off[o]; k < m->adj_off[o + 1]; ++k) one_level(m, m->adj[k], &V, &E);
        }
        ivec_sort_unique(&V);
        ivec_sort_unique(&E);
        for (int64_t i = 0; i < V.n; ++i)
            if (V.a[i] != o) { ivec_push(&allV, V.a[i]); ++nvtot; }
        for (int64_t i = 0; i < E.n; ++i) { ivec_push(&allE, E.a[i]); ++netot; }
        voff[o + 1] = nvtot;
        eoff[o + 1] = netot;
    }
    free(V.a);
    free(E.a);
    m->dv_off = voff;
    m->de_off = eoff;
    m->dv_id = allV.a ? allV.a : (int32_t *)malloc(4);
    m->de_id = allE.a ? allE.a : (int32_t *)malloc(4);
    m->wf = (double *)calloc(nvtot + 1, sizeof(double));
    m->wg = (double *)calloc(nvtot + 1, sizeof(double));
    m->we = (double *)calloc(netot + 1, sizeof(double));
    m->has_w = (uint8_t *)calloc(m->nv, 1);
    return OM_OK;
}

/* ------------------------------------------------------------------ */
/* Least squares (Section 2.2.1): A^+ by one-sided Jacobi SVD          */
/* ------------------------------------------------------------------ */
/* monomials of p(x,y) in the paper's order: x, y, x^2, xy, y^2, x^3, ... */
static int monomials(int degree, double x, double y, double *p) {
    int c = 0;
    for (int d = 1; d <= degree; ++d)
        for (int i = d; i >= 0; --i) p[c++] = pow(x, i) * pow(y, d - i);
    return c;
}

/* pseudo-inverse rows of A (m x n, column-major in A[j*m + i]) via
 * one-sided Jacobi: A = U S V^T, A^+ = V S^-1 U^T.  Returns rows r0 and r1
 * of A^+ summed into out[m].  Fails when sigma_min/sigma_max <= 1e-13. */
static int pinv_rows_sum(double *A, int m, int n, int r0, int r1, double *out) {
    double *V = (double *)calloc((size_t)n * n, sizeof(double));
    for (int j = 0; j < n; ++j) V[j * n + j] = 1;
    for (int sweep = 0; sweep < 60; ++sweep) {
        int rot = 0;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                double al = 0, be = 0, ga = 0;
                for (int i = 0; i < m; ++i) {
                    al += A[p * m + i] * A[p * m + i];
                    be += A[q * m + i] * A[q * m + i];
                    ga += A[p * m + i] * A[q * m + i];
                }
                if (fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
                rot = 1;
                double zeta = (be - al) / (2 * ga);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1 + zeta * zeta));
                double cs = 1 / sqrt(1 + t * t), sn = cs * t;
                for (int i = 0; i < m; ++i) {
                    double x = A[p * m + i], y = A[q * m + i];
                    A[p * m + i] = cs * x - sn * y;
                    A[q * m + i] = sn * x + cs * y;
                }
                for (int i = 0; i < n; ++i) {
                    double x = V[p * n + i], y = V[q * n + i];
                    V[p * n + i] = cs * x - sn * y;
                    V[q * n + i] = sn * x + cs * y;
                }
            }
        if (!rot) break;
    }
    double smax = 0, smin = INFINITY;
    double *sig = (double *)malloc(n * sizeof(double));
    for (int j = 0; j < n; ++j) {
        double s = 0;
        for (int i = 0; i < m; ++i) s += A[j * m + i] * A[j * m + i];
        sig[j] = sqrt(s);
        if (sig[j] > smax) smax = sig[j];
        if (sig[j] < smin) smin = sig[j];
    }
    if (!(smin > 1e-13 * smax)) {
        free(V);
        free(sig);
        return OM_ERR_RANK;
    }
    for (int i = 0; i < m; ++i) out[i] = 0;
    for (int j = 0; j < n; ++j) {
        /* column j of U is A[:,j]/sig_j; row r of A^+ = sum_j V[r][j]/sig_j U[:,j]^T */
        double c = (V[j * n + r0] + V[j * n + r1]) / (sig[j] * sig[j]);
        for (int i = 0; i < m; ++i) out[i] += c * A[j * m + i];
    }
    free(V);
    free(sig);
    return OM_OK;
}

static int lsq_vertex(om_mesh *m, int32_t o) {
    int64_t v0 = m->dv_off[o], J = m->dv_off[o + 1] - v0;
    int64_t e0 = m->de_off[o], K = m->de_off[o + 1] - e0;
    int M = m->degree * (m->degree + 3) / 2, n = 2 * M;
    int rows = (int)(2 * J + K);
    if (rows < n) return fail(OM_ERR_RANK, "divergence stencil has fewer conditions than unknowns");
    /* scale: monomials of degree d are evaluated at (x/h, y/h); the scaled
     * problem has A' = A S with S = diag(h^d), so the rows of A^+ for the
     * degree-1 unknowns a1 and b2 are those of A'^+ divided by h (exact for
     * full column rank). */
    double h = 0;
    for (int64_t j = 0; j < J; ++j) {
        double d[2];
        disp(m, o, m->dv_id[v0 + j], d);
        double r = sqrt(d[0] * d[0] + d[1] * d[1]);
        if (r > h) h = r;
    }
    double *A = (double *)calloc((size_t)rows * n, sizeof(double));
    double p[64];
    for (int64_t j = 0; j < J; ++j) {
        double d[2];
        disp(m, o, m->dv_id[v0 + j], d);
        monomials(m->degree, d[0] / h, d[1] / h, p);
        for (int c = 0; c < M; ++c) {
            A[c * rows + 2 * j] = p[c];
            A[(M + c) * rows + 2 * j + 1] = p[c];
        }
    }
    for (int64_t k = 0; k < K; ++k) {
        int32_t e = m->de_id[e0 + k];
        /* edge midpoint relative to o: o -> v0 of the edge, plus half the edge */
        double d[2], de[2];
        disp(m, o, m->edge[2 * e], d);
        disp(m, m->edge[2 * e], m->edge[2 * e + 1], de);
        double mx = d[0] + 0.5 * de[0], my = d[1] + 0.5 * de[1];
        monomials(m->degree, mx / h, my / h, p);
        for (int c = 0; c < M; ++c) {
            A[c * rows + 2 * J + k] = m->nrm[2 * e] * p[c];
            A[(M + c) * rows + 2 * J + k] = m->nrm[2 * e + 1] * p[c];
        }
    }
    double *wd = (double *)malloc(rows * sizeof(double));
    int st = pinv_rows_sum(A, rows, n, 0, M + 1, wd);
    free(A);
    if (st) {
        free(wd);
        return fail(OM_ERR_RANK, "rank-deficient least-squares system");
    }
    for (int64_t j = 0; j < J; ++j) {
        m->wf[v0 + j] = wd[2 * j] / h;
        m->wg[v0 + j] = wd[2 * j + 1] / h;
    }
    for (int64_t k = 0; k < K; ++k) m->we[e0 + k] = wd[2 * J + k] / h;
    free(wd);
    m->has_w[o] = 1;
    return OM_OK;
}

int om_build_weights(om_mesh *m, const uint8_t *mask) {
    for (int32_t o = 0; o < m->nv; ++o) {
        if (mask && !mask[o]) continue;
        if (m->ghost && m->ghost[o] >= 0) continue;
        if (m->has_w[o]) continue;
        int st = lsq_vertex(m, o);
        if (st) return st;
    }
    return OM_OK;
}

/* ------------------------------------------------------------------ */
/* Mesh construction                                                   */
/* ------------------------------------------------------------------ */
void om_destroy(om_mesh *m) {
    if (!m) return;
    free(m->xy); free(m->edge); free(m->nrm); free(m->mid);
    free(m->adj_off); free(m->adj); free(m->adj_e);
    free(m->sten); free(m->xi); free(m->ghost);
    free(m->dv_off); free(m->dv_id); free(m->de_off); free(m->de_id);
    free(m->wf); free(m->wg); free(m->we); free(m->has_w);
    free(m);
}

/* ghost: [nv] donor ids (-1 for real vertices) or NULL.  On a periodic
 * mesh every edge must have a 1D stencil.  On an open mesh, edges whose
 * walk runs into the boundary are marked with sten = -1; a residual that
 * needs such an edge fails with OM_ERR_STENCIL. */
/* Sorted unique (min id, max id) pairs, in place; returns the count. */
static int64_t unique_pairs(int32_t *pairs, int64_t n) {
    qsort(pairs, n, 2 * sizeof(int32_t), cmp_pair);
    int64_t ne = 0;
    for (int64_t i = 0; i < n; ++i)
        if (ne == 0 || cmp_pair(pairs + 2 * i, pairs + 2 * (ne - 1)) != 0) {
            pairs[2 * ne] = pairs[2 * i];
            pairs[2 * ne + 1] = pairs[2 * i + 1];
            ++ne;
        }
    return ne;
}

static int has_pair(const int32_t *pairs, int64_t n, int32_t a, int32_t b) {
    int32_t key[2] = {a < b ? a : b, a < b ? b : a};
    return bsearch(key, pairs, n, 2 * sizeof(int32_t), cmp_pair) != NULL;
}

static int cell_has(const int32_t *v, int64_t n, int32_t x) {
    for (int64_t i = 0; i < n; ++i)
        if (v[i] == x) return 1;
    return 0;
}

/* Reading of Section 2.2.2 (Figs. l1-hyb, l1-tria4): artificial edges.
 * Mode 1: both diagonals of every quadrilateral cell.  Mode 2: also, for
 * each vertex O whose one-level stencil counts fewer than p(p+3)
 * conditions (two per neighbour, one per edge at O, one per edge joining
 * two neighbours), an edge from O to the third vertex X of every triangle
 * that shares the side opposite O of one of O's triangles, unless X is
 * already a neighbour.  The candidates are found by scanning all cells
 * (slow and plain).  Returns the new pair array (caller frees) and count. */
static int32_t *artificial_pairs(int64_t nv, const int64_t *off, const int32_t *vtx, int64_t nc, int mode,
                                 int degree, int32_t *pairs, int64_t *np) {
    int64_t n = *np;
    if (mode >= 1) {
        int64_t nq = 0;
        for (int64_t c = 0; c < nc; ++c) nq += (off[c + 1] - off[c] == 4);
        pairs = (int32_t *)realloc(pairs, (n + 2 * nq) * 2 * sizeof(int32_t));
        for (int64_t c = 0; c < nc; ++c) {
            if (off[c + 1] - off[c] != 4) continue;
            const int32_t *v = vtx + off[c];
            for (int d = 0; d < 2; ++d) {
                int32_t a = v[d], b = v[d + 2];
                pairs[2 * n] = a < b ? a : b;
                pairs[2 * n + 1] = a < b ? b : a;
                ++n;
            }
        }
        n = unique_pairs(pairs, n);
    }
    if (mode >= 2) {
        const int64_t base = n;
        const int64_t need = (int64_t)degree * (degree + 3);
        for (int32_t o = 0; o < nv; ++o) {
            /* neighbours of o from the pair list */
            int64_t deg = 0, between = 0;
            int32_t *nb = (int32_t *)malloc(base * sizeof(int32_t));
            for (int64_t k = 0; k < base; ++k) {
                if (pairs[2 * k] == o) nb[deg++] = pairs[2 * k + 1];
                else if (pairs[2 * k + 1] == o) nb[deg++] = pairs[2 * k];
            }
            for (int64_t i = 0; i < deg; ++i)
                for (int64_t j = i + 1; j < deg; ++j) between += has_pair(pairs, base, nb[i], nb[j]);
            free(nb);
            if (2 * deg + deg + between >= need) continue;
            for (int64_t c = 0; c < nc; ++c) {
                if (off[c + 1] - off[c] != 3 || !cell_has(vtx + off[c], 3, o)) continue;
                const int32_t *v = vtx + off[c];
                int32_t A = -1, B = -1; /* the side opposite o */
                for (int i = 0; i < 3; ++i)
                    if (v[i] != o) {
                        if (A < 0) A = v[i];
                        else B = v[i];
                    }
                for (int64_t c2 = 0; c2 < nc; ++c2) {
                    if (c2 == c || off[c2 + 1] - off[c2] != 3) continue;
                    const int32_t *u = vtx + off[c2];
                    if (!cell_has(u, 3, A) || !cell_has(u, 3, B) || cell_has(u, 3, o)) continue;
                    int32_t X = -1;
                    for (int i = 0; i < 3; ++i)
                        if (u[i] != A && u[i] != B) X = u[i];
                    if (X < 0 || has_pair(pairs, base, o, X)) continue;
                    pairs = (int32_t *)realloc(pairs, (n + 1) * 2 * sizeof(int32_t));
                    pairs[2 * n] = o < X ? o : X;
                    pairs[2 * n + 1] = o < X ? X : o;
                    ++n;
                }
            }
        }
        n = unique_pairs(pairs, n);
    }
    *np = n;
    return pairs;
}

static int finish_mesh(om_mesh *m, int32_t *pairs, int64_t ne, om_mesh **out);
int om_create_cells(const double *xy, int64_t nv, const int64_t *off, const int32_t *vtx, int64_t nc, int artificial,
                    double Lx, double Ly, int degree, int levels, double gamma, const int32_t *ghost, om_mesh **out);

int om_create(const double *xy, int64_t nv, const int32_t *tri, int64_t nt, double Lx, double Ly, int degree,
              int levels, double gamma, const int32_t *ghost, om_mesh **out) {
    if (!tri || nt < 1) return fail(OM_ERR_ARG, "bad argument");
    int64_t *off = (int64_t *)malloc((nt + 1) * sizeof(int64_t));
    for (int64_t t = 0; t <= nt; ++t) off[t] = 3 * t;
    int r = om_create_cells(xy, nv, off, tri, nt, 0, Lx, Ly, degree, levels, gamma, ghost, out);
    free(off);
    return r;
}

int om_create_cells(const double *xy, int64_t nv, const int64_t *off, const int32_t *vtx, int64_t nc, int artificial,
                    double Lx, double Ly, int degree, int levels, double gamma, const int32_t *ghost, om_mesh **out) {
    if (!xy || !off || !vtx || nv < 3 || nc < 1 || degree < 1 || degree > 6 || levels < 1 || levels > 2 || !out ||
        artificial < 0 || artificial > 2)
        return fail(OM_ERR_ARG, "bad argument");
    om_mesh *m = (om_mesh *)calloc(1, sizeof(om_mesh));
    m->nv = nv; m->nt = nc; m->Lx = Lx; m->Ly = Ly; m->gamma = gamma; m->degree = degree; m->levels = levels;
    m->xy = (double *)malloc(nv * 2 * sizeof(double));
    memcpy(m->xy, xy, nv * 2 * sizeof(double));
    if (ghost) {
        m->ghost = (int32_t *)malloc(nv * sizeof(int32_t));
        memcpy(m->ghost, ghost, nv * sizeof(int32_t));
    }
    /* edges: unique undirected cell sides, (min id, max id), sorted */
    int64_t nside = off[nc];
    int32_t *pairs = (int32_t *)malloc((nside > 0 ? nside : 1) * 2 * sizeof(int32_t));
    for (int64_t c = 0; c < nc; ++c) {
        const int64_t k = off[c + 1] - off[c];
        if (k != 3 && k != 4) {
            free(pairs);
            om_destroy(m);
            return fail(OM_ERR_MESH, "cell with other than 3 or 4 vertices");
        }
        for (int64_t s = 0; s < k; ++s) {
            int32_t a = vtx[off[c] + s], b = vtx[off[c] + (s + 1) % k];
            if (a < 0 || a >= nv || b < 0 || b >= nv || a == b) {
                free(pairs);
                om_destroy(m);
                return fail(OM_ERR_MESH, "cell with a bad vertex id");
            }
            pairs[2 * (off[c] + s)] = a < b ? a : b;
            pairs[2 * (off[c] + s) + 1] = a < b ? b : a;
        }
    }
    int64_t ne = unique_pairs(pairs, nside);
    pairs = artificial_pairs(nv, off, vtx, nc, artificial, degree, pairs, &ne);
    return finish_mesh(m, pairs, ne, out);
}

/* Adjacency, edge geometry, 1D stencils and divergence stencils from the
 * sorted unique edge pairs (takes ownership of `pairs`). */
static int finish_mesh(om_mesh *m, int32_t *pairs, int64_t ne, om_mesh **out) {
    const int64_t nv = m->nv;
    const double Lx = m->Lx, Ly = m->Ly;
    m->ne = ne;
    m->edge = (int32_t *)malloc(ne * 2 * sizeof(int32_t));
    memcpy(m->edge, pairs, ne * 2 * sizeof(int32_t));
    free(pairs);
    /* adjacency, ascending neighbour ids */
    m->adj_off = (int64_t *)calloc(nv + 1, sizeof(int64_t));
    for (int64_t k = 0; k < ne; ++k) {
        m->adj_off[m->edge[2 * k] + 1]++;
        m->adj_off[m->edge[2 * k + 1] + 1]++;
    }
    for (int64_t v = 0; v < nv; ++v) m->adj_off[v + 1] += m->adj_off[v];
    m->adj = (int32_t *)malloc(2 * ne * sizeof(int32_t));
    m->adj_e = (int32_t *)malloc(2 * ne * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc(nv * sizeof(int64_t));
    for (int64_t v = 0; v < nv; ++v) fill[v] = m->adj_off[v];
    for (int64_t k = 0; k < ne; ++k) {
        int32_t a = m->edge[2 * k], b = m->edge[2 * k + 1];
        m->adj[fill[a]] = b; m->adj_e[fill[a]++] = (int32_t)k;
        m->adj[fill[b]] = a; m->adj_e[fill[b]++] = (int32_t)k;
    }
    free(fill);
    for (int64_t v = 0; v < nv; ++v) {
        /* insertion sort of (neighbour, edge) by neighbour id */
        for (int64_t i = m->adj_off[v] + 1; i < m->adj_off[v + 1]; ++i) {
            int32_t a = m->adj[i], e = m->adj_e[i];
            int64_t j = i - 1;
            while (j >= m->adj_off[v] && m->adj[j] > a) {
                m->adj[j + 1] = m->adj[j];
                m->adj_e[j + 1] = m->adj_e[j];
                --j;
            }
            m->adj[j + 1] = a;
            m->adj_e[j + 1] = e;
        }
    }
    /* edge geometry */
    m->nrm = (double *)malloc(ne * 2 * sizeof(double));
    m->mid = (double *)malloc(ne * 2 * sizeof(double));
    for (int64_t k = 0; k < ne; ++k) {
        double d[2];
        disp(m, m->edge[2 * k], m->edge[2 * k + 1], d);
        double l = sqrt(d[0] * d[0] + d[1] * d[1]);
        if (!(l > 0)) {
            om_destroy(m);
            return fail(OM_ERR_MESH, "zero-length edge");
        }
        m->nrm[2 * k] = d[0] / l;
        m->nrm[2 * k + 1] = d[1] / l;
        m->mid[2 * k] = m->xy[2 * m->edge[2 * k]] + 0.5 * d[0];
        m->mid[2 * k + 1] = m->xy[2 * m->edge[2 * k] + 1] + 0.5 * d[1];
    }
    /* 1D stencils and curve coordinates */
    m->sten = (int32_t *)malloc(ne * 6 * sizeof(int32_t));
    m->xi = (double *)malloc(ne * 6 * sizeof(double));
    for (int64_t k = 0; k < ne; ++k) {
        int32_t *s = m->sten + 6 * k;
        if (om_walk_edge(m, k, s) != OM_OK) {
            if (Lx > 0 && Ly > 0) {
                om_destroy(m);
                return fail(OM_ERR_STENCIL, "1D stencil walk found no forward neighbour");
            }
            for (int i = 0; i < 6; ++i) s[i] = -1;
            for (int i = 0; i < 6; ++i) m->xi[6 * k + i] = 0;
            continue;
        }
        double P[12];
        stencil_points(m, s, P);
        om_curve_coords(P, m->xi + 6 * k);
    }
    build_div_stencils(m);
    *out = m;
    return OM_OK;
}

int64_t om_num_edges(const om_mesh *m) { return m->ne; }
void om_get_edges(const om_mesh *m, int32_t *e) { memcpy(e, m->edge, m->ne * 2 * sizeof(int32_t)); }
void om_get_normals(const om_mesh *m, double *n) { memcpy(n, m->nrm, m->ne * 2 * sizeof(double)); }
void om_get_stencils(const om_mesh *m, int32_t *s, double *xi) {
    if (s) memcpy(s, m->sten, m->ne * 6 * sizeof(int32_t));
    if (xi) memcpy(xi, m->xi, m->ne * 6 * sizeof(double));
}
void om_div_sizes(const om_mesh *m, int64_t *nvert, int64_t *nedge) {
    *nvert = m->dv_off[m->nv];
    *nedge = m->de_off[m->nv];
}
void om_get_div(const om_mesh *m, int64_t *voff, int32_t *vid, double *wf, double *wg, int64_t *eoff, int32_t *eid,
                double *we) {
    memcpy(voff, m->dv_off, (m->nv + 1) * sizeof(int64_t));
    memcpy(eoff, m->de_off, (m->nv + 1) * sizeof(int64_t));
    memcpy(vid, m->dv_id, m->dv_off[m->nv] * sizeof(int32_t));
    memcpy(eid, m->de_id, m->de_off[m->nv] * sizeof(int32_t));
    if (wf) memcpy(wf, m->wf, m->dv_off[m->nv] * sizeof(double));
    if (wg) memcpy(wg, m->wg, m->dv_off[m->nv] * sizeof(double));
    if (we) memcpy(we, m->we, m->de_off[m->nv] * sizeof(double));
}

/* ------------------------------------------------------------------ */
/* Residual (Section 2.2.1): dw/dt = -(a1 + b2) per component          */
/* ------------------------------------------------------------------ */
void om_set_positivity(om_mesh *m, double alpha) { m->pos_alpha = alpha; }
/* Reading (the paper uses a CFL number without defining it):
 * dt = cfl * min over real vertices of h_v / (|u_v| + c_v), h_v the
 * shortest edge at v. */
double om_max_dt(const om_mesh *m, const double *w, double cfl) {
    double best = INFINITY;
    for (int64_t v = 0; v < m->nv; ++v) {
        if (m->ghost && m->ghost[v] >= 0) continue;
        double h = INFINITY;
        for (int64_t k = m->adj_off[v]; k < m->adj_off[v + 1]; ++k) {
            double d[2];
            disp(m, v, m->adj[k], d);
            double l = sqrt(d[0] * d[0] + d[1] * d[1]);
            if (l < h) h = l;
        }
        const double *s = w + 4 * v;
        double u = s[1] / s[0], vv = s[2] / s[0];
        double c = sqrt(m->gamma * pressure(s, m->gamma) / s[0]);
        double dt = h / (sqrt(u * u + vv * vv) + c);
        if (dt < best) best = dt;
    }
    return cfl * best;
}

/* smoothness indicators beta_0..2 of the left-state sub-stencils (tests) */
void om_smoothness_all(const double *x, const double *u, double *beta) {
    for (int k = 0; k < 3; ++k) beta[k] = smoothness(x + k, u + k, x[2], x[3]);
}

int64_t om_pos_limited(const om_mesh *m) { return m->pos_limited; }
