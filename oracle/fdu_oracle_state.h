/*
 * fdu_oracle_state.h -- the oracle's state-dependent arithmetic: NU-WENO5
 * (Appendix), the Euler fluxes and the Roe solver (Section 2.1, Section
 * 2.3.1), the edge flux, the residual (Section 2.2.1) and the SSP-RK3 step
 * (Section 3).  TEST INFRASTRUCTURE ONLY, part of the oracle.
 *
 * fdu_oracle.c includes this file twice: with REAL = double it is the
 * oracle; with REAL = double complex it carries complex-step tangents
 * (see fdu_oracle.c).  It has no include guard on purpose.
 */
/* Smoothness indicator of a quadratic through (p[3], q[3]) on [a, b]:
 * sum_{l=1,2} int_a^b dx^{2l-1} (d^l u/dx^l)^2 dx with dx = b - a. */
static REAL OMS(smoothness)(const double *p, const REAL *q, double a, double b) {
    REAL A = 0, B = 0; /* u'(0) and u'' of the interpolating quadratic */
    for (int j = 0; j < 3; ++j) {
        double pa = p[(j + 1) % 3], pb = p[(j + 2) % 3];
        double D = (p[j] - pa) * (p[j] - pb);
        A += q[j] * (-(pa + pb)) / D;
        B += q[j] * 2.0 / D;
    }
    double dx = b - a;
    REAL i1 = A * A * (b - a) + A * B * (b * b - a * a) + B * B * (b * b * b - a * a * a) / 3.0;
    REAL i2 = B * B * (b - a);
    return dx * i1 + dx * dx * dx * i2;
}

/* Left-state interpolation at 0 (mode 0: nonlinear weights, 1: linear). */
REAL OMS(om_nuweno)(const double *x, const REAL *u, double eps, int mode) {
    double lag[9], C[3];
    REAL ut[3], beta[3];
    om_substencil_coeffs(x, lag);
    om_linear_weights(x, C);
    for (int k = 0; k < 3; ++k) {
        ut[k] = lag[3 * k] * u[k] + lag[3 * k + 1] * u[k + 1] + lag[3 * k + 2] * u[k + 2];
        beta[k] = OMS(smoothness)(x + k, u + k, x[2], x[3]);
    }
    if (mode == 1) return C[0] * ut[0] + C[1] * ut[1] + C[2] * ut[2];
    REAL alpha[3], sa = 0;
    for (int k = 0; k < 3; ++k) {
        alpha[k] = C[k] / (beta[k] + eps); /* p = 1 */
        sa += alpha[k];
    }
    REAL r = 0;
    for (int k = 0; k < 3; ++k) r += alpha[k] / sa * ut[k];
    return r;
}

/* ------------------------------------------------------------------ */
/* Euler (Section 2.1) and the Riemann flux                            */
/* ------------------------------------------------------------------ */
static REAL OMS(pressure)(const REAL *w, double g) {
    return (g - 1.0) * (w[3] - 0.5 * (w[1] * w[1] + w[2] * w[2]) / w[0]);
}
static void OMS(flux_fg)(const REAL *w, double g, REAL *f, REAL *gg) {
    REAL rho = w[0], u = w[1] / rho, v = w[2] / rho, p = OMS(pressure)(w, g);
    f[0] = rho * u; f[1] = rho * u * u + p; f[2] = rho * u * v; f[3] = (w[3] + p) * u;
    gg[0] = rho * v; gg[1] = rho * v * u; gg[2] = rho * v * v + p; gg[3] = (w[3] + p) * v;
}

/* Roe average of a and b, then the right eigenvectors of dF_n/dw as
 * columns (order: q_n - c, q_n (entropy), q_n (shear), q_n + c) and the
 * eigenvalues.  Reading: the paper names neither the average nor the
 * eigenvector normalisation. */
static int OMS(roe_eigen)(const REAL *a, const REAL *b, const double *n, double g, REAL R[4][4], REAL lam[4], REAL *cout) {
    REAL ra = a[0], rb = b[0];
    if (!(RE(ra) > 0) || !(RE(rb) > 0)) return OM_ERR_NONPHYSICAL;
    REAL ua = a[1] / ra, va = a[2] / ra, ub = b[1] / rb, vb = b[2] / rb;
    REAL Ha = (a[3] + OMS(pressure)(a, g)) / ra, Hb = (b[3] + OMS(pressure)(b, g)) / rb;
    REAL sa = SQRT(ra), sb = SQRT(rb);
    REAL u = (sa * ua + sb * ub) / (sa + sb);
    REAL v = (sa * va + sb * vb) / (sa + sb);
    REAL H = (sa * Ha + sb * Hb) / (sa + sb);
    REAL q2 = u * u + v * v;
    REAL c2 = (g - 1.0) * (H - 0.5 * q2);
    if (!(RE(c2) > 0)) return OM_ERR_NONPHYSICAL;
    REAL c = SQRT(c2);
    double nx = n[0], ny = n[1];
    REAL qn = u * nx + v * ny, qt = -u * ny + v * nx;
    REAL col[4][4] = {
        {1, u - c * nx, v - c * ny, H - c * qn},
        {1, u, v, 0.5 * q2},
        {0, -ny, nx, qt},
        {1, u + c * nx, v + c * ny, H + c * qn},
    };
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) R[i][j] = col[j][i];
    lam[0] = qn - c; lam[1] = qn; lam[2] = qn; lam[3] = qn + c;
    if (cout) *cout = c;
    return OM_OK;
}

/* Gauss-Jordan inverse with partial pivoting (a plain library-style step) */
static int OMS(inverse4)(REAL A[4][4], REAL X[4][4]) {
    REAL M[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) M[i][j] = j < 4 ? A[i][j] : (j - 4 == i);
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int i = col + 1; i < 4; ++i)
            if (MAGR(M[i][col]) > MAGR(M[piv][col])) piv = i;
        if (M[piv][col] == 0) return -1;
        if (piv != col)
            for (int j = 0; j < 8; ++j) { REAL t = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = t; }
        REAL inv = 1.0 / M[col][col];
        for (int j = 0; j < 8; ++j) M[col][j] *= inv;
        for (int i = 0; i < 4; ++i) {
            if (i == col) continue;
            REAL f = M[i][col];
            for (int j = 0; j < 8; ++j) M[i][j] -= f * M[col][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) X[i][j] = M[i][j + 4];
    return 0;
}

/* Reading (the paper does not name the solver for its method; Roe is the
 * one it pairs with WENO for WCNS in Section 3.2): Roe flux with Harten's
 * entropy fix |l| -> (l^2 + d^2)/(2d) for |l| < d, d = 0.1 c. */
int OMS(om_roe_flux)(const REAL *wl, const REAL *wr, const double *n, double g, REAL *out) {
    REAL R[4][4], L[4][4], lam[4], c;
    int st = OMS(roe_eigen)(wl, wr, n, g, R, lam, &c);
    if (st) return st;
    if (OMS(inverse4)(R, L)) return OM_ERR_NONPHYSICAL;
    REAL fl[4], gl[4], fr[4], gr[4];
    OMS(flux_fg)(wl, g, fl, gl);
    OMS(flux_fg)(wr, g, fr, gr);
    REAL dw[4], al[4];
    for (int i = 0; i < 4; ++i) dw[i] = wr[i] - wl[i];
    for (int k = 0; k < 4; ++k) {
        al[k] = 0;
        for (int j = 0; j < 4; ++j) al[k] += L[k][j] * dw[j];
    }
    REAL delta = 0.1 * c;
    for (int k = 0; k < 4; ++k) {
        REAL a = ABSV(lam[k]);
        if (RE(a) < RE(delta)) a = (lam[k] * lam[k] + delta * delta) / (2 * delta);
        lam[k] = a;
    }
    for (int i = 0; i < 4; ++i) {
        REAL diss = 0;
        for (int k = 0; k < 4; ++k) diss += lam[k] * al[k] * R[i][k];
        REAL fn_l = n[0] * fl[i] + n[1] * gl[i];
        REAL fn_r = n[0] * fr[i] + n[1] * gr[i];
        out[i] = 0.5 * (fn_l + fn_r) - 0.5 * diss;
    }
    return OM_OK;
}

/* ------------------------------------------------------------------ */
/* Edge flux: characteristic NU-WENO5 + Roe (Section 2.3.1, Appendix)  */
/* Reading: characteristics at the Roe average of the two edge end     */
/* states; the right state uses the mirrored stencil.  Positivity      */
/* reading: if an interpolated density or pressure is not positive,    */
/* the edge falls back to the end states (first order) and is counted. */
/* ------------------------------------------------------------------ */
static int OMS(edge_flux)(const om_mesh *m, const REAL *w, int64_t k, double eps, REAL *r, int *fallback) {
    const int32_t *s = m->sten + 6 * k;
    const double *xi = m->xi + 6 * k;
    const REAL *W[6];
    for (int i = 0; i < 6; ++i) W[i] = w + 4 * (int64_t)s[i];
    const double *n = m->nrm + 2 * k;
    REAL R[4][4], L[4][4], lam[4];
    int st = OMS(roe_eigen)(W[2], W[3], n, m->gamma, R, lam, NULL);
    if (st) return st;
    if (OMS(inverse4)(R, L)) return OM_ERR_NONPHYSICAL;
    REAL ch[6][4];
    for (int i = 0; i < 6; ++i)
        for (int f = 0; f < 4; ++f) {
            ch[i][f] = 0;
            for (int j = 0; j < 4; ++j) ch[i][f] += L[f][j] * W[i][j];
        }
    double xl[5] = {xi[0], xi[1], xi[2], xi[3], xi[4]};
    double xr[5] = {-xi[5], -xi[4], -xi[3], -xi[2], -xi[1]};
    REAL cl[4], cr[4];
    for (int f = 0; f < 4; ++f) {
        REAL ul[5] = {ch[0][f], ch[1][f], ch[2][f], ch[3][f], ch[4][f]};
        REAL ur[5] = {ch[5][f], ch[4][f], ch[3][f], ch[2][f], ch[1][f]};
        cl[f] = OMS(om_nuweno)(xl, ul, eps, 0);
        cr[f] = OMS(om_nuweno)(xr, ur, eps, 0);
    }
    REAL wl[4], wr[4];
    for (int i = 0; i < 4; ++i) {
        wl[i] = 0;
        wr[i] = 0;
        for (int f = 0; f < 4; ++f) {
            wl[i] += R[i][f] * cl[f];
            wr[i] += R[i][f] * cr[f];
        }
    }
    *fallback = 0;
    if (!(RE(wl[0]) > 0) || !(RE(wr[0]) > 0) || !(RE(OMS(pressure)(wl, m->gamma)) > 0) ||
        !(RE(OMS(pressure)(wr, m->gamma)) > 0)) {
        memcpy(wl, W[2], sizeof wl);
        memcpy(wr, W[3], sizeof wr);
        *fallback = 1;
    }
    return OMS(om_roe_flux)(wl, wr, n, m->gamma, r);
}

/* r[ne][4] for edges with emask[k] (NULL = all) */
int OMS(om_edge_fluxes)(const om_mesh *m, const REAL *w, double eps, const uint8_t *emask, REAL *r, int64_t *nfallback) {
    int64_t nf = 0;
    for (int64_t k = 0; k < m->ne; ++k) {
        if (emask && !emask[k]) continue;
        if (m->sten[6 * k] < 0) return fail(OM_ERR_STENCIL, "an edge in a divergence stencil has no 1D stencil");
        int fb = 0;
        int st = OMS(edge_flux)(m, w, k, eps, r + 4 * k, &fb);
        if (st) return fail(st, "non-physical state in an edge flux");
        nf += fb;
    }
    if (nfallback) *nfallback = nf;
    return OM_OK;
}

/* ghost fill: a transmissive ghost copies its donor (reading); a ghost
 * that is its own donor is a Dirichlet vertex and keeps its state */
void OMS(om_fill_ghosts)(const om_mesh *m, REAL *w) {
    if (!m->ghost) return;
    for (int64_t v = 0; v < m->nv; ++v)
        if (m->ghost[v] >= 0 && m->ghost[v] != v) memcpy(w + 4 * v, w + 4 * (int64_t)m->ghost[v], 4 * sizeof(REAL));
}

/* dwdt[nv][4] at vertices with vmask[v] (NULL = all real vertices);
 * w must already hold the ghost states.  The edge fluxes needed are
 * computed from scratch. */
int OMS(om_residual)(om_mesh *m, const REAL *w, double eps, const uint8_t *vmask, REAL *dwdt, int64_t *nfallback) {
    int st = om_build_weights(m, vmask);
    if (st) return st;
    uint8_t *emask = (uint8_t *)calloc(m->ne, 1);
    for (int64_t o = 0; o < m->nv; ++o) {
        if (vmask && !vmask[o]) continue;
        for (int64_t i = m->de_off[o]; i < m->de_off[o + 1]; ++i) emask[m->de_id[i]] = 1;
    }
    REAL *r = (REAL *)calloc(m->ne * 4, sizeof(REAL));
    st = OMS(om_edge_fluxes)(m, w, eps, emask, r, nfallback);
    if (st) { free(emask); free(r); return st; }
    for (int64_t o = 0; o < m->nv; ++o) {
        if (vmask && !vmask[o]) continue;
        if (m->ghost && m->ghost[o] >= 0) { for (int c = 0; c < 4; ++c) dwdt[4 * o + c] = 0; continue; }
        REAL f0[4], g0[4], fj[4], gj[4];
        OMS(flux_fg)(w + 4 * o, m->gamma, f0, g0);
        REAL div[4] = {0, 0, 0, 0};
        for (int64_t i = m->dv_off[o]; i < m->dv_off[o + 1]; ++i) {
            OMS(flux_fg)(w + 4 * (int64_t)m->dv_id[i], m->gamma, fj, gj);
            for (int c = 0; c < 4; ++c) div[c] += m->wf[i] * (fj[c] - f0[c]) + m->wg[i] * (gj[c] - g0[c]);
        }
        for (int64_t i = m->de_off[o]; i < m->de_off[o + 1]; ++i) {
            int32_t e = m->de_id[i];
            for (int c = 0; c < 4; ++c)
                div[c] += m->we[i] * (r[4 * e + c] - (m->nrm[2 * e] * f0[c] + m->nrm[2 * e + 1] * g0[c]));
        }
        for (int c = 0; c < 4; ++c) dwdt[4 * o + c] = -div[c];
    }
    free(emask);
    free(r);
    return OM_OK;
}

/* SSP-RK3 stage combination (Shu & Osher), stage = 1, 2, 3:
 *   1: out = wn + dt L
 *   2: out = 3/4 wn + 1/4 (ws + dt L)
 *   3: out = 1/3 wn + 2/3 (ws + dt L)                                  */
void OMS(om_stage_combine)(int64_t n, int stage, const REAL *wn, const REAL *ws, const REAL *L, double dt, REAL *out) {
    for (int64_t i = 0; i < n; ++i) {
        if (stage == 1) out[i] = wn[i] + dt * L[i];
        else if (stage == 2) out[i] = 0.75 * wn[i] + 0.25 * (ws[i] + dt * L[i]);
        else out[i] = (1.0 / 3.0) * wn[i] + (2.0 / 3.0) * (ws[i] + dt * L[i]);
    }
}

/* Positivity safeguard of a stage (a reading: the paper has none, its Sod
 * run overshoots).  The forward-Euler part fe = ws + theta dt L of each
 * vertex's stage uses the largest theta in {1, 1/2, ..., 2^-20, 0} with
 * rho(fe) >= alpha rho(ws) and p(fe) >= alpha p(ws); the stage is then the
 * SSP combination of w_n and fe, which stays physical because the set of
 * physical states is convex.  Returns the number of limited vertices. */
static int64_t OMS(pos_limit)(const om_mesh *m, int64_t nv, const REAL *ws, const REAL *L, double dt, REAL *fe) {
    int64_t lim = 0;
    for (int64_t v = 0; v < nv; ++v) {
        const REAL *s = ws + 4 * v;
        const REAL *l = L + 4 * v;
        REAL *f = fe + 4 * v;
        if (m->ghost && m->ghost[v] >= 0) {
            for (int c = 0; c < 4; ++c) f[c] = s[c] + dt * l[c];
            continue;
        }
        REAL ps = OMS(pressure)(s, m->gamma);
        double theta = 1.0;
        int ok = 0;
        for (int k = 0; k <= 20; ++k) {
            for (int c = 0; c < 4; ++c) f[c] = s[c] + theta * dt * l[c];
            if (RE(f[0]) >= m->pos_alpha * RE(s[0]) && RE(OMS(pressure)(f, m->gamma)) >= m->pos_alpha * RE(ps)) {
                ok = 1;
                break;
            }
            theta *= 0.5;
        }
        if (!ok) {
            theta = 0.0;
            for (int c = 0; c < 4; ++c) f[c] = s[c];
        }
        lim += theta < 1.0;
    }
    return lim;
}


/* one SSP-RK3 step in place on w[nv][4] */
int OMS(om_rk3_step)(om_mesh *m, REAL *w, double dt, double eps, int64_t *nfallback) {
    int64_t n = m->nv * 4, nf = 0, f;
    REAL *wn = (REAL *)malloc(n * sizeof(REAL));
    REAL *L = (REAL *)malloc(n * sizeof(REAL));
    REAL *ws = (REAL *)malloc(n * sizeof(REAL));
    memcpy(wn, w, n * sizeof(REAL));
    memcpy(ws, w, n * sizeof(REAL));
    int st = OM_OK;
    for (int stage = 1; stage <= 3 && st == OM_OK; ++stage) {
        OMS(om_fill_ghosts)(m, ws);
        st = OMS(om_residual)(m, ws, eps, NULL, L, &f);
        nf += f;
        if (st) break;
        if (m->pos_alpha > 0) {
            /* fe = ws + theta dt L, then the stage combination with dt L -> fe - ws */
            REAL *fe = (REAL *)malloc(n * sizeof(REAL));
            m->pos_limited += OMS(pos_limit)(m, m->nv, ws, L, dt, fe);
            for (int64_t i = 0; i < n; ++i) L[i] = fe[i];
            free(fe);
            for (int64_t i = 0; i < n; ++i) {
                if (stage == 1) ws[i] = L[i];
                else if (stage == 2) ws[i] = 0.75 * wn[i] + 0.25 * L[i];
                else ws[i] = (1.0 / 3.0) * wn[i] + (2.0 / 3.0) * L[i];
            }
        } else {
            OMS(om_stage_combine)(n, stage, wn, ws, L, dt, ws);
        }
        if (m->ghost)
            for (int64_t v = 0; v < m->nv; ++v)
                if (m->ghost[v] >= 0) memcpy(ws + 4 * v, wn + 4 * v, 4 * sizeof(REAL));
    }
    if (st == OM_OK) {
        OMS(om_fill_ghosts)(m, ws);
        memcpy(w, ws, n * sizeof(REAL));
    }
    free(wn); free(L); free(ws);
    if (nfallback) *nfallback = nf;
    return st;
}

