// Host preprocessing of libfdu, FP64, done once per static mesh
// ("computed only once at the initial time for static meshes",
// Section 2.2.1):
//   - unique edge list and vertex adjacency;
//   - per edge the six-vertex 1D curvilinear stencil (Section 2.3.1,
//     Fig. weno1d-tri) and its normalised arc-length coordinates along
//     Catmull-Rom curves (Section 2.3.1, Fig. curve_sten);
//   - difference-form NU-WENO5 coefficient blocks (Appendix);
//   - one- or two-level divergence stencils (Section 2.2.2) and their
//     least-squares weights, the a1 and b2 rows of the pseudo-inverse
//     (Section 2.2.1), here by Householder QR of the column-equilibrated
//     system (equal to the SVD pseudo-inverse for full column rank);
//   - a Hilbert-curve locality renumbering of vertices and edges.
// Compiled with -ffp-contract=off so that the stencil walk's cosine
// comparisons give the same bits on every host.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "fdu_internal.h"

namespace fdu {
namespace {

struct Geo {
    const double *xy;
    double Lx, Ly;
    inline void d(int64_t a, int64_t b, double out[2]) const {
        double dx = xy[2 * b] - xy[2 * a];
        double dy = xy[2 * b + 1] - xy[2 * a + 1];
        if (Lx > 0) dx -= Lx * std::rint(dx / Lx);
        if (Ly > 0) dy -= Ly * std::rint(dy / Ly);
        out[0] = dx;
        out[1] = dy;
    }
};

// ---------------------------------------------------------------- edges
inline uint64_t edge_key(int32_t a, int32_t b) {
    uint32_t p = (uint32_t)a, q = (uint32_t)b;
    if (p > q) std::swap(p, q);
    return ((uint64_t)p << 32) | q;
}

// Artificial edges for vertices short of least-squares conditions (Section
// 2.2.2, Fig. l1-tria4): a vertex O whose one-level stencil gives fewer than
// p(p+3) conditions (2 per neighbour, 1 per edge at O or between two
// neighbours) is joined to the far apex X of each triangle across the side
// of O's triangles opposite O, when X is not yet a neighbour.
void far_apex_edges(const CellList &cells, int64_t nv, int degree, std::vector<uint64_t> &keys) {
    std::vector<std::vector<int32_t>> nb(nv);
    for (uint64_t k : keys) {
        const int32_t a = (int32_t)(k >> 32), b = (int32_t)(k & 0xffffffffu);
        nb[a].push_back(b);
        nb[b].push_back(a);
    }
    for (auto &l : nb) std::sort(l.begin(), l.end());
    auto adjacent = [&](int32_t a, int32_t b) { return std::binary_search(nb[a].begin(), nb[a].end(), b); };
    // triangles by side, and by vertex
    std::vector<std::pair<uint64_t, int32_t>> side_apex;  // (side key, apex)
    std::vector<std::vector<int64_t>> tri_of(nv);
    for (int64_t c = 0; c < cells.n; ++c) {
        if (cells.off[c + 1] - cells.off[c] != 3) continue;
        const int32_t *v = cells.vtx + cells.off[c];
        for (int i = 0; i < 3; ++i) {
            side_apex.push_back({edge_key(v[i], v[(i + 1) % 3]), v[(i + 2) % 3]});
            tri_of[v[i]].push_back(c);
        }
    }
    std::sort(side_apex.begin(), side_apex.end());
    const int64_t need = (int64_t)degree * (degree + 3);
    std::vector<uint64_t> extra;
    for (int32_t o = 0; o < (int32_t)nv; ++o) {
        const auto &N = nb[o];
        int64_t between = 0;
        for (size_t i = 0; i < N.size(); ++i)
            for (size_t j = i + 1; j < N.size(); ++j) between += adjacent(N[i], N[j]);
        const int64_t conditions = 2 * (int64_t)N.size() + (int64_t)N.size() + between;
        if (conditions >= need) continue;
        for (int64_t c : tri_of[o]) {
            const int32_t *v = cells.vtx + cells.off[c];
            const int i = v[0] == o ? 0 : (v[1] == o ? 1 : 2);
            const int32_t A = v[(i + 1) % 3], B = v[(i + 2) % 3];
            const uint64_t key = edge_key(A, B);
            auto it = std::lower_bound(side_apex.begin(), side_apex.end(), std::make_pair(key, INT32_MIN));
            for (; it != side_apex.end() && it->first == key; ++it) {
                const int32_t X = it->second;
                if (X != o && !adjacent(o, X)) extra.push_back(edge_key(o, X));
            }
        }
    }
    keys.insert(keys.end(), extra.begin(), extra.end());
}

int build_edges(const CellList &cells, int artificial, int degree, int64_t nv, const Geo &g, HostTables &T,
                std::string &err) {
    std::vector<uint64_t> keys;
    keys.reserve(4 * cells.n);
    for (int64_t t = 0; t < cells.n; ++t) {
        const int64_t nc = cells.off[t + 1] - cells.off[t];
        if (nc != 3 && nc != 4) {
            err = "cell " + std::to_string(t) + " has " + std::to_string(nc) + " vertices (3 or 4 expected)";
            return FDU_ERR_MESH;
        }
        const int32_t *v = cells.vtx + cells.off[t];
        for (int s = 0; s < nc; ++s)
            if (v[s] < 0 || v[s] >= nv) {
                err = "cell " + std::to_string(t) + " has a vertex id out of range";
                return FDU_ERR_MESH;
            }
        for (int s = 0; s < nc; ++s)
            for (int r = s + 1; r < nc; ++r)
                if (v[s] == v[r]) {
                    err = "cell " + std::to_string(t) + " repeats a vertex";
                    return FDU_ERR_MESH;
                }
        for (int s = 0; s < nc; ++s) {  // every corner turns left: convex and counter-clockwise
            double a[2], b[2];
            g.d(v[s], v[(s + 1) % nc], a);
            g.d(v[s], v[(s + nc - 1) % nc], b);
            if (!(a[0] * b[1] - a[1] * b[0] > 0)) {
                err = (nc == 3 ? "triangle " : "cell ") + std::to_string(t) + " is degenerate, clockwise or not convex";
                return FDU_ERR_MESH;
            }
        }
        for (int s = 0; s < nc; ++s) keys.push_back(edge_key(v[s], v[(s + 1) % nc]));
        if (nc == 4 && artificial >= 1) {  // artificial quad diagonals (Fig. l1-hyb)
            keys.push_back(edge_key(v[0], v[2]));
            keys.push_back(edge_key(v[1], v[3]));
        }
    }
    {  // sort and deduplicate: bucket by the smaller id, then sort each short bucket
        std::vector<int64_t> cnt(nv + 1, 0);
        for (uint64_t k : keys) cnt[(k >> 32) + 1]++;
        for (int64_t v = 0; v < nv; ++v) cnt[v + 1] += cnt[v];
        std::vector<uint32_t> q(keys.size());
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (uint64_t k : keys) q[fill[k >> 32]++] = (uint32_t)(k & 0xffffffffu);
        keys.clear();
        for (int64_t v = 0; v < nv; ++v) {
            auto b = q.begin() + cnt[v], e = q.begin() + cnt[v + 1];
            std::sort(b, e);
            e = std::unique(b, e);
            for (auto it = b; it != e; ++it) keys.push_back(((uint64_t)v << 32) | *it);
        }
    }
    if (artificial >= 2) {
        far_apex_edges(cells, nv, degree, keys);
        std::sort(keys.begin(), keys.end());
        keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    }
    T.ne = (int64_t)keys.size();
    T.edge.resize(2 * T.ne);
    T.nrm.resize(2 * T.ne);
    for (int64_t k = 0; k < T.ne; ++k) {
        T.edge[2 * k] = (int32_t)(keys[k] >> 32);
        T.edge[2 * k + 1] = (int32_t)(keys[k] & 0xffffffffu);
        double d[2];
        g.d(T.edge[2 * k], T.edge[2 * k + 1], d);
        double l = std::sqrt(d[0] * d[0] + d[1] * d[1]);
        if (!(l > 0)) {
            err = "zero-length edge";
            return FDU_ERR_MESH;
        }
        T.nrm[2 * k] = d[0] / l;
        T.nrm[2 * k + 1] = d[1] / l;
    }
    // adjacency (CSR): each vertex's (neighbour, edge) pairs in ascending
    // neighbour order; bucketed by vertex, then each short list sorted
    T.adj_off.assign(nv + 1, 0);
    for (int64_t k = 0; k < 2 * T.ne; ++k) T.adj_off[T.edge[k] + 1]++;
    for (int64_t v = 0; v < nv; ++v) T.adj_off[v + 1] += T.adj_off[v];
    {
        std::vector<std::pair<int32_t, int32_t>> nbr(2 * T.ne);  // (neighbour, edge)
        std::vector<int64_t> fill(T.adj_off.begin(), T.adj_off.end() - 1);
        for (int64_t k = 0; k < T.ne; ++k) {
            const int32_t a = T.edge[2 * k], b = T.edge[2 * k + 1];
            nbr[fill[a]++] = {b, (int32_t)k};
            nbr[fill[b]++] = {a, (int32_t)k};
        }
        T.adj.resize(2 * T.ne);
        T.adj_edge.resize(2 * T.ne);
        for (int64_t v = 0; v < nv; ++v) {
            std::sort(nbr.begin() + T.adj_off[v], nbr.begin() + T.adj_off[v + 1]);
            for (int64_t i = T.adj_off[v]; i < T.adj_off[v + 1]; ++i) {
                T.adj[i] = nbr[i].first;
                T.adj_edge[i] = nbr[i].second;
            }
        }
    }
    for (int64_t v = 0; v < nv; ++v)
        if (T.adj_off[v + 1] - T.adj_off[v] < 2) {
            err = "vertex " + std::to_string(v) + " has fewer than two neighbours";
            return FDU_ERR_MESH;
        }
    return FDU_OK;
}

// ---------------------------------------------------------------- 1D stencil walk
// Greedy "as smooth as possible" string (Section 2.3.1): from vertex c
// reached along d, the unused neighbour with the largest cosine between d
// and the next segment; a candidate replaces the best so far only if its
// cosine is larger by more than 1e-12 (neighbours visited in ascending
// original id); the winning cosine must be positive.
bool next_vertex(const HostTables &T, const Geo &g, int32_t from, int32_t at, const int32_t *used, int nused,
                 int32_t &out) {
    double d[2];
    g.d(from, at, d);
    const double dlen = std::sqrt(d[0] * d[0] + d[1] * d[1]);
    int32_t pick = -1;
    double cbest = 0;
    for (int64_t i = T.adj_off[at]; i < T.adj_off[at + 1]; ++i) {
        const int32_t q = T.adj[i];
        if (std::find(used, used + nused, q) != used + nused) continue;
        double e[2];
        g.d(at, q, e);
        const double elen = std::sqrt(e[0] * e[0] + e[1] * e[1]);
        const double c = (d[0] * e[0] + d[1] * e[1]) / (dlen * elen);
        if (pick < 0 || c > cbest + 1e-12) {
            pick = q;
            cbest = c;
        }
    }
    if (pick < 0 || !(cbest > 0)) return false;
    out = pick;
    return true;
}

bool walk(const HostTables &T, const Geo &g, int64_t k, int32_t s[6]) {
    const int32_t a = T.edge[2 * k], b = T.edge[2 * k + 1];
    int32_t used[6] = {a, b, -1, -1, -1, -1};
    int32_t r2, r3, l2, l3;
    if (!next_vertex(T, g, a, b, used, 2, r2)) return false;
    used[2] = r2;
    if (!next_vertex(T, g, b, r2, used, 3, r3)) return false;
    used[3] = r3;
    if (!next_vertex(T, g, b, a, used, 4, l2)) return false;
    used[4] = l2;
    if (!next_vertex(T, g, a, l2, used, 5, l3)) return false;
    s[0] = l3; s[1] = l2; s[2] = a; s[3] = b; s[4] = r2; s[5] = r3;
    return true;
}

// ---------------------------------------------------------------- arc length
// 16-point Gauss-Legendre rule on [0, 1]; nodes from Newton's method on the
// Legendre recurrence started at Tricomi's approximation.
struct GaussLegendre16 {
    double t[16], w[16];
    GaussLegendre16() {
        const int n = 16;
        for (int i = 1; i <= n; ++i) {
            double th = M_PI * (4.0 * i - 1.0) / (4.0 * n + 2.0);
            double x = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(th);
            double pn = 0, pd = 0;
            for (int it = 0; it < 50; ++it) {
                double pm = 1.0, p = x;
                for (int m = 2; m <= n; ++m) {
                    double pnew = ((2.0 * m - 1.0) * x * p - (m - 1.0) * pm) / m;
                    pm = p;
                    p = pnew;
                }
                pn = p;
                pd = n * (pm - x * p) / (1.0 - x * x);
                double step = pn / pd;
                x -= step;
                if (std::fabs(step) <= 4e-16) break;
            }
            {
                double pm = 1.0, p = x;
                for (int m = 2; m <= n; ++m) {
                    double pnew = ((2.0 * m - 1.0) * x * p - (m - 1.0) * pm) / m;
                    pm = p;
                    p = pnew;
                }
                pd = n * (pm - x * p) / (1.0 - x * x);
            }
            t[i - 1] = 0.5 * (x + 1.0);
            w[i - 1] = 1.0 / ((1.0 - x * x) * pd * pd);
        }
    }
};
const GaussLegendre16 &gl16() {
    static const GaussLegendre16 q;
    return q;
}

// length of the cubic Hermite segment p0 -> p1 with end tangents m0, m1
double segment_length(const double p0[2], const double p1[2], const double m0[2], const double m1[2]) {
    const GaussLegendre16 &q = gl16();
    double len = 0;
    for (int i = 0; i < 16; ++i) {
        const double s = q.t[i];
        // derivative of the Hermite basis
        const double a = 6 * s * s - 6 * s;      // coefficient of p0 (and -p1)
        const double b = 3 * s * s - 4 * s + 1;  // of m0
        const double c = 3 * s * s - 2 * s;      // of m1
        const double vx = a * (p0[0] - p1[0]) + b * m0[0] + c * m1[0];
        const double vy = a * (p0[1] - p1[1]) + b * m0[1] + c * m1[1];
        len += q.w[i] * std::sqrt(vx * vx + vy * vy);
    }
    return len;
}

// One side: start A at the middle edge (other end O), then B and C.  The
// curve leaves A along O->A scaled by |B - A|, passes B with the
// Catmull-Rom tangent (C - A)/2 and ends at C with tangent C - B.
void side_arc(const double O[2], const double A[2], const double B[2], const double Cp[2], double &sAB, double &sBC) {
    double u[2] = {A[0] - O[0], A[1] - O[1]};
    const double ul = std::hypot(u[0], u[1]);
    const double chord = std::hypot(B[0] - A[0], B[1] - A[1]);
    const double tA[2] = {u[0] / ul * chord, u[1] / ul * chord};
    const double tB[2] = {0.5 * (Cp[0] - A[0]), 0.5 * (Cp[1] - A[1])};
    const double tC[2] = {Cp[0] - B[0], Cp[1] - B[1]};
    sAB = segment_length(A, B, tA, tB);
    sBC = segment_length(B, Cp, tB, tC);
}

void stencil_coordinates(const Geo &g, const int32_t s[6], double xi[6]) {
    // unwrapped points, L1 at the origin
    double P[6][2];
    double d[2];
    P[2][0] = 0; P[2][1] = 0;
    g.d(s[2], s[3], d); P[3][0] = d[0]; P[3][1] = d[1];
    g.d(s[3], s[4], d); P[4][0] = P[3][0] + d[0]; P[4][1] = P[3][1] + d[1];
    g.d(s[4], s[5], d); P[5][0] = P[4][0] + d[0]; P[5][1] = P[4][1] + d[1];
    g.d(s[2], s[1], d); P[1][0] = d[0]; P[1][1] = d[1];
    g.d(s[1], s[0], d); P[0][0] = P[1][0] + d[0]; P[0][1] = P[1][1] + d[1];
    const double ell = std::hypot(P[3][0], P[3][1]);
    double r1, r2, l1, l2;
    side_arc(P[2], P[3], P[4], P[5], r1, r2);
    side_arc(P[3], P[2], P[1], P[0], l1, l2);
    xi[2] = -0.5;
    xi[3] = 0.5;
    xi[4] = 0.5 + r1 / ell;
    xi[5] = xi[4] + r2 / ell;
    xi[1] = -0.5 - l1 / ell;
    xi[0] = xi[1] - l2 / ell;
}

}  // namespace

// ---------------------------------------------------------------- NU-WENO5 coefficients
// x[5] = x_{i-2..i+2}, origin at the midpoint of [x_i, x_{i+1}].
// Sub-stencil k interpolates points x[k..k+2] by a quadratic (Appendix,
// Eqs. u0-u2); its value, slope and curvature at 0 are written against
// differences from the shared point x_i = x[2].  The linear weights follow
// from their definition (the combination equals the degree-4 interpolant,
// Eq. S5): only S0 holds x_{i-2} and only S2 holds x_{i+2}, so C_0 and C_2
// are ratios of Lagrange values and C_1 = 1 - C_0 - C_2.
void side_coefficients(const double x[5], double out[kSideCoef]) {
    const double dx = x[3] - x[2];
    const double curv = std::sqrt(13.0 / 12.0) * dx * dx;
    // slot of each non-shared point per sub-stencil: local index -> slot
    double val[3][3], der[3][3], sec[3][3];
    for (int k = 0; k < 3; ++k) {
        const double *p = x + k;
        for (int j = 0; j < 3; ++j) {
            const double pa = p[(j + 1) % 3], pb = p[(j + 2) % 3];
            const double den = (p[j] - pa) * (p[j] - pb);
            val[k][j] = pa * pb / den;
            der[k][j] = -(pa + pb) / den;
            sec[k][j] = 2.0 / den;
        }
    }
    // non-shared local indices: k=0 -> (0,1), k=1 -> (0,2), k=2 -> (1,2)
    const int nj[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int k = 0; k < 3; ++k)
        for (int q = 0; q < 2; ++q) {
            const int j = nj[k][q];
            out[2 * k + q] = val[k][j];
            out[6 + 2 * k + q] = dx * der[k][j];
            out[12 + 2 * k + q] = curv * sec[k][j];
        }
    // degree-4 Lagrange weight at 0 of x[0] and x[4]
    double l0 = 1, l4 = 1;
    for (int m = 0; m < 5; ++m) {
        if (m != 0) l0 *= (0.0 - x[m]) / (x[0] - x[m]);
        if (m != 4) l4 *= (0.0 - x[m]) / (x[4] - x[m]);
    }
    const double c0 = l0 / val[0][0];
    const double c2 = l4 / val[2][2];
    out[18] = c0;
    out[19] = 1.0 - c0 - c2;
    out[20] = c2;
}

namespace {

// ---------------------------------------------------------------- divergence stencils
void stencil_of(const HostTables &T, int32_t o, std::vector<int32_t> &V, std::vector<int32_t> &E) {
    V.clear();
    E.clear();
    auto one_level = [&](int32_t c) {
        const int64_t b = T.adj_off[c], e = T.adj_off[c + 1];
        for (int64_t i = b; i < e; ++i) {
            V.push_back(T.adj[i]);
            E.push_back(T.adj_edge[i]);
        }
        // edges between two neighbours of c: merge the sorted neighbour lists
        for (int64_t i = b; i < e; ++i) {
            const int32_t a = T.adj[i];
            int64_t p = T.adj_off[a], pe = T.adj_off[a + 1], q = b;
            while (p < pe && q < e) {
                if (T.adj[p] < T.adj[q]) ++p;
                else if (T.adj[p] > T.adj[q]) ++q;
                else {
                    if (a < T.adj[p]) E.push_back(T.adj_edge[p]);
                    ++p;
                    ++q;
                }
            }
        }
    };
    if (T.levels == 1) {
        one_level(o);
    } else {
        for (int64_t i = T.adj_off[o]; i < T.adj_off[o + 1]; ++i) one_level(T.adj[i]);
    }
    std::sort(V.begin(), V.end());
    V.erase(std::unique(V.begin(), V.end()), V.end());
    V.erase(std::remove(V.begin(), V.end(), o), V.end());
    std::sort(E.begin(), E.end());
    E.erase(std::unique(E.begin(), E.end()), E.end());
}

// ---------------------------------------------------------------- least squares
// Rows of the linear system (Section 2.2.1, Eq. eLinearSystem), unknowns
// [a; b] with monomials ordered x, y, x^2, xy, y^2, ...  Columns are
// scaled to unit norm, the scaled matrix is factorised A S = Q R by
// Householder reflections, and the requested row sum of A^+ = S R^-1 Q^T
// is Q R^-T S e (e = unit vectors of a1 and b2).
int lsq_weights(const HostTables &T, const Geo &g, int32_t o, const int64_t vb, const int64_t nvj, const int64_t eb,
                const int64_t nek, std::vector<double> &w_out, std::vector<double> &A, std::vector<double> &hv) {
    const int p = T.degree;
    const int M = p * (p + 3) / 2, n = 2 * M;  // n <= 54 for p <= 6 (the per-unknown arrays below hold 64)
    const int m = (int)(2 * nvj + nek);
    if (m < n) return FDU_ERR_RANK_DEFICIENT;
    A.assign((size_t)m * n, 0.0);  // column-major
    double mono[64];
    auto monos = [&](double x, double y) {
        int c = 0;
        for (int d = 1; d <= p; ++d) {
            for (int i = d; i >= 0; --i) {
                double v = 1;
                for (int a = 0; a < i; ++a) v *= x;
                for (int b = 0; b < d - i; ++b) v *= y;
                mono[c++] = v;
            }
        }
    };
    for (int64_t j = 0; j < nvj; ++j) {
        double d[2];
        g.d(o, T.vid[vb + j], d);
        monos(d[0], d[1]);
        for (int c = 0; c < M; ++c) {
            A[(size_t)c * m + 2 * j] = mono[c];
            A[(size_t)(M + c) * m + 2 * j + 1] = mono[c];
        }
    }
    for (int64_t k = 0; k < nek; ++k) {
        const int32_t e = T.eid[eb + k];
        double d0[2], de[2];
        g.d(o, T.edge[2 * e], d0);
        g.d(T.edge[2 * e], T.edge[2 * e + 1], de);
        monos(d0[0] + 0.5 * de[0], d0[1] + 0.5 * de[1]);
        const double nx = T.nrm[2 * e], ny = T.nrm[2 * e + 1];
        for (int c = 0; c < M; ++c) {
            A[(size_t)c * m + 2 * nvj + k] = nx * mono[c];
            A[(size_t)(M + c) * m + 2 * nvj + k] = ny * mono[c];
        }
    }
    // column equilibration
    double scale[64];
    for (int c = 0; c < n; ++c) {
        double s = 0;
        for (int i = 0; i < m; ++i) s += A[(size_t)c * m + i] * A[(size_t)c * m + i];
        s = std::sqrt(s);
        if (!(s > 0)) return FDU_ERR_RANK_DEFICIENT;
        scale[c] = 1.0 / s;
        for (int i = 0; i < m; ++i) A[(size_t)c * m + i] *= scale[c];
    }
    // Householder QR in place; reflector k stored in hv (length m-k) with beta
    hv.assign((size_t)m * n, 0.0);
    double beta[64], rdiag[64];
    for (int k = 0; k < n; ++k) {
        double *col = &A[(size_t)k * m];
        double nrm2 = 0;
        for (int i = k; i < m; ++i) nrm2 += col[i] * col[i];
        const double nrm = std::sqrt(nrm2);
        const double alpha = col[k] >= 0 ? -nrm : nrm;
        double *v = &hv[(size_t)k * m];
        for (int i = 0; i < m; ++i) v[i] = 0;
        v[k] = col[k] - alpha;
        for (int i = k + 1; i < m; ++i) v[i] = col[i];
        double vv = 0;
        for (int i = k; i < m; ++i) vv += v[i] * v[i];
        beta[k] = vv > 0 ? 2.0 / vv : 0.0;
        rdiag[k] = alpha;
        // two columns per pass: two independent dot products in flight, each
        // summed in the same order as alone (same bits)
        int c = k;
        for (; c + 1 < n; c += 2) {
            double *a = &A[(size_t)c * m], *a2 = &A[(size_t)(c + 1) * m];
            double dot = 0, dot2 = 0;
            for (int i = k; i < m; ++i) {
                dot += v[i] * a[i];
                dot2 += v[i] * a2[i];
            }
            dot *= beta[k];
            dot2 *= beta[k];
            for (int i = k; i < m; ++i) {
                a[i] -= dot * v[i];
                a2[i] -= dot2 * v[i];
            }
        }
        if (c < n) {
            double *a = &A[(size_t)c * m];
            double dot = 0;
            for (int i = k; i < m; ++i) dot += v[i] * a[i];
            dot *= beta[k];
            for (int i = k; i < m; ++i) a[i] -= dot * v[i];
        }
    }
    double rmax = 0, rmin = INFINITY;
    for (int k = 0; k < n; ++k) {
        rmax = std::max(rmax, std::fabs(rdiag[k]));
        rmin = std::min(rmin, std::fabs(rdiag[k]));
    }
    if (!(rmin > 1e-13 * rmax)) return FDU_ERR_RANK_DEFICIENT;
    // R^T y = S e  (R upper triangular, A now holds R in rows 0..n-1)
    double y[64];
    for (int c = 0; c < n; ++c) y[c] = 0;
    y[0] = scale[0];
    y[M + 1] += scale[M + 1];
    for (int i = 0; i < n; ++i) {
        double s = y[i];
        for (int j = 0; j < i; ++j) s -= A[(size_t)i * m + j] * y[j];  // R[j][i] sits in column i, row j
        y[i] = s / A[(size_t)i * m + i];
    }
    // w = Q [y; 0] = H_0 H_1 ... H_{n-1} [y; 0]
    w_out.assign(m, 0.0);
    for (int i = 0; i < n; ++i) w_out[i] = y[i];
    for (int k = n - 1; k >= 0; --k) {
        const double *v = &hv[(size_t)k * m];
        double dot = 0;
        for (int i = k; i < m; ++i) dot += v[i] * w_out[i];
        dot *= beta[k];
        for (int i = k; i < m; ++i) w_out[i] -= dot * v[i];
    }
    return FDU_OK;
}

// ---------------------------------------------------------------- Hilbert order
uint64_t hilbert_index(uint32_t x, uint32_t y, int order) {
    const uint32_t n = 1u << order;
    uint64_t d = 0;
    for (uint32_t s = n >> 1; s > 0; s >>= 1) {
        const uint32_t rx = (x & s) ? 1u : 0u;
        const uint32_t ry = (y & s) ? 1u : 0u;
        d += (uint64_t)s * s * ((3u * rx) ^ ry);
        if (ry == 0) {  // rotate the quadrant
            if (rx == 1) {
                x = n - 1 - x;
                y = n - 1 - y;
            }
            std::swap(x, y);
        }
    }
    return d;
}

// f(b, e, thread) over [0, n) in ranges that start at multiples of 256 and
// end at the next multiple or at n (one range [0, n) when run serially).
template <class F>
void parallel_for(int64_t n, int threads, F &&f) {
    if (threads <= 1 || n < 1024) {
        f(0, n, 0);
        return;
    }
    std::vector<std::thread> pool;
    std::atomic<int64_t> next(0);
    const int64_t chunk = 256;
    for (int t = 0; t < threads; ++t)
        pool.emplace_back([&, t] {
            for (;;) {
                int64_t b = next.fetch_add(chunk);
                if (b >= n) break;
                f(b, std::min(n, b + chunk), t);
            }
        });
    for (auto &th : pool) th.join();
}

}  // namespace

int build_host_tables(const double *xy, int64_t nv, const int32_t *tri, int64_t nt, const fdu_mesh_opts &o,
                      HostTables &T, std::string &err, const int32_t *comp) {
    std::vector<int64_t> off(nt + 1);
    for (int64_t t = 0; t <= nt; ++t) off[t] = 3 * t;
    return build_host_tables(xy, nv, CellList{off.data(), tri, nt}, 0, o, T, err, comp);
}

int build_host_tables(const double *xy, int64_t nv, const CellList &cells, int artificial, const fdu_mesh_opts &o,
                      HostTables &T, std::string &err, const int32_t *comp) {
    T.nv = nv;
    T.nt = cells.n;
    T.Lx = o.Lx;
    T.Ly = o.Ly;
    T.gamma = o.gamma;
    T.degree = o.lsq_degree;
    T.levels = o.lsq_levels;
    T.xy.assign(xy, xy + 2 * nv);
    T.ghost.clear();
    T.n_real = nv;
    if (o.ghost_donor) {
        T.ghost.assign(o.ghost_donor, o.ghost_donor + nv);
        T.n_real = 0;
        for (int64_t v = 0; v < nv; ++v) {
            const int32_t d = T.ghost[v];
            if (d >= nv || d < -1 || (d >= 0 && d != v && o.ghost_donor[d] >= 0)) {
                err = "ghost donor must be -1, the id of a non-ghost vertex or the ghost's own id";
                return FDU_ERR_ARG;
            }
            T.n_real += (T.ghost[v] < 0);
        }
    }
    Geo g{T.xy.data(), T.Lx, T.Ly};
    int st = build_edges(cells, artificial, o.lsq_degree, nv, g, T, err);
    if (st) return st;
    int threads = o.host_threads > 0 ? o.host_threads : (int)std::max(1u, std::thread::hardware_concurrency());
    const bool periodic = T.Lx > 0 && T.Ly > 0;

    // 1D stencils and coefficients
    T.sten.assign(6 * T.ne, -1);
    T.xi.assign(6 * T.ne, 0.0);
    T.coef.assign((size_t)kEdgeCoef * T.ne, 0.0);
    std::atomic<int64_t> bad(-1);
    parallel_for(T.ne, threads, [&](int64_t b, int64_t e, int) {
        for (int64_t k = b; k < e; ++k) {
            int32_t *s = &T.sten[6 * k];
            if (!walk(T, g, k, s)) {
                for (int i = 0; i < 6; ++i) s[i] = -1;
                bad.store(k);
                continue;
            }
            double *xi = &T.xi[6 * k];
            stencil_coordinates(g, s, xi);
            double *c = &T.coef[(size_t)kEdgeCoef * k];
            const double xl[5] = {xi[0], xi[1], xi[2], xi[3], xi[4]};
            const double xr[5] = {-xi[5], -xi[4], -xi[3], -xi[2], -xi[1]};
            double L[kSideCoef], R[kSideCoef];
            side_coefficients(xl, L);
            side_coefficients(xr, R);
            // sub-stencil k of a side block: value coefficients at 2k, slope at 6 + 2k,
            // curvature at 12 + 2k.  The block keeps the value pair and the
            // smoothness indicator beta = (p0 x + p1 y)^2 + (q0 x + q1 y)^2 as the
            // quadratic form m0 x^2 + m1 x y + m2 y^2 of the same two differences
            auto put = [&](int dst, const double *side, int k) {
                const double p0 = side[6 + 2 * k], p1 = side[6 + 2 * k + 1];
                const double q0 = side[12 + 2 * k], q1 = side[12 + 2 * k + 1];
                c[dst + 0] = side[2 * k];
                c[dst + 1] = side[2 * k + 1];
                c[dst + 2] = p0 * p0 + q0 * q0;
                c[dst + 3] = 2.0 * (p0 * p1 + q0 * q1);
                c[dst + 4] = p1 * p1 + q1 * q1;
            };
            put(0 * kSubCoef, L, 0);  // S_a
            put(1 * kSubCoef, L, 1);  // S_b
            put(2 * kSubCoef, L, 2);  // S_c
            put(3 * kSubCoef, R, 0);  // S_d
            // linear weights divided by the middle one (C_1 > 0 on ordered points):
            // the nonlinear weights are invariant to a common factor of the C_k
            c[kCoefCL] = L[18] / L[19];
            c[kCoefCL + 1] = L[20] / L[19];
            c[kCoefCR] = R[18] / R[19];
            c[kCoefCR + 1] = R[20] / R[19];
            c[kCoefN] = T.nrm[2 * k];
            c[kCoefN + 1] = T.nrm[2 * k + 1];
        }
    });
    if (periodic && bad.load() >= 0) {
        err = "1D stencil walk found no forward neighbour for edge " + std::to_string(bad.load());
        return FDU_ERR_STENCIL;
    }

    // divergence stencils and weights (both parallel).  Each chunk of
    // vertices collects its stencils in its own buffers; concatenating the
    // chunks in vertex order gives the tables a serial loop would build.
    T.voff.assign(nv + 1, 0);
    T.eoff.assign(nv + 1, 0);
    T.vid.clear();
    T.eid.clear();
    {
        const int64_t chunk = 256, nchunk = (nv + chunk - 1) / chunk;
        std::vector<std::vector<int32_t>> cv(nchunk), ce(nchunk);
        std::atomic<int64_t> first_bad(INT64_MAX);  // lowest vertex with an edge lacking a 1D stencil
        std::vector<int32_t> bad_edge(nchunk, -1);
        // parallel_for hands out vertex ranges that start at multiples of 256
        // and hold whole chunks
        parallel_for(nv, threads, [&](int64_t b, int64_t e, int) {
            std::vector<int32_t> V, E;
            for (int64_t c = b / chunk; c * chunk < e; ++c)
                for (int64_t v = c * chunk; v < std::min(nv, (c + 1) * chunk); ++v) {
                    if (!T.ghost.empty() && T.ghost[v] >= 0) {
                        T.voff[v + 1] = 0;
                        T.eoff[v + 1] = 0;
                        continue;
                    }
                    stencil_of(T, (int32_t)v, V, E);
                    for (int32_t k : E)
                        if (T.sten[6 * (int64_t)k] < 0 && bad_edge[c] < 0) {
                            bad_edge[c] = k;
                            int64_t cur = first_bad.load();
                            while (v < cur && !first_bad.compare_exchange_weak(cur, v)) {
                            }
                        }
                    cv[c].insert(cv[c].end(), V.begin(), V.end());
                    ce[c].insert(ce[c].end(), E.begin(), E.end());
                    T.voff[v + 1] = (int64_t)V.size();  // counts, summed below
                    T.eoff[v + 1] = (int64_t)E.size();
                }
        });
        if (first_bad.load() != INT64_MAX) {
            const int64_t v = first_bad.load();
            err = "edge " + std::to_string(bad_edge[v / chunk]) + " in the divergence stencil of vertex " +
                  std::to_string(v) + " has no 1D stencil";
            return FDU_ERR_STENCIL;
        }
        for (int64_t v = 0; v < nv; ++v) {
            T.voff[v + 1] += T.voff[v];
            T.eoff[v + 1] += T.eoff[v];
        }
        T.vid.reserve(T.voff[nv]);
        T.eid.reserve(T.eoff[nv]);
        for (int64_t c = 0; c < nchunk; ++c) {
            T.vid.insert(T.vid.end(), cv[c].begin(), cv[c].end());
            T.eid.insert(T.eid.end(), ce[c].begin(), ce[c].end());
        }
    }
    T.wf.assign(T.vid.size(), 0.0);
    T.wg.assign(T.vid.size(), 0.0);
    T.we.assign(T.eid.size(), 0.0);
    std::atomic<int64_t> rank_bad(-1);
    parallel_for(nv, threads, [&](int64_t b, int64_t e, int) {
        std::vector<double> w, A, hv;
        for (int64_t v = b; v < e; ++v) {
            if (!T.ghost.empty() && T.ghost[v] >= 0) continue;
            const int64_t vb = T.voff[v], nvj = T.voff[v + 1] - vb;
            const int64_t eb = T.eoff[v], nek = T.eoff[v + 1] - eb;
            if (lsq_weights(T, g, (int32_t)v, vb, nvj, eb, nek, w, A, hv) != FDU_OK) {
                rank_bad.store(v);
                continue;
            }
            for (int64_t j = 0; j < nvj; ++j) {
                T.wf[vb + j] = w[2 * j];
                T.wg[vb + j] = w[2 * j + 1];
            }
            for (int64_t k = 0; k < nek; ++k) T.we[eb + k] = w[2 * nvj + k];
        }
    });
    if (rank_bad.load() >= 0) {
        err = "least-squares system of vertex " + std::to_string(rank_bad.load()) +
              " has too few conditions or is rank deficient";
        return FDU_ERR_RANK_DEFICIENT;
    }

    T.hmin.assign(nv, INFINITY);
    for (int64_t k = 0; k < T.ne; ++k) {
        double d[2];
        g.d(T.edge[2 * k], T.edge[2 * k + 1], d);
        const double l = std::sqrt(d[0] * d[0] + d[1] * d[1]);
        T.hmin[T.edge[2 * k]] = std::min(T.hmin[T.edge[2 * k]], l);
        T.hmin[T.edge[2 * k + 1]] = std::min(T.hmin[T.edge[2 * k + 1]], l);
    }

    // locality renumbering
    T.v_new2old.resize(nv);
    std::iota(T.v_new2old.begin(), T.v_new2old.end(), 0);
    if (o.renumber) {
        double lo[2] = {INFINITY, INFINITY}, hi[2] = {-INFINITY, -INFINITY};
        for (int64_t v = 0; v < nv; ++v)
            for (int c = 0; c < 2; ++c) {
                lo[c] = std::min(lo[c], T.xy[2 * v + c]);
                hi[c] = std::max(hi[c], T.xy[2 * v + c]);
            }
        const int order = 16;
        const double span = std::max(hi[0] - lo[0], hi[1] - lo[1]);
        const double scale = span > 0 ? ((1 << order) - 1) / span : 0;
        std::vector<uint64_t> key(nv);
        for (int64_t v = 0; v < nv; ++v) {
            uint32_t ix = (uint32_t)((T.xy[2 * v] - lo[0]) * scale);
            uint32_t iy = (uint32_t)((T.xy[2 * v + 1] - lo[1]) * scale);
            key[v] = hilbert_index(ix, iy, order);
        }
        std::stable_sort(T.v_new2old.begin(), T.v_new2old.end(),
                         [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    }
    if (comp)
        std::stable_sort(T.v_new2old.begin(), T.v_new2old.end(), [&](int32_t a, int32_t b) { return comp[a] < comp[b]; });
    if (!T.ghost.empty())
        std::stable_partition(T.v_new2old.begin(), T.v_new2old.end(), [&](int32_t v) { return T.ghost[v] < 0; });
    T.v_old2new.resize(nv);
    for (int64_t i = 0; i < nv; ++i) T.v_old2new[T.v_new2old[i]] = (int32_t)i;
    T.e_new2old.resize(T.ne);
    std::iota(T.e_new2old.begin(), T.e_new2old.end(), 0);
    if (o.renumber) {
        std::vector<uint64_t> key(T.ne);
        for (int64_t k = 0; k < T.ne; ++k) {
            uint32_t a = (uint32_t)T.v_old2new[T.edge[2 * k]], b = (uint32_t)T.v_old2new[T.edge[2 * k + 1]];
            if (a > b) std::swap(a, b);
            key[k] = ((uint64_t)a << 32) | b;
        }
        std::sort(T.e_new2old.begin(), T.e_new2old.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    }
    {
        std::vector<uint8_t> active(T.ne, 0);
        for (int32_t e : T.eid) active[e] = 1;
        T.ne_active = 0;
        for (int64_t k = 0; k < T.ne; ++k) T.ne_active += active[k];
        std::stable_partition(T.e_new2old.begin(), T.e_new2old.end(), [&](int32_t e) { return active[e] != 0; });
    }
    T.e_old2new.resize(T.ne);
    for (int64_t i = 0; i < T.ne; ++i) T.e_old2new[T.e_new2old[i]] = (int32_t)i;
    return FDU_OK;
}

}  // namespace fdu
