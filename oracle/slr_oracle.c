/*
 * FP64 CPU oracle for the semi-Lagrangian (SL) level-set step of
 * Preda & Semplice, arXiv 2410.22205. TEST INFRASTRUCTURE ONLY: only the
 * tests, the smoke check and the benchmark's CPU-baseline leg may load it.
 *
 * Plain C99, FP64, one node at a time, compiled with -ffp-contract=off.
 * Optional OpenMP over independent nodes; every reduction is summed per
 * fixed slab and then over slabs in order, so the result does not depend on
 * the thread count. Declarations and the list of unpinned functions are in
 * slr_oracle.h.
 *
 * Readings of passages the paper leaves silent or garbled (each one chosen
 * here, not printed in the paper):
 *  - gradients on the domain boundary: one-sided first-order differences;
 *  - feet outside the domain: the index-space coordinate is clamped to
 *    [0, n-1]; WENO stencil nodes outside the grid replicate the edge value;
 *  - eq. subgrid is read as |φ_j| < γ (strict); eq. ZhaoPDECutOff drops δ,
 *    which is kept as in eq. levelset:pde; the cut-off factor multiplies the
 *    scale factor in both the advective and the diffusive displacement;
 *  - "first neighbours" of eq. SL:2 are the face neighbours inside the grid,
 *    and interpolation at a node returns the node value;
 *  - the 3-D WENO splitting runs z-lines first, then y, then x (the 2-D text
 *    gives y then x);
 *  - energy: zero counts with the positive side; a 2-D cell with four edge
 *    crossings pairs them by the sign of the mean of its four corners;
 *  - the stop test uses k = min(n, kmax) for both running means;
 *  - E_p == 0 with p != 1 gives the scale factor 0 (no motion).
 */
#include "slr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* grid helpers                                                         */
/* ------------------------------------------------------------------ */

long long or_num_nodes(const or_params* g) { return g->n[0] * g->n[1] * g->n[2]; }

static void unflatten(const or_params* g, long long idx, long long ijk[3]) {
    ijk[0] = idx % g->n[0];
    ijk[1] = (idx / g->n[0]) % g->n[1];
    ijk[2] = idx / (g->n[0] * g->n[1]);
}

static long long flatten(const or_params* g, long long i, long long j, long long k) {
    return i + g->n[0] * (j + g->n[1] * k);
}

static long long clampi(long long v, long long lo, long long hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* node coordinate x = lo + i*h (§3: uniform mesh width Δx) */
void or_node_coord(const or_params* g, long long idx, double x[3]) {
    long long ijk[3];
    unflatten(g, idx, ijk);
    for (int a = 0; a < 3; ++a) x[a] = (a < g->dim) ? g->lo[a] + (double)ijk[a] * g->h : 0.0;
}

int or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------ */
/* §2 and §3.4: distance to the cloud                                   */
/* ------------------------------------------------------------------ */

/* d(x) = min over Q in S of |x - Q|. The squared distance is summed as
 * (x-qx)^2 + (y-qy)^2 [+ (z-qz)^2] in that order; the minimiser with the
 * lowest index wins ties (strict < over ascending point index). */
void or_distance(const or_params* g, const double* pts, long long npts,
                 const long long* nodes, long long m, double* d_out, int* arg_out) {
    long long count = nodes ? m : or_num_nodes(g);
    int dim = g->dim;
#pragma omp parallel for schedule(dynamic, 64)
    for (long long t = 0; t < count; ++t) {
        long long idx = nodes ? nodes[t] : t;
        double x[3];
        or_node_coord(g, idx, x);
        double best = INFINITY;
        long long arg = -1;
        for (long long q = 0; q < npts; ++q) {
            const double* Q = pts + q * dim;
            double s = 0.0;
            for (int a = 0; a < dim; ++a) {
                double diff = x[a] - Q[a];
                s = s + diff * diff;
            }
            if (s < best) {
                best = s;
                arg = q;
            }
        }
        d_out[t] = sqrt(best);
        if (arg_out) arg_out[t] = (int)arg;
    }
}

/* k-d tree search with the same decisions as the scan above. Median split
 * on the widest axis, leaves of at most 8 points; every tree node keeps the
 * bounding box [bmin, bmax] of its points. A subtree is skipped only when
 *   fl(..fl(o_0^2 + o_1^2) + ..) > best,  o_a = fl(bmin_a - q_a) if q_a < bmin_a,
 *                                          fl(q_a - bmax_a) if q_a > bmax_a, else 0,
 * summed in the same order as a point's squared distance: for a point x of
 * the box, |fl(q_a - x_a)| >= o_a (x_a lies beyond the box face, rounding is
 * monotone and symmetric), squares and sums of non-negative terms keep the
 * order, so each point there has a computed squared distance at least that
 * bound and can neither win nor tie. The nearer child is visited first; the
 * result (smallest squared distance, then lowest index) does not depend on
 * the visiting order. */
typedef struct {
    int axis;          /* -1 for a leaf */
    double split;
    int left, right;
    long long lo, hi;  /* range in the permutation */
    double bmin[3], bmax[3];
} kd_node;

typedef struct {
    const double* pts;
    int dim;
    long long* perm;
    kd_node* nodes;
    int count;
} kd_tree;

static double kd_coord(const kd_tree* t, long long i, int a) { return t->pts[t->perm[i] * t->dim + a]; }

static void kd_select(kd_tree* t, long long lo, long long hi, long long k, int a) {
    /* Hoare-style quickselect: afterwards perm[lo..k) <= perm[k] <= perm[k+1..hi) on axis a */
    while (hi - lo > 1) {
        double pivot = kd_coord(t, lo + (hi - lo) / 2, a);
        long long i = lo, j = hi - 1;
        while (i <= j) {
            while (kd_coord(t, i, a) < pivot) ++i;
            while (kd_coord(t, j, a) > pivot) --j;
            if (i <= j) {
                long long tmp = t->perm[i];
                t->perm[i] = t->perm[j];
                t->perm[j] = tmp;
                ++i;
                --j;
            }
        }
        if (k <= j)
            hi = j + 1;
        else if (k >= i)
            lo = i;
        else
            return;
    }
}

static int kd_build(kd_tree* t, long long lo, long long hi) {
    int id = t->count++;
    kd_node* nd = &t->nodes[id];
    nd->lo = lo;
    nd->hi = hi;
    nd->axis = -1;
    int best_a = 0;
    double best_w = -1.0;
    for (int a = 0; a < 3; ++a) {
        nd->bmin[a] = 0.0;
        nd->bmax[a] = 0.0;
    }
    for (int a = 0; a < t->dim; ++a) {
        double mn = INFINITY, mx = -INFINITY;
        for (long long i = lo; i < hi; ++i) {
            double v = kd_coord(t, i, a);
            if (v < mn) mn = v;
            if (v > mx) mx = v;
        }
        nd->bmin[a] = mn;
        nd->bmax[a] = mx;
        if (mx - mn > best_w) {
            best_w = mx - mn;
            best_a = a;
        }
    }
    if (hi - lo <= 8) return id;
    long long mid = lo + (hi - lo) / 2;
    kd_select(t, lo, hi, mid, best_a);
    double split = kd_coord(t, mid, best_a);
    int left = kd_build(t, lo, mid);
    int right = kd_build(t, mid, hi);
    nd = &t->nodes[id];
    nd->axis = best_a;
    nd->split = split;
    nd->left = left;
    nd->right = right;
    return id;
}

static double kd_box_bound(const kd_tree* t, const kd_node* nd, const double x[3]) {
    double s = 0.0;
    for (int a = 0; a < t->dim; ++a) {
        double o = 0.0;
        if (x[a] < nd->bmin[a])
            o = nd->bmin[a] - x[a];
        else if (x[a] > nd->bmax[a])
            o = x[a] - nd->bmax[a];
        s = s + o * o;
    }
    return s;
}

static void kd_query_ex(const kd_tree* t, int id, const double x[3], long long excl, double* best, long long* arg);

static void kd_query(const kd_tree* t, int id, const double x[3], double* best, long long* arg) {
    kd_query_ex(t, id, x, -1, best, arg);
}

/* the same search, never returning point excl */
static void kd_query_ex(const kd_tree* t, int id, const double x[3], long long excl, double* best, long long* arg) {
    const kd_node* nd = &t->nodes[id];
    if (nd->axis < 0) {
        for (long long i = nd->lo; i < nd->hi; ++i) {
            long long q = t->perm[i];
            if (q == excl) continue;
            const double* Q = t->pts + q * t->dim;
            double s = 0.0;
            for (int a = 0; a < t->dim; ++a) {
                double diff = x[a] - Q[a];
                s = s + diff * diff;
            }
            if (s < *best || (s == *best && q < *arg)) {
                *best = s;
                *arg = q;
            }
        }
        return;
    }
    const double bl = kd_box_bound(t, &t->nodes[nd->left], x);
    const double br = kd_box_bound(t, &t->nodes[nd->right], x);
    const int first = bl <= br ? nd->left : nd->right, second = bl <= br ? nd->right : nd->left;
    const double b1 = bl <= br ? bl : br, b2 = bl <= br ? br : bl;
    if (!(b1 > *best)) kd_query_ex(t, first, x, excl, best, arg);
    if (!(b2 > *best)) kd_query_ex(t, second, x, excl, best, arg);
}

void or_distance_kd(const or_params* g, const double* pts, long long npts,
                    const long long* nodes, long long m, double* d_out, int* arg_out) {
    kd_tree t;
    t.pts = pts;
    t.dim = g->dim;
    t.perm = (long long*)malloc(sizeof(long long) * (size_t)npts);
    t.nodes = (kd_node*)malloc(sizeof(kd_node) * (size_t)(2 * (npts / 4 + 2)));
    t.count = 0;
    for (long long i = 0; i < npts; ++i) t.perm[i] = i;
    kd_build(&t, 0, npts);
    long long count = nodes ? m : or_num_nodes(g);
#pragma omp parallel for schedule(dynamic, 256)
    for (long long k = 0; k < count; ++k) {
        long long idx = nodes ? nodes[k] : k;
        double x[3];
        or_node_coord(g, idx, x);
        double best = INFINITY;
        long long arg = 0x7fffffffffffffffll;
        kd_query(&t, 0, x, &best, &arg);
        d_out[k] = sqrt(best);
        if (arg_out) arg_out[k] = (int)arg;
    }
    free(t.perm);
    free(t.nodes);
}

/* §4 (eq. dxdt) cloud resolution h_S: mean over the sample of the distance
 * from each sampled point to its nearest other point (a duplicate counts, at
 * distance 0), summed in sample order */
double or_cloud_spacing(int dim, const double* pts, long long npts, const long long* sample, long long m) {
    kd_tree t;
    t.pts = pts;
    t.dim = dim;
    t.perm = (long long*)malloc(sizeof(long long) * (size_t)npts);
    t.nodes = (kd_node*)malloc(sizeof(kd_node) * (size_t)(2 * (npts / 4 + 2)));
    t.count = 0;
    for (long long i = 0; i < npts; ++i) t.perm[i] = i;
    kd_build(&t, 0, npts);
    double* dist = (double*)malloc(sizeof(double) * (size_t)m);
#pragma omp parallel for schedule(dynamic, 256)
    for (long long s = 0; s < m; ++s) {
        const long long p = sample[s];
        double x[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < dim; ++a) x[a] = pts[p * dim + a];
        double best = INFINITY;
        long long arg = -1;
        kd_query_ex(&t, 0, x, p, &best, &arg);
        dist[s] = sqrt(best);
    }
    double acc = 0.0;
    for (long long s = 0; s < m; ++s) acc += dist[s];
    free(dist);
    free(t.perm);
    free(t.nodes);
    return acc / (double)m;
}

/* ------------------------------------------------------------------ */
/* §3: centred finite differences                                       */
/* ------------------------------------------------------------------ */

void or_gradient(const or_params* g, const double* v, long long idx, double grad[3]) {
    long long ijk[3];
    unflatten(g, idx, ijk);
    for (int a = 0; a < 3; ++a) grad[a] = 0.0;
    for (int a = 0; a < g->dim; ++a) {
        long long lo_ijk[3] = {ijk[0], ijk[1], ijk[2]};
        long long hi_ijk[3] = {ijk[0], ijk[1], ijk[2]};
        if (ijk[a] > 0 && ijk[a] < g->n[a] - 1) {
            lo_ijk[a] -= 1;
            hi_ijk[a] += 1;
            grad[a] = (v[flatten(g, hi_ijk[0], hi_ijk[1], hi_ijk[2])] -
                       v[flatten(g, lo_ijk[0], lo_ijk[1], lo_ijk[2])]) / (2.0 * g->h);
        } else if (ijk[a] == 0) {
            hi_ijk[a] += 1;
            grad[a] = (v[flatten(g, hi_ijk[0], hi_ijk[1], hi_ijk[2])] - v[idx]) / g->h;
        } else {
            lo_ijk[a] -= 1;
            grad[a] = (v[idx] - v[flatten(g, lo_ijk[0], lo_ijk[1], lo_ijk[2])]) / g->h;
        }
    }
}

/* ------------------------------------------------------------------ */
/* §3.2: interpolators                                                  */
/* ------------------------------------------------------------------ */

/* index-space coordinate of x on axis a, clamped to [0, n-1]; returns the
 * cell index i0 in [0, n-2] and the local coordinate t = xi - i0 in [0, 1] */
static void locate(const or_params* g, const double x[3], int a, long long* i0, double* t) {
    double xi = (x[a] - g->lo[a]) / g->h;
    double top = (double)(g->n[a] - 1);
    if (xi < 0.0) xi = 0.0;
    if (xi > top) xi = top;
    long long c = (long long)floor(xi);
    if (c > g->n[a] - 2) c = g->n[a] - 2;
    *i0 = c;
    *t = xi - (double)c;
}

/* eq. IQ1: Q1 finite-element interpolation. Inside the cell holding x the
 * tensor-product shape functions reduce to linear interpolation along x, then
 * along y, then along z. */
double or_interp_q1(const or_params* g, const double* v, const double x[3]) {
    long long c[3] = {0, 0, 0};
    double t[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < g->dim; ++a) locate(g, x, a, &c[a], &t[a]);
    double vz[2];
    int nz = (g->dim == 3) ? 2 : 1;
    for (int dz = 0; dz < nz; ++dz) {
        double vy[2];
        for (int dy = 0; dy < 2; ++dy) {
            double v0 = v[flatten(g, c[0], c[1] + dy, c[2] + dz)];
            double v1 = v[flatten(g, c[0] + 1, c[1] + dy, c[2] + dz)];
            vy[dy] = (1.0 - t[0]) * v0 + t[0] * v1;
        }
        vz[dz] = (1.0 - t[1]) * vy[0] + t[1] * vy[1];
    }
    if (g->dim == 2) return vz[0];
    return (1.0 - t[2]) * vz[0] + t[2] * vz[1];
}

/* eq. IWENO with n = 2 on the cell [x_j, x_{j+1}] of a uniform mesh of
 * width h. v = (v_{j-1}, v_j, v_{j+1}, v_{j+2}); theta = (x - x_j)/h.
 *  - P_L interpolates v on S_L = {x_{j-1}, x_j, x_{j+1}}, P_R on
 *    S_R = {x_j, x_{j+1}, x_{j+2}} (Lagrange form, nodes at -1,0,1 / 0,1,2);
 *  - linear weights, eq. ckgamma: C_k(x) = γ_k (x - x̂_k)/Δx with
 *    γ_L = -1/3, x̂_L = x_{j+2} and γ_R = 1/3, x̂_R = x_{j-1};
 *  - regularity indicators, eq. ind:1d, as the quadratic forms
 *    I_k = V^T A_k V / Δx^2 with the matrices A_L, A_R of §3.2;
 *  - α_k = C_k / (I_k + ε)^2 with ε = Δx^2; w_k = α_k / Σ α; I = Σ w_k P_k.
 * w (may be NULL) receives (w_L, w_R). */
double or_weno1d_weights(const double v[4], double theta, double h, double w[2]) {
    static const double A_L[4][4] = {{1, -2, 1, 0}, {-2, 4, -2, 0}, {1, -2, 1, 0}, {0, 0, 0, 0}};
    static const double A_R[4][4] = {{0, 0, 0, 0}, {0, 1, -2, 1}, {0, -2, 4, -2}, {0, 1, -2, 1}};
    double s = theta;
    /* Lagrange basis on nodes -1, 0, 1 (P_L) and 0, 1, 2 (P_R) */
    double PL = v[0] * (s * (s - 1.0) / 2.0) + v[1] * ((1.0 - s) * (1.0 + s)) + v[2] * (s * (s + 1.0) / 2.0);
    double PR = v[1] * ((s - 1.0) * (s - 2.0) / 2.0) + v[2] * (s * (2.0 - s)) + v[3] * (s * (s - 1.0) / 2.0);
    double IL = 0.0, IR = 0.0;
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            IL += v[r] * A_L[r][c] * v[c];
            IR += v[r] * A_R[r][c] * v[c];
        }
    IL /= h * h;
    IR /= h * h;
    /* positions in units of h relative to x_j: x_{j-1} = -1, x_{j+2} = 2 */
    double CL = (-1.0 / 3.0) * (s - 2.0);
    double CR = (1.0 / 3.0) * (s - (-1.0));
    double eps = h * h;
    double aL = CL / ((IL + eps) * (IL + eps));
    double aR = CR / ((IR + eps) * (IR + eps));
    double wL = aL / (aL + aR);
    double wR = aR / (aL + aR);
    if (w) {
        w[0] = wL;
        w[1] = wR;
    }
    return wL * PL + wR * PR;
}

double or_weno1d(const double v[4], double theta, double h) { return or_weno1d_weights(v, theta, h, NULL); }

/* §3.2, multi-dimensional WENO by dimension splitting: in 3-D, 16 one-
 * dimensional interpolations along z (one per (x,y) stencil column), then 4
 * along y, then 1 along x; in 2-D, 4 along y then 1 along x. Stencil nodes
 * outside the grid take the nearest edge value. */
double or_interp_weno(const or_params* g, const double* v, const double x[3]) {
    long long c[3] = {0, 0, 0};
    double t[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < g->dim; ++a) locate(g, x, a, &c[a], &t[a]);
    double colx[4];
    for (int a = 0; a < 4; ++a) {
        long long ii = clampi(c[0] - 1 + a, 0, g->n[0] - 1);
        double coly[4];
        for (int b = 0; b < 4; ++b) {
            long long jj = clampi(c[1] - 1 + b, 0, g->n[1] - 1);
            if (g->dim == 3) {
                double line[4];
                for (int e = 0; e < 4; ++e) {
                    long long kk = clampi(c[2] - 1 + e, 0, g->n[2] - 1);
                    line[e] = v[flatten(g, ii, jj, kk)];
                }
                coly[b] = or_weno1d(line, t[2], g->h);
            } else {
                coly[b] = v[flatten(g, ii, jj, 0)];
            }
        }
        colx[a] = or_weno1d(coly, t[1], g->h);
    }
    return or_weno1d(colx, t[0], g->h);
}

double or_interp(const or_params* g, const double* v, const double x[3]) {
    return g->interp == 1 ? or_interp_weno(g, v, x) : or_interp_q1(g, v, x);
}

/* ------------------------------------------------------------------ */
/* §3.8: band, cut, cut-off                                             */
/* ------------------------------------------------------------------ */

/* γ as represented in the storage precision */
static double gamma_s(const or_params* g) { return g->prec == 32 ? (double)(float)g->gamma : g->gamma; }

/* eq. subgrid, read as |φ_j| < γ, decided in the storage precision */
int or_in_band(const or_params* g, double u) {
    if (g->prec == 32) return (float)fabs(u) < (float)g->gamma;
    return fabs(u) < g->gamma;
}

/* eq. cut */
double or_cut(const or_params* g, double u) {
    double gm = gamma_s(g);
    if (u > gm) return gm;
    if (u < -gm) return -gm;
    return u;
}

void or_cut_all(const or_params* g, double* u) {
    long long N = or_num_nodes(g);
    for (long long i = 0; i < N; ++i) u[i] = or_cut(g, u[i]);
}

long long or_band(const or_params* g, const double* u, long long* list_out) {
    long long N = or_num_nodes(g), m = 0;
    for (long long i = 0; i < N; ++i)
        if (or_in_band(g, u[i])) {
            if (list_out) list_out[m] = i;
            ++m;
        }
    return m;
}

/* eq. cutoff */
double or_cutoff(const or_params* g, double u) {
    double a = fabs(u), gm = g->gamma, b = g->beta;
    if (a <= b) return 1.0;
    if (a <= gm) return (a - gm) * (a - gm) * (2.0 * a + gm - 3.0 * b) / ((gm - b) * (gm - b) * (gm - b));
    return 0.0;
}

/* ------------------------------------------------------------------ */
/* §3.1: tangent directions and feet                                    */
/* ------------------------------------------------------------------ */

/* eq. sigma2d: σ = (∂2φ, -∂1φ) / |∇φ| */
void or_sigma2d(const double grad[3], double sigma[3]) {
    double nrm = sqrt(grad[0] * grad[0] + grad[1] * grad[1]);
    sigma[0] = grad[1] / nrm;
    sigma[1] = -grad[0] / nrm;
    sigma[2] = 0.0;
}

/* eq. sigma3d with the regularisation of §3.1: ν1 = (1,0,0), ν2 = (0,0,1)
 * when sqrt((∂1φ)^2 + (∂3φ)^2) == 0. Returns 1 when regularised. */
int or_tangent_basis(const double grad[3], double nu1[3], double nu2[3]) {
    double g1 = grad[0], g2 = grad[1], g3 = grad[2];
    double r = sqrt(g1 * g1 + g3 * g3);
    if (r == 0.0) {
        nu1[0] = 1.0; nu1[1] = 0.0; nu1[2] = 0.0;
        nu2[0] = 0.0; nu2[1] = 0.0; nu2[2] = 1.0;
        return 1;
    }
    double nrm = sqrt(g1 * g1 + g2 * g2 + g3 * g3);
    nu1[0] = -g3 / r;
    nu1[1] = 0.0;
    nu1[2] = g1 / r;
    nu2[0] = (1.0 / nrm) * (-g1 * g2 / r);
    nu2[1] = (1.0 / nrm) * r;
    nu2[2] = (1.0 / nrm) * (-g2 * g3 / r);
    return 0;
}

/* eq. SL2d / SL3d: x* = x_j + C Δt ∇d(x_j) + sqrt(C δ d(x_j) Δt / p) σ λ_i,
 * λ over {-1, +1} (2-D) or {(-,-), (-,+), (+,-), (+,+)} (3-D), σλ = λ1 ν1 + λ2 ν2. */
int or_feet(const or_params* g, const double xj[3], const double grad_u[3], const double grad_d[3],
            double dj, double ct, double feet[4][3]) {
    double base[3];
    for (int a = 0; a < 3; ++a) base[a] = xj[a] + ct * g->dt * grad_d[a];
    double s = sqrt(ct * g->delta * dj * g->dt / g->p);
    if (g->dim == 2) {
        double sigma[3];
        or_sigma2d(grad_u, sigma);
        static const double lam[2] = {-1.0, 1.0};
        for (int i = 0; i < 2; ++i)
            for (int a = 0; a < 3; ++a) feet[i][a] = base[a] + s * sigma[a] * lam[i];
        return 2;
    }
    double nu1[3], nu2[3];
    or_tangent_basis(grad_u, nu1, nu2);
    static const double lam[4][2] = {{-1, -1}, {-1, 1}, {1, -1}, {1, 1}};
    for (int i = 0; i < 4; ++i)
        for (int a = 0; a < 3; ++a) feet[i][a] = base[a] + s * (lam[i][0] * nu1[a] + lam[i][1] * nu2[a]);
    return 4;
}

/* C^n_j = (d(x_j) / E_p(φ^n))^(p-1) (§3.1); C = 1 for p = 1 (§4) */
double or_scale_factor(const or_params* g, double dj, double Ep) {
    if (g->p == 1.0) return 1.0;
    if (!(Ep > 0.0)) return 0.0;
    return pow(dj / Ep, g->p - 1.0);
}

/* ------------------------------------------------------------------ */
/* §3.1: one SL update                                                  */
/* ------------------------------------------------------------------ */

double or_sl_node(const or_params* g, const double* u, const double* d, double Ep, long long idx, int* flags) {
    int f = 0;
    double gu[3], gd[3], x[3];
    or_gradient(g, u, idx, gu);
    double nrm = sqrt(gu[0] * gu[0] + gu[1] * gu[1] + gu[2] * gu[2]);
    double thr = g->c_sing * pow(g->dt, g->alpha);
    if (fabs(nrm - thr) <= 1e-6 * thr) f |= OR_FLAG_MARGIN;
    if (nrm < thr) {
        /* eq. SL:2: mean over the first (face) neighbours inside the grid */
        long long ijk[3];
        unflatten(g, idx, ijk);
        double sum = 0.0;
        int cnt = 0;
        for (int a = 0; a < g->dim; ++a)
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                long long nb[3] = {ijk[0], ijk[1], ijk[2]};
                nb[a] += sgn;
                if (nb[a] < 0 || nb[a] >= g->n[a]) continue;
                sum += u[flatten(g, nb[0], nb[1], nb[2])];
                ++cnt;
            }
        if (flags) *flags = f | OR_FLAG_FALLBACK;
        return sum / (double)cnt;
    }
    or_gradient(g, d, idx, gd);
    or_node_coord(g, idx, x);
    double dj = d[idx];
    double ct = or_scale_factor(g, dj, Ep);
    if (g->band) ct = or_cutoff(g, u[idx]) * ct;
    if (g->dim == 3 && gu[0] == 0.0 && gu[2] == 0.0) f |= OR_FLAG_REGULAR;
    double feet[4][3];
    int nf = or_feet(g, x, gu, gd, dj, ct, feet);
    double sum = 0.0;
    for (int i = 0; i < nf; ++i) sum += or_interp(g, u, feet[i]);
    if (flags) *flags = f;
    return sum / (double)nf;
}

void or_sl_nodes(const or_params* g, const double* u, const double* d, double Ep,
                 const long long* nodes, long long m, double* out, int* flags) {
#pragma omp parallel for schedule(dynamic, 256)
    for (long long t = 0; t < m; ++t) out[t] = or_sl_node(g, u, d, Ep, nodes[t], flags ? flags + t : NULL);
}

/* One iteration of Algorithm 1 without the reinitialisation: band, SL update, cut */
double or_sl_step(const or_params* g, const double* u, const double* d, double Ep, double* u_out, int* flags_out) {
    long long N = or_num_nodes(g);
    long long slab = g->n[0] * g->n[1];
    long long nslab = g->n[2];
    double* part = (double*)calloc((size_t)nslab, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (long long k = 0; k < nslab; ++k) {
        double acc = 0.0;
        for (long long idx = k * slab; idx < (k + 1) * slab; ++idx) {
            double v;
            int f = 0;
            if (!g->band || or_in_band(g, u[idx]))
                v = or_sl_node(g, u, d, Ep, idx, &f);
            else
                v = u[idx];
            if (g->band) v = or_cut(g, v);
            u_out[idx] = v;
            if (flags_out) flags_out[idx] = f;
            acc += fabs(v - u[idx]);
        }
        part[k] = acc;
    }
    double total = 0.0;
    for (long long k = 0; k < nslab; ++k) total += part[k];
    free(part);
    (void)N;
    return total * pow(g->h, (double)g->dim);
}

/* ------------------------------------------------------------------ */
/* §3.5: energy                                                         */
/* ------------------------------------------------------------------ */

static int negative(double v) { return v < 0.0; }

/* 2-D: the front crosses the cell edges where φ changes sign (linear
 * interpolation of φ along the edge); d at a crossing is interpolated
 * linearly along the edge; trapezoid rule on the segment(s). */
static double energy_cell_2d(const or_params* g, const double* u, const double* d, double p,
                             long long i, long long j) {
    /* corners in the order 00, 10, 11, 01; edge e joins corner e and e+1 */
    long long id[4] = {flatten(g, i, j, 0), flatten(g, i + 1, j, 0), flatten(g, i + 1, j + 1, 0),
                       flatten(g, i, j + 1, 0)};
    double cx[4] = {0, 1, 1, 0}, cy[4] = {0, 0, 1, 1};
    double uv[4], dv[4];
    for (int c = 0; c < 4; ++c) {
        uv[c] = u[id[c]];
        dv[c] = d[id[c]];
    }
    double px[4], py[4], pd[4];
    int has[4] = {0, 0, 0, 0}, nc = 0;
    for (int e = 0; e < 4; ++e) {
        int a = e, b = (e + 1) % 4;
        if (negative(uv[a]) != negative(uv[b])) {
            double t = uv[a] / (uv[a] - uv[b]);
            px[e] = (cx[a] + t * (cx[b] - cx[a])) * g->h;
            py[e] = (cy[a] + t * (cy[b] - cy[a])) * g->h;
            pd[e] = dv[a] + t * (dv[b] - dv[a]);
            has[e] = 1;
            ++nc;
        }
    }
    if (nc == 0) return 0.0;
    int pairs[2][2], np = 0;
    if (nc == 2) {
        int k = 0;
        for (int e = 0; e < 4; ++e)
            if (has[e]) pairs[0][k++] = e;
        np = 1;
    } else {
        /* four crossings: corners 00 and 11 share a sign. If the cell mean
         * has that sign too, the segments cut off corners 10 (edges 0,1) and
         * 01 (edges 2,3); otherwise corners 00 (edges 3,0) and 11 (edges 1,2). */
        double mean = (uv[0] + uv[1] + uv[2] + uv[3]) / 4.0;
        if (negative(mean) == negative(uv[0])) {
            pairs[0][0] = 0; pairs[0][1] = 1;
            pairs[1][0] = 2; pairs[1][1] = 3;
        } else {
            pairs[0][0] = 3; pairs[0][1] = 0;
            pairs[1][0] = 1; pairs[1][1] = 2;
        }
        np = 2;
    }
    double acc = 0.0;
    for (int s = 0; s < np; ++s) {
        int e1 = pairs[s][0], e2 = pairs[s][1];
        double len = sqrt((px[e1] - px[e2]) * (px[e1] - px[e2]) + (py[e1] - py[e2]) * (py[e1] - py[e2]));
        acc += len * (pow(fabs(pd[e1]), p) + pow(fabs(pd[e2]), p)) / 2.0;
    }
    return acc;
}

/* 3-D, eq. energyApproxFiner: the front cell is split into R^3 subcells of
 * width Δx' = Δx/R; a subcell counts when the reconstruction of φ at its
 * centre (the active interpolator) satisfies |φ(x')| < (√3/2) Δx'; it adds
 * |d(x')|^p (Δx')^2 with d interpolated by Q1. */
static double energy_cell_3d(const or_params* g, const double* u, const double* d, double p, int R,
                             long long i, long long j, long long k, double amb_tol, double* amb) {
    double hp = g->h / (double)R;
    double thr = sqrt(3.0) / 2.0 * hp;
    or_params gq = *g;
    gq.interp = 0;
    double x0[3];
    or_node_coord(g, flatten(g, i, j, k), x0);
    double acc = 0.0;
    for (int c = 0; c < R; ++c)
        for (int b = 0; b < R; ++b)
            for (int a = 0; a < R; ++a) {
                double xp[3] = {x0[0] + ((double)a + 0.5) * hp, x0[1] + ((double)b + 0.5) * hp,
                                x0[2] + ((double)c + 0.5) * hp};
                double up = or_interp(g, u, xp);
                double contrib = pow(fabs(or_interp_q1(&gq, d, xp)), p) * hp * hp;
                if (fabs(up) < thr) acc += contrib;
                if (fabs(fabs(up) - thr) <= amb_tol) *amb += contrib;
            }
    return acc;
}

static int front_cell(const or_params* g, const double* u, long long i, long long j, long long k) {
    int nz = g->dim == 3 ? 2 : 1;
    int seen_neg = 0, seen_pos = 0;
    for (int dz = 0; dz < nz; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                if (negative(u[flatten(g, i + dx, j + dy, k + dz)]))
                    seen_neg = 1;
                else
                    seen_pos = 1;
            }
    return seen_neg && seen_pos;
}

void or_energy(const or_params* g, const double* u, const double* d, double p, int R, double amb_tol, double out[4]) {
    long long nk = g->dim == 3 ? g->n[2] - 1 : 1;
    double* part = (double*)calloc((size_t)nk, sizeof(double));
    double* pamb = (double*)calloc((size_t)nk, sizeof(double));
    long long* pcnt = (long long*)calloc((size_t)nk, sizeof(long long));
#pragma omp parallel for schedule(dynamic, 1)
    for (long long k = 0; k < nk; ++k) {
        double acc = 0.0, amb = 0.0;
        long long cnt = 0;
        for (long long j = 0; j < g->n[1] - 1; ++j)
            for (long long i = 0; i < g->n[0] - 1; ++i) {
                if (!front_cell(g, u, i, j, k)) continue;
                ++cnt;
                if (g->dim == 2)
                    acc += energy_cell_2d(g, u, d, p, i, j);
                else
                    acc += energy_cell_3d(g, u, d, p, R, i, j, k, amb_tol, &amb);
            }
        part[k] = acc;
        pamb[k] = amb;
        pcnt[k] = cnt;
    }
    double total = 0.0, amb = 0.0;
    long long cnt = 0;
    for (long long k = 0; k < nk; ++k) {
        total += part[k];
        amb += pamb[k];
        cnt += pcnt[k];
    }
    free(part);
    free(pamb);
    free(pcnt);
    out[0] = total;
    out[1] = pow(total, 1.0 / p);
    out[2] = amb;
    out[3] = (double)cnt;
}

/* ------------------------------------------------------------------ */
/* §4: stopping criterion, evolution loop, diagnostics                 */
/* ------------------------------------------------------------------ */

/* eq. deltaEn: ē_n = (1/k) Σ_{i=n-k+1..n} E_2(φ^i), k = min(n, kmax);
 * stop when Δ_E^n = |ē_{n-1} - ē_n| / ē_n < tol and n >= min_iters, or when
 * n reaches max_iters. */
int or_stop(const double* E2, int n, int kmax, double tol, int min_iters, int max_iters, double* delta_out) {
    double delta = -1.0;
    if (n >= 1) {
        int k = n < kmax ? n : kmax;
        double en = 0.0, em = 0.0;
        for (int i = n - k + 1; i <= n; ++i) en += E2[i];
        for (int i = n - k; i <= n - 1; ++i) em += E2[i];
        en /= (double)k;
        em /= (double)k;
        if (en > 0.0)
            delta = fabs(em - en) / en;
        else
            delta = (em == en) ? 0.0 : INFINITY;
    }
    if (delta_out) *delta_out = delta;
    if (n >= max_iters) return 1;
    if (n >= min_iters && delta >= 0.0 && delta < tol) return 1;
    return 0;
}

/* ------------------------------------------------------------------ */
/* §3.7 reinitialisation (Algorithm 1)                                  */
/* ------------------------------------------------------------------ */

/* The paper runs the constrained reinitialisation of Hartmann, Meinke and
 * Schröder (2008) on Ḡ = G̃ and its first neighbours: one explicit step sets
 * the signed distance on the nodes next to the interface (a sign change of
 * φ̃ to a face neighbour); then forward-Euler steps in pseudo-time τ of the
 * first-order discretisation of eq. reinit, φ_τ + sign(φ̃)(|∇φ| - 1) = 0
 * (Sussman, Smereka and Osher 1994), reinitialise the rest of Ḡ while the
 * interface nodes stay fixed; then eq. cut. The paper gives no formulas for
 * either part; the readings taken here:
 *  - sign classes: φ < 0 and φ >= 0 (zero with the positive side, as in the
 *    energy of §3.5); sign(φ̃) in eq. reinit is -1, 0, +1;
 *  - explicit step on an interface node j ("one step", keeping the
 *    interface where φ̃ puts it), in two parts:
 *    (a) the subcell estimate of Russo and Smereka (2000) on every interface
 *        node k: D_k = φ̃_k / Δ_k with Δ_k the largest of the norm of the
 *        gradient (centred components (φ̃_{k+e} - φ̃_{k-e})/(2h), one-sided
 *        on the domain boundary) and the one-sided differences
 *        |φ̃_{k±e} - φ̃_k|/h (those that exist); D_k = φ̃_k if Δ_k = 0.
 *        Exact for any plane, scaled or not;
 *    (b) the constraint of the constrained reinitialisation: with S_j the
 *        face neighbours of j of the other sign class, φ_j = φ̃_j Σ_{k∈S_j}
 *        D_k / Σ_{k∈S_j} φ̃_k, so that j keeps against its neighbours across
 *        the interface the ratio it has in φ̃ (the zero crossings of the
 *        linear interpolant do not move, on average over S_j); D_j if the
 *        sum of φ̃ over S_j is 0;
 *  - first-order discretisation: Godunov's upwind Hamiltonian with the
 *    one-sided differences a = (ψ_j - ψ_{j-e})/h, b = (ψ_{j+e} - ψ_j)/h per
 *    axis (a missing neighbour outside the grid gives a difference of 0):
 *    sign > 0: |∇ψ|^2 = Σ_a max(max(a,0)^2, min(b,0)^2),
 *    sign < 0: |∇ψ|^2 = Σ_a max(min(a,0)^2, max(b,0)^2);
 *  - Jacobi sweeps ψ^{m+1}_j = ψ^m_j - Δτ sign(φ̃_j)(|∇ψ^m|_j - 1) on
 *    Ḡ minus the interface nodes and minus the nodes on the domain boundary
 *    (no upwind data enters from outside the grid: they keep φ̃, which
 *    keeps the scheme from drifting there), Δτ = h/2 (within h/sqrt(dim), the
 *    stability limit of the scheme), for M = 4(γ/h + 1) sweeps: information
 *    moves h/2 per sweep, so 2(γ/h + 1) sweeps reach across the band and its
 *    first neighbours, and as many again bring the band to within about
 *    10^-4 h of the steady state of eq. reinit ("until steady state");
 *    nodes outside Ḡ keep their values;
 *  - the band G̃ whose neighbours form Ḡ is the one the SL step used,
 *    {j : |φ^n_j| < γ}, given here by phi_band.
 * Returns |Ḡ|. out receives φ̃ outside Ḡ and the cut reinitialised values
 * in Ḡ. flags_out (may be NULL): bit 0 node in Ḡ, bit 1 interface node. */
static int sign_class(double v) { return v < 0.0 ? -1 : 1; }

/* (a) the Russo-Smereka estimate at node idx (of v = φ̃) */
static double reinit_rs_estimate(const or_params* g, const double* v, long long idx) {
    long long stride[3] = {1, g->n[0], g->n[0] * g->n[1]};
    long long c[3] = {idx % g->n[0], (idx / g->n[0]) % g->n[1], idx / (g->n[0] * g->n[1])};
    double vj = v[idx], cn = 0.0, mx = 0.0;
    for (int a = 0; a < g->dim; ++a) {
        int has_m = c[a] > 0, has_p = c[a] < g->n[a] - 1;
        if (has_m) mx = fmax(mx, fabs(vj - v[idx - stride[a]]) / g->h);
        if (has_p) mx = fmax(mx, fabs(v[idx + stride[a]] - vj) / g->h);
        /* the gradient component: centred, one-sided on the domain boundary (reading of §3) */
        double ce = 0.0;
        if (has_m && has_p)
            ce = (v[idx + stride[a]] - v[idx - stride[a]]) / (2.0 * g->h);
        else if (has_p)
            ce = (v[idx + stride[a]] - vj) / g->h;
        else if (has_m)
            ce = (vj - v[idx - stride[a]]) / g->h;
        cn = cn + ce * ce;
    }
    double den = fmax(sqrt(cn), mx);
    if (!(den > 0.0)) return vj;
    return vj / den;
}

/* the explicit value of interface node idx: (a), then the constraint (b) */
static double reinit_one_step(const or_params* g, const double* v, long long idx) {
    long long stride[3] = {1, g->n[0], g->n[0] * g->n[1]};
    long long c[3] = {idx % g->n[0], (idx / g->n[0]) % g->n[1], idx / (g->n[0] * g->n[1])};
    int cj = v[idx] < 0.0 ? -1 : 1;
    double sd = 0.0, sp = 0.0;
    for (int a = 0; a < g->dim; ++a)
        for (int side = -1; side <= 1; side += 2) {
            long long q = c[a] + side;
            if (q < 0 || q >= g->n[a]) continue;
            long long k = idx + side * stride[a];
            if ((v[k] < 0.0 ? -1 : 1) == cj) continue;
            sd = sd + reinit_rs_estimate(g, v, k);
            sp = sp + v[k];
        }
    if (sp == 0.0) return reinit_rs_estimate(g, v, idx);
    return v[idx] * sd / sp;
}

static int reinit_is_interface(const or_params* g, const double* v, long long idx) {
    long long stride[3] = {1, g->n[0], g->n[0] * g->n[1]};
    long long c[3] = {idx % g->n[0], (idx / g->n[0]) % g->n[1], idx / (g->n[0] * g->n[1])};
    int cj = sign_class(v[idx]);
    for (int a = 0; a < g->dim; ++a)
        for (int side = -1; side <= 1; side += 2) {
            long long q = c[a] + side;
            if (q < 0 || q >= g->n[a]) continue;
            if (sign_class(v[idx + side * stride[a]]) != cj) return 1;
        }
    return 0;
}

/* node idx is not on the domain boundary: all 2·dim face neighbours exist */
static double godunov_norm(const or_params* g, const double* v, long long idx, int sgn) {
    long long stride[3] = {1, g->n[0], g->n[0] * g->n[1]};
    double vj = v[idx], s2 = 0.0;
    for (int a = 0; a < g->dim; ++a) {
        double am = (vj - v[idx - stride[a]]) / g->h;
        double bp = (v[idx + stride[a]] - vj) / g->h;
        double t1, t2;
        if (sgn > 0) {
            t1 = am > 0.0 ? am : 0.0;
            t2 = bp < 0.0 ? bp : 0.0;
        } else {
            t1 = am < 0.0 ? am : 0.0;
            t2 = bp > 0.0 ? bp : 0.0;
        }
        t1 = t1 * t1;
        t2 = t2 * t2;
        s2 = s2 + (t1 > t2 ? t1 : t2);
    }
    return sqrt(s2);
}

int or_reinit_sweeps(const or_params* g) { return 4 * ((int)floor(g->gamma / g->h + 0.5) + 1); }

long long or_reinit(const or_params* g, const double* phi_band, const double* phi_tilde, int sweeps, double dtau,
                    double* out, unsigned char* flags_out) {
    long long N = or_num_nodes(g);
    long long stride[3] = {1, g->n[0], g->n[0] * g->n[1]};
    if (sweeps <= 0) sweeps = or_reinit_sweeps(g);
    if (!(dtau > 0.0)) dtau = 0.5 * g->h;
    unsigned char* fl = (unsigned char*)calloc((size_t)N, 1);
    /* Ḡ: the band and its face neighbours */
    for (long long i = 0; i < N; ++i) {
        if (!or_in_band(g, phi_band[i])) continue;
        fl[i] |= 1;
        long long c[3] = {i % g->n[0], (i / g->n[0]) % g->n[1], i / (g->n[0] * g->n[1])};
        for (int a = 0; a < g->dim; ++a) {
            if (c[a] > 0) fl[i - stride[a]] |= 1;
            if (c[a] < g->n[a] - 1) fl[i + stride[a]] |= 1;
        }
    }
    long long m = 0;
    for (long long i = 0; i < N; ++i) m += fl[i] & 1;
    double* psi = (double*)malloc((size_t)N * sizeof(double));
    double* nxt = (double*)malloc((size_t)N * sizeof(double));
    memcpy(psi, phi_tilde, (size_t)N * sizeof(double));
    /* explicit step on the interface nodes of Ḡ */
    for (long long i = 0; i < N; ++i)
        if ((fl[i] & 1) && reinit_is_interface(g, phi_tilde, i)) fl[i] |= 2;
    for (long long i = 0; i < N; ++i)
        if (fl[i] & 2) psi[i] = reinit_one_step(g, phi_tilde, i);
    /* forward-Euler Jacobi sweeps on the rest of Ḡ */
    for (int it = 0; it < sweeps; ++it) {
        memcpy(nxt, psi, (size_t)N * sizeof(double));
#pragma omp parallel for schedule(static)
        for (long long i = 0; i < N; ++i) {
            if ((fl[i] & 3) != 1) continue;
            long long c[3] = {i % g->n[0], (i / g->n[0]) % g->n[1], i / (g->n[0] * g->n[1])};
            int edge = 0;
            for (int a = 0; a < g->dim; ++a) edge |= (c[a] == 0 || c[a] == g->n[a] - 1);
            if (edge) continue;
            double v = phi_tilde[i];
            int sgn = v > 0.0 ? 1 : (v < 0.0 ? -1 : 0);
            if (sgn == 0) continue;
            nxt[i] = psi[i] - dtau * (double)sgn * (godunov_norm(g, psi, i, sgn) - 1.0);
        }
        double* t = psi;
        psi = nxt;
        nxt = t;
    }
    for (long long i = 0; i < N; ++i) out[i] = (fl[i] & 1) ? or_cut(g, psi[i]) : phi_tilde[i];
    if (flags_out) memcpy(flags_out, fl, (size_t)N);
    free(fl);
    free(psi);
    free(nxt);
    return m;
}

/* ------------------------------------------------------------------ */
/* §3.6 initial data: external marking, then fast sweeping               */
/* ------------------------------------------------------------------ */

/* Readings (the paper describes the steps in words):
 *  - marking: every node on the grid boundary is external; then one round of
 *    directional sweeps along the grid lines, in the order +x, -x, +y, -y
 *    (+z, -z): a sweep in direction +x visits each line in increasing x and
 *    marks a node external when the node before it is external and its own
 *    d >= γ_S ("until we find a point for which d < γ_S"). The paper
 *    iterates the round only in parallel runs, to reproduce this serial
 *    result;
 *  - φ0 = d - γ_S on external nodes, 1e30 (the "artificially high value")
 *    on the others;
 *  - fast sweeping (Zhao 2005) on the internal nodes: Gauss-Seidel sweeps in
 *    the 2^dim orderings (x, y, z each increasing or decreasing; the sign
 *    patterns in binary order, bit a set = axis a decreasing, x fastest in
 *    every ordering), two rounds; the update is the Godunov local solution
 *    of |∇φ| = 1 with a_a = min(φ_{j-e_a}, φ_{j+e_a}) (the one that exists on
 *    the boundary), sorted a_1 <= a_2 <= a_3:
 *      x = a_1 + h; if x > a_2: x = (a_1 + a_2 + sqrt(2h² - (a_1 - a_2)²))/2;
 *      if x > a_3 (3-D): x = (s + sqrt(s² - 3(a_1² + a_2² + a_3² - h²)))/3,
 *      s = a_1 + a_2 + a_3; and φ_j = min(φ_j, x); external nodes keep theirs;
 *  - finally φ0 = -φ on the internal nodes.
 * out: φ0 on every node; ext_out (may be NULL): 1 on external nodes.
 * Returns the number of external nodes. */
/* Godunov local solution of |∇φ| = 1 from the per-axis upwind values a[0..m) */
double or_fsm_solve(const double* a_in, int m, double h) {
    double a[3];
    for (int i = 0; i < m; ++i) a[i] = a_in[i];
    /* sort ascending (insertion, at most 3 values) */
    for (int i = 1; i < m; ++i)
        for (int j = i; j > 0 && a[j] < a[j - 1]; --j) {
            double t = a[j];
            a[j] = a[j - 1];
            a[j - 1] = t;
        }
    double x = a[0] + h;
    if (m > 1 && x > a[1]) {
        double df = a[0] - a[1];
        x = (a[0] + a[1] + sqrt(2.0 * h * h - df * df)) / 2.0;
        if (m > 2 && x > a[2]) {
            double sm = a[0] + a[1] + a[2];
            double q = a[0] * a[0] + a[1] * a[1] + a[2] * a[2] - h * h;
            x = (sm + sqrt(sm * sm - 3.0 * q)) / 3.0;
        }
    }
    return x;
}

static double fsm_local(const or_params* g, const double* v, long long idx, const long long c[3],
                        const long long stride[3]) {
    double a[3];
    int m = 0;
    for (int ax = 0; ax < g->dim; ++ax) {
        double lo = c[ax] > 0 ? v[idx - stride[ax]] : INFINITY;
        double hi = c[ax] < g->n[ax] - 1 ? v[idx + stride[ax]] : INFINITY;
        a[m++] = lo < hi ? lo : hi;
    }
    return or_fsm_solve(a, m, g->h);
}

long long or_init_marking(const or_params* g, const double* d, double gamma_s, double* out, unsigned char* ext_out) {
    long long N = or_num_nodes(g);
    long long n[3] = {g->n[0], g->n[1], g->dim == 3 ? g->n[2] : 1};
    long long stride[3] = {1, g->n[0], g->n[0] * g->n[1]};
    unsigned char* ext = (unsigned char*)calloc((size_t)N, 1);
    for (long long k = 0; k < n[2]; ++k)
        for (long long j = 0; j < n[1]; ++j)
            for (long long i = 0; i < n[0]; ++i) {
                int b = i == 0 || i == n[0] - 1 || j == 0 || j == n[1] - 1;
                if (g->dim == 3) b = b || k == 0 || k == n[2] - 1;
                if (b) ext[i + stride[1] * j + stride[2] * k] = 1;
            }
    /* one round of directional sweeps */
    for (int ax = 0; ax < g->dim; ++ax)
        for (int dir = 0; dir < 2; ++dir) {
            int o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
            for (long long q2 = 0; q2 < n[o2]; ++q2)
                for (long long q1 = 0; q1 < n[o1]; ++q1) {
                    long long base = q1 * stride[o1] + q2 * stride[o2];
                    for (long long t = 1; t < n[ax]; ++t) {
                        long long cur = dir == 0 ? t : n[ax] - 1 - t;
                        long long prev = dir == 0 ? t - 1 : n[ax] - t;
                        long long ic = base + cur * stride[ax], ip = base + prev * stride[ax];
                        if (!ext[ic] && ext[ip] && d[ic] >= gamma_s) ext[ic] = 1;
                    }
                }
        }
    long long next = 0;
    for (long long i = 0; i < N; ++i) {
        out[i] = ext[i] ? d[i] - gamma_s : 1e30;
        next += ext[i];
    }
    /* fast sweeping on the internal nodes */
    int nord = 1 << g->dim;
    for (int round = 0; round < 2; ++round)
        for (int o = 0; o < nord; ++o) {
            long long c[3];
            for (long long kk = 0; kk < n[2]; ++kk) {
                c[2] = (o & 4) ? n[2] - 1 - kk : kk;
                for (long long jj = 0; jj < n[1]; ++jj) {
                    c[1] = (o & 2) ? n[1] - 1 - jj : jj;
                    for (long long ii = 0; ii < n[0]; ++ii) {
                        c[0] = (o & 1) ? n[0] - 1 - ii : ii;
                        long long idx = c[0] + stride[1] * c[1] + stride[2] * c[2];
                        if (ext[idx]) continue;
                        double x = fsm_local(g, out, idx, c, stride);
                        if (x < out[idx]) out[idx] = x;
                    }
                }
            }
        }
    for (long long i = 0; i < N; ++i)
        if (!ext[i]) out[i] = -out[i];
    if (ext_out) memcpy(ext_out, ext, (size_t)N);
    free(ext);
    return next;
}

/* §3.4: d exact (eq. distance, the whole cloud) on the nodes of a box of 4
 * (2-D: 4 x 4; 3-D: 4 x 4 x 4) grid points around each point, the fast
 * sweeping method (Zhao 2005) on every other node.
 * Readings: the box of Q holds, per axis, the nodes i0-1 .. i0+2 with
 * i0 = floor((Q_a - lo_a)/h), those outside the grid dropped; the other nodes
 * start at +inf and take the Godunov local solution of |∇d| = 1 in the
 * 2^dim orderings, two rounds, box nodes kept (the sweeps of or_init_marking).
 * d_out: FP64 on every node; fixed_out (may be NULL): 1 on box nodes.
 * Returns the number of box nodes (0: no point within a cell of the grid,
 * d_out untouched). */
long long or_distance_fsm(const or_params* g, const double* pts, long long npts, double* d_out,
                          unsigned char* fixed_out) {
    long long N = or_num_nodes(g);
    long long n[3] = {g->n[0], g->n[1], g->dim == 3 ? g->n[2] : 1};
    long long stride[3] = {1, g->n[0], g->n[0] * g->n[1]};
    unsigned char* fix = (unsigned char*)calloc((size_t)N, 1);
    for (long long q = 0; q < npts; ++q) {
        long long b0[3] = {0, 0, 0}, b1[3] = {0, 0, 0};
        int empty = 0;
        for (int a = 0; a < g->dim; ++a) {
            double xi = floor((pts[q * g->dim + a] - g->lo[a]) / g->h);
            double lo = xi - 1.0, hi = xi + 2.0;
            if (lo < 0.0) lo = 0.0;
            if (hi > (double)(n[a] - 1)) hi = (double)(n[a] - 1);
            if (lo > hi) empty = 1;
            else {
                b0[a] = (long long)lo;
                b1[a] = (long long)hi;
            }
        }
        if (empty) continue;
        for (long long k = b0[2]; k <= b1[2]; ++k)
            for (long long j = b0[1]; j <= b1[1]; ++j)
                for (long long i = b0[0]; i <= b1[0]; ++i) fix[i + stride[1] * j + stride[2] * k] = 1;
    }
    long long m = 0;
    for (long long i = 0; i < N; ++i) m += fix[i];
    if (m == 0) {
        free(fix);
        return 0;
    }
    long long* list = (long long*)malloc(sizeof(long long) * (size_t)m);
    double* dv = (double*)malloc(sizeof(double) * (size_t)m);
    int* arg = (int*)malloc(sizeof(int) * (size_t)m);
    m = 0;
    for (long long i = 0; i < N; ++i)
        if (fix[i]) list[m++] = i;
    or_distance_kd(g, pts, npts, list, m, dv, arg);
    for (long long i = 0; i < N; ++i) d_out[i] = INFINITY;
    for (long long t = 0; t < m; ++t) d_out[list[t]] = dv[t];
    free(list);
    free(dv);
    free(arg);
    int nord = 1 << g->dim;
    for (int round = 0; round < 2; ++round)
        for (int o = 0; o < nord; ++o) {
            long long c[3];
            for (long long kk = 0; kk < n[2]; ++kk) {
                c[2] = (o & 4) ? n[2] - 1 - kk : kk;
                for (long long jj = 0; jj < n[1]; ++jj) {
                    c[1] = (o & 2) ? n[1] - 1 - jj : jj;
                    for (long long ii = 0; ii < n[0]; ++ii) {
                        c[0] = (o & 1) ? n[0] - 1 - ii : ii;
                        long long idx = c[0] + stride[1] * c[1] + stride[2] * c[2];
                        if (fix[idx]) continue;
                        double x = fsm_local(g, d_out, idx, c, stride);
                        if (x < d_out[idx]) d_out[idx] = x;
                    }
                }
            }
        }
    if (fixed_out) memcpy(fixed_out, fix, (size_t)N);
    free(fix);
    return m;
}

int or_evolve(const or_params* g, double* u, const double* d, int R, double stop_tol, int kmax,
              int min_iters, int max_iters, double* E2_hist, double* dphi_hist, int* converged) {
    return or_evolve_reinit(g, u, d, R, stop_tol, kmax, min_iters, max_iters, 0, 0, 0.0, E2_hist, dphi_hist, converged);
}

int or_evolve_reinit(const or_params* g, double* u, const double* d, int R, double stop_tol, int kmax,
                     int min_iters, int max_iters, int reinit, int sweeps, double dtau, double* E2_hist,
                     double* dphi_hist, int* converged) {
    long long N = or_num_nodes(g);
    double* next = (double*)malloc((size_t)N * sizeof(double));
    double* re = reinit ? (double*)malloc((size_t)N * sizeof(double)) : NULL;
    double e[4];
    or_energy(g, u, d, 2.0, R, 0.0, e);
    E2_hist[0] = e[1];
    int n = 0, conv = 0;
    for (;;) {
        double Ep = E2_hist[n];
        if (g->p != 2.0 && g->p != 1.0) {
            double ep[4];
            or_energy(g, u, d, g->p, R, 0.0, ep);
            Ep = ep[1];
        }
        double dphi = or_sl_step(g, u, d, Ep, next, NULL);
        if (reinit) {
            /* the reinitialisation of Algorithm 1; Δ_φ then measures the whole update */
            or_reinit(g, u, next, sweeps, dtau, re, NULL);
            double acc = 0.0;
            for (long long i = 0; i < N; ++i) acc += fabs(re[i] - u[i]);
            dphi = acc * pow(g->h, (double)g->dim);
            memcpy(u, re, (size_t)N * sizeof(double));
        } else {
            memcpy(u, next, (size_t)N * sizeof(double));
        }
        dphi_hist[n] = dphi;
        ++n;
        or_energy(g, u, d, 2.0, R, 0.0, e);
        E2_hist[n] = e[1];
        double delta;
        if (or_stop(E2_hist, n, kmax, stop_tol, min_iters, max_iters, &delta)) {
            conv = (n >= min_iters && delta >= 0.0 && delta < stop_tol);
            break;
        }
    }
    free(next);
    free(re);
    if (converged) *converged = conv;
    return n;
}

/* §4: the L^1 norm of the error against the exact level set, read as
 * Δx^dim Σ_j |c(u_j) - c(φ*_j)| over every node, c the cut at γ in band mode
 * (the identity on the whole grid) */
double or_l1_error(const or_params* g, const double* u, const double* exact) {
    long long N = or_num_nodes(g);
    double s = 0.0;
    for (long long j = 0; j < N; ++j) {
        double a = u[j], b = exact[j];
        if (g->band) {
            a = fmin(fmax(a, -g->gamma), g->gamma);
            b = fmin(fmax(b, -g->gamma), g->gamma);
        }
        s += fabs(a - b);
    }
    double vol = g->h * g->h;
    if (g->dim == 3) vol *= g->h;
    return s * vol;
}

/* signed distance |x - c| - r to a circle (2-D) / sphere (3-D) on every node */
void or_sdf_sphere(const or_params* g, const double* sphere, double* out) {
    long long N = or_num_nodes(g);
    for (long long j = 0; j < N; ++j) {
        double x[3];
        or_node_coord(g, j, x);
        double s2 = (x[0] - sphere[0]) * (x[0] - sphere[0]) + (x[1] - sphere[1]) * (x[1] - sphere[1]);
        if (g->dim == 3) s2 += (x[2] - sphere[2]) * (x[2] - sphere[2]);
        out[j] = sqrt(s2) - sphere[3];
    }
}

/* ------------------------------------------------------------------ */
/* §4 runs from coarse to fine (eq. dxdt, Tab. param)                    */
/* ------------------------------------------------------------------ */

/* splitmix64 (Steele, Lea and Flood 2014), counter form: the i-th output of
 * the stream started at `seed` */
unsigned long long or_splitmix64(unsigned long long seed, unsigned long long i) {
    unsigned long long z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double or_grid_nodes(int dim, const double* bmin, const double* bmax, double dx, double margin,
                               long long nn[3]) {
    double tot = 1.0;
    for (int a = 0; a < 3; ++a) nn[a] = 1;
    for (int a = 0; a < dim; ++a) {
        /* clamped (far above any grid the budget admits) so that the
         * conversion and the product stay finite for any cloud extent */
        double q = fmin(ceil(((bmax[a] - bmin[a]) + 2.0 * margin) / dx) + 1.0, 4e9);
        nn[a] = q < 8.0 ? 8 : (long long)q;
        tot *= (double)nn[a];
    }
    return tot;
}

/* Readings: the sample draws point i when splitmix64(seed, i) < frac·2^64
 * (every point when frac >= 1; point 0 if none); the box is the cloud's
 * bounding box widened by γ_S + 8 Δx(1), Δx(1) = h_S coarsened (×
 * (N/max_nodes)^(1/dim)·1.0001 until it fits; γ_S = K_S Δx(1), which is
 * K_S h_S unless coarsened); run r has Δx = Δx(1)/2^(r-1),
 * coarsened the same way, over the bounding box widened by 8 Δx(r), plus
 * γ_S in run 1 (the box that gives the grids printed for the circle test,
 * Tab. errGlobCircle), (p, δ) = (1, 0), (2, 0), then (2, 1), Δt = Δx/4,
 * band, reinitialisation; φ0 of run 1 by or_init_marking at γ_S,
 * of later runs by Q1 (or_interp_q1) of the previous state at the new nodes;
 * both rounded to the storage type and cut; d exact, or by or_distance_fsm
 * when distance_fsm is set. phi_out receives the last run's
 * field (at most phi_cap values). Returns 0, or -1 (bad input / capacity). */
int or_reconstruct(int dim, int prec, int interp, int runs, double K_s, double sample_frac,
                   unsigned long long seed, long long max_nodes, int max_iters, int distance_fsm, int exact_sphere,
                   const double* sphere, const double* pts, long long npts, double* phi_out, long long phi_cap,
                   or_multirun_report* rep) {
    memset(rep, 0, sizeof(*rep));
    if (dim != 2 && dim != 3) return -1;
    double bmin[3] = {0, 0, 0}, bmax[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
        bmin[a] = INFINITY;
        bmax[a] = -INFINITY;
    }
    for (long long i = 0; i < npts; ++i)
        for (int a = 0; a < dim; ++a) {
            double v = pts[i * dim + a];
            if (v < bmin[a]) bmin[a] = v;
            if (v > bmax[a]) bmax[a] = v;
        }
    long long* sample = (long long*)malloc(sizeof(long long) * (size_t)npts);
    long long m = 0;
    double limd = sample_frac * 18446744073709551616.0;
    if (limd > 18446744073709549568.0) limd = 18446744073709549568.0;
    unsigned long long lim = (unsigned long long)limd;
    for (long long i = 0; i < npts; ++i)
        if (sample_frac >= 1.0 || or_splitmix64(seed, (unsigned long long)i) < lim) sample[m++] = i;
    if (m == 0) sample[m++] = 0;
    double hs = or_cloud_spacing(dim, pts, npts, sample, m);
    free(sample);
    rep->h_s = hs;
    rep->sample_size = m;
    long long nn[3];
    double dx1 = hs;
    for (int it = 0; it < 200; ++it) {
        double tot = or_grid_nodes(dim, bmin, bmax, dx1, (K_s + 8.0) * dx1, nn);
        if (tot <= (double)max_nodes) break;
        dx1 *= pow(tot / (double)max_nodes, 1.0 / dim) * 1.0001;
    }
    /* γ_S = K_S h_S, or K_S Δx(1) on a coarsened first grid (the marked
     * shell must stay closed on the grid) */
    double gamma_s = K_s * dx1;
    double* prev = NULL;
    or_params pp;
    memset(&pp, 0, sizeof(pp));
    for (int r = 1; r <= runs; ++r) {
        double dx = dx1 / (double)(1ll << (r - 1));
        for (int it = 0; it < 200; ++it) {
            double tot = or_grid_nodes(dim, bmin, bmax, dx, 8.0 * dx + (r == 1 ? gamma_s : 0.0), nn);
            if (tot <= (double)max_nodes) break;
            dx *= pow(tot / (double)max_nodes, 1.0 / dim) * 1.0001;
        }
        double margin = 8.0 * dx + (r == 1 ? gamma_s : 0.0);
        double lo[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) lo[a] = bmin[a] - margin;
        or_params P;
        memset(&P, 0, sizeof(P));
        P.dim = dim;
        for (int a = 0; a < 3; ++a) {
            P.n[a] = a < dim ? nn[a] : 1;
            P.lo[a] = a < dim ? lo[a] : 0.0;
        }
        double hi0 = lo[0] + (double)(nn[0] - 1) * dx;
        P.h = (hi0 - lo[0]) / (double)(nn[0] - 1);
        P.interp = interp;
        P.p = r == 1 ? 1.0 : 2.0;
        P.delta = r <= 2 ? 0.0 : 1.0;
        P.dt = P.h / 4.0;
        P.band = 1;
        P.gamma = (dim == 2 ? 4.0 : 6.0) * P.h;
        P.beta = (dim == 2 ? 2.0 : 3.0) * P.h;
        P.c_sing = 1e-3;
        P.alpha = 1.0;
        P.prec = prec;
        long long N = or_num_nodes(&P);
        double* d = (double*)malloc(sizeof(double) * (size_t)N);
        double* u = (double*)malloc(sizeof(double) * (size_t)N);
        if (distance_fsm) {
            if (or_distance_fsm(&P, pts, npts, d, NULL) == 0) {
                free(d);
                free(u);
                free(prev);
                return -1;
            }
        } else {
            or_distance_kd(&P, pts, npts, NULL, 0, d, NULL);
        }
        if (prec == 32)
            for (long long i = 0; i < N; ++i) d[i] = (double)(float)d[i];
        if (r == 1) {
            or_init_marking(&P, d, gamma_s, u, NULL);
        } else {
            for (long long i = 0; i < N; ++i) {
                double x[3];
                or_node_coord(&P, i, x);
                u[i] = or_interp_q1(&pp, prev, x);
            }
            free(prev);
        }
        for (long long i = 0; i < N; ++i) {
            double v = prec == 32 ? (double)(float)u[i] : u[i];
            u[i] = or_cut(&P, v);
        }
        double* E2 = (double*)malloc(sizeof(double) * (size_t)(max_iters + 1));
        double* dphi = (double*)malloc(sizeof(double) * (size_t)(max_iters + 1));
        int conv = 0;
        int it = or_evolve_reinit(&P, u, d, 5, 1e-4, 10, 10, max_iters, 1, 0, 0.0, E2, dphi, &conv);
        rep->run_energy[r - 1] = E2[it];
        rep->run_err_cloud[r - 1] = or_err_cloud(&P, u, pts, npts);
        rep->run_l1_err[r - 1] = NAN;
        if (exact_sphere) {
            double* ex = (double*)malloc(sizeof(double) * (size_t)N);
            or_sdf_sphere(&P, sphere, ex);
            rep->run_l1_err[r - 1] = or_l1_error(&P, u, ex);
            free(ex);
        }
        for (int a = 0; a < 3; ++a) rep->run_lo[r - 1][a] = P.lo[a];
        free(E2);
        free(dphi);
        free(d);
        rep->runs_done = r;
        rep->run_dx[r - 1] = dx;
        for (int a = 0; a < 3; ++a) rep->run_n[r - 1][a] = P.n[a];
        rep->run_iters[r - 1] = it;
        rep->run_converged[r - 1] = conv;
        prev = u;
        pp = P;
    }
    long long N = or_num_nodes(&pp);
    if (N > phi_cap) {
        free(prev);
        return -1;
    }
    memcpy(phi_out, prev, sizeof(double) * (size_t)N);
    free(prev);
    return 0;
}

long long or_extract(const or_params* g, const double* u, double width, long long* idx_out, double* u_out) {
    long long N = or_num_nodes(g), m = 0;
    for (long long i = 0; i < N; ++i)
        if (fabs(u[i]) < width) {
            if (idx_out) idx_out[m] = i;
            if (u_out) u_out[m] = u[i];
            ++m;
        }
    return m;
}

/* eq. errCloud */
double or_err_cloud(const or_params* g, const double* u, const double* pts, long long npts) {
    double acc = 0.0;
    for (long long q = 0; q < npts; ++q) {
        double x[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < g->dim; ++a) x[a] = pts[q * g->dim + a];
        acc += fabs(or_interp(g, u, x));
    }
    return acc / (double)npts;
}
