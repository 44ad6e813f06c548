/*
 * cmg_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, sequential, FP64 CPU restatement of the cascadic multigrid (CMG)
 * Fiedler-vector method of Urschel, Hu, Xu and Zikatanov, "A cascadic multigrid
 * algorithm for computing the Fiedler vector of graph Laplacians"
 * (arXiv 1412.0565).  It exists to check the CUDA library against, and only
 * the test-suite, the package smoke check and the benchmark's CPU-baseline leg
 * may load it.  It shares no code, header, table or generator with the CUDA
 * library; the two sides implement the same written readings independently.
 *
 * Every routine follows the paper's steps in the paper's order, with no
 * blocking, fusion or reordering:
 *   - Laplacian and g:          Sec. 2, Definition 2.1; Alg. 3 (Gershgorin shift)
 *   - heaviest neighbour m(v):  Alg. 2 (argmin of the column L(:,v))
 *   - visit order p = randperm: Alg. 2, restated as a keyed Feistel permutation
 *   - heavy edge coarsening:    Alg. 2, executed literally and sequentially
 *   - Galerkin coarse matrix:   Sec. 2 Step 1, L^{i+1} = I L I^T (Proposition 2.7)
 *   - power iteration:          Alg. 3 (projection against 1 as in Sec. 2.2)
 *   - cascade driver:           Alg. 1 (setup, coarsest solve, refinement)
 *   - error metric:             Sec. 4, ||(L - r I) y|| with r = y^T L y
 *
 * Readings where the paper is silent or garbled (they are listed, with the
 * reason for each, in the project's design notes):
 *   R1  heaviest neighbour: strict '>' on the FP64 weight, ties -> lowest column.
 *   R2  coarsening stops when n_i <= coarse_size, when HEC returns c < 2, or at
 *       max_levels levels.
 *   R3  randperm is replaced by a 4-round balanced Feistel permutation keyed by
 *       splitmix64 (published generator of Steele, Lea and Flood, 2014), with
 *       cycle walking onto [0, n).
 *   R4  randn(n_J) is Box-Muller on splitmix64-derived uniforms in (0, 1].
 *   R5  Galerkin sums: for a < b, w_ab is the left-to-right FP64 sum over fine
 *       pairs (i, j), agg(i) = a, agg(j) = b, in ascending (i, then j) order;
 *       w_ba = w_ab; the coarse diagonal is the row sum of the off-diagonals.
 *   R6  stopping: while cos(u, v) < 1 - tol, at least one sweep, capped.
 *   R7  Alg. 3's printed projection is read as Gram-Schmidt against 1 and is
 *       applied after every sweep (equal to Alg. 3 in exact arithmetic).
 *   R8  g = max_i (|l_ii| + sum_j |l_ij|) = max_i 2 d_i for a Laplacian.
 *   R9  lambda = (1/2) sum_i sum_j w_ij (u_i - u_j)^2 / ||u||^2.
 *   R10 if a sweep returns, after projection, a vector of norm at most
 *       64 eps g (rounding level; the iterate has norm 1), the previous
 *       iterate is an eigenvector with B_g v = 0 (lambda = g, e.g. n = 2)
 *       and the iteration stops there, keeping it.
 *   R11 the returned vector is scaled so that its largest-magnitude entry
 *       (lowest index on ties) is positive.
 *   R12 a vertex without neighbours (possible on a coarse level of a
 *       disconnected graph) has no heaviest neighbour and forms an aggregate
 *       of its own when it is visited.
 */
#include <float.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------ */
/* R3/R4: splitmix64.  One output of the SplitMix64 generator whose state is x:
 * the state is advanced by the golden gamma and the result is passed through
 * the MIX13 finaliser (Steele, Lea, Flood, OOPSLA 2014).                      */
ORC_EXPORT uint64_t orc_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* R3: the visit rank r_l(v) of vertex v at level l (Alg. 2's randperm).
 * Width k = smallest even integer >= 2 with 2^k >= n, halves of k/2 bits.
 * Round t (t = 0..3):  (L, R) -> (R, L xor F_t(R)),
 *   F_t(R) = low k/2 bits of splitmix64(R xor K_t),
 *   K_t    = splitmix64(seed xor (l * 0x9E3779B97F4A7C15) xor t).
 * The permutation of [0, 2^k) is restricted to [0, n) by cycle walking.    */
ORC_EXPORT int64_t orc_visit_rank(uint64_t seed, int32_t level, int64_t n, int64_t v)
{
    int k = 2;
    while (((int64_t)1 << k) < n) k += 2;
    int half = k / 2;
    uint64_t mask = ((uint64_t)1 << half) - 1;
    uint64_t key[4];
    for (int t = 0; t < 4; t++)
        key[t] = orc_splitmix64(seed ^ ((uint64_t)(int64_t)level * 0x9E3779B97F4A7C15ULL) ^ (uint64_t)t);
    uint64_t x = (uint64_t)v;
    do {
        uint64_t L = x >> half, R = x & mask;
        for (int t = 0; t < 4; t++) {
            uint64_t F = orc_splitmix64(R ^ key[t]) & mask;
            uint64_t nl = R, nr = L ^ F;
            L = nl;
            R = nr;
        }
        x = (L << half) | R;
    } while (x >= (uint64_t)n);
    return (int64_t)x;
}

ORC_EXPORT void orc_visit_ranks(uint64_t seed, int32_t level, int64_t n, int64_t *rank_out)
{
    for (int64_t v = 0; v < n; v++) rank_out[v] = orc_visit_rank(seed, level, n, v);
}

/* R4: the Gaussian start randn(n_J) of Alg. 1 Step 2.  For entry i,
 *   a = splitmix64(seed ^ 0xC0A45E ^ 2i),  b = splitmix64(seed ^ 0xC0A45E ^ (2i+1)),
 *   u1 = ((a >> 11) + 1) 2^-53,  u2 = ((b >> 11) + 1) 2^-53   (both in (0, 1]),
 *   x_i = sqrt(-2 ln u1) cos(2 pi u2)                          (Box-Muller).   */
ORC_EXPORT void orc_gaussian_start(uint64_t seed, int64_t n, double *x)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = 0; i < n; i++) {
        uint64_t a = orc_splitmix64(seed ^ 0xC0A45EULL ^ (uint64_t)(2 * i));
        uint64_t b = orc_splitmix64(seed ^ 0xC0A45EULL ^ (uint64_t)(2 * i + 1));
        double u1 = (double)((a >> 11) + 1) * (1.0 / 9007199254740992.0);
        double u2 = (double)((b >> 11) + 1) * (1.0 / 9007199254740992.0);
        x[i] = sqrt(-2.0 * log(u1)) * cos(two_pi * u2);
    }
}

/* ------------------------------------------------------------------ */
/* Definition 2.1: d_i = sum_j w_ij (left to right over the row).             */
static void weighted_degrees(int64_t n, const int64_t *rp, const double *w, double *d)
{
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) s += w[e];
        d[i] = s;
    }
}

/* Alg. 3, first line with R8: g = max_i sum_j |l_ij| = max_i (d_i + d_i).     */
ORC_EXPORT double orc_gershgorin(int64_t n, const int64_t *rp, const double *w)
{
    double g = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) s += w[e];
        double row_abs = s + s;
        if (row_abs > g) g = row_abs;
    }
    return g;
}

/* Alg. 2, line "m <- argmin(L(:, p(i)))" with R1.  Off-diagonal entries of
 * column v are -w_jv < 0 < d_v, so the argmin is the neighbour of maximum
 * weight; among equal maxima the lowest index is taken (MATLAB's min returns
 * the first).  A vertex without neighbours gets -1.                           */
ORC_EXPORT void orc_heaviest_neighbour(int64_t n, const int64_t *rp, const int32_t *col,
                                       const double *w, int32_t *m_out)
{
    for (int64_t v = 0; v < n; v++) {
        int32_t best_j = -1;
        double best_w = 0.0;
        for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
            if (best_j < 0 || w[e] > best_w || (w[e] == best_w && col[e] < best_j)) {
                best_w = w[e];
                best_j = col[e];
            }
        }
        m_out[v] = best_j;
    }
}

/* Alg. 2 (heavy edge coarsening), executed literally with 0-based labels.
 * The visit order p is the inverse of the rank array: vertex p(t) is visited
 * at step t.  q(v) = -1 plays the role of the paper's q(v) = 0 ("unmapped").
 * Returns c, the number of aggregates; agg_out[v] = q(v) in 0..c-1.           */
ORC_EXPORT int64_t orc_hec(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                           const int64_t *rank, int32_t *agg_out)
{
    int64_t *p = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int32_t *m = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; v++) p[rank[v]] = v;
    orc_heaviest_neighbour(n, rp, col, w, m);
    int64_t c = 0;
    for (int64_t v = 0; v < n; v++) agg_out[v] = -1;
    for (int64_t t = 0; t < n; t++) {
        int64_t v = p[t];
        if (agg_out[v] != -1) continue;          /* already mapped: skip       */
        int32_t mv = m[v];
        if (mv < 0) {                            /* R12: no neighbour at all   */
            agg_out[v] = (int32_t)c;
            c++;
        } else if (agg_out[mv] == -1) {          /* heavy neighbour unmapped:  */
            agg_out[mv] = (int32_t)c;            /* new aggregate {v, m(v)}    */
            agg_out[v] = (int32_t)c;
            c++;
        } else {
            agg_out[v] = agg_out[mv];            /* join m(v)'s aggregate      */
        }
    }
    free(p);
    free(m);
    return c;
}

/* ------------------------------------------------------------------ */
/* Galerkin product L^{i+1} = I L I^T (Sec. 2 Step 1; Proposition 2.7) with R5.
 * The coarse graph is stored as CSR of the off-diagonal weights, columns
 * ascending; the diagonal (coarse degree) is implied by the row sums.         */
typedef struct {
    int64_t a, b, e; /* coarse row, coarse column, fine entry index (order key) */
} orc_triple;

static int cmp_triple(const void *x, const void *y)
{
    const orc_triple *s = (const orc_triple *)x, *t = (const orc_triple *)y;
    if (s->a != t->a) return s->a < t->a ? -1 : 1;
    if (s->b != t->b) return s->b < t->b ? -1 : 1;
    if (s->e != t->e) return s->e < t->e ? -1 : 1;
    return 0;
}

typedef struct {
    int64_t col;
    double w;
} orc_entry;

static int cmp_entry(const void *x, const void *y)
{
    const orc_entry *s = (const orc_entry *)x, *t = (const orc_entry *)y;
    return (s->col > t->col) - (s->col < t->col);
}

/* Returns the coarse nnz; *rp_c, *col_c, *w_c are malloc'ed (free with orc_free_buf). */
static int64_t galerkin(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                        const int32_t *agg, int64_t c, int64_t **rp_c, int32_t **col_c, double **w_c)
{
    /* fine entries (i, j) whose aggregates satisfy a < b, in CSR order */
    int64_t nt = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t e = rp[i]; e < rp[i + 1]; e++)
            if (agg[i] < agg[col[e]]) nt++;
    orc_triple *t = (orc_triple *)malloc(sizeof(orc_triple) * (size_t)(nt > 0 ? nt : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < n; i++)
        for (int64_t e = rp[i]; e < rp[i + 1]; e++)
            if (agg[i] < agg[col[e]]) {
                t[k].a = agg[i];
                t[k].b = agg[col[e]];
                t[k].e = e;
                k++;
            }
    /* group equal (a, b); inside a group the fine entries stay in (i, j) order */
    qsort(t, (size_t)nt, sizeof(orc_triple), cmp_triple);
    /* left-to-right sums per (a, b) */
    int64_t nu = 0;
    orc_entry *ua = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(nt > 0 ? nt : 1));
    int64_t *urow = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nt > 0 ? nt : 1));
    for (int64_t s = 0; s < nt;) {
        int64_t u = s;
        double acc = 0.0;
        while (u < nt && t[u].a == t[s].a && t[u].b == t[s].b) {
            acc += w[t[u].e];
            u++;
        }
        urow[nu] = t[s].a;
        ua[nu].col = t[s].b;
        ua[nu].w = acc;
        nu++;
        s = u;
    }
    /* mirror: w_ba = w_ab, then per-row column sort */
    int64_t *cnt = (int64_t *)calloc((size_t)c + 1, sizeof(int64_t));
    for (int64_t s = 0; s < nu; s++) {
        cnt[urow[s]]++;
        cnt[ua[s].col]++;
    }
    int64_t *rpc = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c + 1));
    rpc[0] = 0;
    for (int64_t a = 0; a < c; a++) rpc[a + 1] = rpc[a] + cnt[a];
    int64_t nnzc = rpc[c];
    orc_entry *ent = (orc_entry *)malloc(sizeof(orc_entry) * (size_t)(nnzc > 0 ? nnzc : 1));
    int64_t *fill = (int64_t *)calloc((size_t)c + 1, sizeof(int64_t));
    for (int64_t s = 0; s < nu; s++) {
        int64_t a = urow[s], b = ua[s].col;
        ent[rpc[a] + fill[a]].col = b;
        ent[rpc[a] + fill[a]].w = ua[s].w;
        fill[a]++;
        ent[rpc[b] + fill[b]].col = a;
        ent[rpc[b] + fill[b]].w = ua[s].w;
        fill[b]++;
    }
    for (int64_t a = 0; a < c; a++)
        qsort(ent + rpc[a], (size_t)(rpc[a + 1] - rpc[a]), sizeof(orc_entry), cmp_entry);
    int32_t *colc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnzc > 0 ? nnzc : 1));
    double *wc = (double *)malloc(sizeof(double) * (size_t)(nnzc > 0 ? nnzc : 1));
    for (int64_t s = 0; s < nnzc; s++) {
        colc[s] = (int32_t)ent[s].col;
        wc[s] = ent[s].w;
    }
    free(t);
    free(ua);
    free(urow);
    free(cnt);
    free(fill);
    free(ent);
    *rp_c = rpc;
    *col_c = colc;
    *w_c = wc;
    return nnzc;
}

/* ------------------------------------------------------------------ */
/* Alg. 3 building blocks.                                                     */

/* (B_g v)_i = g v_i - (L v)_i with (L v)_i = d_i v_i - sum_j w_ij v_j (Def. 2.1). */
static void apply_bg(int64_t n, const int64_t *rp, const int32_t *col, const double *w,
                     const double *d, double g, const double *v, double *out)
{
    for (int64_t i = 0; i < n; i++) {
        double lv = d[i] * v[i];
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) lv -= w[e] * v[col[e]];
        out[i] = g * v[i] - lv;
    }
}

/* R7: Gram-Schmidt against 1, then division by the 2-norm.  Returns the norm
 * after projection (0 means the vector was a multiple of 1).                 */
static double project_normalise(int64_t n, double *u)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += u[i];
    double mean = s / (double)n;
    for (int64_t i = 0; i < n; i++) u[i] -= mean;
    double q = 0.0;
    for (int64_t i = 0; i < n; i++) q += u[i] * u[i];
    double nrm = sqrt(q);
    if (nrm > 0.0)
        for (int64_t i = 0; i < n; i++) u[i] /= nrm;
    return nrm;
}

/* R6: cosine of the angle between the stored vectors u and v. */
static double cosine(int64_t n, const double *u, const double *v)
{
    double uv = 0.0, uu = 0.0, vv = 0.0;
    for (int64_t i = 0; i < n; i++) {
        uv += u[i] * v[i];
        uu += u[i] * u[i];
        vv += v[i] * v[i];
    }
    return uv / sqrt(uu * vv);
}

/* R9: lambda = (1/2) sum_i sum_j w_ij (u_i - u_j)^2 / ||u||^2, and the error
 * metric of Sec. 4, ||(L - lambda I) u|| / ||u||.                           */
ORC_EXPORT void orc_rayleigh_residual(int64_t n, const int64_t *rp, const int32_t *col,
                                      const double *w, const double *u, double *lambda_out,
                                      double *residual_out)
{
    double num = 0.0, uu = 0.0;
    for (int64_t i = 0; i < n; i++) {
        uu += u[i] * u[i];
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
            double df = u[i] - u[col[e]];
            num += w[e] * df * df;
        }
    }
    double lam = 0.5 * num / uu;
    double rr = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double di = 0.0, lu = 0.0;
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) di += w[e];
        lu = di * u[i];
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) lu -= w[e] * u[col[e]];
        double r = lu - lam * u[i];
        rr += r * r;
    }
    if (lambda_out) *lambda_out = lam;
    if (residual_out) *residual_out = sqrt(rr / uu);
}

/* Alg. 3 (power iteration on B_g = g I - L).
 * mode 0: run while cos(u, v) < 1 - tol (R6), at most max_sweeps sweeps;
 * mode 1: run exactly k_fixed sweeps (a fixed schedule, Sec. 3's k_j).
 * y0 is the initial guess (length n, not modified); u_out receives the result.
 * Returns the number of sweeps; *capped = 1 if max_sweeps stopped the loop.  */
ORC_EXPORT int64_t orc_power_iteration(int64_t n, const int64_t *rp, const int32_t *col,
                                       const double *w, double g, const double *y0, double tol,
                                       int32_t mode, int64_t k_fixed, int64_t max_sweeps,
                                       double *u_out, double *cos_out, int32_t *capped)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *u = u_out;
    weighted_degrees(n, rp, w, d);
    /* u = y0 - (1^T y0 / n) 1 ;  u = u / ||u||   (R7) */
    for (int64_t i = 0; i < n; i++) u[i] = y0[i];
    project_normalise(n, u);
    /* v = zeros(n, 1) */
    for (int64_t i = 0; i < n; i++) v[i] = 0.0;
    int64_t k = 0;
    double c = 0.0;
    if (capped) *capped = 0;
    for (;;) {
        if (mode == 1) {
            if (k >= k_fixed) break;
        } else {
            /* u^T v with v = 0 on entry; the cosine of R6 afterwards */
            c = (k == 0) ? 0.0 : cosine(n, u, v);
            if (!(c < 1.0 - tol)) break;
            if (k >= max_sweeps) {
                if (capped) *capped = 1;
                break;
            }
        }
        /* v <- u ; u = B_g v ; u <- u / ||u||  (with R7's projection) */
        memcpy(v, u, sizeof(double) * (size_t)n);
        apply_bg(n, rp, col, w, d, g, v, u);
        double nrm = project_normalise(n, u);
        k++;
        if (nrm <= 64.0 * DBL_EPSILON * g) { /* R10: v is an eigenvector with B_g v = 0 */
            memcpy(u, v, sizeof(double) * (size_t)n);
            c = 1.0;
            break;
        }
    }
    if (mode == 1 && k > 0) c = cosine(n, u, v);
    if (cos_out) *cos_out = c;
    free(d);
    free(v);
    return k;
}

/* ------------------------------------------------------------------ */
/* Alg. 1 (multilevel cascadic eigensolver).                                   */
typedef struct {
    int64_t n, nnz;
    int64_t *rp;
    int32_t *col;
    double *w;
    double g;
    int32_t *agg; /* restriction of this level to the next (NULL at the coarsest) */
    int64_t sweeps;
    double cos_final;
} orc_level;

typedef struct {
    int32_t levels;
    orc_level lv[64];
} orc_hierarchy;

static int64_t *copy_i64(const int64_t *x, int64_t n)
{
    int64_t *y = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    memcpy(y, x, sizeof(int64_t) * (size_t)n);
    return y;
}

/* Step 1 (setup phase) with R2.  Returns NULL on n < 2. */
ORC_EXPORT orc_hierarchy *orc_setup(int64_t n, const int64_t *rp, const int32_t *col,
                                    const double *w, uint64_t seed, int32_t coarse_size,
                                    int32_t max_levels)
{
    if (n < 2) return NULL;
    if (max_levels > 64) max_levels = 64;
    if (max_levels < 1) max_levels = 1;
    orc_hierarchy *h = (orc_hierarchy *)calloc(1, sizeof(orc_hierarchy));
    orc_level *L0 = &h->lv[0];
    L0->n = n;
    L0->nnz = rp[n];
    L0->rp = copy_i64(rp, n + 1);
    L0->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(rp[n] > 0 ? rp[n] : 1));
    memcpy(L0->col, col, sizeof(int32_t) * (size_t)rp[n]);
    L0->w = (double *)malloc(sizeof(double) * (size_t)(rp[n] > 0 ? rp[n] : 1));
    memcpy(L0->w, w, sizeof(double) * (size_t)rp[n]);
    L0->g = orc_gershgorin(n, rp, w);
    int32_t i = 0;
    while (h->lv[i].n > coarse_size && i + 1 < max_levels) {
        orc_level *f = &h->lv[i];
        int64_t *rank = (int64_t *)malloc(sizeof(int64_t) * (size_t)f->n);
        int32_t *agg = (int32_t *)malloc(sizeof(int32_t) * (size_t)f->n);
        orc_visit_ranks(seed, i, f->n, rank);
        int64_t c = orc_hec(f->n, f->rp, f->col, f->w, rank, agg);
        free(rank);
        if (c < 2) {
            free(agg);
            break;
        }
        f->agg = agg;
        orc_level *cl = &h->lv[i + 1];
        cl->n = c;
        cl->nnz = galerkin(f->n, f->rp, f->col, f->w, agg, c, &cl->rp, &cl->col, &cl->w);
        cl->g = orc_gershgorin(c, cl->rp, cl->w);
        i++;
    }
    h->levels = i + 1;
    return h;
}

ORC_EXPORT int32_t orc_levels(const orc_hierarchy *h) { return h->levels; }

ORC_EXPORT void orc_level_info(const orc_hierarchy *h, int32_t l, int64_t *n, int64_t *nnz,
                               double *g)
{
    *n = h->lv[l].n;
    *nnz = h->lv[l].nnz;
    *g = h->lv[l].g;
}

ORC_EXPORT void orc_level_csr(const orc_hierarchy *h, int32_t l, int64_t *rp, int32_t *col,
                              double *w)
{
    const orc_level *L = &h->lv[l];
    memcpy(rp, L->rp, sizeof(int64_t) * (size_t)(L->n + 1));
    memcpy(col, L->col, sizeof(int32_t) * (size_t)L->nnz);
    memcpy(w, L->w, sizeof(double) * (size_t)L->nnz);
}

/* agg of level l (maps level l to level l+1); returns 0 if l is the coarsest. */
ORC_EXPORT int32_t orc_level_agg(const orc_hierarchy *h, int32_t l, int32_t *agg)
{
    const orc_level *L = &h->lv[l];
    if (!L->agg) return 0;
    memcpy(agg, L->agg, sizeof(int32_t) * (size_t)L->n);
    return 1;
}

ORC_EXPORT void orc_free(orc_hierarchy *h)
{
    if (!h) return;
    for (int32_t l = 0; l < h->levels; l++) {
        free(h->lv[l].rp);
        free(h->lv[l].col);
        free(h->lv[l].w);
        free(h->lv[l].agg);
    }
    free(h);
}

/* Steps 2 and 3 of Alg. 1.
 * schedule 0 (tolerance): Alg. 3 with tol at every level.
 * schedule 1 (fixed):     k_j = ceil(k0 * beta^j) sweeps at level j < J (Sec. 3),
 *                         tolerance mode at the coarsest level.
 * schedule 2 (replay):    exactly replay[j] sweeps at level j (j = 0..J).
 * converged != 0: after level 0's sweeps, keep sweeping level 0 until
 *                 ||(L - lambda I) u|| <= conv_rtol * g_0 (test use only).
 * start_level < 0: Step 2 from the Gaussian start keyed by `seed`, then Step 3.
 * start_level = s in 0..J: the cascade starts on level s from x0 (length n_s,
 *                 level s's numbering) instead: PI(L^s, x0), then Step 3 from
 *                 level s-1 down to 0; levels above s are not visited (0 sweeps).
 *                 This is the re-solve with a new start vector on a kept
 *                 hierarchy that the Remark after Alg. 1 has in mind for
 *                 repeated computations.
 * trace_start, trace_end (nullable, length sum_j n_j, level j at offset
 *                 n_0 + ... + n_{j-1}): the vector each visited level's PI
 *                 starts from (the Gaussian, x0, or the prolongation
 *                 (I_j^{j+1})^T y~^(j+1) before Gram-Schmidt) and the vector it
 *                 returns, y~^(j) (before the sign rule).  Unvisited levels are
 *                 left untouched.
 * Outputs: u (length n_0, R11 sign), lambda, residual, sweeps[j], cosines[j].
 * Returns 1 if a sweep cap was reached, else 0.                              */
ORC_EXPORT int32_t orc_solve_ex(orc_hierarchy *h, uint64_t seed, double tol, int32_t schedule,
                                double beta, int32_t k0, const int64_t *replay,
                                int64_t max_sweeps, int64_t max_sweeps_coarsest,
                                int32_t converged, double conv_rtol, int32_t start_level,
                                const double *x0, double *u, double *lambda_out,
                                double *residual_out, int64_t *sweeps_out, double *cos_out,
                                double *trace_start, double *trace_end)
{
    int32_t J = h->levels - 1;
    int32_t warn = 0;
    int32_t top = (start_level >= 0 && start_level <= J) ? start_level : J;
    int64_t off[65];
    off[0] = 0;
    for (int32_t j = 0; j <= J; j++) off[j + 1] = off[j] + h->lv[j].n;
    for (int32_t j = top + 1; j <= J; j++) {
        h->lv[j].sweeps = 0;
        h->lv[j].cos_final = 0.0;
    }
    /* Step 2: PI(L^J, randn(n_J)), or PI(L^s, x0) for a given start */
    orc_level *c = &h->lv[top];
    double *y = (double *)malloc(sizeof(double) * (size_t)c->n);
    double *yt = (double *)malloc(sizeof(double) * (size_t)c->n);
    if (top == start_level)
        memcpy(y, x0, sizeof(double) * (size_t)c->n);
    else
        orc_gaussian_start(seed, c->n, y);
    if (trace_start) memcpy(trace_start + off[top], y, sizeof(double) * (size_t)c->n);
    int32_t capped = 0;
    int32_t mode = 0;
    int64_t kf = 0;
    if (schedule == 2) {
        mode = 1;
        kf = replay[top];
    } else if (schedule == 1 && top < J) {
        mode = 1;
        kf = (int64_t)ceil((double)k0 * pow(beta, (double)top));
    }
    c->sweeps = orc_power_iteration(c->n, c->rp, c->col, c->w, c->g, y, tol, mode, kf,
                                    top == J ? max_sweeps_coarsest : max_sweeps, yt,
                                    &c->cos_final, &capped);
    warn |= capped;
    if (trace_end) memcpy(trace_end + off[top], yt, sizeof(double) * (size_t)c->n);
    free(y);
    y = yt;
    /* Step 3: for j = top-1 down to 0: prolongate, then PI */
    for (int32_t j = top - 1; j >= 0; j--) {
        orc_level *f = &h->lv[j];
        double *yh = (double *)malloc(sizeof(double) * (size_t)f->n);
        double *yn = (double *)malloc(sizeof(double) * (size_t)f->n);
        for (int64_t i = 0; i < f->n; i++) yh[i] = y[f->agg[i]]; /* (I_j^{j+1})^T y */
        if (trace_start) memcpy(trace_start + off[j], yh, sizeof(double) * (size_t)f->n);
        int32_t md = 0;
        int64_t k = 0;
        if (schedule == 1) {
            md = 1;
            k = (int64_t)ceil((double)k0 * pow(beta, (double)j));
        } else if (schedule == 2) {
            md = 1;
            k = replay[j];
        }
        f->sweeps = orc_power_iteration(f->n, f->rp, f->col, f->w, f->g, yh, tol, md, k,
                                        max_sweeps, yn, &f->cos_final, &capped);
        warn |= capped;
        if (trace_end) memcpy(trace_end + off[j], yn, sizeof(double) * (size_t)f->n);
        free(yh);
        free(y);
        y = yn;
    }
    orc_level *f = &h->lv[0];
    if (converged) {
        double lam = 0.0, res = 0.0;
        double *yn = (double *)malloc(sizeof(double) * (size_t)f->n);
        for (int64_t it = 0; it < 4000000; it++) {
            orc_rayleigh_residual(f->n, f->rp, f->col, f->w, y, &lam, &res);
            if (res <= conv_rtol * f->g) break;
            double cf;
            orc_power_iteration(f->n, f->rp, f->col, f->w, f->g, y, tol, 1, 64, 64, yn, &cf, NULL);
            memcpy(y, yn, sizeof(double) * (size_t)f->n);
        }
        free(yn);
    }
    /* R11: largest |u_i| positive, ties to the lowest index */
    int64_t imax = 0;
    for (int64_t i = 1; i < f->n; i++)
        if (fabs(y[i]) > fabs(y[imax])) imax = i;
    double sg = (y[imax] < 0.0) ? -1.0 : 1.0;
    for (int64_t i = 0; i < f->n; i++) u[i] = sg * y[i];
    orc_rayleigh_residual(f->n, f->rp, f->col, f->w, u, lambda_out, residual_out);
    for (int32_t j = 0; j <= J; j++) {
        if (sweeps_out) sweeps_out[j] = h->lv[j].sweeps;
        if (cos_out) cos_out[j] = h->lv[j].cos_final;
    }
    free(y);
    return warn;
}

/* Alg. 1 Steps 2-3 from the Gaussian start (orc_solve_ex without a given
 * start vector and without traces).                                          */
ORC_EXPORT int32_t orc_solve(orc_hierarchy *h, uint64_t seed, double tol, int32_t schedule,
                             double beta, int32_t k0, const int64_t *replay,
                             int64_t max_sweeps, int64_t max_sweeps_coarsest, int32_t converged,
                             double conv_rtol, double *u, double *lambda_out,
                             double *residual_out, int64_t *sweeps_out, double *cos_out)
{
    return orc_solve_ex(h, seed, tol, schedule, beta, k0, replay, max_sweeps, max_sweeps_coarsest,
                        converged, conv_rtol, -1, NULL, u, lambda_out, residual_out, sweeps_out,
                        cos_out, NULL, NULL);
}

/* ------------------------------------------------------------------ */
/* Geometric cascadic multigrid, Alg. 4 (Sec. 3), on the structured grid of
 * the Table 4 experiment (Sec. 4): the unit-weight grid graph on N^dim
 * vertices (dim = 2: 5-point, dim = 3: 7-point; vertex (x, y, z) has id
 * (z N + y) N + x), nested by taking every other vertex, N_j = (N - 1)/2^j + 1
 * (N - 1 divisible by 2^J).  A_j is that level's graph Laplacian.
 * Readings:
 *   G1 the coarsest level J is solved exactly by its eigenvector for
 *      lambda_2 that varies along x only, phi(x) = cos(pi (x + 1/2) / N_J)
 *      (lambda_2 = 2 - 2 cos(pi / N_J) has multiplicity dim; this is one of
 *      its eigenvectors, written out from the separable grid spectrum);
 *   G2 prolongation is multilinear interpolation between the nested grids
 *      (coarse vertex I sits at fine vertex 2I; a fine vertex between coarse
 *      ones takes the average of its two (four, eight) coarse neighbours);
 *   G3 after prolongation the vector is made orthogonal to 1 (Gram-Schmidt,
 *      as Alg. 1 Step 3 keeps the iterates) and normalised;
 *   G4 the smoother u <- (I - omega_j A_j) u with omega_j = 1 / ||A_j||_inf
 *      runs k_j = ceil(k0 beta^j) times, each step followed by Gram-Schmidt
 *      against 1 and normalisation ("with appropriate scaling").
 * Outputs per level j = 0..J-1: r0[j] = Rayleigh quotient of the prolonged
 * start, rk[j] = Rayleigh quotient after the k_j smoothing steps (the two
 * columns of Table 4 are |lambda_2^(j) - r0[j]| and |lambda_2^(j) - rk[j]|),
 * ks[j] = k_j; r0[J] = rk[J] = the coarsest Rayleigh quotient.  u (N^dim):
 * the level-0 result.  Returns 0, or -1 for invalid sizes.                  */
static int64_t grid_n(int32_t dim, int64_t N) { return dim == 2 ? N * N : N * N * N; }

/* CSR of the unit grid graph, columns ascending. */
static void grid_csr(int32_t dim, int64_t N, int64_t **rp_o, int32_t **col_o, double **w_o)
{
    int64_t n = grid_n(dim, N);
    int64_t *rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int32_t *col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * dim * n));
    double *w = (double *)malloc(sizeof(double) * (size_t)(2 * dim * n));
    int64_t e = 0;
    for (int64_t v = 0; v < n; v++) {
        int64_t x = v % N, y = (v / N) % N, z = dim == 3 ? v / (N * N) : 0;
        rp[v] = e;
        /* neighbours in ascending id order: -z, -y, -x, +x, +y, +z */
        if (dim == 3 && z > 0) col[e++] = (int32_t)(v - N * N);
        if (y > 0) col[e++] = (int32_t)(v - N);
        if (x > 0) col[e++] = (int32_t)(v - 1);
        if (x < N - 1) col[e++] = (int32_t)(v + 1);
        if (y < N - 1) col[e++] = (int32_t)(v + N);
        if (dim == 3 && z < N - 1) col[e++] = (int32_t)(v + N * N);
    }
    rp[n] = e;
    for (int64_t k = 0; k < e; k++) w[k] = 1.0;
    *rp_o = rp;
    *col_o = col;
    *w_o = w;
}

/* Multilinear interpolation from the Nc-grid to the (2 Nc - 1)-grid (G2). */
static void grid_prolong(int32_t dim, int64_t Nc, const double *yc, double *yf)
{
    int64_t Nf = 2 * Nc - 1;
    int64_t nf = grid_n(dim, Nf);
    for (int64_t v = 0; v < nf; v++) {
        int64_t c[3] = {v % Nf, (v / Nf) % Nf, dim == 3 ? v / (Nf * Nf) : 0};
        /* per axis: the one or two coarse indices this fine index lies between */
        int64_t lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = c[a] / 2;
            hi[a] = (c[a] % 2) ? c[a] / 2 + 1 : c[a] / 2;
        }
        double s = 0.0;
        int cnt = 0;
        for (int iz = 0; iz < (dim == 3 ? 2 : 1); iz++)
            for (int iy = 0; iy < 2; iy++)
                for (int ix = 0; ix < 2; ix++) {
                    int64_t X = ix ? hi[0] : lo[0], Y = iy ? hi[1] : lo[1];
                    int64_t Z = (dim == 3) ? (iz ? hi[2] : lo[2]) : 0;
                    s += yc[(Z * Nc + Y) * Nc + X];
                    cnt++;
                }
        yf[v] = s / (double)cnt;
    }
}

/* Rayleigh quotient u^T A u / u^T u of the unit grid graph (edge form, R9). */
static double grid_rq(int64_t n, const int64_t *rp, const int32_t *col, const double *u)
{
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < n; i++) {
        den += u[i] * u[i];
        for (int64_t e = rp[i]; e < rp[i + 1]; e++) {
            double d = u[i] - u[col[e]];
            num += d * d;
        }
    }
    return 0.5 * num / den;
}

ORC_EXPORT int32_t orc_gcmg_grid(int32_t dim, int64_t N, int32_t J, double beta, int32_t k0,
                                 double *r0, double *rk, int64_t *ks, double *u_out)
{
    if ((dim != 2 && dim != 3) || J < 0 || N < 3 || ((N - 1) % ((int64_t)1 << J)) != 0 ||
        (N - 1) / ((int64_t)1 << J) < 1)
        return -1;
    const double pi = 3.14159265358979323846264338327950288;
    /* level J: the exact eigenvector (G1) */
    int64_t Nj = (N - 1) / ((int64_t)1 << J) + 1;
    int64_t nj = grid_n(dim, Nj);
    double *y = (double *)malloc(sizeof(double) * (size_t)nj);
    for (int64_t v = 0; v < nj; v++) y[v] = cos(pi * ((double)(v % Nj) + 0.5) / (double)Nj);
    {
        int64_t *rp;
        int32_t *col;
        double *w;
        grid_csr(dim, Nj, &rp, &col, &w);
        project_normalise(nj, y);
        r0[J] = rk[J] = grid_rq(nj, rp, col, y);
        ks[J] = 0;
        free(rp);
        free(col);
        free(w);
    }
    for (int32_t j = J - 1; j >= 0; j--) {
        int64_t Nf = 2 * Nj - 1, nf = grid_n(dim, Nf);
        double *u = (double *)malloc(sizeof(double) * (size_t)nf);
        double *t = (double *)malloc(sizeof(double) * (size_t)nf);
        int64_t *rp;
        int32_t *col;
        double *w;
        grid_csr(dim, Nf, &rp, &col, &w);
        grid_prolong(dim, Nj, y, u); /* G2 */
        project_normalise(nf, u);    /* G3 */
        r0[j] = grid_rq(nf, rp, col, u);
        /* G4: omega = 1 / ||A||_inf = 1 / max_i 2 d_i */
        double g = orc_gershgorin(nf, rp, w);
        double *d = (double *)malloc(sizeof(double) * (size_t)nf);
        weighted_degrees(nf, rp, w, d);
        int64_t k = (int64_t)ceil((double)k0 * pow(beta, (double)j));
        for (int64_t s = 0; s < k; s++) {
            for (int64_t i = 0; i < nf; i++) {
                double au = d[i] * u[i];
                for (int64_t e = rp[i]; e < rp[i + 1]; e++) au -= w[e] * u[col[e]];
                t[i] = u[i] - au / g;
            }
            memcpy(u, t, sizeof(double) * (size_t)nf);
            project_normalise(nf, u);
        }
        rk[j] = grid_rq(nf, rp, col, u);
        ks[j] = k;
        free(d);
        free(rp);
        free(col);
        free(w);
        free(t);
        free(y);
        y = u;
        Nj = Nf;
    }
    memcpy(u_out, y, sizeof(double) * (size_t)grid_n(dim, N));
    free(y);
    return 0;
}

/* ------------------------------------------------------------------ */
/* k eigenpairs (the Remark after Alg. 4): the cascade of Alg. 1 carries k
 * vectors instead of one.  On the coarsest level k Gaussian vectors
 * (vector i from randn keyed by seed + i, R4); on every level, after each
 * power-iteration sweep (each vector multiplied by B_g), the vectors are
 * orthogonalised -- modified Gram-Schmidt in their order, each first
 * against 1 (R7) and then against the earlier ones, then normalised -- and
 * after the last level each vector's Rayleigh quotient is computed.
 * Readings:
 *   K1 orthogonalisation after every sweep (as R7 does for 1), so the k
 *      vectors span the dominant k-dimensional invariant subspace of B_g on
 *      the complement of 1, i.e. tend to the eigenvectors of lambda_2 ..
 *      lambda_{k+1} (orthogonal iteration); the prolonged vectors are
 *      orthogonalised before the first sweep of their level;
 *   K2 stopping: a level stops when every vector's cosine with its previous
 *      iterate is at least 1 - tol (R6 for each vector); at least one sweep;
 *   K3 the sign rule R11 is applied to each returned vector.
 * X holds the k vectors of length n one after another (vector i at X + i n). */
static double mgs(int64_t n, int32_t k, double *X)
{
    double min_nrm = 1e300;
    for (int32_t i = 0; i < k; i++) {
        double *xi = X + (size_t)i * (size_t)n;
        double s = 0.0;
        for (int64_t r = 0; r < n; r++) s += xi[r];
        double mean = s / (double)n;
        for (int64_t r = 0; r < n; r++) xi[r] -= mean;
        for (int32_t j = 0; j < i; j++) {
            const double *xj = X + (size_t)j * (size_t)n;
            double d = 0.0;
            for (int64_t r = 0; r < n; r++) d += xi[r] * xj[r];
            for (int64_t r = 0; r < n; r++) xi[r] -= d * xj[r];
        }
        double q = 0.0;
        for (int64_t r = 0; r < n; r++) q += xi[r] * xi[r];
        double nrm = sqrt(q);
        if (nrm < min_nrm) min_nrm = nrm;
        if (nrm > 0.0)
            for (int64_t r = 0; r < n; r++) xi[r] /= nrm;
    }
    return min_nrm;
}

/* Block power iteration on one level (K1, K2).  X: in the start vectors,
 * out the result.  mode 0: tolerance rule (cap max_sweeps); mode 1: exactly
 * k_fixed sweeps.  Returns the sweeps; *capped = 1 if the cap stopped it. */
static int64_t block_power_iteration(int64_t n, const int64_t *rp, const int32_t *col,
                                     const double *w, double g, int32_t k, double *X,
                                     double tol, int32_t mode, int64_t k_fixed,
                                     int64_t max_sweeps, int32_t *capped)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)n);
    double *V = (double *)malloc(sizeof(double) * (size_t)n * (size_t)k);
    weighted_degrees(n, rp, w, d);
    mgs(n, k, X);
    int64_t s = 0;
    if (capped) *capped = 0;
    for (;;) {
        if (mode == 1) {
            if (s >= k_fixed) break;
        } else if (s >= 1) {
            /* every vector's cosine with its previous iterate (K2) */
            int done = 1;
            for (int32_t i = 0; i < k && done; i++)
                if (!(cosine(n, X + (size_t)i * (size_t)n, V + (size_t)i * (size_t)n) >= 1.0 - tol))
                    done = 0;
            if (done) break;
            if (s >= max_sweeps) {
                if (capped) *capped = 1;
                break;
            }
        }
        memcpy(V, X, sizeof(double) * (size_t)n * (size_t)k);
        for (int32_t i = 0; i < k; i++)
            apply_bg(n, rp, col, w, d, g, V + (size_t)i * (size_t)n, X + (size_t)i * (size_t)n);
        mgs(n, k, X);
        s++;
    }
    free(d);
    free(V);
    return s;
}

/* Alg. 1 Steps 2-3 for k vectors on hierarchy h (schedule 0 tolerance, 2
 * replay).  converged != 0: after level 0, sweep level 0 until every
 * vector's residual ||(L - lambda_i I) u_i|| <= conv_rtol g_0 (test use).
 * Outputs: U (k vectors of n_0, R11 sign each), lam[k], res[k] (Sec. 4 error
 * metric per vector), sweeps[J+1].  Returns 1 if a cap was reached, 0, or -1
 * when k is outside 1 .. n_J - 1.                                           */
ORC_EXPORT int32_t orc_solve_block(orc_hierarchy *h, int32_t k, uint64_t seed, double tol,
                                   int32_t schedule, const int64_t *replay, int64_t max_sweeps,
                                   int64_t max_sweeps_coarsest, int32_t converged,
                                   double conv_rtol, double *U, double *lam, double *res,
                                   int64_t *sweeps_out)
{
    int32_t J = h->levels - 1;
    if (k < 1 || (int64_t)k > h->lv[J].n - 1) return -1;
    int32_t warn = 0, capped = 0;
    orc_level *c = &h->lv[J];
    double *Y = (double *)malloc(sizeof(double) * (size_t)c->n * (size_t)k);
    for (int32_t i = 0; i < k; i++)
        orc_gaussian_start(seed + (uint64_t)i, c->n, Y + (size_t)i * (size_t)c->n);
    int32_t mode = (schedule == 2) ? 1 : 0;
    c->sweeps = block_power_iteration(c->n, c->rp, c->col, c->w, c->g, k, Y, tol, mode,
                                      mode ? replay[J] : 0, max_sweeps_coarsest, &capped);
    warn |= capped;
    for (int32_t j = J - 1; j >= 0; j--) {
        orc_level *f = &h->lv[j];
        int64_t nc = h->lv[j + 1].n;
        double *X = (double *)malloc(sizeof(double) * (size_t)f->n * (size_t)k);
        for (int32_t i = 0; i < k; i++)
            for (int64_t r = 0; r < f->n; r++)
                X[(size_t)i * (size_t)f->n + (size_t)r] = Y[(size_t)i * (size_t)nc + (size_t)f->agg[r]];
        f->sweeps = block_power_iteration(f->n, f->rp, f->col, f->w, f->g, k, X, tol, mode,
                                          mode ? replay[j] : 0, max_sweeps, &capped);
        warn |= capped;
        free(Y);
        Y = X;
    }
    orc_level *f = &h->lv[0];
    if (converged) {
        for (int64_t it = 0; it < 100000; it++) {
            double worst = 0.0;
            for (int32_t i = 0; i < k; i++) {
                double l, r;
                orc_rayleigh_residual(f->n, f->rp, f->col, f->w, Y + (size_t)i * (size_t)f->n, &l, &r);
                if (r > worst) worst = r;
            }
            if (worst <= conv_rtol * f->g) break;
            block_power_iteration(f->n, f->rp, f->col, f->w, f->g, k, Y, tol, 1, 64, 64, NULL);
        }
    }
    for (int32_t i = 0; i < k; i++) {
        double *y = Y + (size_t)i * (size_t)f->n;
        int64_t imax = 0;
        for (int64_t r = 1; r < f->n; r++)
            if (fabs(y[r]) > fabs(y[imax])) imax = r;
        double sg = (y[imax] < 0.0) ? -1.0 : 1.0;
        double *u = U + (size_t)i * (size_t)f->n;
        for (int64_t r = 0; r < f->n; r++) u[r] = sg * y[r];
        orc_rayleigh_residual(f->n, f->rp, f->col, f->w, u, lam + i, res + i);
    }
    for (int32_t j = 0; j <= J; j++)
        if (sweeps_out) sweeps_out[j] = h->lv[j].sweeps;
    free(Y);
    return warn;
}
