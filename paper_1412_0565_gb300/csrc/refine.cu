// refine.cu -- power iteration (Alg. 3 of arXiv 1412.0565), the final vector,
// its sign, and the Rayleigh quotient / residual of Sec. 4.
//
// A sweep computes u <- B_g v = g v - L v, projects u against 1 and
// normalises it (Alg. 3; the projection is repeated every sweep, which equals
// Alg. 3 in exact arithmetic and keeps rounding from growing along 1, the
// dominant eigenvector of B_g).  The normalised iterate is never stored: a
// buffer holds the raw vector y and scalars (mu, 1/s) with u = (y - mu) / s,
// and the next sweep applies B_g to u on the fly,
//     (B_g u)_i = [ g (y_i - mu) - sum_j w_ij (y_i - y_j) ] / s
// (edge-difference form of L; mu cancels inside the differences).  The same
// pass accumulates sum y, sum y^2, sum y u_prev, sum u_prev, sum u_prev^2 in
// FP64, from which the next (mu, s) and the stopping cosine cos(u^k, u^{k-1})
// follow.  Every combination of partial sums runs in a fixed order, so results
// are bitwise reproducible and all CTAs take the same stop decision.
//
// Two kernels:
//   k_power_tiled  large levels: a cooperative persistent kernel, one grid
//                  barrier per sweep.  The rows are cut into tiles of at most
//                  kTileRows rows and about kChunk entries; a tile's column
//                  indices and weights are streamed with coalesced loads, all
//                  its x gathers are in flight at once, and the products are
//                  summed per row, left to right, in shared memory.
//   k_power_small  small levels: one CTA holds the level's CSR and both
//                  vectors in shared memory; a sweep costs two __syncthreads.
#include <algorithm>
#include <math.h>

#include "internal.h"

namespace cmg {

// Loads of data written by other CTAs of the same launch go through L2.
#define LDX(p) __ldcg(p)

constexpr int kNumPartials = 5;
constexpr int kTileThreads = 512;
constexpr int kTileRows = 1024;      // rows per tile (cost units: 4 per row)
constexpr int kChunk = 4096;         // entries per chunk of a tile
constexpr int kTileCost = 4096;      // cost of a tile: entries + 4 * rows
constexpr int kSmallThreads = 1024;
constexpr int kFinThreads = 256;

struct PiArgs {
    int n;
    const int *rp;
    const int *col;
    const double *w;
    const float *w32;
    double g;
    const int *tile_row;
    int ntiles;
    int mode;
    int k_fixed;
    int max_sweeps;
    double tol;
    uint64_t seed;
    int start;             // 0 Gaussian, 1 prolongation, 2 explicit
    const void *cbuf0;     // coarse level buffers (start = 1)
    const void *cbuf1;
    const PiResult *cres;
    const int *agg;
    const double *x_init;  // start = 2
    void *buf0;
    void *buf1;
    PiResult *res;
    double *partials;      // [2][gridDim.x][kNumPartials]
};

__device__ __forceinline__ uint64_t sm64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Alg. 1 Step 2's randn: Box-Muller on two splitmix64 uniforms in (0, 1]:
// a = splitmix64(seed ^ 0xC0A45E ^ 2i), b = splitmix64(seed ^ 0xC0A45E ^ (2i+1)).
__device__ __forceinline__ double gaussian_entry(uint64_t seed, long long i) {
    const uint64_t a = sm64(seed ^ 0xC0A45Eull ^ (uint64_t)(2 * i));
    const uint64_t b = sm64(seed ^ 0xC0A45Eull ^ (uint64_t)(2 * i + 1));
    const double u1 = (double)((a >> 11) + 1) * (1.0 / 9007199254740992.0);
    const double u2 = (double)((b >> 11) + 1) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

// Start value of row i: Gaussian (Alg. 1 Step 2), prolongation (I^T y of
// Alg. 1 Step 3) of the coarse result, or an explicit vector.
template <typename T>
__device__ __forceinline__ double start_value(const PiArgs &a, int i, const T *cb, double cmu,
                                              double cinv) {
    if (a.start == 0) return gaussian_entry(a.seed, i);
    if (a.start == 1) return ((double)cb[a.agg[i]] - cmu) * cinv;
    return a.x_init[i];
}

// Iteration state shared by both kernels.
struct SweepState {
    double mu, inv_s, mu_prev, inv_prev, cosv;
    int cur, k, zero;
};

// Scalars after a sweep from the sums S; returns true when the iteration stops.
__device__ __forceinline__ bool after_sweep(const PiArgs &a, const double *S, int n, SweepState &st) {
    st.k++;
    const double muy = S[0] / (double)n;
    double ss = S[1] - (double)n * muy * muy;
    if (ss < 0.0) ss = 0.0;
    const double den = sqrt(ss * S[4]);
    st.cosv = den > 0.0 ? (S[2] - muy * S[3]) / den : 1.0;
    // B_g annihilated the unit iterate to rounding level: it is an
    // eigenvector of L with eigenvalue g (e.g. n = 2); keep it and stop
    if (sqrt(ss) <= 64.0 * 2.220446049250313e-16 * a.g) {
        st.zero = 1;
        return true;
    }
    st.mu_prev = st.mu;
    st.inv_prev = st.inv_s;
    st.mu = muy;
    st.inv_s = 1.0 / sqrt(ss);
    st.cur ^= 1;
    if (a.mode == 1) return st.k >= a.k_fixed;
    if (!(st.cosv < 1.0 - a.tol)) return true;
    return st.k >= a.max_sweeps;
}

__device__ __forceinline__ void write_result(const PiArgs &a, const SweepState &st, bool run) {
    PiResult r;
    r.mu = st.mu;
    r.inv_s = st.inv_s;
    r.cos = st.cosv;
    r.mu_prev = st.mu_prev;
    r.inv_s_prev = st.inv_prev;
    r.buf = st.cur;
    r.sweeps = st.k;
    r.capped = (a.mode == 0 && run && !st.zero && st.cosv < 1.0 - a.tol) ? 1 : 0;
    r.zero = st.zero;
    *a.res = r;
}

// Sum of K per-thread doubles over the CTA, result in out[] of every thread
// (fixed order).  sm: 32*K doubles.  Two __syncthreads.
template <int K>
__device__ __forceinline__ void block_allsum(double (&v)[K], double *sm, double (&out)[K]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sm[warp * K + k] = v[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; k++) {
        double t = (lane < nw) ? sm[lane * K + k] : 0.0;
        out[k] = warp_sum(t);
    }
    __syncthreads();
}

// Grid-wide sum of K doubles per thread, result in out[] of every thread.
template <int K>
__device__ __forceinline__ bool grid_allsum(double (&v)[K], double *sm, double *part,
                                            double (&out)[K], GridSync *gs) {
    double tot[K];
    block_allsum<K>(v, sm, tot);
    if (gridDim.x == 1) {
#pragma unroll
        for (int k = 0; k < K; k++) out[k] = tot[k];
        return true;
    }
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < K; k++) part[blockIdx.x * K + k] = tot[k];
    if (!grid_sync(gs)) return false;
    const int lane = threadIdx.x & 31;
    double s[K];
#pragma unroll
    for (int k = 0; k < K; k++) s[k] = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32)
#pragma unroll
        for (int k = 0; k < K; k++) s[k] += LDX(part + b * K + k);
#pragma unroll
    for (int k = 0; k < K; k++) out[k] = warp_sum(s[k]);
    return true;
}

template <typename T>
__device__ __forceinline__ const T *wsel(const PiArgs &a);
template <>
__device__ __forceinline__ const double *wsel<double>(const PiArgs &a) { return a.w; }
template <>
__device__ __forceinline__ const float *wsel<float>(const PiArgs &a) { return a.w32; }

// ================================================================== tiled kernel
template <typename T>
__global__ void __launch_bounds__(kTileThreads, 2) k_power_tiled(PiArgs a, GridSync *gs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s_prod = reinterpret_cast<T *>(smem_raw);                       // kChunk
    T *s_x = s_prod + kChunk;                                         // kTileRows
    T *s_acc = s_x + kTileRows;                                       // kTileRows
    int *s_rp = reinterpret_cast<int *>(s_acc + kTileRows);           // kTileRows + 1
    unsigned short *s_row = reinterpret_cast<unsigned short *>(s_rp + kTileRows + 4);  // kChunk
    __shared__ double sm[32 * kNumPartials];

    const int n = a.n;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int tb = (int)((long long)a.ntiles * blockIdx.x / gridDim.x);
    const int te = (int)((long long)a.ntiles * (blockIdx.x + 1) / gridDim.x);
    const int r0 = a.tile_row[tb], r1 = a.tile_row[te];
    T *buf0 = (T *)a.buf0, *buf1 = (T *)a.buf1;
    const T *__restrict__ wv = wsel<T>(a);
    double *part0 = a.partials;
    double *part1 = a.partials + (size_t)gridDim.x * kNumPartials;

    // ---- start vector into buf0; Gram-Schmidt against 1; norm
    double p[kNumPartials] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double S[kNumPartials];
    {
        const T *cb = nullptr;
        double cmu = 0.0, cinv = 0.0;
        if (a.start == 1) {
            cb = (const T *)(a.cres->buf ? a.cbuf1 : a.cbuf0);
            cmu = a.cres->mu;
            cinv = a.cres->inv_s;
        }
        for (int i = r0 + tid; i < r1; i += nt) {
            const T xt = (T)start_value<T>(a, i, cb, cmu, cinv);
            buf0[i] = xt;
            p[0] += (double)xt;
        }
    }
    if (!grid_allsum<kNumPartials>(p, sm, part0, S, gs)) return;
    const double mu0 = S[0] / (double)n;
    p[0] = 0.0;
    for (int i = r0 + tid; i < r1; i += nt) {
        const double d = (double)buf0[i] - mu0;
        p[0] += d * d;
    }
    if (!grid_allsum<kNumPartials>(p, sm, part1, S, gs)) return;
    SweepState st;
    st.mu = mu0;
    st.inv_s = S[0] > 0.0 ? 1.0 / sqrt(S[0]) : 0.0;
    st.mu_prev = st.mu;
    st.inv_prev = st.inv_s;
    st.cosv = 0.0;
    st.cur = 0;
    st.k = 0;
    st.zero = 0;
    const bool run = !(a.mode == 1 && a.k_fixed <= 0);
    const T gT = (T)a.g;
    constexpr int U = kChunk / kTileThreads;

    while (run) {
        const T *x = st.cur ? buf1 : buf0;
        T *y = st.cur ? buf0 : buf1;
        const T muT = (T)st.mu, invT = (T)st.inv_s;
        const double mu = st.mu, inv_s = st.inv_s;
#pragma unroll
        for (int q = 0; q < kNumPartials; q++) p[q] = 0.0;
        for (int t = tb; t < te; t++) {
            const int t0 = a.tile_row[t], t1 = a.tile_row[t + 1];
            const int nr = t1 - t0;
            if (nr <= 0) continue;
            const int e0 = __ldg(a.rp + t0);
            const int ne = __ldg(a.rp + t1) - e0;
            for (int k = tid; k < nr; k += nt) {
                s_rp[k] = __ldg(a.rp + t0 + k) - e0;
                s_x[k] = LDX(x + t0 + k);
                s_acc[k] = (T)0;
            }
            if (tid == 0) s_rp[nr] = ne;
            __syncthreads();
            for (int c0 = 0; c0 < ne; c0 += kChunk) {
                const int cn = min(kChunk, ne - c0);
                // row of every entry of the chunk
                for (int r = tid; r < nr; r += nt) {
                    const int lo = max(s_rp[r], c0), hi = min(s_rp[r + 1], c0 + cn);
                    for (int q = lo; q < hi; q++) s_row[q - c0] = (unsigned short)r;
                }
                __syncthreads();
                // products w_ij (x_i - x_j): all loads of the chunk issued first
                int jj[U];
                T ww[U], xj[U];
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int k = tid + u * kTileThreads;
                    jj[u] = 0;
                    ww[u] = (T)0;
                    if (k < cn) {
                        jj[u] = __ldg(a.col + e0 + c0 + k);
                        ww[u] = __ldg(wv + e0 + c0 + k);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int k = tid + u * kTileThreads;
                    xj[u] = (T)0;
                    if (k < cn) xj[u] = LDX(x + jj[u]);
                }
#pragma unroll
                for (int u = 0; u < U; u++) {
                    const int k = tid + u * kTileThreads;
                    if (k < cn) s_prod[k] = ww[u] * (s_x[s_row[k]] - xj[u]);
                }
                __syncthreads();
                // per-row sums, left to right
                for (int r = tid; r < nr; r += nt) {
                    const int lo = max(s_rp[r], c0), hi = min(s_rp[r + 1], c0 + cn);
                    T acc = s_acc[r];
                    for (int q = lo; q < hi; q++) acc += s_prod[q - c0];
                    s_acc[r] = acc;
                }
                __syncthreads();
            }
            for (int r = tid; r < nr; r += nt) {
                const T xi = s_x[r];
                const T yv = (gT * (xi - muT) - s_acc[r]) * invT;
                y[t0 + r] = yv;
                const double yd = (double)yv;
                const double xs = ((double)xi - mu) * inv_s;
                p[0] += yd;
                p[1] += yd * yd;
                p[2] += yd * xs;
                p[3] += xs;
                p[4] += xs * xs;
            }
            __syncthreads();
        }
        if (!grid_allsum<kNumPartials>(p, sm, (st.k & 1) ? part1 : part0, S, gs)) return;
        if (after_sweep(a, S, n, st)) break;
    }
    if (blockIdx.x == 0 && tid == 0) write_result(a, st, run);
}

// ================================================================== small kernel
// Shared memory: w[m] T, x[n] T, y[n] T, rp[n+1] int, col[m] int.
template <typename T>
constexpr size_t small_smem_bytes(long long n, long long m) {
    return (size_t)(4 * (n + 1) + 4 * m + sizeof(T) * m + 2 * sizeof(T) * n + 64);
}

template <typename T, int G>
__global__ void __launch_bounds__(kSmallThreads) k_power_small(PiArgs a, GridSync *) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n;
    const int m = a.rp[n];
    T *s_w = reinterpret_cast<T *>(smem_raw);
    T *s_x0 = s_w + m;
    T *s_x1 = s_w + m + n;
    int *s_rp = reinterpret_cast<int *>(s_w + m + 2 * n);
    int *s_col = s_rp + n + 1;
    __shared__ double sm[32 * kNumPartials];
    const int tid = threadIdx.x, nt = blockDim.x;
    const T *__restrict__ wv = wsel<T>(a);

    for (int i = tid; i <= n; i += nt) s_rp[i] = a.rp[i];
    for (int e = tid; e < m; e += nt) {
        s_col[e] = a.col[e];
        s_w[e] = wv[e];
    }
    double p[kNumPartials] = {0.0, 0.0, 0.0, 0.0, 0.0};
    double S[kNumPartials];
    {
        const T *cb = nullptr;
        double cmu = 0.0, cinv = 0.0;
        if (a.start == 1) {
            cb = (const T *)(a.cres->buf ? a.cbuf1 : a.cbuf0);
            cmu = a.cres->mu;
            cinv = a.cres->inv_s;
        }
        for (int i = tid; i < n; i += nt) {
            const T xt = (T)start_value<T>(a, i, cb, cmu, cinv);
            s_x0[i] = xt;
            p[0] += (double)xt;
        }
    }
    block_allsum<kNumPartials>(p, sm, S);
    const double mu0 = S[0] / (double)n;
    p[0] = 0.0;
    for (int i = tid; i < n; i += nt) {
        const double d = (double)s_x0[i] - mu0;
        p[0] += d * d;
    }
    block_allsum<kNumPartials>(p, sm, S);
    SweepState st;
    st.mu = mu0;
    st.inv_s = S[0] > 0.0 ? 1.0 / sqrt(S[0]) : 0.0;
    st.mu_prev = st.mu;
    st.inv_prev = st.inv_s;
    st.cosv = 0.0;
    st.cur = 0;
    st.k = 0;
    st.zero = 0;
    const bool run = !(a.mode == 1 && a.k_fixed <= 0);
    const T gT = (T)a.g;
    const int lane = tid & (G - 1);
    const int groups = nt / G;
    while (run) {
        const T *x = st.cur ? s_x1 : s_x0;
        T *y = st.cur ? s_x0 : s_x1;
        const T muT = (T)st.mu, invT = (T)st.inv_s;
        const double mu = st.mu, inv_s = st.inv_s;
#pragma unroll
        for (int q = 0; q < kNumPartials; q++) p[q] = 0.0;
        for (int base = tid / G;; base += groups) {
            if (__shfl_sync(0xffffffffu, base, 0) >= n) break;
            const int i = base;
            T acc = (T)0, xi = (T)0;
            if (i < n) {
                xi = x[i];
                for (int e = s_rp[i] + lane, e1 = s_rp[i + 1]; e < e1; e += G)
                    acc += s_w[e] * (xi - x[s_col[e]]);
            }
            acc = group_sum<G>(acc);
            if (i < n && lane == 0) {
                const T yv = (gT * (xi - muT) - acc) * invT;
                y[i] = yv;
                const double yd = (double)yv;
                const double xs = ((double)xi - mu) * inv_s;
                p[0] += yd;
                p[1] += yd * yd;
                p[2] += yd * xs;
                p[3] += xs;
                p[4] += xs * xs;
            }
        }
        block_allsum<kNumPartials>(p, sm, S);
        if (after_sweep(a, S, n, st)) break;
    }
    // result -> buf0, previous iterate -> buf1 (for the FP64 final recompute)
    T *out0 = (T *)a.buf0, *out1 = (T *)a.buf1;
    const T *res = st.cur ? s_x1 : s_x0;
    const T *prv = st.cur ? s_x0 : s_x1;
    for (int i = tid; i < n; i += nt) {
        out0[i] = res[i];
        out1[i] = prv[i];
    }
    if (tid == 0) {
        SweepState r = st;
        r.cur = 0;
        write_result(a, r, run);
    }
}

// ================================================================== host side
__global__ void k_tiles(int n, const int *__restrict__ rp, int ntiles, int *__restrict__ tile_row) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= ntiles; k += gridDim.x * blockDim.x) {
        if (k == ntiles) {
            tile_row[k] = n;
            continue;
        }
        const long long target = (long long)k * kTileCost;
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if ((long long)rp[mid] + 4ll * mid < target) lo = mid + 1;
            else hi = mid;
        }
        tile_row[k] = lo;
    }
}

int tile_count(int n, long long nnz) { return (int)((nnz + 4ll * n + kTileCost - 1) / kTileCost); }

cmg_status_t build_tiles(int n, long long nnz, const int *rp, int *tile_row, cudaStream_t s) {
    const int nt = tile_count(n, nnz);
    k_tiles<<<grid_for(nt + 1, 256), 256, 0, s>>>(n, rp, nt, tile_row);
    return launch_status();
}

static size_t tiled_smem(bool fp32) {
    const size_t e = fp32 ? sizeof(float) : sizeof(double);
    return e * (kChunk + 2 * kTileRows) + sizeof(int) * (kTileRows + 4) + 2 * kChunk;
}

template <typename T>
static const void *small_kernel(int G) {
    switch (G) {
        case 1: return (const void *)k_power_small<T, 1>;
        case 2: return (const void *)k_power_small<T, 2>;
        case 4: return (const void *)k_power_small<T, 4>;
        case 8: return (const void *)k_power_small<T, 8>;
        case 16: return (const void *)k_power_small<T, 16>;
        default: return (const void *)k_power_small<T, 32>;
    }
}

// Lanes per row in the small kernel: about 4 entries per lane, and one row
// per lane group when the level has at most kSmallThreads / G rows.
static int small_lanes(int n, long long nnz) {
    const double avg = (double)nnz / (double)std::max(1, n);
    int g = 1;
    while (g < 32 && g * 4 < avg) g <<= 1;
    while (g > 1 && (long long)(kSmallThreads / g) < n) g >>= 1;
    return g;
}

bool small_level_fits(int n, long long nnz, int fp32) {
    DeviceInfo d;
    if (device_info(&d) != CMG_OK) return false;
    const size_t b = fp32 ? small_smem_bytes<float>(n, nnz) : small_smem_bytes<double>(n, nnz);
    return b + 32 * kNumPartials * 8 + 256 <= (size_t)d.max_smem_optin;
}

cmg_status_t power_iteration(const PiRun &run, GridSync *gs, cudaStream_t s, const PiWorkspace *ws) {
    const PiLevel &lv = *run.lv;
    Scratch scr(s);
    PiArgs a;
    a.n = lv.n;
    a.rp = lv.rp;
    a.col = lv.col;
    a.w = lv.w;
    a.w32 = lv.w32;
    a.g = lv.g;
    a.tile_row = lv.tile_row;
    a.ntiles = lv.ntiles;
    a.mode = run.mode;
    a.k_fixed = run.k_fixed;
    a.max_sweeps = run.max_sweeps;
    a.tol = run.tol;
    a.seed = run.seed;
    a.start = run.x_init ? 2 : (run.coarse_res ? 1 : 0);
    a.cbuf0 = run.coarse_buf;
    a.cbuf1 = run.coarse_buf1;
    a.cres = run.coarse_res;
    a.agg = run.coarse_agg;
    a.x_init = run.x_init;
    a.buf0 = run.bufs[0];
    a.buf1 = run.bufs[1];
    a.res = run.res;
    a.partials = nullptr;
    void *args[] = {&a, &gs};
    if (small_level_fits(lv.n, lv.nnz, run.fp32)) {
        const int G = small_lanes(lv.n, lv.nnz);
        const void *kern = run.fp32 ? small_kernel<float>(G) : small_kernel<double>(G);
        const size_t smem = run.fp32 ? small_smem_bytes<float>(lv.n, lv.nnz)
                                     : small_smem_bytes<double>(lv.n, lv.nnz);
        CMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        return coop_launch(kern, 1, kSmallThreads, smem, s, args, gs);
    }
    if (!a.tile_row) {
        int *tr;
        if (ws) {
            if (tile_count(lv.n, lv.nnz) + 1 > ws->tile_cap) return CMG_ERR_TOO_LARGE;
            tr = ws->tile_row;
        } else {
            CMG_TRY(scr.get(&tr, (size_t)tile_count(lv.n, lv.nnz) + 1));
        }
        CMG_TRY(build_tiles(lv.n, lv.nnz, lv.rp, tr, s));
        a.tile_row = tr;
        a.ntiles = tile_count(lv.n, lv.nnz);
    }
    const void *kern = run.fp32 ? (const void *)k_power_tiled<float> : (const void *)k_power_tiled<double>;
    const size_t smem = tiled_smem(run.fp32 != 0);
    CMG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int maxb = 0;
    CMG_TRY(coop_max_blocks(kern, kTileThreads, smem, &maxb));
    // at least 4 tiles per CTA where possible, never more CTAs than co-resident
    int blocks = std::max(1, std::min(maxb, (a.ntiles + 3) / 4));
    double *partials;
    if (ws) {
        if (2 * blocks * kNumPartials > ws->partials_cap) return CMG_ERR_TOO_LARGE;
        partials = ws->partials;
    } else {
        CMG_TRY(scr.get(&partials, (size_t)2 * blocks * kNumPartials));
    }
    a.partials = partials;
    return coop_launch(kern, blocks, kTileThreads, smem, s, args, gs);
}

// ================================================================== finalisation
// Rows [r0, r1) of CTA b out of nb, balanced by 3 * nnz + 5 * rows.
__device__ __forceinline__ void cta_rows(const int *rp, int n, int b, int nb, int *r0, int *r1) {
    const long long total = 3ll * rp[n] + 5ll * n;
    auto first_at = [&](long long target) {
        int lo = 0, hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (3ll * rp[mid] + 5ll * mid < target) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    *r0 = (b == 0) ? 0 : first_at((total * b + nb - 1) / nb);
    *r1 = (b == nb - 1) ? n : first_at((total * (b + 1) + nb - 1) / nb);
}

struct FinArgs {
    int n;
    const int *rp;
    const int *col;
    const double *w;
    double g;
    int fp32;
    const void *buf0;
    const void *buf1;
    const PiResult *res;
    double *u;
    double *tmp;
    double *part;      // [3][gridDim.x][4]
    double *out;       // [2]: lambda, residual
    int sign;          // apply the canonical sign
    int fresh;         // u already holds the vector (skip the vector phase)
};

// (|v|, index) order of the sign rule: larger magnitude first, lower index on ties.
__device__ __forceinline__ bool better(double v, int i, double bv, int bi) {
    return v > bv || (v == bv && i < bi);
}

template <int G>
__global__ void __launch_bounds__(kFinThreads) k_finalize(FinArgs a, GridSync *gs) {
    __shared__ double sm[32 * 4];
    __shared__ double s_best[32], s_bval[32];
    __shared__ int s_bidx[32];
    const int n = a.n;
    int r0, r1;
    cta_rows(a.rp, n, blockIdx.x, gridDim.x, &r0, &r1);
    const int lane = threadIdx.x & (G - 1);
    const int groups = blockDim.x / G;
    double *part0 = a.part, *part1 = a.part + (size_t)gridDim.x * 4,
           *part2 = a.part + (size_t)gridDim.x * 8;
    double p[4], S[4];

    if (!a.fresh) {
        const PiResult r = *a.res;
        const bool recompute = a.fp32 && r.sweeps > 0 && !r.zero;
        if (recompute) {
            // FP64 recomputation of the last sweep from the previous (FP32) iterate
            const float *x = (const float *)(r.buf ? a.buf0 : a.buf1);
            p[0] = p[1] = p[2] = p[3] = 0.0;
            for (int base = r0 + threadIdx.x / G;; base += groups) {
                if (__shfl_sync(0xffffffffu, base, 0) >= r1) break;
                const int i = base;
                double acc = 0.0, xi = 0.0;
                if (i < r1) {
                    xi = ((double)x[i] - r.mu_prev) * r.inv_s_prev;
                    const int e1 = __ldg(a.rp + i + 1);
                    for (int e = __ldg(a.rp + i) + lane; e < e1; e += G) {
                        const double xj = ((double)x[__ldg(a.col + e)] - r.mu_prev) * r.inv_s_prev;
                        acc += __ldg(a.w + e) * (xi - xj);
                    }
                }
                acc = group_sum<G>(acc);
                if (i < r1 && lane == 0) {
                    const double yv = a.g * xi - acc;
                    a.tmp[i] = yv;
                    p[0] += yv;
                    p[1] += yv * yv;
                }
            }
            if (!grid_allsum<4>(p, sm, part0, S, gs)) return;
            const double mu = S[0] / (double)n;
            const double ss = S[1] - (double)n * mu * mu;
            const double inv = ss > 0.0 ? 1.0 / sqrt(ss) : 0.0;
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) a.u[i] = (a.tmp[i] - mu) * inv;
        } else if (a.fp32) {
            const float *y = (const float *)(r.buf ? a.buf1 : a.buf0);
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x)
                a.u[i] = ((double)y[i] - r.mu) * r.inv_s;
        } else {
            const double *y = (const double *)(r.buf ? a.buf1 : a.buf0);
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) a.u[i] = (y[i] - r.mu) * r.inv_s;
        }
    }
    // ---- canonical sign: the entry of largest |u_i| (lowest index on ties) is
    // made positive.  Its signed value travels with the reduction, so no CTA
    // reads u after another may have negated it.
    if (a.sign) {
        double best = -1.0, bval = 0.0;
        int bidx = 0x7fffffff;
        for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const double v = a.u[i];
            if (better(fabs(v), i, best, bidx)) {
                best = fabs(v);
                bidx = i;
                bval = v;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
            const double ov = __shfl_xor_sync(0xffffffffu, bval, o);
            if (better(ob, oi, best, bidx)) {
                best = ob;
                bidx = oi;
                bval = ov;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            s_best[threadIdx.x >> 5] = best;
            s_bidx[threadIdx.x >> 5] = bidx;
            s_bval[threadIdx.x >> 5] = bval;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < (int)blockDim.x / 32; q++)
                if (better(s_best[q], s_bidx[q], best, bidx)) {
                    best = s_best[q];
                    bidx = s_bidx[q];
                    bval = s_bval[q];
                }
            part1[blockIdx.x * 4 + 0] = best;
            part1[blockIdx.x * 4 + 1] = (double)bidx;
            part1[blockIdx.x * 4 + 2] = bval;
        }
        if (!grid_sync(gs)) return;
        __syncthreads();
        if (threadIdx.x == 0) {
            double bb = -1.0, bv = 0.0;
            int bi = 0x7fffffff;
            for (int b = 0; b < (int)gridDim.x; b++) {
                const double v = LDX(part1 + b * 4 + 0);
                const int ii = (int)LDX(part1 + b * 4 + 1);
                if (better(v, ii, bb, bi)) {
                    bb = v;
                    bi = ii;
                    bv = LDX(part1 + b * 4 + 2);
                }
            }
            s_bval[0] = bv;
        }
        __syncthreads();
        if (s_bval[0] < 0.0)
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) a.u[i] = -a.u[i];
        if (!grid_sync(gs)) return;
    } else if (!a.fresh) {
        if (!grid_sync(gs)) return;
    }
    // ---- Rayleigh quotient: lambda = (1/2) sum_i sum_j w_ij (u_i - u_j)^2 / ||u||^2
    p[0] = p[1] = p[2] = p[3] = 0.0;
    for (int base = r0 + threadIdx.x / G;; base += groups) {
        if (__shfl_sync(0xffffffffu, base, 0) >= r1) break;
        const int i = base;
        double acc = 0.0, ui = 0.0;
        if (i < r1) {
            ui = LDX(a.u + i);
            const int e1 = __ldg(a.rp + i + 1);
            for (int e = __ldg(a.rp + i) + lane; e < e1; e += G) {
                const double d = ui - LDX(a.u + __ldg(a.col + e));
                acc += __ldg(a.w + e) * d * d;
            }
        }
        acc = group_sum<G>(acc);
        if (i < r1 && lane == 0) {
            p[0] += acc;
            p[1] += ui * ui;
        }
    }
    if (!grid_allsum<4>(p, sm, part2, S, gs)) return;
    const double uu = S[1];
    const double lam = 0.5 * S[0] / uu;
    // ---- residual ||(L - lambda I) u|| / ||u||, (L u)_i = sum_j w_ij (u_i - u_j)
    p[0] = p[1] = p[2] = p[3] = 0.0;
    for (int base = r0 + threadIdx.x / G;; base += groups) {
        if (__shfl_sync(0xffffffffu, base, 0) >= r1) break;
        const int i = base;
        double acc = 0.0, ui = 0.0;
        if (i < r1) {
            ui = LDX(a.u + i);
            const int e1 = __ldg(a.rp + i + 1);
            for (int e = __ldg(a.rp + i) + lane; e < e1; e += G)
                acc += __ldg(a.w + e) * (ui - LDX(a.u + __ldg(a.col + e)));
        }
        acc = group_sum<G>(acc);
        if (i < r1 && lane == 0) {
            const double rr = acc - lam * ui;
            p[0] += rr * rr;
        }
    }
    if (!grid_allsum<4>(p, sm, part0, S, gs)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out[0] = lam;
        a.out[1] = sqrt(S[0] / uu);
    }
}

static const void *finalize_kernel(int G) {
    switch (G) {
        case 2: return (const void *)k_finalize<2>;
        case 4: return (const void *)k_finalize<4>;
        case 8: return (const void *)k_finalize<8>;
        case 16: return (const void *)k_finalize<16>;
        default: return (const void *)k_finalize<32>;
    }
}

cmg_status_t finalize(const PiLevel &lv, int fp32, const void *buf0, const void *buf1,
                      const PiResult *res, double *u, int sign, int fresh, double *out2,
                      GridSync *gs, cudaStream_t s, const PiWorkspace *ws) {
    const int G = lanes_for_avg((double)lv.nnz / (double)std::max(1, lv.n));
    const void *kern = finalize_kernel(G);
    int maxb = 0;
    CMG_TRY(coop_max_blocks(kern, kFinThreads, 0, &maxb));
    DeviceInfo d;
    CMG_TRY(device_info(&d));
    const long long bytes = 12 * lv.nnz + 20ll * lv.n;
    int blocks = (int)std::min<long long>((bytes + 65535) / 65536, (long long)std::min(maxb, 2 * d.sms));
    blocks = std::max(1, blocks);
    Scratch scr(s);
    double *part, *tmp = nullptr;
    if (ws) {
        if (12 * blocks > ws->fin_part_cap || (fp32 && !fresh)) return CMG_ERR_TOO_LARGE;
        part = ws->fin_part;
    } else {
        CMG_TRY(scr.get(&part, (size_t)12 * blocks));
        if (fp32 && !fresh) CMG_TRY(scr.get(&tmp, (size_t)lv.n));
    }
    FinArgs a;
    a.n = lv.n;
    a.rp = lv.rp;
    a.col = lv.col;
    a.w = lv.w;
    a.g = lv.g;
    a.fp32 = fp32;
    a.buf0 = buf0;
    a.buf1 = buf1;
    a.res = res;
    a.u = u;
    a.tmp = tmp;
    a.part = part;
    a.out = out2;
    a.sign = sign;
    a.fresh = fresh;
    void *args[] = {&a, &gs};
    return coop_launch(kern, blocks, kFinThreads, 0, s, args, gs);
}

}  // namespace cmg
