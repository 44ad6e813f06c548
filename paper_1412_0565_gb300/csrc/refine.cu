// refine.cu -- power iteration (Alg. 3 of arXiv 1412.0565), the final vector,
// its sign, and the Rayleigh quotient / residual of Sec. 4.
//
// Alg. 3 iterates u <- B_g v / ||B_g v|| with B_g = g I - L, after one
// Gram-Schmidt step against 1, and stops when cos(u^k, u^{k-1}) >= 1 - tol.
// Here the iterate is kept unnormalised, y_s = sigma_{s-1} (B_g y_{s-1} -
// g m_{s-1} 1), with sigma = 2^e / g (an exact power-of-two rescale keeps
// ||y|| near 1) and m an estimate of the mean of y_{s-1}, so that u_s is
// (y_s - mean(y_s)) / ||y_s - mean(y_s)||: the same vector as Alg. 3's in exact
// arithmetic, since 1 is an eigenvector of B_g.  Each sweep accumulates
//     A_s = sum y_s,  B_s = sum y_s^2,  C_s = sum y_s y_{s-1}
// from which mean, norm and the stopping cosine follow:
//     mu_s = A_s / n,  ss_s = B_s - n mu_s^2,
//     cos_s = (C_s - n mu_s mu_{s-1}) / sqrt(ss_s ss_{s-1}).
// Those sums are reduced by a dedicated control warp while the other warps
// compute the next sweep, so no reduction is on the critical path: the stop
// decision for sweep s is taken during sweep s+1 (whose result is then
// discarded; the iterates live in a ring of three buffers), and the mean
// estimate for sweep s+2 is m_{s+1} = 2^{e_s} (mu_s - m_s), the propagated
// 1-component of y_s, which keeps that component at rounding level.
//
// Sums and scalars are float-float (ffloat.cuh) on the FP32 pipe; FP64 is
// used where the FP64 form computes its sweeps, and for the final scalars.
//
// Two kernels:
//   k_power_tiled  large levels: cooperative persistent kernel, one grid
//                  barrier per sweep.  Rows are cut into tiles (at most
//                  kTileRows rows, about kChunk entries); a tile's column
//                  indices and weights stream in with coalesced loads, all
//                  its x gathers are issued at once, and per-row sums run left
//                  to right in shared memory.
//   k_power_small  small levels: one CTA holds the CSR and the iterate ring in
//                  shared memory; one __syncthreads per sweep.
#include <algorithm>
#include <functional>
#include <math.h>

#include "ffloat.cuh"
#include "internal.h"
#include "pi_common.cuh"

namespace cmg {

#ifdef CMG_TRACE
// cycle stamps of the first sweeps of the last small-kernel launch:
// [sweep][0] loop top, [1] control done, [2] first row warp done, [3] last row warp done
__device__ long long g_trace[256][8];
#define TRACE(s, k) do { if ((s) < 256) g_trace[(s)][(k)] = clock64(); } while (0)
// cycle stamps of the phases of the two-phase kernel's third sweep, per CTA
// and pass: [b][t][0] pass top, [2] phase 1 done, [3] after the barrier,
// [5] the last dest block's list summed, [6] its rows completed
__device__ long long g_x2t[160][32][8];
#define X2T(s, t, k) do { if ((s) == 2 && (t) < 32 && threadIdx.x == 32 && blockIdx.x < 160) g_x2t[blockIdx.x][(t)][(k)] = clock64(); } while (0)
extern "C" int cmg_debug_x2_trace(long long *host, int count) {
    return (int)cudaMemcpyFromSymbol(host, g_x2t, sizeof(long long) * (size_t)count);
}
// cycle stamps of the cluster kernel's first sweeps (rank 0, thread 0):
// [s][0] loop top, [1] rows done, [2] sums stored, [3] after the barrier
__device__ long long g_clt[256][4];
#define CLT(s, k) do { if ((s) < 256 && threadIdx.x == 0 && cluster_rank() == 0) g_clt[(s)][(k)] = clock64(); } while (0)
extern "C" int cmg_debug_cluster_trace(long long *host, int count) {
    return (int)cudaMemcpyFromSymbol(host, g_clt, sizeof(long long) * (size_t)count);
}
#else
#define TRACE(s, k) do { } while (0)
#define X2T(s, t, k) do { } while (0)
#define CLT(s, k) do { } while (0)
#endif

// Loads of data written by other CTAs of the same launch go through L2.
#define LDX(p) __ldcg(p)
// Gathers of the iterate: ordinary (L1-cached) loads.  The iterate read in a
// sweep was written before the preceding grid barrier, whose acquire by the
// CTA's thread 0 (followed by __syncthreads) orders these loads after the
// writes; the parity tests check this bit for bit against L2-only loads.
#ifdef CMG_X_LDCG
#define LDXG(p) __ldcg(p)
#else
#define LDXG(p) (*(p))
#endif

constexpr int kTileThreads = 512;                 // warp 0: control, 15 row warps
constexpr int kStageThreads = 1024;               // slice kernel with a staged iterate
#ifndef CMG_OCT32
#define CMG_OCT32 2
#endif
constexpr int kOct32 = CMG_OCT32;                 // FP32 heavy rows: octets per lane per round trip
constexpr int kRowThreads = kTileThreads - 32;
constexpr int kU = 8;                             // entries per row thread per chunk
constexpr int kChunk = kRowThreads * kU;          // 3840 entries
constexpr int kTileRows = 960;
constexpr int kTileCost = 3840;                   // entries + 4 * rows per tile
constexpr int kSmallMaxThreads = 1024;
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
    int start;              // 0 Gaussian, 1 prolongation, 2 explicit
    const void *cbuf[3];    // coarse ring (start = 1)
    int cfp64;              // the coarse ring holds doubles (else floats)
    const PiResult *cres;
    const int *agg;
    const double *x_init;   // start = 2
    void *buf[3];           // iterate ring
    double *gd;             // FP64 form: g - d_i
    PiResult *res;
    ff *partials;           // [2][gridDim.x][3] (tiled kernel)
    float zero_tol2;        // (64 eps)^2 of the sweep precision
    long long sell_nnz;     // SELL-32 size of the level (0: unknown)
    const int *cinvp;       // coarse level's layout order (start = 1), or nullptr
    // slice kernel: the level's sweep layout (rows in layout order)
    const int *perm;
    int lay_h, lay_nsl;
    const int *lay_meta;
    const void *lay_col;
    const void *lay_w;
    const int *hchunk;      // heavy rows: first chunk per row ([h+1]), or nullptr
    const int *crow;        // heavy row of each chunk
    int *hcount;            // chunks finished per heavy row
    void *cpart;            // chunk partial sums
    int nchunks;
    int stream_hint;        // the layout is larger than L2: read it evict-first
    int stage_n;            // iterate entries 0..stage_n-1 copied to shared memory per sweep
    // two-phase kernel: the level's XLayout (see internal.h)
    int x_T, x_Q, x_SB, x_VMAX;
    const uint16_t *x_src, *x_dst;
    const void *x_w;
    const int *x_ps, *x_sal, *x_qoff, *x_ndb, *x_dbr, *x_dbl, *x_cdel, *x_choff;
    const uint2 *x_chk;
    double *x_pmax;
    void *x_buf[2];
    int cl_emax;            // cluster kernel: SELL-32 entries each CTA holds (at most)
};


// Start value of row i: Gaussian (Alg. 1 Step 2), prolongation (I^T y of
// Alg. 1 Step 3) of the coarse result, or an explicit vector.
// The coarse ring has the coarse level's own sweep precision (a level held in
// one CTA keeps FP64 sweeps in the FP32 form).
__device__ __forceinline__ double start_value(const PiArgs &a, int i, const void *cb, double cmu,
                                              double cinv) {
    if (a.start == 0) return gaussian_entry(a.seed, i);
    if (a.start == 1) {
        const int c = a.agg[i];
        const int k = a.cinvp ? a.cinvp[c] : c;
        const double v = a.cfp64 ? reinterpret_cast<const double *>(cb)[k]
                                 : (double)reinterpret_cast<const float *>(cb)[k];
        return (v - cmu) * cinv;
    }
    return a.x_init[i];
}


// ------------------------------------------------------------------ control
// Sweep parameters and decisions, double-buffered by sweep parity in shared
// memory.  Slot for sweep t holds what the rows of sweep t need (m_{t-1},
// e_{t-1}) and the stop decision taken for sweep t-2.
struct Slot {
    // FP64 rows: the same scalars as doubles, formed once per sweep by the
    // control warp (an FP64 operation issues at 2 per SM per clock: per-row-
    // thread copies of this arithmetic cost every row warp FP64 issue slots)
    double m_d;     // m as a double
    double sig_d;   // 2^e / g
    double gm_d;    // g m
    ff m;           // mean estimate to subtract
    int e;          // power-of-two rescale exponent
    int stop;       // decision for sweep t-2: 0 continue, 1 stop
    int zero;       // that sweep annihilated the iterate
    int pad;
};

// fp64: also form the doubles (the FP32 kernels leave them unused)
__device__ __forceinline__ Slot slot_make(ff m, int e, double g, bool fp64) {
    Slot sl;
    sl.m = m;
    sl.e = e;
    sl.stop = 0;
    sl.zero = 0;
    sl.pad = 0;
    sl.m_d = sl.sig_d = sl.gm_d = 0.0;
    if (fp64) {
        sl.m_d = ff_to_double(m);
        sl.sig_d = ldexp(1.0 / g, e);
        sl.gm_d = g * sl.m_d;
    }
    return sl;
}

// Scalars of the reduced sweeps, kept by the control warp (all lanes hold
// the same values).
struct Ctl {
    ff mu_prev, ss_prev;   // mean and squared norm of y_{s-1}
    ff m_cur;              // m_s: used by sweep s+1
    ff inv_n, omt2;        // 1/n and (1 - tol)^2
    int e_cur, e_prev;     // e_s, e_{s-1}
    // result of the decision (valid once `stopped`)
    int stopped, zero, res_sweep, capped;
    double mu_res, ss_res, mu_res_prev, ss_res_prev, cos_res;
};


// One control step for sweep s (s >= 1) with its reduced sums P.  Decides,
// and fills the slot for sweep s+2 (m_{s+1}, e_{s+1}).  `count_exit`: the
// loop ends after sweep s regardless (fixed count or sweep cap reached).
__device__ __forceinline__ void ctrl_step(const PiArgs &a, int s, const Part &P, Ctl &c,
                                          Slot *next, bool count_exit, bool fp64) {
    const float nf = (float)a.n;
    // the mean is at rounding level: n mu^2 and n mu mu_prev need no extra
    // precision, mu itself does (it is subtracted from the iterate)
    const ff mu = ff_mul(P.A, c.inv_n);
    const ff ss = ff_add_f(P.B, -nf * mu.hi * mu.hi);
    const ff cs = ff_add_f(P.C, -nf * mu.hi * c.mu_prev.hi);
    // annihilated: ||proj y_s|| <= 64 eps 2^{e_{s-1}} ||proj y_{s-1}||
    const bool zero = ss.hi <= a.zero_tol2 * ldexpf(c.ss_prev.hi, 2 * c.e_prev);
    // cos_s >= 1 - tol  <=>  cs > 0 and cs^2 >= (1 - tol)^2 ss_s ss_{s-1}
    const bool conv = cs.hi > 0.f && !ff_lt(ff_mul(cs, cs), ff_mul(ff_mul(ss, c.ss_prev), c.omt2));
    bool stop = zero;
    if (a.mode == 0) stop = stop || conv || count_exit;
    else stop = stop || count_exit;
    if (stop && !c.stopped) {
        c.stopped = 1;
        c.zero = zero;
        c.res_sweep = s;
        if (zero) {
            c.mu_res = to_d(c.mu_prev);
            c.ss_res = to_d(c.ss_prev);
            c.cos_res = 1.0;
        } else {
            c.mu_res = to_d(mu);
            c.ss_res = to_d(ss);
            c.mu_res_prev = to_d(c.mu_prev);
            c.ss_res_prev = to_d(c.ss_prev);
            const double den = sqrt(c.ss_res * c.ss_res_prev);
            c.cos_res = den > 0.0 ? to_d(cs) / den : 1.0;
        }
        c.capped = (a.mode == 0 && !zero && !conv) ? 1 : 0;
    }
    // parameters of sweep s+2 (exact power-of-two scaling of mu_s - m_s)
    const ff dm = ff_sub(mu, c.m_cur);
    const ff m_next = ff_make(ldexpf(dm.hi, c.e_cur), ldexpf(dm.lo, c.e_cur));
    int e_next = 0;
    {
        // predicted log2 ||y_{s+1}|| <= log2 ||y_s|| + e_s; lift it back to ~1
        const float l2 = 0.5f * log2f(fmaxf(ss.hi, 1e-37f)) + (float)c.e_cur;
        if (l2 < -24.f) e_next = (int)(-l2);
    }
    if (next) {
        *next = slot_make(m_next, e_next, a.g, fp64);
        next->stop = stop ? 1 : 0;
        next->zero = zero ? 1 : 0;
    }
    c.mu_prev = mu;
    c.ss_prev = ss;
    c.m_cur = m_next;
    c.e_prev = c.e_cur;
    c.e_cur = e_next;
}

__device__ __forceinline__ void ctl_init(Ctl &c, const PiArgs &a, double mu0, double ss0, int e0) {
    c.mu_prev = ff_from_double(mu0);
    c.ss_prev = ff_from_double(ss0);
    c.m_cur = ff_zero();   // m_1: the start was projected exactly
    c.inv_n = ff_from_double(1.0 / (double)a.n);
    const double omt = 1.0 - a.tol;
    c.omt2 = ff_from_double(omt * omt);
    c.e_cur = 0;
    c.e_prev = e0;
    c.stopped = 0;
    c.zero = 0;
    c.res_sweep = 0;
    c.capped = 0;
    c.mu_res = mu0;
    c.ss_res = ss0;
    c.mu_res_prev = mu0;
    c.ss_res_prev = ss0;
    c.cos_res = 0.0;
}


__device__ __forceinline__ void write_result(const PiArgs &a, const Ctl &c, int buf, int buf_prev) {
    PiResult r;
    r.mu = c.mu_res;
    r.inv_s = c.ss_res > 0.0 ? 1.0 / sqrt(c.ss_res) : 0.0;
    r.cos = c.cos_res;
    r.mu_prev = c.mu_res_prev;
    r.inv_s_prev = c.ss_res_prev > 0.0 ? 1.0 / sqrt(c.ss_res_prev) : 0.0;
    r.buf = buf;
    r.buf_prev = buf_prev;
    r.sweeps = c.res_sweep;
    r.capped = c.capped;
    r.zero = c.zero;
    r.pad = 0;
    *a.res = r;
}

template <typename T>
__device__ __forceinline__ const T *wsel(const PiArgs &a);
template <>
__device__ __forceinline__ const double *wsel<double>(const PiArgs &a) { return a.w; }
template <>
__device__ __forceinline__ const float *wsel<float>(const PiArgs &a) { return a.w32; }


template <typename P>
__device__ __forceinline__ P pick3(P p0, P p1, P p2, int k) {
    return k == 0 ? p0 : (k == 1 ? p1 : p2);
}

__device__ __forceinline__ void bar_rows(int nthreads) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// ================================================================== tiled kernel
template <typename T>
struct TileSmem;
// FP32: products; FP64: weights and gathered x (the row sum is an FMA chain)
template <>
struct TileSmem<float> {
    float prod[kChunk];
};
template <>
struct TileSmem<double> {
    double wv[kChunk];
    double xj[kChunk];
};

template <typename T>
__global__ void __launch_bounds__(kTileThreads, 2) k_power_tiled(PiArgs a, GridSync *gs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TileSmem<T> &ts = *reinterpret_cast<TileSmem<T> *>(smem_raw);
    T *s_x = reinterpret_cast<T *>(smem_raw + sizeof(TileSmem<T>));     // kTileRows
    T *s_acc = s_x + kTileRows;                                         // kTileRows
    int *s_rp = reinterpret_cast<int *>(s_acc + kTileRows);             // kTileRows + 1
    unsigned short *s_row = reinterpret_cast<unsigned short *>(s_rp + kTileRows + 4);  // kChunk
    __shared__ Part s_pw[kTileThreads / 32];
    __shared__ Slot s_slot[2];

    const int n = a.n;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tb = (int)((long long)a.ntiles * blockIdx.x / gridDim.x);
    const int te = (int)((long long)a.ntiles * (blockIdx.x + 1) / gridDim.x);
    const int r0 = a.tile_row[tb], r1 = a.tile_row[te];
    T *const ring0 = (T *)a.buf[0], *const ring1 = (T *)a.buf[1], *const ring2 = (T *)a.buf[2];
    const T *__restrict__ wv = wsel<T>(a);
    const bool fp64 = sizeof(T) == 8;
    const T g = (T)a.g;
    const float inv_gf = 1.0f / (float)a.g;
    const double inv_gd = 1.0 / a.g;

    // ---------------------------------------------------------- start phase
    // y_0 (and g - d_i for the FP64 form); then one blocking reduction.
    {
        const void *cb = nullptr;
        double cmu = 0.0, cinv = 0.0;
        if (a.start == 1) {
            cb = a.cbuf[a.cres->buf];
            cmu = a.cres->mu;
            cinv = a.cres->inv_s;
        }
        // start sums: A = sum y_0 (not small after a prolongation), B = sum y_0^2
        Part acc = part_zero();
        for (int i = r0 + tid; i < r1; i += blockDim.x) {
            const T xt = (T)start_value(a, i, cb, cmu, cinv);
            ring0[i] = xt;
            if (fp64) {
                double d = 0.0;
                for (int e = __ldg(a.rp + i), e1 = __ldg(a.rp + i + 1); e < e1; e++) d += __ldg(a.w + e);
                a.gd[i] = a.g - d;
            }
            const ff v = fp64 ? ff_from_double((double)xt) : ff_make((float)xt, 0.f);
            acc.A = ff_add(acc.A, v);
            acc.B = ff_add(acc.B, ff_mul(v, v));
        }
        Part p = warp_sum_part(acc);
        if (lane == 0) s_pw[warp] = p;
        __syncthreads();
        if (warp == 0) {
            Part q = (lane < (int)(blockDim.x >> 5)) ? s_pw[lane] : part_zero();
            q = warp_sum_part(q);
            if (lane == 0) {
                ff *dst = a.partials + (size_t)blockIdx.x * 3;
                dst[0] = q.A;
                dst[1] = q.B;
                dst[2] = q.C;
            }
        }
    }
    if (!grid_sync(gs)) return;
    Ctl c;
    if (warp == 0) {
        Part q = part_zero();
        for (int b = lane; b < (int)gridDim.x; b += 32) {
            const ff *src = a.partials + (size_t)b * 3;
            Part t;
            t.A = ff_make(LDX(&src[0].hi), LDX(&src[0].lo));
            t.B = ff_make(LDX(&src[1].hi), LDX(&src[1].lo));
            t.C = ff_zero();
            q = part_add(q, t);
        }
        q = warp_sum_part(q);
        const double mu0 = to_d(q.A) / (double)n;
        double ss0 = to_d(q.B) - (double)n * mu0 * mu0;
        if (ss0 < 0.0) ss0 = 0.0;
        const int e0 = start_exponent(ss0);
        ctl_init(c, a, mu0, ss0, e0);
        if (lane == 0) {
            s_slot[1] = slot_make(ff_from_double(mu0), e0, a.g, fp64);  // sweep 1: exact mean of y_0
            s_slot[0] = slot_make(ff_zero(), 0, a.g, fp64);             // sweep 2: m_1 = 0
        }
    }
    __syncthreads();

    const bool no_sweeps = (a.mode == 1 && a.k_fixed <= 0);
    int s = 0;
    int exit_kind = no_sweeps ? 2 : 0;   // 1: decided stop, 2: count exit
    while (!no_sweeps) {
        const Slot sl = s_slot[(s + 1) & 1];
        if (sl.stop) {
            exit_kind = 1;
            break;
        }
        if ((a.mode == 1 && s >= a.k_fixed) || (a.mode == 0 && s >= a.max_sweeps)) {
            exit_kind = 2;
            break;
        }
        const T *x = pick3<T *>(ring0, ring1, ring2, s % 3);
        T *y = pick3<T *>(ring0, ring1, ring2, (s + 1) % 3);
        if (warp == 0) {
            // ---- control: reduce sweep s over all CTAs, decide, plan sweep s+2
            if (s >= 1) {
                Part q = part_zero();
                const ff *base = a.partials + (size_t)(s & 1) * gridDim.x * 3;
                for (int b = lane; b < (int)gridDim.x; b += 32) {
                    const ff *src = base + (size_t)b * 3;
                    Part t;
                    t.A = ff_make(LDX(&src[0].hi), LDX(&src[0].lo));
                    t.B = ff_make(LDX(&src[1].hi), LDX(&src[1].lo));
                    t.C = ff_make(LDX(&src[2].hi), LDX(&src[2].lo));
                    q = part_add(q, t);
                }
                q = warp_sum_part(q);
                Slot nx;
                ctrl_step(a, s, q, c, &nx, false, fp64);
                if (lane == 0) s_slot[s & 1] = nx;
            }
        } else {
            // ---- rows of sweep s+1
            const int rt = tid - 32;
            const T m = fp64 ? (T)sl.m_d : (T)sl.m.hi;
            const T sig = fp64 ? (T)sl.sig_d : (T)scale2f(inv_gf, sl.e);
            const T gm = fp64 ? (T)sl.gm_d : g * m;
            Acc<T> acc;
            acc.reset();
            for (int t = tb; t < te; t++) {
                const int t0 = a.tile_row[t], t1 = a.tile_row[t + 1];
                const int nr = t1 - t0;
                if (nr <= 0) continue;
                const int e0 = __ldg(a.rp + t0);
                const int ne = __ldg(a.rp + t1) - e0;
                for (int k = rt; k < nr; k += kRowThreads) {
                    s_rp[k] = __ldg(a.rp + t0 + k) - e0;
                    s_x[k] = LDXG(x + t0 + k);
                    s_acc[k] = (T)0;
                }
                if (rt == 0) s_rp[nr] = ne;
                bar_rows(kRowThreads);
                for (int c0 = 0; c0 < ne; c0 += kChunk) {
                    const int cn = min(kChunk, ne - c0);
                    if (!fp64) {
                        for (int r = rt; r < nr; r += kRowThreads) {
                            const int lo = max(s_rp[r], c0), hi = min(s_rp[r + 1], c0 + cn);
                            for (int q = lo; q < hi; q++) s_row[q - c0] = (unsigned short)r;
                        }
                        bar_rows(kRowThreads);
                    }
                    int jj[kU];
                    T ww[kU], xj[kU];
#pragma unroll
                    for (int u = 0; u < kU; u++) {
                        const int k = rt + u * kRowThreads;
                        jj[u] = 0;
                        ww[u] = (T)0;
                        if (k < cn) {
                            jj[u] = __ldg(a.col + e0 + c0 + k);
                            ww[u] = __ldg(wv + e0 + c0 + k);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kU; u++) {
                        const int k = rt + u * kRowThreads;
                        xj[u] = (T)0;
                        if (k < cn) xj[u] = LDXG(x + jj[u]);
                    }
                    if (fp64) {
                        double *swv = reinterpret_cast<double *>(&ts);
                        double *sxj = swv + kChunk;
#pragma unroll
                        for (int u = 0; u < kU; u++) {
                            const int k = rt + u * kRowThreads;
                            if (k < cn) {
                                swv[k] = (double)ww[u];
                                sxj[k] = (double)xj[u];
                            }
                        }
                    } else {
                        float *sp = reinterpret_cast<float *>(&ts);
#pragma unroll
                        for (int u = 0; u < kU; u++) {
                            const int k = rt + u * kRowThreads;
                            if (k < cn) sp[k] = (float)ww[u] * ((float)s_x[s_row[k]] - (float)xj[u]);
                        }
                    }
                    bar_rows(kRowThreads);
                    for (int r = rt; r < nr; r += kRowThreads) {
                        const int lo = max(s_rp[r], c0), hi = min(s_rp[r + 1], c0 + cn);
                        T ac = s_acc[r];
                        if (fp64) {
                            const double *swv = reinterpret_cast<const double *>(&ts);
                            const double *sxj = swv + kChunk;
                            for (int q = lo; q < hi; q++) ac = fma((double)swv[q - c0], (double)sxj[q - c0], (double)ac);
                        } else {
                            const float *sp = reinterpret_cast<const float *>(&ts);
                            for (int q = lo; q < hi; q++) ac += (T)sp[q - c0];
                        }
                        s_acc[r] = ac;
                    }
                    bar_rows(kRowThreads);
                }
                for (int r = rt; r < nr; r += kRowThreads) {
                    const T xi = s_x[r];
                    T yv;
                    if (fp64) yv = (T)((fma(a.gd[t0 + r], (double)xi, (double)s_acc[r]) - (double)gm) * (double)sig);
                    else yv = (g * (xi - m) - s_acc[r]) * sig;
                    y[t0 + r] = yv;
                    acc.add(yv, xi);
                }
                bar_rows(kRowThreads);
            }
            Part p = warp_sum_part(acc.get());
            if (lane == 0) s_pw[warp] = p;
        }
        __syncthreads();
        if (warp == 0) {
            Part q = (lane >= 1 && lane < (int)(blockDim.x >> 5)) ? s_pw[lane] : part_zero();
            q = warp_sum_part(q);
            if (lane == 0) {
                ff *dst = a.partials + ((size_t)((s + 1) & 1) * gridDim.x + blockIdx.x) * 3;
                dst[0] = q.A;
                dst[1] = q.B;
                dst[2] = q.C;
            }
        }
        if (!grid_sync(gs)) return;
        s++;
    }
    // ---------------------------------------------------------- result
    if (warp == 0) {
        if (exit_kind == 2 && !no_sweeps) {
            // the last sweep s ended the loop by count: reduce it now
            Part q = part_zero();
            const ff *base = a.partials + (size_t)(s & 1) * gridDim.x * 3;
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                const ff *src = base + (size_t)b * 3;
                Part t;
                t.A = ff_make(LDX(&src[0].hi), LDX(&src[0].lo));
                t.B = ff_make(LDX(&src[1].hi), LDX(&src[1].lo));
                t.C = ff_make(LDX(&src[2].hi), LDX(&src[2].lo));
                q = part_add(q, t);
            }
            q = warp_sum_part(q);
            ctrl_step(a, s, q, c, nullptr, true, fp64);
        }
        if (blockIdx.x == 0 && lane == 0) {
            const int rs = c.res_sweep;
            const int rb = c.zero ? (rs - 1) % 3 : rs % 3;
            write_result(a, c, rb, (rs + 2) % 3);
        }
    }
}

// ================================================================== slice kernel
// Large levels with a sweep layout (rows renumbered by decreasing degree;
// heavy rows in CSR form, the rest in 32-row slices with interleaved entries):
// cooperative persistent kernel with the control warp of k_power_tiled.  A
// row warp takes a chunk of a heavy row (32 lanes over its octets) or a slice
// (one lane per row; entry k of the slice's rows is one coalesced load), so
// the loads of a sweep do not wait on one another and no CTA barrier is
// needed inside a sweep.  The iterates are stored in layout order.
//
// STAGE: one 1024-thread CTA per SM; at the top of each sweep the row warps
// copy the iterate's first stage_n entries (the highest-degree rows, which
// take the largest share of the gathers) into shared memory and gather from
// there.  A gather of 32 scattered words from L1 or L2 costs about one cycle
// per distinct line; from shared memory it costs the bank conflicts, a few
// cycles per 32 words.
template <typename T, typename IDX, bool CHUNKS, bool STREAM, bool STAGE>
__global__ void __launch_bounds__(STAGE ? kStageThreads : kTileThreads, STAGE ? 1 : 2)
    k_power_sell(PiArgs a, GridSync *gs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const s_x = reinterpret_cast<T *>(smem_raw);
    __shared__ Part s_pw[kStageThreads / 32];
    __shared__ Slot s_slot[2];
    const int n = a.n;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    T *const ring0 = (T *)a.buf[0], *const ring1 = (T *)a.buf[1], *const ring2 = (T *)a.buf[2];
    const bool fp64 = sizeof(T) == 8;
    const T g = (T)a.g;
    const float inv_gf = 1.0f / (float)a.g;
    const double inv_gd = 1.0 / a.g;
    const int h = a.lay_h, nsl = a.lay_nsl;
    const int *__restrict__ M = a.lay_meta;
    const int *__restrict__ SO = M + h;
    const IDX *__restrict__ C = reinterpret_cast<const IDX *>(a.lay_col);
    const T *__restrict__ W = reinterpret_cast<const T *>(a.lay_w);
    // work of this CTA: a contiguous range of slices holding about 1/gridDim
    // of the slice entries (the slices are sorted by width, so equal slice
    // counts would not balance); heavy rows go round robin over all warps
    __shared__ int s_range[2];
    if (threadIdx.x < 2) {
        const long long tot = (long long)SO[nsl] - SO[0];
        const long long target = SO[0] + tot * (blockIdx.x + threadIdx.x) / gridDim.x;
        int lo = 0, hi = nsl;   // first slice starting at or after the target
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (SO[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        s_range[threadIdx.x] = (blockIdx.x + threadIdx.x == gridDim.x) ? nsl : lo;
    }
    __syncthreads();
    const int sb = s_range[0], se = s_range[1];
    const int r0 = (int)((long long)n * blockIdx.x / gridDim.x);
    const int r1 = (int)((long long)n * (blockIdx.x + 1) / gridDim.x);

    // ---------------------------------------------------------- start phase
    {
        const void *cb = nullptr;
        double cmu = 0.0, cinv = 0.0;
        if (a.start == 1) {
            cb = a.cbuf[a.cres->buf];
            cmu = a.cres->mu;
            cinv = a.cres->inv_s;
        }
        Part acc = part_zero();
        for (int p = r0 + tid; p < r1; p += blockDim.x) {
            const int old = a.perm[p];
            const T xt = (T)start_value(a, old, cb, cmu, cinv);
            ring0[p] = xt;
            if (fp64) {
                double d = 0.0;
                for (int e = __ldg(a.rp + old), e1 = __ldg(a.rp + old + 1); e < e1; e++) d += __ldg(a.w + e);
                a.gd[p] = a.g - d;
            }
            const ff v = fp64 ? ff_from_double((double)xt) : ff_make((float)xt, 0.f);
            acc.A = ff_add(acc.A, v);
            acc.B = ff_add(acc.B, ff_mul(v, v));
        }
        Part p = warp_sum_part(acc);
        if (lane == 0) s_pw[warp] = p;
        __syncthreads();
        if (warp == 0) {
            Part q = (lane < (int)(blockDim.x >> 5)) ? s_pw[lane] : part_zero();
            q = warp_sum_part(q);
            if (lane == 0) {
                ff *dst = a.partials + (size_t)blockIdx.x * 3;
                dst[0] = q.A;
                dst[1] = q.B;
                dst[2] = q.C;
            }
        }
    }
    if (!grid_sync(gs)) return;
    Ctl c;
    if (warp == 0) {
        Part q = part_zero();
        for (int b = lane; b < (int)gridDim.x; b += 32) {
            const ff *src = a.partials + (size_t)b * 3;
            Part t;
            t.A = ff_make(LDX(&src[0].hi), LDX(&src[0].lo));
            t.B = ff_make(LDX(&src[1].hi), LDX(&src[1].lo));
            t.C = ff_zero();
            q = part_add(q, t);
        }
        q = warp_sum_part(q);
        const double mu0 = to_d(q.A) / (double)n;
        double ss0 = to_d(q.B) - (double)n * mu0 * mu0;
        if (ss0 < 0.0) ss0 = 0.0;
        const int e0 = start_exponent(ss0);
        ctl_init(c, a, mu0, ss0, e0);
        if (lane == 0) {
            s_slot[1] = slot_make(ff_from_double(mu0), e0, a.g, fp64);
            s_slot[0] = slot_make(ff_zero(), 0, a.g, fp64);
        }
    }
    __syncthreads();

    const bool no_sweeps = (a.mode == 1 && a.k_fixed <= 0);
    int s = 0;
    int exit_kind = no_sweeps ? 2 : 0;
    const int rw = warp - 1, nrw = (int)(blockDim.x >> 5) - 1;            // row warps of this CTA
    // heavy-row chunks are dealt CTA by CTA (chunk k to CTA k mod grid), so
    // a level with few chunks still spreads them over all SMs
    const int gw = rw * (int)gridDim.x + blockIdx.x, ngw = (int)gridDim.x * nrw;
    while (!no_sweeps) {
        const Slot sl = s_slot[(s + 1) & 1];
        if (sl.stop) {
            exit_kind = 1;
            break;
        }
        if ((a.mode == 1 && s >= a.k_fixed) || (a.mode == 0 && s >= a.max_sweeps)) {
            exit_kind = 2;
            break;
        }
        const T *x = pick3<T *>(ring0, ring1, ring2, s % 3);
        T *y = pick3<T *>(ring0, ring1, ring2, (s + 1) % 3);
        if (warp == 0) {
            if (s >= 1) {
                Part q = part_zero();
                const ff *base = a.partials + (size_t)(s & 1) * gridDim.x * 3;
                for (int b = lane; b < (int)gridDim.x; b += 32) {
                    const ff *src = base + (size_t)b * 3;
                    Part t;
                    t.A = ff_make(LDX(&src[0].hi), LDX(&src[0].lo));
                    t.B = ff_make(LDX(&src[1].hi), LDX(&src[1].lo));
                    t.C = ff_make(LDX(&src[2].hi), LDX(&src[2].lo));
                    q = part_add(q, t);
                }
                q = warp_sum_part(q);
                Slot nx;
                ctrl_step(a, s, q, c, &nx, false, fp64);
                if (lane == 0) s_slot[s & 1] = nx;
            }
        } else {
            const T m = fp64 ? (T)sl.m_d : (T)sl.m.hi;
            const T sig = fp64 ? (T)sl.sig_d : (T)scale2f(inv_gf, sl.e);
            const T gm = fp64 ? (T)sl.gm_d : g * m;
            Acc<T> acc;
            acc.reset();
            auto finish = [&](int i, T xi, T ac) {
                T yv;
                if (fp64) yv = (T)((fma(a.gd[i], (double)xi, (double)ac) - (double)gm) * (double)sig);
                else yv = (g * (xi - m) - ac) * sig;
                y[i] = yv;
                acc.add(yv, xi);
            };
            const int S = STAGE ? a.stage_n : 0;
            if (STAGE) {
                // 16-byte copies of x[0, S) into shared memory, then the row
                // warps meet (the control warp does not take part)
                const int nrt = (int)blockDim.x - 32;
                const int nv = ((reinterpret_cast<uintptr_t>(x) & 15) == 0) ? (int)(((long long)S * sizeof(T)) / 16) : 0;
                const float4 *src = reinterpret_cast<const float4 *>(x);
                float4 *dst = reinterpret_cast<float4 *>(s_x);
                for (int k = tid - 32; k < nv; k += nrt) dst[k] = __ldcg(src + k);
                for (int k = nv * (16 / (int)sizeof(T)) + tid - 32; k < S; k += nrt) s_x[k] = __ldcg(x + k);
                bar_rows(nrt);
            }
            auto ldx = [&](int c) { return (STAGE && c < S) ? s_x[c] : LDXG(x + c); };
            // heavy rows: a row of len entries (a multiple of 8) is cut into
            // nc = ceil(len / kHeavyChunk) chunks of equal length rounded up
            // to whole octets, a warp per chunk, lanes taking octets; the
            // warp of a row's last chunk waits for the row's other chunks,
            // sums the chunk partials in chunk order and completes the row
            const bool vec = ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(W)) & 15) == 0;
            for (int cidx = gw; CHUNKS && cidx < a.nchunks; cidx += ngw) {
                const int r = a.crow[cidx], c0 = a.hchunk[r], nc = a.hchunk[r + 1] - c0;
                const int len = M[r + 1] - M[r];
                const int per = (((len + nc - 1) / nc) + 7) & ~7;
                const int f0 = min(M[r + 1], M[r] + (cidx - c0) * per);
                const int f1 = min(M[r + 1], f0 + per);
                const T xi = ldx(r);
                T ac = vec ? row_sum_octets<T, IDX, sizeof(T) == 4 ? kOct32 : 1>(C, W, (f0 >> 3) + lane, f1 >> 3, xi, ldx,
                                                                        STREAM)
                           : row_sum_grouped<T, IDX>(C, W, f0 + lane, f1, 32, xi, ldx, STREAM);
                ac = warp_sum(ac);
                if (nc == 1) {
                    if (lane == 0) finish(r, xi, ac);
                } else if (lane == 0) {
                    // the warp of the row's last chunk completes the row (a
                    // fixed thread, so the sweep's partial sums group the
                    // same way in every run); the others publish their partial
                    T *cp = reinterpret_cast<T *>(a.cpart);
                    unsigned int *cnt = reinterpret_cast<unsigned int *>(a.hcount + r);
                    if (cidx < c0 + nc - 1) {
                        cp[cidx] = ac;
                        red_add_release_gpu(cnt, 1u);
                    } else {
                        // the other chunks have lower indices: their warps
                        // never wait on this one, so the wait ends; bounded
                        // all the same (GridSync::err, like a barrier)
                        const unsigned int want = (unsigned int)((s + 1) * (nc - 1));
                        unsigned long long t0 = 0;
                        for (unsigned int spin = 0; ld_acquire_gpu(cnt) < want; spin++) {
                            if ((spin & 255u) == 255u) {
                                const unsigned long long t = global_ns();
                                if (t0 == 0) {
                                    t0 = t;
                                } else if (t - t0 > kBarrierTimeoutNs || ld_relaxed_gpu(&gs->err)) {
                                    atomicExch(&gs->err, 1u);
                                    break;
                                }
                            }
                        }
                        T tot = (T)0;
                        for (int c = c0; c < c0 + nc - 1; c++) tot += __ldcg(cp + c);
                        finish(r, xi, tot + ac);
                    }
                }
                __syncwarp();
            }
            // slices: a lane per row, entries in groups of 8 (row_sum_grouped)
            for (int q = sb + rw; q < se; q += nrw) {
                const int i = h + 32 * q + lane;
                const int so = SO[q] + lane, wd = (SO[q + 1] - SO[q]) >> 5;
                const T xi = (i < n) ? ldx(i) : (T)0;
                const T ac = row_sum_grouped<T, IDX>(C, W, so, so + 32 * wd, 32, xi, ldx, STREAM);
                if (i < n) finish(i, xi, ac);
            }
            Part p = warp_sum_part(acc.get());
            if (lane == 0) s_pw[warp] = p;
        }
        __syncthreads();
        if (warp == 0) {
            Part q = (lane >= 1 && lane < (int)(blockDim.x >> 5)) ? s_pw[lane] : part_zero();
            q = warp_sum_part(q);
            if (lane == 0) {
                ff *dst = a.partials + ((size_t)((s + 1) & 1) * gridDim.x + blockIdx.x) * 3;
                dst[0] = q.A;
                dst[1] = q.B;
                dst[2] = q.C;
            }
        }
        if (!grid_sync(gs)) return;
        s++;
    }
    // ---------------------------------------------------------- result
    if (warp == 0) {
        if (exit_kind == 2 && !no_sweeps) {
            Part q = part_zero();
            const ff *base = a.partials + (size_t)(s & 1) * gridDim.x * 3;
            for (int b = lane; b < (int)gridDim.x; b += 32) {
                const ff *src = base + (size_t)b * 3;
                Part t;
                t.A = ff_make(LDX(&src[0].hi), LDX(&src[0].lo));
                t.B = ff_make(LDX(&src[1].hi), LDX(&src[1].lo));
                t.C = ff_make(LDX(&src[2].hi), LDX(&src[2].lo));
                q = part_add(q, t);
            }
            q = warp_sum_part(q);
            ctrl_step(a, s, q, c, nullptr, true, fp64);
        }
        if (blockIdx.x == 0 && lane == 0) {
            const int rs = c.res_sweep;
            const int rb = c.zero ? (rs - 1) % 3 : rs % 3;
            write_result(a, c, rb, (rs + 2) % 3);
        }
    }
}

// ================================================================== two-phase kernel
// Sweeps of a level with a two-phase layout (XLayout, internal.h): one
// 1024-thread CTA per SM (grid = the layout's P), warp 0 the control warp,
// warps 1..31 the row warps.  Per pass: phase 1 (source blocks staged in
// shared memory, xbuf written in list order), a grid barrier, phase 2 (the
// CTA's dest blocks: terms added into 64-bit fixed-point row accumulators in
// shared memory, then the rows completed).  The two xbufs alternate between
// passes, so phase 1 of pass t+1 follows phase 2 of pass t without a
// barrier: the buffer it overwrites was last read in pass t-1, which every
// CTA finished before the barrier of pass t.
//
// Fixed point: a sweep's terms are w x_c (FP64 form) or w (x_r - x_c) (FP32
// form), so every partial sum of a row is at most g max|x| in magnitude (g
// is twice the largest weighted degree).  With sc = 61 - e, g max|x| < 2^e,
// the terms scaled by 2^sc and rounded to integers sum in int64 without
// overflow; integer addition is associative, so the sum does not depend on
// the order of the shared-memory atomics.  max|x| of the sweep's iterate is
// the exact maximum of the previous sweep's per-CTA maxima.
constexpr int kXRows = kStageThreads / 32 - 1;   // row warps

// round(v 2^sc) for a double, by integer arithmetic (round half away from
// zero; values below 2^-sc / 2 and subnormals give 0): the FP64 pipe is
// left to the product that forms v
__device__ __forceinline__ long long fix64(double v, int sc) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int ef = (int)((b >> 52) & 0x7ffu);
    if (ef == 0) return 0;
    const long long mant = (long long)((b & 0xfffffffffffffull) | 0x10000000000000ull);
    const int sh = ef - 1075 + sc;   // v 2^sc = mant 2^sh; sh <= 8 by the choice of sc
    long long r;
    if (sh >= 0) r = mant << min(sh, 10);
    else if (sh > -64) r = (mant + (1ll << (-sh - 1))) >> (-sh);
    else r = 0;
    return (b >> 63) ? -r : r;
}

__device__ __forceinline__ long long fix_term(float v, int sc, float scf) { return __float2ll_rn(v * scf); }
__device__ __forceinline__ long long fix_term(double v, int sc, float) { return fix64(v, sc); }

__device__ __forceinline__ int fix_scale(double g, double xmax) {
    if (!(xmax > 0.0)) return 0;
    int ex;
    frexp(g * xmax, &ex);   // g xmax < 2^ex
    return max(-120, min(120, 61 - ex));
}

template <typename T>
__global__ void __launch_bounds__(kStageThreads, 1) k_power_2p(PiArgs a, GridSync *gs) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sm = reinterpret_cast<T *>(smem_raw);
    __shared__ Part s_pw[kStageThreads / 32];
    __shared__ double s_mx[kStageThreads / 32];
    __shared__ Slot s_slot[2];
    __shared__ int s_sc;
    __shared__ Ctl s_ctl;   // the control warp's state (kept out of every thread's registers)
    const int n = a.n;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int rt = tid - 32, nrt = (int)blockDim.x - 32, rw = warp - 1;   // row threads and warps
    T *const ring0 = (T *)a.buf[0], *const ring1 = (T *)a.buf[1], *const ring2 = (T *)a.buf[2];
    const bool fp64 = sizeof(T) == 8;
    const T g = (T)a.g;
    const float inv_gf = 1.0f / (float)a.g;
    const int P = (int)gridDim.x, b = (int)blockIdx.x;
    const int r0 = (int)((long long)n * b / P), r1 = (int)((long long)n * (b + 1) / P);
    const T *__restrict__ XW = reinterpret_cast<const T *>(a.x_w);
    auto cta_max = [&](double v, double *dst) {   // max over the CTA into *dst (thread 0 writes)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) s_mx[warp] = v;
        __syncthreads();
        if (warp == 0) {
            double u = lane < (int)(blockDim.x >> 5) ? s_mx[lane] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) u = fmax(u, __shfl_xor_sync(0xffffffffu, u, o));
            if (lane == 0) *dst = u;
        }
    };
    auto grid_max = [&](const double *src) {      // warp 0: max of the P per-CTA values
        double u = 0.0;
        for (int k = lane; k < P; k += 32) u = fmax(u, __ldcg(src + k));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) u = fmax(u, __shfl_xor_sync(0xffffffffu, u, o));
        return u;
    };

    // ---------------------------------------------------------- start phase
    {
        const void *cb = nullptr;
        double cmu = 0.0, cinv = 0.0;
        if (a.start == 1) {
            cb = a.cbuf[a.cres->buf];
            cmu = a.cres->mu;
            cinv = a.cres->inv_s;
        }
        Part acc = part_zero();
        double mx = 0.0;
        for (int p = r0 + tid; p < r1; p += blockDim.x) {
            const int old = a.perm[p];
            const T xt = (T)start_value(a, old, cb, cmu, cinv);
            ring0[p] = xt;
            mx = fmax(mx, fabs((double)xt));
            if (fp64) {
                double d = 0.0;
                for (int e = __ldg(a.rp + old), e1 = __ldg(a.rp + old + 1); e < e1; e++) d += __ldg(a.w + e);
                a.gd[p] = a.g - d;
            }
            const ff v = fp64 ? ff_from_double((double)xt) : ff_make((float)xt, 0.f);
            acc.A = ff_add(acc.A, v);
            acc.B = ff_add(acc.B, ff_mul(v, v));
        }
        Part p = warp_sum_part(acc);
        if (lane == 0) s_pw[warp] = p;
        cta_max(mx, a.x_pmax + b);   // its __syncthreads also publishes s_pw
        if (warp == 0) {
            Part q = (lane < (int)(blockDim.x >> 5)) ? s_pw[lane] : part_zero();
            q = warp_sum_part(q);
            if (lane == 0) {
                ff *dst = a.partials + (size_t)blockIdx.x * 3;
                dst[0] = q.A;
                dst[1] = q.B;
                dst[2] = q.C;
            }
        }
    }
    if (!grid_sync(gs)) return;
    if (warp == 0) {
        Ctl c;
        Part q = part_zero();
        for (int k = lane; k < P; k += 32) {
            const ff *src = a.partials + (size_t)k * 3;
            Part t;
            t.A = ff_make(LDX(&src[0].hi), LDX(&src[0].lo));
            t.B = ff_make(LDX(&src[1].hi), LDX(&src[1].lo));
            t.C = ff_zero();
            q = part_add(q, t);
        }
        q = warp_sum_part(q);
        const double xmax = grid_max(a.x_pmax);
        const double mu0 = to_d(q.A) / (double)n;
        double ss0 = to_d(q.B) - (double)n * mu0 * mu0;
        if (ss0 < 0.0) ss0 = 0.0;
        const int e0 = start_exponent(ss0);
        ctl_init(c, a, mu0, ss0, e0);
        if (lane == 0) {
            s_ctl = c;
            s_slot[1] = slot_make(ff_from_double(mu0), e0, a.g, fp64);
            s_slot[0] = slot_make(ff_zero(), 0, a.g, fp64);
            s_sc = fix_scale(a.g, xmax);
        }
    }
    __syncthreads();

    const bool no_sweeps = (a.mode == 1 && a.k_fixed <= 0);
    int s = 0;
    int exit_kind = no_sweeps ? 2 : 0;
    while (!no_sweeps) {
        const Slot sl = s_slot[(s + 1) & 1];
        if (sl.stop) {
            exit_kind = 1;
            break;
        }
        if ((a.mode == 1 && s >= a.k_fixed) || (a.mode == 0 && s >= a.max_sweeps)) {
            exit_kind = 2;
            break;
        }
        const T *x = pick3<T *>(ring0, ring1, ring2, s % 3);
        T *y = pick3<T *>(ring0, ring1, ring2, (s + 1) % 3);
        if (warp == 0 && s >= 1) {
            // decisions of sweep s-1 and the fixed-point scale of sweep s,
            // overlapped with phase 1 of pass 0 (published by its barrier)
            Part q = part_zero();
            const ff *base = a.partials + (size_t)(s & 1) * P * 3;
            for (int k = lane; k < P; k += 32) {
                const ff *src = base + (size_t)k * 3;
                Part t;
                t.A = ff_make(LDX(&src[0].hi), LDX(&src[0].lo));
                t.B = ff_make(LDX(&src[1].hi), LDX(&src[1].lo));
                t.C = ff_make(LDX(&src[2].hi), LDX(&src[2].lo));
                q = part_add(q, t);
            }
            q = warp_sum_part(q);
            Slot nx;
            Ctl c = s_ctl;
            ctrl_step(a, s, q, c, &nx, false, fp64);
            const double xmax = grid_max(a.x_pmax + (size_t)(s & 1) * P);
            __syncwarp();
            if (lane == 0) {
                s_ctl = c;
                s_slot[s & 1] = nx;
                s_sc = fix_scale(a.g, xmax);
            }
        }
        const T m = fp64 ? (T)sl.m_d : (T)sl.m.hi;
        const T sig = fp64 ? (T)sl.sig_d : (T)scale2f(inv_gf, sl.e);
        const T gm = fp64 ? (T)sl.gm_d : g * m;
        Acc<T> acc;
        acc.reset();
        T ymax = (T)0;
        auto finish = [&](int i, T xi, T ac) {
            T yv;
            if (fp64) yv = (T)((fma(a.gd[i], (double)xi, (double)ac) - (double)gm) * (double)sig);
            else yv = (g * (xi - m) - ac) * sig;
            y[i] = yv;
            acc.add(yv, xi);
            ymax = max(ymax, abs(yv));
        };
        for (int t = 0; t < a.x_T; t++) {
            // xbuf holds pass t's list positions from ps0 & ~7 on, so that 8
            // list entries at a multiple of 8 sit at a multiple of 8 there
            T *const xb = reinterpret_cast<T *>(a.x_buf[t & 1]);
            const int ps0 = __ldg(a.x_ps + t), xsh = ps0 & 7, xb0 = ps0 - xsh;
            X2T(s, t, 0);
            if (warp > 0) {
                // ------------------------------------------------ phase 1
                // this CTA's share of the pass's stream, source block by
                // source block; entry j goes to its list position, found
                // from its 32-entry chunk's cell and cell-start bits
                const long long Et = (long long)__ldg(a.x_ps + t + 1) - ps0;
                int e = (int)(Et * b / P);
                const int e1 = (int)(Et * (b + 1) / P);
                const int *qo = a.x_qoff + (size_t)t * (a.x_Q + 1);
                const uint2 *chk = a.x_chk + __ldg(a.x_choff + t);
                const uint16_t *srcp = a.x_src + __ldg(a.x_sal + t);
                int lo = 0, hi = a.x_Q - 1;   // last block q with qo[q] <= e
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (__ldg(qo + mid) <= e) lo = mid;
                    else hi = mid - 1;
                }
                for (int q = lo; e < e1; q++) {
                    const int qe = min(e1, __ldg(qo + q + 1));
                    if (qe > e) {
                        const int base = q * a.x_SB, cnt = min(a.x_SB, n - base);
                        const T *xs = x + base;
                        // 16-byte asynchronous copies (L2 only: x was written
                        // by other CTAs before the last barrier), then the tail
                        const int nv16 = ((reinterpret_cast<uintptr_t>(xs) & 15) == 0) ? (int)((cnt * sizeof(T)) / 16) : 0;
                        for (int k = rt; k < nv16; k += nrt) {
                            const unsigned dsm = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char *>(sm) + 16 * (size_t)k);
                            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dsm),
                                         "l"(reinterpret_cast<const char *>(xs) + 16 * (size_t)k)
                                         : "memory");
                        }
                        asm volatile("cp.async.wait_all;" ::: "memory");
                        for (int k = nv16 * (int)(16 / sizeof(T)) + rt; k < cnt; k += nrt) sm[k] = __ldcg(xs + k);
                        bar_rows(nrt);
                        // 8 consecutive stream entries per row thread (one
                        // vector load of their source offsets); an entry's
                        // cell comes from its 32-entry chunk's bits
                        for (int gi = (e >> 3) + rt; 8 * gi < qe; gi += nrt) {
                            const int j0 = 8 * gi;
                            const uint4 sv = __ldcs(reinterpret_cast<const uint4 *>(srcp + j0));
                            const uint2 ci = __ldg(chk + (j0 >> 5));
                            const unsigned sw[4] = {sv.x, sv.y, sv.z, sv.w};
                            int lastc = -1, dl = 0;
#pragma unroll
                            for (int u = 0; u < 8; u++) {
                                const int j = j0 + u;
                                if (j < e || j >= qe) continue;
                                const int cell = (int)ci.x + __popc(ci.y & ((2u << (j & 31)) - 1u));
                                if (cell != lastc) {
                                    dl = __ldg(a.x_cdel + cell);
                                    lastc = cell;
                                }
                                xb[j + xsh + dl] = sm[(sw[u >> 1] >> (16 * (u & 1))) & 0xffffu];
                            }
                        }
                        bar_rows(nrt);
                    }
                    e = qe;
                }
            }
            X2T(s, t, 2);
            if (!grid_sync(gs)) return;
            X2T(s, t, 3);
            if (warp > 0) {
                // ------------------------------------------------ phase 2
                const int sc = s_sc;
                const float scf = ldexpf(1.0f, sc);
                long long *const accs = reinterpret_cast<long long *>(smem_raw);
                T *const xv = reinterpret_cast<T *>(accs + a.x_VMAX);
                const int g0 = __ldg(a.x_ndb + t), g1 = __ldg(a.x_ndb + t + 1);
                for (int gb = g0 + b; gb < g1; gb += P) {
                    const int R0 = __ldg(a.x_dbr + gb), R1 = __ldg(a.x_dbr + gb + 1);
                    const int L0 = __ldg(a.x_dbl + gb), L1 = __ldg(a.x_dbl + gb + 1);
                    for (int p = R0 + rt; p < R1; p += nrt) {
                        xv[p - R0] = __ldcg(x + p);
                        accs[p - R0] = 0;
                    }
                    bar_rows(nrt);
                    // 8 consecutive list entries per lane (vector loads from
                    // a multiple of 8); a run of one row's entries is summed
                    // in a register and added to its accumulator once
                    for (int pb = (L0 & ~7) + 256 * rw; pb < L1; pb += 256 * kXRows) {
                        const int base = pb + 8 * lane;
                        if (base + 8 <= L0 || base >= L1) continue;
                        const uint4 dv = __ldcs(reinterpret_cast<const uint4 *>(a.x_dst + base));
                        const unsigned dw[4] = {dv.x, dv.y, dv.z, dv.w};
                        T wv[8], xvv[8];
                        if (fp64) {
#pragma unroll
                            for (int h = 0; h < 4; h++) {
                                const double2 w2 = __ldcs(reinterpret_cast<const double2 *>(XW + base) + h);
                                const double2 x2 = __ldcg(reinterpret_cast<const double2 *>(xb + (base - xb0)) + h);
                                wv[2 * h] = (T)w2.x;
                                wv[2 * h + 1] = (T)w2.y;
                                xvv[2 * h] = (T)x2.x;
                                xvv[2 * h + 1] = (T)x2.y;
                            }
                        } else {
#pragma unroll
                            for (int h = 0; h < 2; h++) {
                                const float4 w4 = __ldcs(reinterpret_cast<const float4 *>(XW + base) + h);
                                const float4 x4 = __ldcg(reinterpret_cast<const float4 *>(xb + (base - xb0)) + h);
                                wv[4 * h] = (T)w4.x;
                                wv[4 * h + 1] = (T)w4.y;
                                wv[4 * h + 2] = (T)w4.z;
                                wv[4 * h + 3] = (T)w4.w;
                                xvv[4 * h] = (T)x4.x;
                                xvv[4 * h + 1] = (T)x4.y;
                                xvv[4 * h + 2] = (T)x4.z;
                                xvv[4 * h + 3] = (T)x4.w;
                            }
                        }
                        int rd = -1;
                        long long ra = 0;
#pragma unroll
                        for (int k = 0; k < 8; k++) {
                            const int pos = base + k;
                            if (pos < L0 || pos >= L1) continue;
                            const int d = (int)((dw[k >> 1] >> (16 * (k & 1))) & 0xffffu);
                            const T v = fp64 ? wv[k] * xvv[k] : wv[k] * (xv[d] - xvv[k]);
                            const long long iv = fix_term(v, sc, scf);
                            if (d != rd) {
                                if (rd >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(accs + rd), (unsigned long long)ra);
                                rd = d;
                                ra = iv;
                            } else {
                                ra += iv;
                            }
                        }
                        if (rd >= 0) atomicAdd(reinterpret_cast<unsigned long long *>(accs + rd), (unsigned long long)ra);
                    }
                    bar_rows(nrt);
                    X2T(s, t, 5);
                    for (int p = R0 + rt; p < R1; p += nrt) {
                        T ac;
                        if (fp64) ac = (T)((double)accs[p - R0] * ldexp(1.0, -sc));
                        else ac = (T)(__ll2float_rn(accs[p - R0]) * ldexpf(1.0f, -sc));
                        finish(p, xv[p - R0], ac);
                    }
                    bar_rows(nrt);
                }
                X2T(s, t, 6);
            }
        }
        if (warp > 0) {
            Part p = warp_sum_part(acc.get());
            if (lane == 0) s_pw[warp] = p;
        }
        cta_max((double)ymax, a.x_pmax + (size_t)((s + 1) & 1) * P + b);   // its __syncthreads publishes s_pw
        if (warp == 0) {
            Part q = (lane >= 1 && lane < (int)(blockDim.x >> 5)) ? s_pw[lane] : part_zero();
            q = warp_sum_part(q);
            if (lane == 0) {
                ff *dst = a.partials + ((size_t)((s + 1) & 1) * P + blockIdx.x) * 3;
                dst[0] = q.A;
                dst[1] = q.B;
                dst[2] = q.C;
            }
        }
        if (!grid_sync(gs)) return;
        s++;
    }
    // ---------------------------------------------------------- result
    if (warp == 0) {
        Ctl c = s_ctl;
        if (exit_kind == 2 && !no_sweeps) {
            Part q = part_zero();
            const ff *base = a.partials + (size_t)(s & 1) * P * 3;
            for (int k = lane; k < P; k += 32) {
                const ff *src = base + (size_t)k * 3;
                Part t;
                t.A = ff_make(LDX(&src[0].hi), LDX(&src[0].lo));
                t.B = ff_make(LDX(&src[1].hi), LDX(&src[1].lo));
                t.C = ff_make(LDX(&src[2].hi), LDX(&src[2].lo));
                q = part_add(q, t);
            }
            q = warp_sum_part(q);
            ctrl_step(a, s, q, c, nullptr, true, fp64);
        }
        if (blockIdx.x == 0 && lane == 0) {
            const int rs = c.res_sweep;
            const int rb = c.zero ? (rs - 1) % 3 : rs % 3;
            write_result(a, c, rb, (rs + 2) % 3);
        }
    }
}

// ================================================================== small kernel
// Shared memory: ring[3][n] T, gd[n] (FP64 form), w[E] T, rp[n+1] int,
// col[E] int, slice offsets[n/32 + 2] int.  E = nnz (CSR) or the SELL-32
// size (one lane per row: each 32-row slice stores entry k of its rows
// contiguously, rows padded to the slice's longest with zero weights, so the
// lanes of a warp read consecutive words -- no bank conflicts).
// ================================================================== slot order
// The one-CTA and cluster kernels hold a level's rows in "slot" order: rows by
// decreasing degree, ties by row number, so that the 32 rows of a SELL-32
// slice have about the same length and the slices carry little padding (a
// padded entry costs an FP64 FMA like a stored one).  The iterate, g - d_i
// and the columns are renumbered to slots; rows are mapped back on output.
// The order is taken when it shrinks the SELL-32 size by at least 1/16 and
// every row holds fewer than n entries; otherwise slots are rows.  Sorted
// order never needs more entries than row order: in any order, at least k+1
// slices hold a row at least as long as the sorted row at position 32k, so
// the k-th widest slice is at least as wide as the sorted order's k-th slice,
// and a buffer sized for row order holds either.
__host__ __device__ __forceinline__ bool slot_order_pays(long long natural, long long sorted) {
    return sorted * 16 <= natural * 15;
}

// perm[p] = row of slot p and inv[i] = slot of row i (n ints each, shared
// memory); hist: n ints of shared scratch.  A stable counting sort: bucket
// maxdeg - d_i, bucket starts by one warp's scan, rows placed by one warp in
// row order (rows of equal degree keep their order).  Every thread of the CTA
// calls it; the CTA is synchronised on return.
__device__ __noinline__ void slot_order(int n, const int *rp, int *perm, int *inv, int *hist) {
    __shared__ int s_maxd, s_sorted;
    __shared__ unsigned long long s_nat;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31;
    if (tid == 0) {
        s_maxd = 0;
        s_sorted = 0;
        s_nat = 0;
    }
    __syncthreads();
    int md = 0;
    unsigned long long nat = 0;
    for (int i = tid; i < n; i += nt) md = max(md, rp[i + 1] - rp[i]);
    for (int q = tid; q < (n + 31) / 32; q += nt) {
        int L = 0;
        for (int r = 32 * q; r < min(n, 32 * q + 32); r++) L = max(L, rp[r + 1] - rp[r]);
        nat += 32ull * (unsigned long long)L;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        md = max(md, __shfl_xor_sync(0xffffffffu, md, o));
        nat += __shfl_xor_sync(0xffffffffu, nat, o);
    }
    if (lane == 0) {
        atomicMax(&s_maxd, md);
        atomicAdd(&s_nat, nat);
    }
    __syncthreads();
    const int D = s_maxd;
    if (D < n) {
        for (int b = tid; b <= D; b += nt) hist[b] = 0;
        __syncthreads();
        for (int i = tid; i < n; i += nt) {
            const int b = D - (rp[i + 1] - rp[i]);
            inv[i] = b;   // the row's bucket, read back by the placing warp
            atomicAdd(&hist[b], 1);
        }
        __syncthreads();
        if (tid < 32) {
            // bucket starts (exclusive scan) and the SELL-32 size in slot
            // order: a slice is as wide as the degree of its first slot
            int carry = 0;
            unsigned long long tot = 0;
            for (int b0 = 0; b0 <= D; b0 += 32) {
                const int b = b0 + lane;
                const int c = (b <= D) ? hist[b] : 0;
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                const int st = carry + incl - c;
                if (b <= D) {
                    hist[b] = st;
                    const int starts = (st + c + 31) / 32 - (st + 31) / 32;
                    tot += 32ull * (unsigned long long)(D - b) * (unsigned long long)starts;
                }
                carry += __shfl_sync(0xffffffffu, incl, 31);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
            if (lane == 0) s_sorted = slot_order_pays((long long)s_nat, (long long)tot) ? 1 : 0;
        }
        __syncthreads();
    }
    if (s_sorted) {
        if (tid < 32) {
            for (int i0 = 0; i0 < n; i0 += 32) {
                const int i = i0 + lane;
                const unsigned act = __ballot_sync(0xffffffffu, i < n);
                if (i < n) {
                    const int b = inv[i];
                    const unsigned peers = __match_any_sync(act, b);
                    const int r = __popc(peers & ((1u << lane) - 1u));
                    const int base = hist[b];
                    perm[base + r] = i;
                    __syncwarp(act);
                    if (r == 0) hist[b] = base + __popc(peers);
                }
                __syncwarp();
            }
        }
    } else {
        for (int p = tid; p < n; p += nt) perm[p] = p;
    }
    __syncthreads();
    for (int p = tid; p < n; p += nt) inv[perm[p]] = p;
    __syncthreads();
}

// Prefix sums pre[0..nsl] of the SELL-32 slice sizes in the order slot_order
// takes, from the host copy of the row pointers (the same arithmetic; the
// sorted widths come from the degree counts: slice q of the sorted rows is as
// wide as the degree at sorted position 32q).
static void slot_sell_prefix(int n, const int *rph, std::vector<int> &pre) {
    const int nsl = (n + 31) / 32;
    std::vector<int> wid(nsl, 0);
    int D = 0;
    long long nat = 0;
    for (int q = 0; q < nsl; q++) {
        for (int r = 32 * q; r < std::min(n, 32 * q + 32); r++) wid[q] = std::max(wid[q], rph[r + 1] - rph[r]);
        nat += 32ll * wid[q];
        D = std::max(D, wid[q]);
    }
    if (D < n) {
        std::vector<int> cnt((size_t)D + 1, 0), sw(nsl, 0);
        for (int i = 0; i < n; i++) cnt[rph[i + 1] - rph[i]]++;
        long long tot = 0;
        int pos = 0;   // sorted position of the first row of degree d
        for (int d = D; d >= 0; d--) {
            for (int q = (pos + 31) / 32; 32 * q < pos + cnt[d]; q++) {
                sw[q] = d;
                tot += 32ll * d;
            }
            pos += cnt[d];
        }
        if (slot_order_pays(nat, tot)) wid.swap(sw);
    }
    pre.assign(nsl + 1, 0);
    for (int q = 0; q < nsl; q++) pre[q + 1] = pre[q] + 32 * wid[q];
}

template <typename T>
constexpr size_t small_smem_bytes(long long n, long long e) {
    return (size_t)(sizeof(T) * (3 * n + e) + (sizeof(T) == 8 ? 8 * n : 0) + 4 * (n + 1) + 4 * e +
                    4 * (n / 32 + 2) + 4 * n + 64);
}

template <typename T, int G>
__global__ void __launch_bounds__(kSmallMaxThreads) k_power_small(PiArgs a, GridSync *) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n;
    const int m = a.rp[n];
    const bool sell = (G == 1) && a.sell_nnz > 0;
    const int E = sell ? (int)a.sell_nnz : m;
    const bool fp64 = sizeof(T) == 8;
    T *ring0 = reinterpret_cast<T *>(smem_raw);
    double *s_gd = reinterpret_cast<double *>(ring0 + 3 * n);
    T *s_w = fp64 ? reinterpret_cast<T *>(s_gd + n) : ring0 + 3 * n;
    int *s_rp = reinterpret_cast<int *>(s_w + E);
    int *s_col = s_rp + n + 1;
    int *s_soff = s_col + E;
    // SELL-32 form: the row of each slot (the iterate, g - d_i and the
    // columns are held by slot)
    int *s_perm = s_soff + (n / 32 + 2);
    // FP64 form: every row thread's stop sums (A, B, C as doubles), by sweep
    // parity; the control warp reduces them (one float-float conversion per
    // control lane, instead of one per row thread: conversions issue on the
    // FP64 pipe)
    double *s_dacc = reinterpret_cast<double *>(
        (reinterpret_cast<uintptr_t>(s_perm + n) + 7) & ~(uintptr_t)7);
    __shared__ Part s_pw[2][32];
    __shared__ Slot s_slot[2];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nw = blockDim.x >> 5;
    // the control warp's sums of the row warps' partials of parity `par`, in
    // a fixed order (rows warps in order per lane, then the lanes' xor tree)
    auto ctl_part = [&](int par) -> Part {
        if constexpr (sizeof(T) == 8) {
            double A = 0.0, B = 0.0, C = 0.0;
            for (int w = 1; w < nw; w++) {
                const double *src = s_dacc + ((size_t)par * blockDim.x + 32 * w + lane) * 3;
                A += src[0];
                B += src[1];
                C += src[2];
            }
            Part p;
            p.A = ff_from_double(A);
            p.B = ff_from_double(B);
            p.C = ff_from_double(C);
            return warp_sum_part(p);
        } else {
            const Part q = (lane >= 1 && lane < nw) ? s_pw[par][lane] : part_zero();
            return warp_sum_part(q, 1, pow2_at_least(nw));
        }
    };
    const T *__restrict__ wv = wsel<T>(a);
    const T g = (T)a.g;
    const float inv_gf = 1.0f / (float)a.g;
    const double inv_gd = 1.0 / a.g;

    for (int i = tid; i <= n; i += blockDim.x) s_rp[i] = a.rp[i];
    const int nsl = (n + 31) / 32;
    if (sell) {
        __syncthreads();
        // slot order; inv and the sort's scratch borrow ring slots 1 and 2
        // (n values each), which the first sweep overwrites
        int *s_inv = reinterpret_cast<int *>(ring0 + n);
        slot_order(n, s_rp, s_perm, s_inv, reinterpret_cast<int *>(ring0 + 2 * (size_t)n));
        for (int q = tid; q < nsl; q += blockDim.x) {
            int L = 0;
            for (int p = 32 * q; p < min(n, 32 * q + 32); p++) {
                const int r = s_perm[p];
                L = max(L, s_rp[r + 1] - s_rp[r]);
            }
            s_soff[q + 1] = 32 * L;
        }
        __syncthreads();
        if (tid == 0) {
            s_soff[0] = 0;
            for (int q = 0; q < nsl; q++) s_soff[q + 1] += s_soff[q];
        }
        __syncthreads();
        for (int p = tid; p < 32 * nsl; p += blockDim.x) {
            const int q = p >> 5, l = p & 31;
            const int L = (s_soff[q + 1] - s_soff[q]) >> 5;
            const int r = (p < n) ? s_perm[p] : 0;
            const int e0 = (p < n) ? s_rp[r] : 0;
            const int len = (p < n) ? s_rp[r + 1] - e0 : 0;
            for (int k = 0; k < L; k++) {
                const int idx = s_soff[q] + 32 * k + l;
                if (k < len) {
                    s_col[idx] = s_inv[a.col[e0 + k]];
                    s_w[idx] = wv[e0 + k];
                } else {
                    s_col[idx] = (p < n) ? p : 0;   // zero weight: no contribution
                    s_w[idx] = (T)0;
                }
            }
        }
        __syncthreads();
    } else {
        for (int e = tid; e < m; e += blockDim.x) {
            s_col[e] = a.col[e];
            s_w[e] = wv[e];
        }
    }
    {
        const void *cb = nullptr;
        double cmu = 0.0, cinv = 0.0;
        if (a.start == 1) {
            cb = a.cbuf[a.cres->buf];
            cmu = a.cres->mu;
            cinv = a.cres->inv_s;
        }
        Part acc = part_zero();
        for (int i = tid; i < n; i += blockDim.x) {
            const int r = sell ? s_perm[i] : i;
            const T xt = (T)start_value(a, r, cb, cmu, cinv);
            ring0[i] = xt;
            if (fp64) {
                double d = 0.0;
                for (int e = a.rp[r], e1 = a.rp[r + 1]; e < e1; e++) d += a.w[e];
                s_gd[i] = a.g - d;
            }
            const ff v = fp64 ? ff_from_double((double)xt) : ff_make((float)xt, 0.f);
            acc.A = ff_add(acc.A, v);
            acc.B = ff_add(acc.B, ff_mul(v, v));
        }
        Part p = warp_sum_part(acc);
        if (lane == 0) s_pw[0][warp] = p;
    }
    __syncthreads();
    Ctl c;
    if (warp == 0) {
        Part q = (lane < nw) ? s_pw[0][lane] : part_zero();
        q = warp_sum_part(q);
        const double mu0 = to_d(q.A) / (double)n;
        double ss0 = to_d(q.B) - (double)n * mu0 * mu0;
        if (ss0 < 0.0) ss0 = 0.0;
        const int e0 = start_exponent(ss0);
        ctl_init(c, a, mu0, ss0, e0);
        if (lane == 0) {
            s_slot[1] = slot_make(ff_from_double(mu0), e0, a.g, fp64);
            s_slot[0] = slot_make(ff_zero(), 0, a.g, fp64);
        }
    }
    __syncthreads();

    const bool no_sweeps = (a.mode == 1 && a.k_fixed <= 0);
    int s = 0;
    int exit_kind = no_sweeps ? 2 : 0;
    const int rt = tid - 32, nrt = blockDim.x - 32;
    const int rlane = rt & (G - 1);
    const int groups = nrt / G;
    while (!no_sweeps) {
        const Slot sl = s_slot[(s + 1) & 1];
        if (sl.stop) {
            exit_kind = 1;
            break;
        }
        if ((a.mode == 1 && s >= a.k_fixed) || (a.mode == 0 && s >= a.max_sweeps)) {
            exit_kind = 2;
            break;
        }
        const T *x = ring0 + (size_t)(s % 3) * n;
        T *y = ring0 + (size_t)((s + 1) % 3) * n;
        if (warp == 0) {
            if (lane == 0) TRACE(s, 0);
            if (s >= 1) {
                const Part q = ctl_part(s & 1);
                Slot nx;
                ctrl_step(a, s, q, c, &nx, false, fp64);
                if (lane == 0) s_slot[s & 1] = nx;
            }
            if (lane == 0) TRACE(s, 1);
        } else {
            if (lane == 0 && warp == 1) TRACE(s, 4);
            const T mT = fp64 ? (T)sl.m_d : (T)sl.m.hi;
            const T sig = fp64 ? (T)sl.sig_d : (T)scale2f(inv_gf, sl.e);
            const T gm = fp64 ? (T)sl.gm_d : g * mT;
            Acc<T> acc;
            acc.reset();
            for (int base = rt / G;; base += groups) {
                if (__shfl_sync(0xffffffffu, base, 0) >= n) break;
                const int i = base;
                T ac = (T)0, xi = (T)0;
                if (sell) {
                    // one lane per row, 32 rows per warp = one slice; padded
                    // entries have zero weight
                    const int q = base >> 5;
                    const int off = s_soff[q] + (base & 31);
                    const int L = (s_soff[q + 1] - s_soff[q]) >> 5;
                    xi = (i < n) ? x[i] : (T)0;
                    T a0 = (T)0, a1 = (T)0;
                    int k = 0;
                    for (; k + 1 < L; k += 2) {
                        const int c0 = s_col[off + 32 * k], c1 = s_col[off + 32 * k + 32];
                        const T w0 = s_w[off + 32 * k], w1 = s_w[off + 32 * k + 32];
                        const T x0 = x[c0], x1 = x[c1];
                        if (fp64) {
                            a0 = fma(w0, x0, a0);
                            a1 = fma(w1, x1, a1);
                        } else {
                            a0 += w0 * (xi - x0);
                            a1 += w1 * (xi - x1);
                        }
                    }
                    if (k < L) {
                        const T w0 = s_w[off + 32 * k], x0 = x[s_col[off + 32 * k]];
                        if (fp64) a0 = fma(w0, x0, a0);
                        else a0 += w0 * (xi - x0);
                    }
                    ac = a0 + a1;
                } else if (i < n) {
                    xi = x[i];
                    // four independent accumulators: the loads of four entries
                    // are in flight together
                    T a0 = (T)0, a1 = (T)0, a2 = (T)0, a3 = (T)0;
                    int e = s_rp[i] + rlane;
                    const int e1 = s_rp[i + 1];
                    for (; e + 3 * G < e1; e += 4 * G) {
                        const int c0 = s_col[e], c1 = s_col[e + G], c2 = s_col[e + 2 * G], c3 = s_col[e + 3 * G];
                        const T w0 = s_w[e], w1 = s_w[e + G], w2 = s_w[e + 2 * G], w3 = s_w[e + 3 * G];
                        const T x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
                        if (fp64) {
                            a0 = fma(w0, x0, a0);
                            a1 = fma(w1, x1, a1);
                            a2 = fma(w2, x2, a2);
                            a3 = fma(w3, x3, a3);
                        } else {
                            a0 += w0 * (xi - x0);
                            a1 += w1 * (xi - x1);
                            a2 += w2 * (xi - x2);
                            a3 += w3 * (xi - x3);
                        }
                    }
                    for (; e < e1; e += G) {
                        if (fp64) a0 = fma(s_w[e], x[s_col[e]], a0);
                        else a0 += s_w[e] * (xi - x[s_col[e]]);
                    }
                    ac = (a0 + a1) + (a2 + a3);
                }
                ac = group_sum<G>(ac);
                if (lane == 0 && warp == 1) TRACE(s, 5);
                if (i < n && rlane == 0) {
                    T yv;
                    if (fp64) yv = (T)((fma(s_gd[i], (double)xi, (double)ac) - (double)gm) * (double)sig);
                    else yv = (g * (xi - mT) - ac) * sig;
                    y[i] = yv;
                    acc.add(yv, xi);
                }
                if (lane == 0 && warp == 1) TRACE(s, 6);
            }
            // only the lanes leading a row group hold sums
            if constexpr (sizeof(T) == 8) {
                double *dst = s_dacc + ((size_t)((s + 1) & 1) * blockDim.x + tid) * 3;
                dst[0] = acc.A;
                dst[1] = acc.B;
                dst[2] = acc.C;
            } else {
                const Part p = warp_sum_part(acc.get(), G);
                if (lane == 0) s_pw[(s + 1) & 1][warp] = p;
            }
            if (lane == 0 && warp == 1) TRACE(s, 2);
            if (lane == 0 && warp == nw - 1) TRACE(s, 3);
        }
        __syncthreads();
        s++;
    }
    __shared__ int s_rb, s_rbp;
    if (warp == 0) {
        if (exit_kind == 2 && !no_sweeps) {
            const Part q = ctl_part(s & 1);
            ctrl_step(a, s, q, c, nullptr, true, fp64);
        }
        if (lane == 0) {
            const int rs = c.res_sweep;
            s_rb = c.zero ? (rs + 2) % 3 : rs % 3;
            s_rbp = (rs + 2) % 3;
            write_result(a, c, 0, 1);
        }
    }
    __syncthreads();
    // result -> buf[0], previous iterate -> buf[1]
    T *o0 = (T *)a.buf[0], *o1 = (T *)a.buf[1];
    const T *rr = ring0 + (size_t)s_rb * n, *rp = ring0 + (size_t)s_rbp * n;
    for (int i = tid; i < n; i += blockDim.x) {
        const int r = sell ? s_perm[i] : i;
        o0[r] = rr[i];
        o1[r] = rp[i];
    }
}

// ================================================================== cluster kernel
// FP64 sweeps of a level spread over one thread-block cluster of C CTAs
// (2..8, one per SM).  Every CTA holds the whole iterate ring (3 x n rows
// rounded up to whole slices) and g - d_i of every row, and the SELL-32
// slices of its share of the rows (rows in slot order, slices split into C
// ranges of about equal SELL size).  A sweep: the row warps compute their rows from the
// local iterate (each warp's stop sums summed over its lanes as float-
// float); then all threads copy the CTA's row block, in 16-byte pieces, into
// every other CTA's ring (distributed shared memory) while the control warp
// sums the warps' stop sums and stores the total into every CTA's slot
// [sweep parity][rank]; then the cluster meets at its barrier.  Every
// CTA's control warp sums the C slots in rank order and takes the same
// decisions, so all CTAs run the same sweeps and reach the same barriers.
// A CTA is at most one sweep ahead of another (one barrier per sweep), so
// two slot parities and the ring of three keep stores and reads apart.
constexpr int kClusterMax = 8;

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ unsigned cluster_ctas() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
// every thread of every CTA of the cluster; orders the distributed
// shared-memory stores before it with the reads after it
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ unsigned cluster_addr(const void *local, unsigned cta) {
    const unsigned la = (unsigned)__cvta_generic_to_shared(local);
    unsigned ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(la), "r"(cta));
    return ra;
}
__device__ __forceinline__ void st_cluster_f32(float *local, unsigned cta, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(cluster_addr(local, cta)), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster_v2f64(double2 *local, unsigned cta, double2 v) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(cluster_addr(local, cta)), "d"(v.x), "d"(v.y)
                 : "memory");
}

// First slice of each of C ranges of about equal SELL-32 size, from the
// prefix sums pre[0..nsl] of the slices' sizes (the host plans with the same
// arithmetic).
__host__ __device__ __forceinline__ int cluster_split(const int *pre, int nsl, int C, int r) {
    if (r <= 0) return 0;
    if (r >= C) return nsl;
    const long long target = (long long)pre[nsl] * r / C;
    int lo = 0, hi = nsl;   // first q with pre[q] >= target
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((long long)pre[mid] < target) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(kSmallMaxThreads) k_power_cluster(PiArgs a, GridSync *) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.n, nsl = (n + 31) / 32, nr = 32 * nsl;   // ring slots hold whole slices
    const int C = (int)cluster_ctas();
    const unsigned rank = cluster_rank();
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nw = blockDim.x >> 5, nrw = nw - 1, rw = warp - 1;
    double *ring0 = reinterpret_cast<double *>(smem_raw);      // [3][nr]
    double *s_gd = ring0 + 3 * (size_t)nr;                      // [nr]
    Part *s_cpart = reinterpret_cast<Part *>(s_gd + nr);        // [2][kClusterMax]: CTAs' stop sums
    double *s_w = reinterpret_cast<double *>(s_cpart + 2 * kClusterMax);   // [emax]
    int *s_col = reinterpret_cast<int *>(s_w + a.cl_emax);
    int *s_pre = s_col + a.cl_emax;                             // [nsl + 1]
    int *s_perm = s_pre + nsl + 1;                              // [n]: row of each slot
    __shared__ Part s_pw[32];
    __shared__ Slot s_slot[2];
    __shared__ int s_q[2];
    const double g = a.g;

    // ---- slot order (the same in every CTA); inv and the sort's scratch
    // borrow ring slots 1 and 2, cleared below
    const int *s_inv = reinterpret_cast<const int *>(ring0 + nr);
    slot_order(n, a.rp, s_perm, reinterpret_cast<int *>(ring0 + nr), reinterpret_cast<int *>(ring0 + 2 * (size_t)nr));
    // ---- the slices' SELL-32 sizes, this CTA's range and its entries
    for (int q = tid; q < nsl; q += blockDim.x) {
        int L = 0;
        for (int p = 32 * q; p < min(n, 32 * q + 32); p++) {
            const int r = s_perm[p];
            L = max(L, a.rp[r + 1] - a.rp[r]);
        }
        s_pre[q + 1] = 32 * L;
    }
    __syncthreads();
    if (tid == 0) {
        s_pre[0] = 0;
        for (int q = 0; q < nsl; q++) s_pre[q + 1] += s_pre[q];
        s_q[0] = cluster_split(s_pre, nsl, C, (int)rank);
        s_q[1] = cluster_split(s_pre, nsl, C, (int)rank + 1);
    }
    __syncthreads();
    const int q0 = s_q[0], q1 = s_q[1], e_base = s_pre[q0];
    for (int p = 32 * q0 + tid; p < 32 * q1; p += blockDim.x) {
        const int q = p >> 5, l = p & 31;
        const int L = (s_pre[q + 1] - s_pre[q]) >> 5;
        const int r = (p < n) ? s_perm[p] : 0;
        const int e0 = (p < n) ? a.rp[r] : 0;
        const int len = (p < n) ? a.rp[r + 1] - e0 : 0;
        for (int k = 0; k < L; k++) {
            const int idx = s_pre[q] - e_base + 32 * k + l;
            if (k < len) {
                s_col[idx] = s_inv[a.col[e0 + k]];
                s_w[idx] = a.w[e0 + k];
            } else {
                s_col[idx] = (p < n) ? p : 0;   // zero weight: no contribution
                s_w[idx] = 0.0;
            }
        }
    }
    __syncthreads();   // inv read before ring slots 1 and 2 are cleared
    // ---- start vector and g - d_i of every slot (the same in every CTA)
    {
        const void *cb = nullptr;
        double cmu = 0.0, cinv = 0.0;
        if (a.start == 1) {
            cb = a.cbuf[a.cres->buf];
            cmu = a.cres->mu;
            cinv = a.cres->inv_s;
        }
        Part acc = part_zero();
        for (int i = tid; i < nr; i += blockDim.x) {
            double xt = 0.0, gd = 0.0;
            if (i < n) {
                const int r = s_perm[i];
                xt = start_value(a, r, cb, cmu, cinv);
                double d = 0.0;
                for (int e = a.rp[r], e1 = a.rp[r + 1]; e < e1; e++) d += a.w[e];
                gd = g - d;
                const ff v = ff_from_double(xt);
                acc.A = ff_add(acc.A, v);
                acc.B = ff_add(acc.B, ff_mul(v, v));
            }
            ring0[i] = xt;
            ring0[nr + i] = 0.0;
            ring0[2 * (size_t)nr + i] = 0.0;
            s_gd[i] = gd;
        }
        Part p = warp_sum_part(acc);
        if (lane == 0) s_pw[warp] = p;
    }
    __syncthreads();
    Ctl c;
    if (warp == 0) {
        Part q = (lane < nw) ? s_pw[lane] : part_zero();
        q = warp_sum_part(q);
        const double mu0 = to_d(q.A) / (double)n;
        double ss0 = to_d(q.B) - (double)n * mu0 * mu0;
        if (ss0 < 0.0) ss0 = 0.0;
        const int e0 = start_exponent(ss0);
        ctl_init(c, a, mu0, ss0, e0);
        if (lane == 0) {
            s_slot[1] = slot_make(ff_from_double(mu0), e0, a.g, true);
            s_slot[0] = slot_make(ff_zero(), 0, a.g, true);
        }
    }
    __syncthreads();
    // every CTA's shared memory is set up before any CTA stores into it
    cluster_barrier();

    // the C CTAs' stop sums of parity par, in rank order (every lane)
    auto cluster_part = [&](int par) -> Part {
        Part q = part_zero();
        for (int r = 0; r < C; r++) q = part_add(q, s_cpart[par * kClusterMax + r]);
        return q;
    };
    // this CTA's row block, in 16-byte pieces, into every other CTA's ring
    const int rb0 = 32 * q0, rb_pairs = 16 * (q1 - q0);

    const bool no_sweeps = (a.mode == 1 && a.k_fixed <= 0);
    int s = 0;
    int exit_kind = no_sweeps ? 2 : 0;
    while (!no_sweeps) {
        const Slot sl = s_slot[(s + 1) & 1];
        if (sl.stop) {
            exit_kind = 1;
            break;
        }
        if ((a.mode == 1 && s >= a.k_fixed) || (a.mode == 0 && s >= a.max_sweeps)) {
            exit_kind = 2;
            break;
        }
        const double *x = ring0 + (size_t)(s % 3) * nr;
        double *y = ring0 + (size_t)((s + 1) % 3) * nr;
        CLT(s, 0);
        if (warp == 0) {
            if (s >= 1) {
                const Part q = cluster_part((s - 1) & 1);
                Slot nx;
                ctrl_step(a, s, q, c, &nx, false, true);
                if (lane == 0) s_slot[s & 1] = nx;
            }
        } else {
            const double mT = sl.m_d, sig = sl.sig_d, gm = sl.gm_d;
            Acc<double> acc;
            acc.reset();
            for (int q = q0 + rw; q < q1; q += nrw) {
                const int i = 32 * q + lane;
                const int off = s_pre[q] - e_base + lane;
                const int L = (s_pre[q + 1] - s_pre[q]) >> 5;
                const double xi = x[i];
                double a0 = 0.0, a1 = 0.0;
                int k = 0;
                for (; k + 1 < L; k += 2) {
                    a0 = fma(s_w[off + 32 * k], x[s_col[off + 32 * k]], a0);
                    a1 = fma(s_w[off + 32 * k + 32], x[s_col[off + 32 * k + 32]], a1);
                }
                if (k < L) a0 = fma(s_w[off + 32 * k], x[s_col[off + 32 * k]], a0);
                if (i < n) {
                    const double yv = (fma(s_gd[i], xi, a0 + a1) - gm) * sig;
                    y[i] = yv;
                    acc.add(yv, xi);
                }
            }
            // the warp's stop sums as float-float, summed over its lanes
            const Part p = warp_sum_part(acc.get());
            if (lane == 0) s_pw[warp] = p;
        }
        __syncthreads();
        CLT(s, 1);
        if (warp == 0) {
            // this CTA's stop sums (row warps in order) into every CTA's slot
            Part q = (lane >= 1 && lane < nw) ? s_pw[lane] : part_zero();
            q = warp_sum_part(q);
            if (lane < C) {
                Part *slot = s_cpart + (s & 1) * kClusterMax + rank;
                if (lane == (int)rank) {
                    *slot = q;
                } else {
                    const float *src = reinterpret_cast<const float *>(&q);
                    float *dst = reinterpret_cast<float *>(slot);
                    for (int k = 0; k < 6; k++) st_cluster_f32(dst + k, (unsigned)lane, src[k]);
                }
            }
        }
        for (int k = tid; k < (C - 1) * rb_pairs; k += blockDim.x) {
            const int pr = k / rb_pairs, j = k - pr * rb_pairs;
            const unsigned peer = (unsigned)(pr < (int)rank ? pr : pr + 1);
            const double2 v = reinterpret_cast<const double2 *>(y + rb0)[j];
            st_cluster_v2f64(reinterpret_cast<double2 *>(y + rb0) + j, peer, v);
        }
        CLT(s, 2);
        cluster_barrier();
        CLT(s, 3);
        s++;
    }
    __shared__ int s_rb, s_rbp;
    if (warp == 0) {
        if (exit_kind == 2 && !no_sweeps) {
            const Part q = cluster_part((s - 1) & 1);
            ctrl_step(a, s, q, c, nullptr, true, true);
        }
        if (lane == 0) {
            const int rs = c.res_sweep;
            s_rb = c.zero ? (rs + 2) % 3 : rs % 3;
            s_rbp = (rs + 2) % 3;
            if (rank == 0) write_result(a, c, 0, 1);
        }
    }
    __syncthreads();
    if (rank == 0) {
        // result -> buf[0], previous iterate -> buf[1]
        double *o0 = (double *)a.buf[0], *o1 = (double *)a.buf[1];
        const double *rr = ring0 + (size_t)s_rb * nr, *rp = ring0 + (size_t)s_rbp * nr;
        for (int i = tid; i < n; i += blockDim.x) {
            o0[s_perm[i]] = rr[i];
            o1[s_perm[i]] = rp[i];
        }
    }
}

static size_t cluster_smem(int n, int, int emax) {
    const int nsl = (n + 31) / 32, nr = 32 * nsl;
    return 8 * (4 * (size_t)nr + (size_t)emax) + sizeof(Part) * 2 * kClusterMax +
           4 * ((size_t)emax + nsl + 1 + (size_t)n) + 16;
}

// Shared memory a cluster CTA may take (0: unknown).
static long long cluster_room() {
    DeviceInfo d;
    if (device_info(&d) != CMG_OK) return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, (const void *)k_power_cluster) != cudaSuccess) return 0;
    return (long long)d.max_smem_optin - (long long)fa.sharedSizeBytes - 1024;
}

bool cluster_may_hold(int n) {
    return n >= 128 && n <= 65536 && (long long)cluster_smem(n, 0, 0) <= cluster_room();
}

void cluster_plan(PiLevel *lv, const int *rph) {
    lv->cl_ctas = 0;
    const int n = lv->n;
    if (!cluster_may_hold(n)) return;
    const long long room = cluster_room();
    const int nsl = (n + 31) / 32;
    std::vector<int> pre;
    slot_sell_prefix(n, rph, pre);
    // about 96 rows per CTA: enough FP64 work per SM to repay the barrier
    for (int C = std::max(2, std::min(kClusterMax, (n + 95) / 96)); C <= kClusterMax; C++) {
        int emax = 0, smax = 0;
        for (int r = 0; r < C; r++) {
            const int a0 = cluster_split(pre.data(), nsl, C, r), a1 = cluster_split(pre.data(), nsl, C, r + 1);
            emax = std::max(emax, pre[a1] - pre[a0]);
            smax = std::max(smax, a1 - a0);
        }
        const int threads = 32 * (1 + std::max(1, std::min(31, smax)));
        const size_t smem = cluster_smem(n, threads, emax);
        if ((long long)smem > room) continue;
        if (allow_max_dynamic_smem((const void *)k_power_cluster) != CMG_OK) return;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)C;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, (const void *)k_power_cluster, &cfg) != cudaSuccess || ncl < 1) {
            cudaGetLastError();
            return;
        }
        lv->cl_ctas = C;
        lv->cl_threads = threads;
        lv->cl_emax = emax;
        lv->cl_smem = smem;
        return;
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
    const size_t ts = fp32 ? sizeof(TileSmem<float>) : sizeof(TileSmem<double>);
    return ts + e * 2 * kTileRows + sizeof(int) * (kTileRows + 4) + 2 * kChunk;
}

template <typename T, typename IDX, bool STAGE>
static const void *sell_kernel_tis(bool chunks, bool stream) {
    if (chunks)
        return stream ? (const void *)k_power_sell<T, IDX, true, true, STAGE>
                      : (const void *)k_power_sell<T, IDX, true, false, STAGE>;
    return stream ? (const void *)k_power_sell<T, IDX, false, true, STAGE>
                  : (const void *)k_power_sell<T, IDX, false, false, STAGE>;
}

template <typename T, typename IDX>
static const void *sell_kernel_ti(bool chunks, bool stream, bool stage) {
    return stage ? sell_kernel_tis<T, IDX, true>(chunks, stream) : sell_kernel_tis<T, IDX, false>(chunks, stream);
}

static const void *sell_kernel(int fp32, int col16, bool chunks, bool stream, bool stage) {
    if (fp32)
        return col16 ? sell_kernel_ti<float, uint16_t>(chunks, stream, stage)
                     : sell_kernel_ti<float, int>(chunks, stream, stage);
    return col16 ? sell_kernel_ti<double, uint16_t>(chunks, stream, stage)
                 : sell_kernel_ti<double, int>(chunks, stream, stage);
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

// Lanes per row in the small kernel: about 4 entries per lane, fewer lanes
// when that leaves more row groups than rows would need.
static int small_lanes(int n, long long nnz, int fp32) {
    const double avg = (double)nnz / (double)std::max(1, n);
    int g = 1;
    if (fp32) {
        // a row per lane while a lane's (unrolled) entry loop stays short:
        // every lane that holds a row pays its share of the per-sweep
        // float-float reduction
        while (g < 32 && g * 32 < avg) g <<= 1;
    } else {
        // FP64: every lane-operation costs FP64 issue slots, so use the fewest
        // lanes that keep each lane's dependent FMA chain short
        while (g < 32 && g * 16 < avg) g <<= 1;
    }
    return g;
}

// Threads of the small kernel: the control warp plus enough row warps for
// one row per lane group (at most 31 row warps).
static int small_threads(int n, int G) {
    long long lanes = (long long)n * G;
    int w = (int)std::min<long long>(31, std::max<long long>(1, (lanes + 31) / 32));
    return 32 * (w + 1);
}

// Entries the small kernel stores: the SELL-32 size with one lane per row
// (when known), else the CSR size.
static long long small_entries(const PiLevel &lv, int G) {
    return (G == 1 && lv.sell_nnz > 0) ? lv.sell_nnz : lv.nnz;
}

static size_t small_bytes(const PiLevel &lv, int G, int fp32) {
    const long long e = small_entries(lv, G);
    if (fp32) return small_smem_bytes<float>(lv.n, e);
    // plus the row threads' FP64 stop sums: 2 parities x 3 doubles per thread
    return small_smem_bytes<double>(lv.n, e) + 8 + 48 * (size_t)small_threads(lv.n, G);
}

size_t xsweep_smem(int fp32) {
    DeviceInfo d;
    if (device_info(&d) != CMG_OK) return 0;
    cudaFuncAttributes fa;
    const void *k = fp32 ? (const void *)k_power_2p<float> : (const void *)k_power_2p<double>;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return 0;
    const long long room = (long long)d.max_smem_optin - (long long)fa.sharedSizeBytes - 256;
    // 192 KB: a 48K-vertex FP32 (24K FP64) source block, 24K (12K) vrows
    const long long want = 192ll << 10;
    if (room < (64ll << 10)) return 0;
    return (size_t)(std::min(room, want) & ~255ll);
}

int stage_capacity(int fp32) {
    DeviceInfo d;
    if (device_info(&d) != CMG_OK) return 0;
    cudaFuncAttributes fa;
    const void *k = fp32 ? (const void *)k_power_sell<float, int, true, true, true>
                         : (const void *)k_power_sell<double, int, true, true, true>;
    if (cudaFuncGetAttributes(&fa, k) != cudaSuccess) return 0;
    const long long room = (long long)d.max_smem_optin - (long long)fa.sharedSizeBytes - 256;
    if (room <= 0) return 0;
    const long long cap = room / (fp32 ? (long long)sizeof(float) : (long long)sizeof(double));
    return (int)(cap & ~3ll);
}

// Lanes per row with which the small kernel holds the level (0: it cannot).
static int small_config(const PiLevel &lv, int fp32) {
    DeviceInfo d;
    if (device_info(&d) != CMG_OK) return 0;
    const int G = small_lanes(lv.n, lv.nnz, fp32);
    return small_bytes(lv, G, fp32) + 4096 <= (size_t)d.max_smem_optin ? G : 0;
}

bool small_level_fits(const PiLevel &lv, int fp32) { return small_config(lv, fp32) > 0; }

__global__ void k_sell_size(int n_static, const int *__restrict__ n_dev, const int *__restrict__ rp,
                            unsigned long long *out) {
    const int n = n_dev ? *n_dev : n_static;
    const int nsl = (n + 31) / 32;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nsl; q += gridDim.x * blockDim.x) {
        int L = 0;
        for (int r = 32 * q; r < min(n, 32 * q + 32); r++) L = max(L, rp[r + 1] - rp[r]);
        atomicAdd(out, (unsigned long long)(32 * L));
    }
}

cmg_status_t sell_size(int n, const int *rp, unsigned long long *dev_counter, long long *out,
                       cudaStream_t s) {
    CMG_CUDA(cudaMemsetAsync(dev_counter, 0, sizeof(unsigned long long), s));
    k_sell_size<<<grid_for((n + 31) / 32, 256), 256, 0, s>>>(n, nullptr, rp, dev_counter);
    CMG_TRY(launch_status());
    unsigned long long v = 0;
    CMG_CUDA(cudaMemcpyAsync(&v, dev_counter, sizeof(v), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    *out = (long long)v;
    return CMG_OK;
}

cmg_status_t sell_size_async(const int *n_dev, int n_cap, const int *rp,
                             unsigned long long *dev_counter, cudaStream_t s) {
    CMG_CUDA(cudaMemsetAsync(dev_counter, 0, sizeof(unsigned long long), s));
    k_sell_size<<<grid_for((n_cap + 31) / 32, 256), 256, 0, s>>>(n_cap, n_dev, rp, dev_counter);
    return launch_status();
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
    for (int k = 0; k < 3; k++) {
        a.cbuf[k] = run.coarse_bufs[k];
        a.cfp64 = run.coarse_fp64;
        a.buf[k] = run.bufs[k];
    }
    a.cres = run.coarse_res;
    a.agg = run.coarse_agg;
    a.x_init = run.x_init;
    a.gd = run.gd;
    a.res = run.res;
    a.partials = nullptr;
    a.zero_tol2 = run.fp32 ? kZeroTol2_32 : kZeroTol2_64;
    a.sell_nnz = lv.sell_nnz;
    a.cinvp = run.coarse_inv;
    a.perm = nullptr;
    a.lay_h = a.lay_nsl = 0;
    a.lay_meta = nullptr;
    a.lay_col = a.lay_w = nullptr;
    a.hchunk = nullptr;
    a.crow = nullptr;
    a.hcount = nullptr;
    a.cpart = nullptr;
    a.nchunks = 0;
    a.stream_hint = 0;
    a.stage_n = 0;
    void *args[] = {&a, &gs};
    if (lv.cl_ctas > 0 && !run.fp32 && !lv.lay) {
        // FP64 sweeps in one thread-block cluster
        a.cl_emax = lv.cl_emax;
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = (unsigned)lv.cl_ctas;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3((unsigned)lv.cl_ctas);
        cfg.blockDim = dim3((unsigned)lv.cl_threads);
        cfg.dynamicSmemBytes = lv.cl_smem;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        CMG_TRY(allow_max_dynamic_smem((const void *)k_power_cluster));
        CMG_CUDA(cudaLaunchKernelExC(&cfg, (const void *)k_power_cluster, args));
        return launch_status();
    }
    if (small_level_fits(lv, run.fp32)) {
        const int G = small_config(lv, run.fp32);
        const void *kern = run.fp32 ? small_kernel<float>(G) : small_kernel<double>(G);
        const size_t smem = small_bytes(lv, G, run.fp32);
        CMG_TRY(allow_max_dynamic_smem(kern));
        return coop_launch(kern, 1, small_threads(lv.n, G), smem, s, args, gs);
    }
    if (!run.fp32 && !run.gd) return CMG_ERR_INVALID_ARG;
    if (lv.xl && lv.lay) {
        // two-phase kernel: one 1024-thread CTA per SM, the layout's P CTAs
        const XLayout &X = *lv.xl;
        a.perm = reinterpret_cast<const int *>(lv.lay->perm);
        a.x_T = X.T;
        a.x_Q = X.Q;
        a.x_SB = X.SB;
        a.x_VMAX = X.VMAX;
        a.x_src = X.src;
        a.x_dst = X.dst;
        a.x_w = X.w;
        a.x_ps = X.pass_s;
        a.x_sal = X.sal;
        a.x_qoff = X.qoff;
        a.x_ndb = X.ndb;
        a.x_dbr = X.dbr;
        a.x_dbl = X.dbl;
        a.x_cdel = X.cdel;
        a.x_choff = X.choff;
        a.x_chk = X.chk;
        a.x_pmax = X.pmax;
        a.x_buf[0] = X.xbuf[0];
        a.x_buf[1] = X.xbuf[1];
        const void *kern = run.fp32 ? (const void *)k_power_2p<float> : (const void *)k_power_2p<double>;
        CMG_TRY(allow_max_dynamic_smem(kern));
        int maxb = 0;
        CMG_TRY(coop_max_blocks(kern, kStageThreads, X.smem, &maxb));
        if (maxb < X.P) return CMG_ERR_TOO_LARGE;
        double *partials;
        if (ws) {
            if (2 * X.P * 3 > ws->partials_cap) return CMG_ERR_TOO_LARGE;
            partials = ws->partials;
        } else {
            CMG_TRY(scr.get(&partials, (size_t)2 * X.P * 3));
        }
        a.partials = reinterpret_cast<ff *>(partials);
        return coop_launch(kern, X.P, kStageThreads, X.smem, s, args, gs);
    }
    if (lv.lay) {
        // slice kernel over the level's sweep layout (one graph)
        const SweepLayout &L = *lv.lay;
        a.perm = reinterpret_cast<const int *>(L.perm);
        a.lay_h = L.hheavy[0];
        a.lay_nsl = (lv.n - a.lay_h + 31) / 32;
        {
            // layout bytes against L2: only a stream that cannot stay in L2
            // is read evict-first
            DeviceInfo di;
            CMG_TRY(device_info(&di));
            const int l2 = di.l2_bytes;
            const long long lay_bytes = L.entries * (long long)((L.col16 ? 2 : 4) + (run.fp32 ? 4 : 8));
            a.stream_hint = (l2 > 0 && lay_bytes > (long long)l2) ? 1 : 0;
        }
        a.lay_meta = L.meta;
        a.lay_col = L.bcol;
        a.lay_w = L.bw;
        a.hchunk = L.hchunk;
        a.crow = L.crow;
        a.hcount = L.hcount;
        a.cpart = L.cpart;
        a.nchunks = L.nchunks;
        if (a.lay_h > 0) {
            if (!L.hchunk) return CMG_ERR_INVALID_ARG;
            CMG_CUDA(cudaMemsetAsync(L.hcount, 0, sizeof(int) * (size_t)a.lay_h, s));
        }
        a.stage_n = std::min(L.stage_n, lv.n);
        const bool stage = a.stage_n > 0;
        const void *kern = sell_kernel(run.fp32, L.col16, a.lay_h > 0, a.stream_hint != 0, stage);
        const int threads = stage ? kStageThreads : kTileThreads;
        const size_t smem = stage ? (size_t)a.stage_n * (run.fp32 ? sizeof(float) : sizeof(double)) : 0;
        if (stage) CMG_TRY(allow_max_dynamic_smem(kern));
        int maxb = 0;
        CMG_TRY(coop_max_blocks(kern, threads, smem, &maxb));
        const int row_warps = threads / 32 - 1;
        const long long tasks = (long long)a.lay_nsl + a.nchunks;
        const int blocks = (int)std::max<long long>(1, std::min<long long>(maxb, (tasks + row_warps - 1) / row_warps));
        double *partials;
        if (ws) {
            if (2 * blocks * 3 > ws->partials_cap) return CMG_ERR_TOO_LARGE;
            partials = ws->partials;
        } else {
            CMG_TRY(scr.get(&partials, (size_t)2 * blocks * 3));
        }
        a.partials = reinterpret_cast<ff *>(partials);
        return coop_launch(kern, blocks, threads, smem, s, args, gs);
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
    CMG_TRY(allow_max_dynamic_smem(kern));
    int maxb = 0;
    CMG_TRY(coop_max_blocks(kern, kTileThreads, smem, &maxb));
    // one tile per CTA where possible (each tile's phases are latency-bound),
    // never more CTAs than co-resident
    const int blocks = std::max(1, std::min(maxb, a.ntiles));
    // partial sums: [2][blocks][3] float-float values (6 floats = 3 doubles each)
    double *partials;
    if (ws) {
        if (2 * blocks * 3 > ws->partials_cap) return CMG_ERR_TOO_LARGE;
        partials = ws->partials;
    } else {
        CMG_TRY(scr.get(&partials, (size_t)2 * blocks * 3));
    }
    a.partials = reinterpret_cast<ff *>(partials);
    return coop_launch(kern, blocks, kTileThreads, smem, s, args, gs);
}

// Sum of K per-thread doubles over the CTA, result in out[] of every thread
// (fixed order).  sm: 32*K doubles.  Two __syncthreads.  (Used once per
// solve by the final pass.)
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
    const void *buf[3];
    const PiResult *res;
    double *u;
    double *tmp;
    double *part;      // [3][gridDim.x][4]
    double *out;       // [2]: lambda, residual
    int sign;          // apply the canonical sign
    int fresh;         // u already holds the vector (skip the vector phase)
    const int *inv;    // the iterates are in layout order: row i is at inv[i] (nullptr: natural)
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
            const float *x = (const float *)a.buf[r.buf_prev];
            p[0] = p[1] = p[2] = p[3] = 0.0;
            for (int base = r0 + threadIdx.x / G;; base += groups) {
                if (__shfl_sync(0xffffffffu, base, 0) >= r1) break;
                const int i = base;
                double acc = 0.0, xi = 0.0;
                if (i < r1) {
                    xi = ((double)x[a.inv ? a.inv[i] : i] - r.mu_prev) * r.inv_s_prev;
                    const int e1 = __ldg(a.rp + i + 1);
                    for (int e = __ldg(a.rp + i) + lane; e < e1; e += G) {
                        const int j = __ldg(a.col + e);
                        const double xj = ((double)x[a.inv ? a.inv[j] : j] - r.mu_prev) * r.inv_s_prev;
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
            const float *y = (const float *)a.buf[r.buf];
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x)
                a.u[i] = ((double)y[a.inv ? a.inv[i] : i] - r.mu) * r.inv_s;
        } else {
            const double *y = (const double *)a.buf[r.buf];
            for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x)
                a.u[i] = (y[a.inv ? a.inv[i] : i] - r.mu) * r.inv_s;
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

cmg_status_t finalize(const PiLevel &lv, int fp32, void *const bufs[3], const PiResult *res,
                      double *u, int sign, int fresh, double *out2, GridSync *gs, cudaStream_t s,
                      const PiWorkspace *ws) {
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
    for (int k = 0; k < 3; k++) a.buf[k] = bufs ? bufs[k] : nullptr;
    a.res = res;
    a.u = u;
    a.tmp = tmp;
    a.part = part;
    a.out = out2;
    a.sign = sign;
    a.fresh = fresh;
    a.inv = lv.lay ? lv.lay->inv : nullptr;
    void *args[] = {&a, &gs};
    return coop_launch(kern, blocks, kFinThreads, 0, s, args, gs);
}

}  // namespace cmg

#ifdef CMG_TRACE
extern "C" int cmg_debug_trace(long long *out) {
    return (int)cudaMemcpyFromSymbol(out, cmg::g_trace, sizeof(cmg::g_trace));
}
#endif
