// batch.cu -- the batched form: Alg. 1 of arXiv 1412.0565 for many
// independent graphs at once.
//
// Setup.  The batch is one block-diagonal union per level.  Visit ranks are
// taken per graph and offset by the graph's first union row (graph-major
// rank space), so one HEC pass over the union numbers every graph's
// aggregates contiguously and in that graph's own creator order; one
// Galerkin pass then yields the union of the coarse Laplacians, bit for bit
// the ones the single-graph setup builds.  A graph leaves the cascade where
// Alg. 1 stops it (n <= coarse_size, fewer than 2 aggregates, or the level
// cap); its block keeps shrinking in later unions but is never solved.
//
// Solve.  One persistent launch per union level: groups of `threads per
// graph` threads take graphs from an atomic queue (largest first) and run
// Alg. 3 on each graph alone -- start vector (Gaussian on the graph's
// coarsest level, else the prolongated coarse result), sweeps until
// cos >= 1 - tol (or the schedule's count), then the normalised result.  A
// group stages its graph's vectors, and its CSR when they fit, in shared
// memory, so a sweep costs one group barrier.  On level 0 the group also
// forms the final vector (FP64 recomputation of the last sweep for the FP32
// form), fixes its sign and computes the Rayleigh quotient and residual.
// The per-level launches are captured once into a CUDA graph and replayed.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "pi_common.cuh"

namespace cmg {

// ------------------------------------------------------------------ setup kernels
// First union row of every graph on the coarse level: the smallest aggregate
// id among the graph's fine rows (ids are graph-major).  coff[G] = c.
__global__ void k_batch_coff(int G, const int *__restrict__ voff, const int *__restrict__ agg,
                             const LevelCounts *__restrict__ cnt, int *__restrict__ coff) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < G; q += warps) {
        int lo = 0x7fffffff;
        for (int v = voff[q] + lane; v < voff[q + 1]; v += 32) lo = min(lo, agg[v]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        if (lane == 0) coff[q] = lo;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) coff[G] = cnt->c;
}

// Per-graph Gershgorin shift g = max_i (d_i + d_i) over the graph's rows,
// d_i summed left to right (Alg. 3, first line): the single-graph value.
__global__ void k_batch_gersh(int G, const int *__restrict__ off, const int *__restrict__ rp,
                              const double *__restrict__ w, double *__restrict__ gout) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int q = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < G; q += warps) {
        double best = 0.0;
        for (int i = off[q] + lane; i < off[q + 1]; i += 32) {
            double d = 0.0;
            for (int e = rp[i]; e < rp[i + 1]; e++) d += w[e];
            best = fmax(best, d + d);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) gout[q] = best;
    }
}

// out[q] = rp[off[q]] for q = 0..G (the graphs' first entries).
__global__ void k_gather_at(int G, const int *__restrict__ off, const int *__restrict__ rp,
                            int *__restrict__ out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q <= G; q += gridDim.x * blockDim.x)
        out[q] = rp[off[q]];
}

// Every entry of a row stays inside the row's graph.
__global__ void k_batch_check(int n, int G, const int *__restrict__ voff, const int *__restrict__ rp,
                              const int *__restrict__ col, unsigned *__restrict__ flag) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int lo = 0, hi = G - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (voff[mid] <= v) lo = mid;
            else hi = mid - 1;
        }
        const int a = voff[lo], b = voff[lo + 1];
        for (int e = rp[v]; e < rp[v + 1]; e++) {
            const int j = col[e];
            if (j < a || j >= b) {
                atomicOr(flag, 1u);
                break;
            }
        }
    }
}

// ------------------------------------------------------------------ solve kernel
constexpr int kGroupHeader = 4096;   // per-group control area in shared memory
constexpr int kOffDred = 2 * 32 * (int)sizeof(Part);
constexpr int kOffInt = kOffDred + 32 * 4 * (int)sizeof(double);
constexpr int kBatchMaxThreads = 1024;
static_assert(kOffInt + 64 <= kGroupHeader, "group header too small");


struct BatchPiArgs {
    int level;
    const int *rp;        // the level's CSR (original numbering): finalisation
    const int *col;
    const double *w;
    const int *perm;      // new union position -> original union vertex
    const int *inv;       // original union vertex -> new union position
    const int *heavy;     // [G] heavy rows per graph
    const int *eoff;      // [G] first layout entry of each graph
    const int *moff;      // [G] first meta word of each graph
    const int *meta;
    const void *bcol;     // layout columns (uint16 or int32)
    const void *bw;       // layout weights (T)
    const int *voff;      // [G+1] union offsets of the graphs on this level
    const double *gsh;    // [G]   Gershgorin shift per graph
    const int *list;      // graphs solved on this level (largest first)
    int count;
    int *queue;           // work counter (zero at launch)
    const int *J;         // [G]   coarsest level per graph
    const int *agg;       // this level -> level + 1 (union ids)
    const void *uc;       // normalised results of level + 1 (in that level's precision)
    int uc_fp64;          // uc holds doubles (else floats)
    void *uo;             // T[n_level] normalised results (level > 0)
    double *uf;           // double[n_0] final vectors (level 0)
    void *vscr;           // T[2 n_level] iterates of graphs too large for shared memory
    double *gdscr;        // double[n_level] g - d_i of those graphs (FP64 form)
    int tg;               // threads per graph
    int smem_group;       // shared bytes per group, header included
    int stage;            // copy the layout to shared memory when it fits
    int fixed;            // schedule FIXED: k_fixed sweeps below the coarsest level
    int k_fixed;
    const int *replay;    // schedule REPLAY: [G][CMG_MAX_LEVELS] sweep counts
    int force_k;          // >= 0: Gaussian start and exactly force_k sweeps (autotuner)
    int max_sweeps, max_sweeps_coarsest;
    double tol;
    uint64_t seed;
    float zero_tol2;
    int *sweeps;          // [G] results of this level
    double *cosv;
    int *flags;           // bit 0 sweep cap reached, bit 1 iterate annihilated
    double *lam, *res;    // [G] (level 0)
};

// Barrier of one group: the warp itself, or named barrier `id` of tg threads.
__device__ __forceinline__ void gbar(int id, int tg) {
    if (tg == 32) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(tg) : "memory");
}

// Group sum of the sweep sums; only lanes leading a row (lane % G == 0) may
// hold non-zero values.  Every thread of the group receives the same bits.
// Contains a group barrier.
template <int G>
__device__ __forceinline__ Part gsum_part(const Part &mine, Part *slots, int lane, int wg, int nwg,
                                          int bid, int tg) {
    Part p = warp_sum_part(mine, G);
    if (tg == 32) {
        __syncwarp();
        p.A = ff_make(__shfl_sync(0xffffffffu, p.A.hi, 0), __shfl_sync(0xffffffffu, p.A.lo, 0));
        p.B = ff_make(__shfl_sync(0xffffffffu, p.B.hi, 0), __shfl_sync(0xffffffffu, p.B.lo, 0));
        p.C = ff_make(__shfl_sync(0xffffffffu, p.C.hi, 0), __shfl_sync(0xffffffffu, p.C.lo, 0));
        return p;
    }
    if (lane == 0) slots[wg] = p;
    gbar(bid, tg);
    Part q = (lane < nwg) ? slots[lane] : part_zero();
    return warp_sum_part(q, 1, 32);
}

// Group sum of K doubles per thread (all threads receive the same bits).
template <int K>
__device__ __forceinline__ void gsum_d(double (&v)[K], double *sm, int lane, int wg, int nwg, int bid,
                                       int tg) {
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = warp_sum(v[k]);
    if (tg == 32) {
        __syncwarp();
        return;
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sm[wg * K + k] = v[k];
    gbar(bid, tg);
#pragma unroll
    for (int k = 0; k < K; k++) {
        const double t = (lane < nwg) ? sm[lane * K + k] : 0.0;
        v[k] = warp_sum(t);
    }
    gbar(bid, tg);
}

// (|v|, index) order of the sign rule: larger magnitude first, lower index on ties.
__device__ __forceinline__ bool sign_better(double v, int i, double bv, int bi) {
    return v > bv || (v == bv && i < bi);
}

template <typename T, typename IDX, int G>
__global__ void __launch_bounds__(kBatchMaxThreads, 1) k_batch_pi(BatchPiArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool fp64 = sizeof(T) == 8;
    const int tg = a.tg;
    const int grp = threadIdx.x / tg;
    const int gt = threadIdx.x - grp * tg;
    const int lane = threadIdx.x & 31;
    const int wg = gt >> 5, nwg = tg >> 5;
    const int bid = 1 + grp;
    unsigned char *gbase = smem_raw + (size_t)grp * a.smem_group;
    Part *s_part = reinterpret_cast<Part *>(gbase);
    double *s_dred = reinterpret_cast<double *>(gbase + kOffDred);
    int *s_int = reinterpret_cast<int *>(gbase + kOffInt);
    unsigned char *data = gbase + kGroupHeader;
    const long long data_bytes = (long long)a.smem_group - kGroupHeader;
    const int rg = gt / G, rl = gt & (G - 1), ngr = tg / G;
    constexpr int kRpw = 32 / G;   // heavy rows per warp pass

    for (;;) {
        // ---- next graph from the queue
        int k;
        if (tg == 32) {
            k = 0;
            if (lane == 0) k = atomicAdd(a.queue, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
        } else {
            if (gt == 0) s_int[0] = atomicAdd(a.queue, 1);
            gbar(bid, tg);
            k = s_int[0];
        }
        if (k >= a.count) break;
        const int q = a.list[k];
        const int v0 = a.voff[q], n = a.voff[q + 1] - v0;
        const int h = a.heavy[q];
        const int nsl = (n - h + 31) >> 5;
        const int *gmeta = a.meta + a.moff[q];
        const int nm = h + nsl + 1;
        const int ne = gmeta[nm - 1];
        const double gsh = a.gsh[q];
        const bool coarsest = a.level == a.J[q];
        int mode = 0, kfix = 0;   // 0: until cos >= 1 - tol, 1: exactly kfix sweeps
        if (a.force_k >= 0) {
            mode = 1;
            kfix = a.force_k;
        } else if (a.replay) {
            mode = 1;
            kfix = a.replay[(size_t)q * CMG_MAX_LEVELS + a.level];
        } else if (a.fixed && !coarsest) {
            mode = 1;
            kfix = a.k_fixed;
        }
        const int maxs = coarsest ? a.max_sweeps_coarsest : a.max_sweeps;
        const bool gauss = coarsest || a.force_k >= 0;

        // ---- placement: iterates (and the layout) in shared memory when they fit
        const long long vbytes = (long long)n * (2 * (long long)sizeof(T) + (fp64 ? 8 : 0));
        const long long cbytes = (long long)ne * (long long)(sizeof(T) + sizeof(IDX)) + 4ll * nm + 16;
        T *X0, *X1;
        double *GD = nullptr;
        const int *M;
        const IDX *C;
        const T *W;
        if (a.stage && vbytes + cbytes <= data_bytes) {
            X0 = reinterpret_cast<T *>(data);
            X1 = X0 + n;
            unsigned char *p = reinterpret_cast<unsigned char *>(X1 + n);
            if (fp64) {
                GD = reinterpret_cast<double *>(p);
                p += 8ll * n;
            }
            T *sW = reinterpret_cast<T *>(p);
            int *sM = reinterpret_cast<int *>(sW + ne);
            IDX *sC = reinterpret_cast<IDX *>(sM + nm);
            const T *gw = reinterpret_cast<const T *>(a.bw) + a.eoff[q];
            const IDX *gc = reinterpret_cast<const IDX *>(a.bcol) + a.eoff[q];
            for (int e = gt; e < ne; e += tg) {
                sW[e] = gw[e];
                sC[e] = gc[e];
            }
            for (int m = gt; m < nm; m += tg) sM[m] = gmeta[m];
            M = sM;
            C = sC;
            W = sW;
        } else {
            if (vbytes <= data_bytes) {
                X0 = reinterpret_cast<T *>(data);
                X1 = X0 + n;
                if (fp64) GD = reinterpret_cast<double *>(X1 + n);
            } else {
                X0 = reinterpret_cast<T *>(a.vscr) + 2ll * v0;
                X1 = X0 + n;
                if (fp64) GD = a.gdscr + v0;
            }
            M = gmeta;
            C = reinterpret_cast<const IDX *>(a.bcol) + a.eoff[q];
            W = reinterpret_cast<const T *>(a.bw) + a.eoff[q];
        }
        const int *SO = M + h;       // slice offsets
        gbar(bid, tg);

        // ---- start vector (renumbered rows): Gaussian (Alg. 1 Step 2) or
        // I^T y (Alg. 1 Step 3) of the original vertex
        Part p0;
        p0.A = ff_zero();
        p0.B = ff_zero();
        p0.C = ff_zero();
        {
            for (int i = gt; i < n; i += tg) {
                const int old = a.perm[v0 + i];
                double xv;
                if (gauss) xv = gaussian_entry(a.seed, old - v0);
                else if (a.uc_fp64) xv = reinterpret_cast<const double *>(a.uc)[a.agg[old]];
                else xv = (double)reinterpret_cast<const float *>(a.uc)[a.agg[old]];
                const T xt = (T)xv;
                X0[i] = xt;
                if (fp64) {
                    double d = 0.0;
                    if (i < h) {
                        for (int e = M[i], e1 = M[i + 1]; e < e1; e++) d += (double)W[e];
                    } else {
                        const int sl = (i - h) >> 5, l = (i - h) & 31;
                        const int so = SO[sl], wd = (SO[sl + 1] - so) >> 5;
                        for (int kk = 0; kk < wd; kk++) d += (double)W[so + 32 * kk + l];
                    }
                    GD[i] = gsh - d;
                }
                const ff v = fp64 ? ff_from_double((double)xt) : ff_make((float)xt, 0.f);
                p0.A = ff_add(p0.A, v);
                p0.B = ff_add(p0.B, ff_mul(v, v));
            }
        }
        const Part P0 = gsum_part<1>(p0, s_part, lane, wg, nwg, bid, tg);
        const double mu0 = to_d(P0.A) / (double)n;
        double ss0 = to_d(P0.B) - (double)n * mu0 * mu0;
        if (ss0 < 0.0) ss0 = 0.0;
        int e = start_exponent(ss0);
        ff mu = ff_from_double(mu0), ss = ff_from_double(ss0);
        ff mu_p = mu, ss_p = ss, cs_last = ff_zero();

        // ---- Alg. 3: y_{s+1} = 2^e / g (B_g y_s - g mu_s 1), mean and norm of
        // y_s applied lazily; one group barrier per sweep
        const ff inv_n = ff_from_double(1.0 / (double)n);
        const double omt = 1.0 - a.tol;
        const ff omt2 = ff_from_double(omt * omt);
        const float inv_gf = 1.0f / (float)gsh;
        const double inv_gd = 1.0 / gsh;
        const float nf = (float)n;
        int s = 0, cur = 0, zero_hit = 0, capped = 0;
        for (;;) {
            if (mode == 1 ? s >= kfix : s >= maxs) {
                capped = (mode == 0) ? 1 : 0;
                break;
            }
            const T *x = cur ? X1 : X0;
            T *y = cur ? X0 : X1;
            const T mT = fp64 ? (T)ff_to_double(mu) : (T)mu.hi;
            const T sig = fp64 ? (T)ldexp(inv_gd, e) : (T)scale2f(inv_gf, e);
            const T gm = (T)gsh * mT;
            Acc<T> acc;
            acc.reset();
            auto finish_row = [&](int i, T xi, T ac) {
                T yv;
                if (fp64) yv = (T)((fma((double)GD[i], (double)xi, (double)ac) - (double)gm) * (double)sig);
                else yv = ((T)gsh * (xi - mT) - ac) * sig;
                y[i] = yv;
                acc.add(yv, xi);
            };
            // heavy rows: G lanes per row
            for (int base = wg * kRpw;; base += nwg * kRpw) {
                if (base >= h) break;
                const int i = base + lane / G;
                T ac = (T)0, xi = (T)0;
                if (i < h) {
                    xi = x[i];
                    ac = row_sum_grouped<T, IDX>(C, W, M[i] + rl, M[i + 1], G, xi,
                                                 [&](int c) { return x[c]; });
                }
                ac = group_sum<G>(ac);
                if (i < h && rl == 0) finish_row(i, xi, ac);
            }
            // light rows: one warp per slice of 32 rows, coalesced entries
            for (int sl = wg; sl < nsl; sl += nwg) {
                const int i = h + 32 * sl + lane;
                const int so = SO[sl] + lane, wd = (SO[sl + 1] - SO[sl]) >> 5;
                const T xi = (i < n) ? x[i] : (T)0;
                const T ac = row_sum_grouped<T, IDX>(C, W, so, so + 32 * wd, 32, xi,
                                                     [&](int c) { return x[c]; });
                if (i < n) finish_row(i, xi, ac);
            }
            const Part P = gsum_part<1>(acc.get(), s_part + 32 * ((s + 1) & 1), lane, wg, nwg, bid, tg);
            const ff mu1 = ff_mul(P.A, inv_n);
            const ff ss1 = ff_add_f(P.B, -nf * mu1.hi * mu1.hi);
            const ff cs = ff_add_f(P.C, -nf * mu1.hi * mu.hi);
            // annihilated: ||proj y_{s+1}|| <= 64 eps 2^e ||proj y_s||
            const bool zero = ss1.hi <= a.zero_tol2 * ldexpf(ss.hi, 2 * e);
            // cos >= 1 - tol  <=>  cs > 0 and cs^2 >= (1 - tol)^2 ss_{s+1} ss_s
            const bool conv = cs.hi > 0.f && !ff_lt(ff_mul(cs, cs), ff_mul(ff_mul(ss1, ss), omt2));
            s++;
            if (zero) {
                zero_hit = 1;   // keep y_s
                break;
            }
            mu_p = mu;
            ss_p = ss;
            mu = mu1;
            ss = ss1;
            cs_last = cs;
            cur ^= 1;
            if (mode == 0 && conv) break;
            // exact power-of-two rescale: ||proj y|| back near 1
            e = -(int)floorf(0.5f * log2f(fmaxf(ss.hi, 1e-37f)) + 0.5f);
        }

        // ---- result of this level, back in the original numbering
        const T *Yr = cur ? X1 : X0;
        const T *Yp = cur ? X0 : X1;
        const double r_mu = to_d(mu), r_ss = to_d(ss);
        const double r_inv = r_ss > 0.0 ? 1.0 / sqrt(r_ss) : 0.0;
        double r_cos = 0.0;
        if (zero_hit) {
            r_cos = 1.0;
        } else if (s > 0) {
            const double den = sqrt(r_ss * to_d(ss_p));
            r_cos = den > 0.0 ? to_d(cs_last) / den : 1.0;
        }
        if (a.level > 0) {
            T *uo = reinterpret_cast<T *>(a.uo);
            for (int i = gt; i < n; i += tg) uo[a.perm[v0 + i]] = (T)(((double)Yr[i] - r_mu) * r_inv);
        } else {
            double *u = a.uf + v0;
            if (!fp64 && s > 0 && !zero_hit) {
                // FP64 recomputation of the last sweep from the previous (FP32)
                // iterate, over the original CSR
                const double mp = to_d(mu_p), sp = to_d(ss_p);
                const double ip = sp > 0.0 ? 1.0 / sqrt(sp) : 0.0;
                double p2[2] = {0.0, 0.0};
                for (int base = rg;; base += ngr) {
                    if (__shfl_sync(0xffffffffu, base, 0) >= n) break;
                    const int i = base;
                    double accd = 0.0, xi = 0.0;
                    if (i < n) {
                        xi = ((double)Yp[a.inv[v0 + i] - v0] - mp) * ip;
                        for (int f = a.rp[v0 + i] + rl, f1 = a.rp[v0 + i + 1]; f < f1; f += G) {
                            const double xj = ((double)Yp[a.inv[a.col[f]] - v0] - mp) * ip;
                            accd += a.w[f] * (xi - xj);
                        }
                    }
                    accd = group_sum<G>(accd);
                    if (i < n && rl == 0) {
                        const double yv = gsh * xi - accd;
                        u[i] = yv;
                        p2[0] += yv;
                        p2[1] += yv * yv;
                    }
                }
                gsum_d<2>(p2, s_dred, lane, wg, nwg, bid, tg);
                const double m2 = p2[0] / (double)n;
                const double s2 = p2[1] - (double)n * m2 * m2;
                const double i2 = s2 > 0.0 ? 1.0 / sqrt(s2) : 0.0;
                for (int i = gt; i < n; i += tg) u[i] = (u[i] - m2) * i2;
            } else {
                for (int i = gt; i < n; i += tg) u[a.perm[v0 + i] - v0] = ((double)Yr[i] - r_mu) * r_inv;
            }
            gbar(bid, tg);
            // canonical sign: largest |u_i| (lowest i on ties) made positive
            {
                double best = -1.0, bval = 0.0;
                int bidx = 0x7fffffff;
                for (int i = gt; i < n; i += tg) {
                    const double v = u[i];
                    if (sign_better(fabs(v), i, best, bidx)) {
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
                    if (sign_better(ob, oi, best, bidx)) {
                        best = ob;
                        bidx = oi;
                        bval = ov;
                    }
                }
                if (tg > 32) {
                    if (lane == 0) {
                        s_dred[wg * 3 + 0] = best;
                        s_dred[wg * 3 + 1] = (double)bidx;
                        s_dred[wg * 3 + 2] = bval;
                    }
                    gbar(bid, tg);
                    best = -1.0;
                    bidx = 0x7fffffff;
                    bval = 0.0;
                    if (lane < nwg) {
                        best = s_dred[lane * 3 + 0];
                        bidx = (int)s_dred[lane * 3 + 1];
                        bval = s_dred[lane * 3 + 2];
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
                        const double ov = __shfl_xor_sync(0xffffffffu, bval, o);
                        if (sign_better(ob, oi, best, bidx)) {
                            best = ob;
                            bidx = oi;
                            bval = ov;
                        }
                    }
                    gbar(bid, tg);
                }
                if (bval < 0.0)
                    for (int i = gt; i < n; i += tg) u[i] = -u[i];
                gbar(bid, tg);
            }
            // Rayleigh quotient (1/2) sum_ij w_ij (u_i - u_j)^2 / ||u||^2 and
            // residual ||(L - lambda I) u|| / ||u||
            double p2[2] = {0.0, 0.0};
            for (int base = rg;; base += ngr) {
                if (__shfl_sync(0xffffffffu, base, 0) >= n) break;
                const int i = base;
                double accd = 0.0, ui = 0.0;
                if (i < n) {
                    ui = u[i];
                    for (int f = a.rp[v0 + i] + rl, f1 = a.rp[v0 + i + 1]; f < f1; f += G) {
                        const double d = ui - u[a.col[f] - v0];
                        accd += a.w[f] * d * d;
                    }
                }
                accd = group_sum<G>(accd);
                if (i < n && rl == 0) {
                    p2[0] += accd;
                    p2[1] += ui * ui;
                }
            }
            gsum_d<2>(p2, s_dred, lane, wg, nwg, bid, tg);
            const double uu = p2[1];
            const double lam = 0.5 * p2[0] / uu;
            double p1[1] = {0.0};
            for (int base = rg;; base += ngr) {
                if (__shfl_sync(0xffffffffu, base, 0) >= n) break;
                const int i = base;
                double accd = 0.0, ui = 0.0;
                if (i < n) {
                    ui = u[i];
                    for (int f = a.rp[v0 + i] + rl, f1 = a.rp[v0 + i + 1]; f < f1; f += G)
                        accd += a.w[f] * (ui - u[a.col[f] - v0]);
                }
                accd = group_sum<G>(accd);
                if (i < n && rl == 0) {
                    const double rr = accd - lam * ui;
                    p1[0] += rr * rr;
                }
            }
            gsum_d<1>(p1, s_dred, lane, wg, nwg, bid, tg);
            if (gt == 0) {
                a.lam[q] = lam;
                a.res[q] = sqrt(p1[0] / uu);
            }
        }
        if (gt == 0) {
            a.sweeps[q] = s;
            a.cosv[q] = r_cos;
            a.flags[q] = capped | (zero_hit << 1);
        }
        // the group's shared memory is reused by its next graph
        gbar(bid, tg);
    }
}

// Queue order of a level by predicted work, longest first: the graph's
// sweeps on the next coarser level (just solved) times its rows + entries on
// this level; graphs without a coarser solve keep their size order after the
// others.  One CTA, bitonic sort in shared memory (count <= kOrderMax).
constexpr int kOrderMax = 8192;

__global__ void __launch_bounds__(1024) k_order_level(int count, const int *__restrict__ list_in,
                                                      const int *__restrict__ sweeps_coarse,
                                                      const int *__restrict__ J, int level,
                                                      const int *__restrict__ voff,
                                                      const int *__restrict__ rp, int *__restrict__ list_out) {
    extern __shared__ __align__(16) unsigned char order_smem[];
    unsigned long long *key = reinterpret_cast<unsigned long long *>(order_smem);   // [m]
    int m = 1;
    while (m < count) m <<= 1;
    int *val = reinterpret_cast<int *>(key + m);   // [m]
    for (int t = threadIdx.x; t < m; t += blockDim.x) {
        if (t < count) {
            const int q = list_in[t];
            const unsigned long long size =
                (unsigned long long)(voff[q + 1] - voff[q]) + (unsigned long long)(rp[voff[q + 1]] - rp[voff[q]]);
            const unsigned long long sw = (J[q] > level) ? (unsigned long long)max(sweeps_coarse[q], 1) : 0ull;
            // work (48 bits) then the input position (ties keep the size order)
            const unsigned long long work = min(sw * size, (1ull << 47) - 1);
            key[t] = (work << 16) | (unsigned long long)(0xffff - min(t, 0xffff));
            val[t] = q;
        } else {
            key[t] = 0ull;   // padding sorts last
            val[t] = -1;
        }
    }
    __syncthreads();
    // bitonic sort, descending
    for (int k = 2; k <= m; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < m; t += blockDim.x) {
                const int u = t ^ j;
                if (u > t) {
                    const bool desc = (t & k) == 0;
                    const unsigned long long a = key[t], b = key[u];
                    if (desc ? (a < b) : (a > b)) {
                        key[t] = b;
                        key[u] = a;
                        const int tv = val[t];
                        val[t] = val[u];
                        val[u] = tv;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int t = threadIdx.x; t < count; t += blockDim.x) list_out[t] = val[t];
}

typedef void (*BatchKernel)(BatchPiArgs);

template <typename T, typename IDX>
static BatchKernel batch_kernel_ti(int G) {
    switch (G) {
        case 1: return k_batch_pi<T, IDX, 1>;
        case 2: return k_batch_pi<T, IDX, 2>;
        case 4: return k_batch_pi<T, IDX, 4>;
        case 8: return k_batch_pi<T, IDX, 8>;
        case 16: return k_batch_pi<T, IDX, 16>;
        case 32: return k_batch_pi<T, IDX, 32>;
        default: return nullptr;
    }
}

static BatchKernel batch_kernel(int fp32, int col16, int G) {
    if (fp32) return col16 ? batch_kernel_ti<float, uint16_t>(G) : batch_kernel_ti<float, int>(G);
    return col16 ? batch_kernel_ti<double, uint16_t>(G) : batch_kernel_ti<double, int>(G);
}

}  // namespace cmg

// ================================================================== host side
using namespace cmg;

namespace {

struct BLevel {
    int n = 0;
    long long nnz = 0;
    int *rp = nullptr;
    int *col = nullptr;
    double *w = nullptr;
    int *agg = nullptr;          // onto the next union level
    SweepLayout lay;             // sweep layout of the level
    int *voff = nullptr;         // device int[G+1]
    double *gsh = nullptr;       // device double[G]
    std::vector<int> hvoff;      // host copies
    std::vector<int> heoff;      // row_ptr at hvoff
    std::vector<double> hg;
    int *list = nullptr;         // graphs solved on this level, largest first
    int *order = nullptr;        // the same graphs by predicted work (set per solve)
    int count = 0;
    int kbig = 0;                // graphs of the level's big-graph launch
    long long max_vbytes = 0;    // largest graph on the list: vector bytes
    long long max_cbytes = 0;    //                            CSR bytes
    void *u = nullptr;           // normalised level result (levels > 0)
    void *vscr = nullptr;        // iterates of graphs too large for shared memory
    double *gdscr = nullptr;
    cmg_batch_shape_t shape = {128, 1, 2, 1};
    int smem_group = 0;
};

void free_blevel(BLevel &L, cudaStream_t s) {
    dev_free(L.rp, s);
    dev_free(L.col, s);
    dev_free(L.w, s);
    free_sweep_layout(L.lay, s);
    dev_free(L.agg, s);
    dev_free(L.voff, s);
    dev_free(L.gsh, s);
    dev_free(L.list, s);
    dev_free(L.order, s);
    dev_free(L.u, s);
    dev_free(L.vscr, s);
    dev_free(L.gdscr, s);
    L = BLevel();
}

}  // namespace

struct cmg_batch_s {
    int device = 0;
    cudaStream_t stream = nullptr;    // stream the batch was built on
    cudaStream_t cap = nullptr;       // library stream used for graph capture
    cmg_options_t opts;
    int G = 0;
    std::vector<BLevel> lv;
    std::vector<int> J;
    int *dJ = nullptr;
    int *queue = nullptr;             // [levels]
    int *sweeps = nullptr;            // [levels][G]
    int *flags = nullptr;
    double *cosv = nullptr;
    double *lam = nullptr, *res = nullptr;
    double *uf = nullptr;             // double[N_0]
    int *replay = nullptr;            // [G][CMG_MAX_LEVELS]
    bool solved = false;
    std::vector<int> h_sweeps, h_flags;
    std::vector<double> h_cos, h_lam, h_res;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool dirty = true;
    unsigned long long graph_kernels = 0;
    std::vector<double> level_ms;     // options.timing: device time per union level
    cudaStream_t side = nullptr;      // second stream: the big-graph launch of a level
    std::vector<cudaEvent_t> ev_fork, ev_join;
    int *tune_replay = nullptr;       // autotuner: replayed sweep counts
    size_t bytes = 0;
};

static void drop_graph(cmg_batch_s *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->dirty = true;
}

static void free_batch(cmg_batch_s *b) {
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    drop_graph(b);
    for (auto &L : b->lv) free_blevel(L, b->stream);
    dev_free(b->dJ, b->stream);
    dev_free(b->queue, b->stream);
    dev_free(b->sweeps, b->stream);
    dev_free(b->flags, b->stream);
    dev_free(b->cosv, b->stream);
    dev_free(b->lam, b->stream);
    dev_free(b->res, b->stream);
    dev_free(b->uf, b->stream);
    dev_free(b->replay, b->stream);
    dev_free(b->tune_replay, b->stream);
    cudaStreamSynchronize(b->stream);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->side) cudaStreamDestroy(b->side);
    for (cudaEvent_t e : b->ev_fork) cudaEventDestroy(e);
    for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
    cudaSetDevice(prev);
    delete b;
}

static int threads_for_gpc(const cmg_batch_shape_t &sh) { return sh.threads_per_graph * sh.graphs_per_cta; }

static bool shape_valid(const cmg_batch_shape_t &sh) {
    const int t = sh.threads_per_graph, l = sh.lanes_per_row, g = sh.graphs_per_cta;
    if (t < 32 || t > kBatchMaxThreads || (t & 31)) return false;
    if (l != 1 && l != 2 && l != 4 && l != 8 && l != 16 && l != 32) return false;
    if (g < 1 || t * g > kBatchMaxThreads) return false;
    if (t > 32 && g > 15) return false;   // named barriers 1..15
    if (sh.stage_csr != 0 && sh.stage_csr != 1) return false;
    return true;
}

// Shared bytes per group for a level's shape: the largest graph's needs,
// capped so that two CTAs fit on an SM (each CTA also holds 1 KB of
// system shared memory); graphs beyond the cap keep their iterates in
// global memory.
static int group_smem(const BLevel &L, const cmg_batch_shape_t &sh, int max_optin) {
    const long long need = (sh.stage_csr ? L.max_vbytes + L.max_cbytes : L.max_vbytes) + 16;
    const long long cap = ((long long)max_optin - 1024) / 2 / sh.graphs_per_cta - kGroupHeader;
    const long long d = std::max<long long>(0, std::min(need, cap));
    return (int)((kGroupHeader + d) / 16 * 16);
}


// A level with enough graphs runs its largest-work graphs (a quarter of the
// level, at most kBigGraphs) in a launch of their own, one 1024-thread group
// per graph, so the graphs whose sweeps form the level's longest serial
// chains get the most threads; the rest run concurrently in the level's
// tuned shape.
constexpr int kBigGraphs = 64;

static cmg_batch_shape_t big_shape(const BLevel &L) {
    cmg_batch_shape_t sh;
    sh.threads_per_graph = kBatchMaxThreads;
    sh.lanes_per_row = L.shape.lanes_per_row;
    sh.graphs_per_cta = 1;
    sh.stage_csr = 1;
    return sh;
}

static cmg_batch_shape_t default_shape(const BLevel &L) {
    double avg_n = 0.0, avg_deg = 0.0;
    // per-graph sizes of the listed graphs are not kept on the host; the
    // level totals give the averages
    const int G = (int)L.hvoff.size() - 1;
    avg_n = (double)L.n / std::max(1, G);
    avg_deg = (double)L.nnz / std::max(1, L.n);
    cmg_batch_shape_t sh;
    sh.threads_per_graph = avg_n <= 192 ? 32 : avg_n <= 768 ? 64 : avg_n <= 3072 ? 128 : 256;
    sh.lanes_per_row = avg_deg <= 12 ? 1 : avg_deg <= 24 ? 2 : 4;
    sh.graphs_per_cta = std::max(1, std::min(256 / sh.threads_per_graph, 8));
    sh.stage_csr = 1;
    return sh;
}

// Sweep precision of union level j.  In the FP32 form only level 0 sweeps in
// FP32: it carries most of the bytes and the fewest sweeps.  The coarse
// levels keep FP64 sweeps: each graph's coarse levels are small (its group
// holds them in shared memory), and they run the longest sweep chains
// (thousands of sweeps), along which FP32 rounding accumulates in slowly
// converging components that the finer levels inherit.
static int level_fp32(const cmg_batch_s *b, int j) {
    return (b->opts.precision == CMG_PRECISION_FP32_SWEEP && j == 0) ? 1 : 0;
}

// Workspace of level j for its current shape: the fallback iterate buffers
// are allocated only if some listed graph does not fit in shared memory.
static cmg_status_t level_workspace(cmg_batch_s *b, int j, cudaStream_t s) {
    BLevel &L = b->lv[j];
    const int fp32 = level_fp32(b, j);
    const size_t esz = fp32 ? sizeof(float) : sizeof(double);
    DeviceInfo di;
    CMG_TRY(device_info(&di));
    L.smem_group = group_smem(L, L.shape, di.max_smem_optin);
    const int big_group = group_smem(L, big_shape(L), di.max_smem_optin);
    if (L.max_vbytes > std::min(L.smem_group, big_group) - kGroupHeader && !L.vscr) {
        CMG_TRY(dev_alloc(&L.vscr, 2 * esz * (size_t)std::max(L.n, 1), s));
        b->bytes += 2 * esz * (size_t)L.n;
        if (!fp32) {
            CMG_TRY(dev_alloc_n(&L.gdscr, (size_t)std::max(L.n, 1), s));
            b->bytes += sizeof(double) * (size_t)L.n;
        }
    }
    BatchKernel kern = batch_kernel(fp32, L.lay.col16, L.shape.lanes_per_row);
    if (!kern) return CMG_ERR_INVALID_ARG;
    const int smem = L.smem_group * L.shape.graphs_per_cta;
    if (smem > di.max_smem_optin) return CMG_ERR_INVALID_ARG;
    CMG_TRY(allow_max_dynamic_smem((const void *)kern));
    return CMG_OK;
}

// One launch of level j's kernel over `count` graphs of `list` with the
// given shape and queue counter.
static cmg_status_t launch_part(cmg_batch_s *b, int j, int force_k, cudaStream_t s, const int *list,
                                int count, int *queue, const cmg_batch_shape_t &shape, int smem_group) {
    BLevel &L = b->lv[j];
    if (count <= 0) return CMG_OK;
    const int fp32 = level_fp32(b, j);
    const cmg_options_t &o = b->opts;
    BatchKernel kern = batch_kernel(fp32, L.lay.col16, shape.lanes_per_row);
    const int threads = threads_for_gpc(shape);
    const int smem = smem_group * shape.graphs_per_cta;
    int per_sm = 0;
    CMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)kern, threads, smem));
    if (per_sm < 1) return CMG_ERR_INVALID_ARG;
    DeviceInfo di;
    CMG_TRY(device_info(&di));
    const int blocks = std::max(1, std::min(div_up(count, shape.graphs_per_cta), per_sm * di.sms));
    BatchPiArgs a;
    memset(&a, 0, sizeof(a));
    a.level = j;
    a.rp = L.rp;
    a.col = L.col;
    a.w = L.w;
    a.perm = reinterpret_cast<const int *>(L.lay.perm);
    a.inv = L.lay.inv;
    a.heavy = L.lay.heavy;
    a.eoff = L.lay.eoff;
    a.moff = L.lay.moff;
    a.meta = L.lay.meta;
    a.bcol = L.lay.bcol;
    a.bw = L.lay.bw;
    a.voff = L.voff;
    a.gsh = L.gsh;
    a.list = list;
    a.count = count;
    a.queue = queue;
    a.J = b->dJ;
    a.agg = L.agg;
    a.uc = (j + 1 < (int)b->lv.size()) ? b->lv[j + 1].u : nullptr;
    a.uc_fp64 = (j + 1 < (int)b->lv.size()) ? !level_fp32(b, j + 1) : 1;
    a.uo = L.u;
    a.uf = b->uf;
    a.vscr = L.vscr;
    a.gdscr = L.gdscr;
    a.tg = shape.threads_per_graph;
    a.smem_group = smem_group;
    a.stage = shape.stage_csr;
    a.fixed = o.schedule == CMG_SCHEDULE_FIXED;
    a.k_fixed = (int)ceil((double)o.k0 * pow(o.beta, (double)j));
    a.replay = b->tune_replay ? b->tune_replay : ((o.schedule == CMG_SCHEDULE_REPLAY) ? b->replay : nullptr);
    a.force_k = force_k;
    a.max_sweeps = o.max_sweeps;
    a.max_sweeps_coarsest = o.max_sweeps_coarsest;
    a.tol = o.tol;
    a.seed = o.seed;
    a.zero_tol2 = fp32 ? kZeroTol2_32 : kZeroTol2_64;
    a.sweeps = b->sweeps + (size_t)j * b->G;
    a.cosv = b->cosv + (size_t)j * b->G;
    a.flags = b->flags + (size_t)j * b->G;
    a.lam = b->lam;
    a.res = b->res;
    kern<<<blocks, threads, smem, s>>>(a);
    return launch_status();
}

// All launches of level j.  With a work order (use_order) and big graphs on
// the level, the first kbig graphs of the order run in their own launch on
// the side stream while the rest run on `s` (fork/join through events, so the
// pair is also captured as two parallel graph branches).
static cmg_status_t launch_level(cmg_batch_s *b, int j, int force_k, cudaStream_t s,
                                 bool use_order = false) {
    BLevel &L = b->lv[j];
    if (L.count == 0) return CMG_OK;
    const int *list = (use_order && L.order) ? L.order : L.list;
    const int kbig = use_order ? std::min(L.kbig, L.count) : 0;
    if (kbig == 0)
        return launch_part(b, j, force_k, s, list, L.count, b->queue + 2 * j, L.shape, L.smem_group);
    CMG_CUDA(cudaEventRecord(b->ev_fork[j], s));
    CMG_CUDA(cudaStreamWaitEvent(b->side, b->ev_fork[j], 0));
    DeviceInfo di;
    CMG_TRY(device_info(&di));
    const cmg_batch_shape_t bs = big_shape(L);
    CMG_TRY(launch_part(b, j, force_k, b->side, list, kbig, b->queue + 2 * j + 1, bs,
                        group_smem(L, bs, di.max_smem_optin)));
    CMG_TRY(launch_part(b, j, force_k, s, list + kbig, L.count - kbig, b->queue + 2 * j, L.shape,
                        L.smem_group));
    CMG_CUDA(cudaEventRecord(b->ev_join[j], b->side));
    CMG_CUDA(cudaStreamWaitEvent(s, b->ev_join[j], 0));
    return CMG_OK;
}

// Orders level j's queue by predicted work (see k_order_level).
static cmg_status_t order_level(cmg_batch_s *b, int j, cudaStream_t s, bool *ordered) {
    BLevel &L = b->lv[j];
    *ordered = false;
    if (j + 1 >= (int)b->lv.size() || L.count < 2 || L.count > kOrderMax) return CMG_OK;
    int m = 1;
    while (m < L.count) m <<= 1;
    k_order_level<<<1, 1024, (size_t)m * 12, s>>>(L.count, L.list, b->sweeps + (size_t)(j + 1) * b->G,
                                                 b->dJ, j, L.voff, L.rp, L.order);
    CMG_TRY(launch_status());
    *ordered = true;
    return CMG_OK;
}

static cmg_status_t enqueue_solve(cmg_batch_s *b, int force_k, cudaStream_t s) {
    const int L = (int)b->lv.size();
    CMG_CUDA(cudaMemsetAsync(b->queue, 0, sizeof(int) * 2 * L, s));
    for (int j = L - 1; j >= 0; j--) {
        bool ordered = false;
        if (force_k < 0) CMG_TRY(order_level(b, j, s, &ordered));
        CMG_TRY(launch_level(b, j, force_k, s, ordered));
    }
    return CMG_OK;
}

// Sweep layout of union level j (see SweepLayout).
static cmg_status_t build_layout(cmg_batch_s *b, int j, cudaStream_t s, size_t *bytes) {
    BLevel &L = b->lv[j];
    return build_sweep_layout(b->G, L.voff, L.hvoff, L.n, L.rp, L.col, L.w, level_fp32(b, j), &L.lay,
                              bytes, s);
}

// Level lists: graphs with J >= j, ordered by decreasing n + nnz on level j.
static cmg_status_t build_lists(cmg_batch_s *b, cudaStream_t s) {
    const int G = b->G;
    for (int j = 0; j < (int)b->lv.size(); j++) {
        BLevel &L = b->lv[j];
        std::vector<int> ids;
        L.max_vbytes = L.max_cbytes = 0;
        const int fp32 = level_fp32(b, j);
        const long long esz = fp32 ? 4 : 8;
        for (int q = 0; q < G; q++) {
            if (b->J[q] < j) continue;
            ids.push_back(q);
            const long long n = L.hvoff[q + 1] - L.hvoff[q];
            const long long isz = L.lay.col16 ? 2 : 4;
            L.max_vbytes = std::max(L.max_vbytes, n * (2 * esz + (fp32 ? 0 : 8)));
            L.max_cbytes = std::max(L.max_cbytes, (long long)L.lay.hecnt[q] * (esz + isz) + 4ll * L.lay.hmcnt[q] + 16);
        }
        std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) {
            const long long wx = (L.hvoff[x + 1] - L.hvoff[x]) + (long long)(L.heoff[x + 1] - L.heoff[x]);
            const long long wy = (L.hvoff[y + 1] - L.hvoff[y]) + (long long)(L.heoff[y + 1] - L.heoff[y]);
            return wx > wy;
        });
        L.count = (int)ids.size();
        L.kbig = (L.count >= 16) ? std::min(kBigGraphs, L.count / 4) : 0;
        CMG_TRY(dev_alloc_n(&L.list, std::max<size_t>(ids.size(), 1), s));
        CMG_TRY(dev_alloc_n(&L.order, std::max<size_t>(ids.size(), 1), s));
        if (!ids.empty())
            CMG_CUDA(cudaMemcpyAsync(L.list, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, s));
        b->bytes += sizeof(int) * ids.size();
    }
    return CMG_OK;
}

static cmg_status_t build_batch(cmg_batch_s *b, const int64_t *offs, const int64_t *row_ptr,
                                const int32_t *col, const double *w, int32_t mem) {
    cudaStream_t s = b->stream;
    const cmg_options_t &o = b->opts;
    const int G = b->G;
    const int64_t N = offs[G];
    // ---- level 0
    b->lv.emplace_back();
    {
        BLevel &Z = b->lv.back();
        Z.n = (int)N;
        CMG_TRY(load_level0(N, row_ptr, col, w, mem, o.validate, &Z.rp, &Z.col, &Z.w, &Z.nnz, s));
        Z.hvoff.resize(G + 1);
        for (int q = 0; q <= G; q++) Z.hvoff[q] = (int)offs[q];
        CMG_TRY(dev_alloc_n(&Z.voff, (size_t)G + 1, s));
        CMG_CUDA(cudaMemcpyAsync(Z.voff, Z.hvoff.data(), sizeof(int) * (G + 1), cudaMemcpyHostToDevice, s));
        Scratch scr(s);
        unsigned *flag;
        int *eoff;
        CMG_TRY(scr.get(&flag, 1));
        CMG_TRY(scr.get(&eoff, (size_t)G + 1));
        CMG_CUDA(cudaMemsetAsync(flag, 0, sizeof(unsigned), s));
        if (o.validate) {
            k_batch_check<<<grid_for(N, 256), 256, 0, s>>>((int)N, G, Z.voff, Z.rp, Z.col, flag);
            CMG_TRY(launch_status());
        }
        CMG_TRY(dev_alloc_n(&Z.gsh, (size_t)G, s));
        k_batch_gersh<<<grid_for((long long)G * 32, 256), 256, 0, s>>>(G, Z.voff, Z.rp, Z.w, Z.gsh);
        CMG_TRY(launch_status());
        k_gather_at<<<grid_for(G + 1, 256), 256, 0, s>>>(G, Z.voff, Z.rp, eoff);
        CMG_TRY(launch_status());
        unsigned hf = 0;
        Z.heoff.resize(G + 1);
        Z.hg.resize(G);
        CMG_CUDA(cudaMemcpyAsync(&hf, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaMemcpyAsync(Z.heoff.data(), eoff, sizeof(int) * (G + 1), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaMemcpyAsync(Z.hg.data(), Z.gsh, sizeof(double) * G, cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
        if (hf) return CMG_ERR_BAD_CSR;
    }
    b->J.assign(G, -1);
    // ---- Alg. 1 Step 1 on the union, one host synchronisation per level
    Scratch scr(s);
    LevelCounts *cnt;
    int *coff_t, *eoff_t;
    double *g_t;
    CMG_TRY(scr.get(&cnt, 1));
    CMG_TRY(scr.get(&coff_t, (size_t)G + 1));
    CMG_TRY(scr.get(&eoff_t, (size_t)G + 1));
    CMG_TRY(scr.get(&g_t, (size_t)G));
    std::vector<int> hcoff(G + 1), heoff(G + 1);
    std::vector<double> hg(G);
    for (int level = 0;; level++) {
        const BLevel F = b->lv.back();
        std::vector<int> cand;
        for (int q = 0; q < G; q++) {
            if (b->J[q] >= 0) continue;
            const int nq = F.hvoff[q + 1] - F.hvoff[q];
            if (nq > o.coarse_size && level + 1 < o.max_levels) cand.push_back(q);
            else b->J[q] = level;
        }
        if (cand.empty()) break;
        int *agg = nullptr, *rp_t = nullptr, *col_t = nullptr;
        double *w_t = nullptr;
        uint32_t *rank = nullptr;
        LevelCounts hc;
        auto release = [&]() {
            dev_free(agg, s);
            dev_free(rp_t, s);
            dev_free(col_t, s);
            dev_free(w_t, s);
            dev_free(rank, s);
        };
        cmg_status_t st = CMG_OK;
        do {
            const size_t cap = (size_t)std::max<long long>(F.nnz, 1);
            if ((st = dev_alloc_n(&agg, (size_t)F.n, s)) != CMG_OK) break;
            if ((st = dev_alloc_n(&rank, (size_t)F.n, s)) != CMG_OK) break;
            if ((st = dev_alloc_n(&rp_t, (size_t)F.n + 1, s)) != CMG_OK) break;
            if ((st = dev_alloc_n(&col_t, cap, s)) != CMG_OK) break;
            if ((st = dev_alloc_n(&w_t, cap, s)) != CMG_OK) break;
            if ((st = from_cuda(cudaMemsetAsync(cnt, 0, sizeof(LevelCounts), s))) != CMG_OK) break;
            if ((st = launch_ranks_batch(F.n, G, F.voff, o.seed, level, rank, s)) != CMG_OK) break;
            st = hec_level_async(F.n, F.nnz, F.rp, F.col, F.w, o.seed, level, rank, agg, &cnt->c,
                                 &cnt->gs, s);
            if (st != CMG_OK) break;
            st = galerkin_async(F.n, F.nnz, F.rp, F.col, F.w, agg, bits_for(F.n), cnt, rp_t, col_t,
                                w_t, s);
            if (st != CMG_OK) break;
            k_batch_coff<<<grid_for((long long)G * 32, 256), 256, 0, s>>>(G, F.voff, agg, cnt, coff_t);
            if ((st = launch_status()) != CMG_OK) break;
            k_batch_gersh<<<grid_for((long long)G * 32, 256), 256, 0, s>>>(G, coff_t, rp_t, w_t, g_t);
            if ((st = launch_status()) != CMG_OK) break;
            k_gather_at<<<grid_for(G + 1, 256), 256, 0, s>>>(G, coff_t, rp_t, eoff_t);
            if ((st = launch_status()) != CMG_OK) break;
            cudaError_t ce = cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(hcoff.data(), coff_t, sizeof(int) * (G + 1), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(heoff.data(), eoff_t, sizeof(int) * (G + 1), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(hg.data(), g_t, sizeof(double) * G, cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) st = from_cuda(ce);
            if (st == CMG_OK && hc.gs.err) st = CMG_ERR_DEVICE_TIMEOUT;
        } while (0);
        if (st != CMG_OK) {
            release();
            return st;
        }
        // a graph whose coarsening collapses (c < 2) keeps this level as its coarsest
        bool any = false;
        for (int q : cand) {
            if (hcoff[q + 1] - hcoff[q] < 2) b->J[q] = level;
            else any = true;
        }
        if (!any) {
            release();
            break;
        }
        BLevel C;
        C.n = hc.c;
        C.nnz = hc.nseg;
        C.hvoff = hcoff;
        C.heoff = heoff;
        C.hg = hg;
        st = dev_alloc_n(&C.rp, (size_t)C.n + 1, s);
        if (st == CMG_OK) st = dev_alloc_n(&C.col, (size_t)std::max<long long>(C.nnz, 1), s);
        if (st == CMG_OK) st = dev_alloc_n(&C.w, (size_t)std::max<long long>(C.nnz, 1), s);
        if (st == CMG_OK) st = dev_alloc_n(&C.voff, (size_t)G + 1, s);
        if (st == CMG_OK) st = dev_alloc_n(&C.gsh, (size_t)G, s);
        if (st == CMG_OK)
            st = from_cuda(cudaMemcpyAsync(C.rp, rp_t, sizeof(int) * ((size_t)C.n + 1),
                                           cudaMemcpyDeviceToDevice, s));
        if (st == CMG_OK && C.nnz > 0)
            st = from_cuda(cudaMemcpyAsync(C.col, col_t, sizeof(int) * (size_t)C.nnz,
                                           cudaMemcpyDeviceToDevice, s));
        if (st == CMG_OK && C.nnz > 0)
            st = from_cuda(cudaMemcpyAsync(C.w, w_t, sizeof(double) * (size_t)C.nnz,
                                           cudaMemcpyDeviceToDevice, s));
        if (st == CMG_OK)
            st = from_cuda(cudaMemcpyAsync(C.voff, coff_t, sizeof(int) * (G + 1), cudaMemcpyDeviceToDevice, s));
        if (st == CMG_OK)
            st = from_cuda(cudaMemcpyAsync(C.gsh, g_t, sizeof(double) * G, cudaMemcpyDeviceToDevice, s));
        b->lv.back().agg = agg;
        agg = nullptr;
        release();
        b->lv.push_back(C);  // freed with the batch, also on error
        if (st != CMG_OK) return st;
    }
    for (int q = 0; q < G; q++)
        if (b->J[q] < 0) b->J[q] = (int)b->lv.size() - 1;
    // ---- solve workspace
    const int L = (int)b->lv.size();
    size_t bytes = 0;
    for (int j = 0; j < L; j++) {
        BLevel &V = b->lv[j];
        const size_t esz = level_fp32(b, j) ? sizeof(float) : sizeof(double);
        bytes += sizeof(int) * ((size_t)V.n + 1) + (sizeof(int) + sizeof(double)) * (size_t)V.nnz;
        bytes += sizeof(int) * (G + 1) + sizeof(double) * G;
        if (V.agg) bytes += sizeof(int) * (size_t)V.n;
        CMG_TRY(build_layout(b, j, s, &bytes));
        if (j > 0) {
            CMG_TRY(dev_alloc(&V.u, esz * (size_t)std::max(V.n, 1), s));
            bytes += esz * (size_t)V.n;
        }
    }
    CMG_TRY(dev_alloc_n(&b->dJ, (size_t)G, s));
    CMG_CUDA(cudaMemcpyAsync(b->dJ, b->J.data(), sizeof(int) * G, cudaMemcpyHostToDevice, s));
    CMG_TRY(dev_alloc_n(&b->queue, (size_t)2 * L, s));
    CMG_TRY(dev_alloc_n(&b->sweeps, (size_t)L * G, s));
    CMG_TRY(dev_alloc_n(&b->flags, (size_t)L * G, s));
    CMG_TRY(dev_alloc_n(&b->cosv, (size_t)L * G, s));
    CMG_CUDA(cudaMemsetAsync(b->sweeps, 0, sizeof(int) * (size_t)L * G, s));
    CMG_CUDA(cudaMemsetAsync(b->flags, 0, sizeof(int) * (size_t)L * G, s));
    CMG_CUDA(cudaMemsetAsync(b->cosv, 0, sizeof(double) * (size_t)L * G, s));
    CMG_TRY(dev_alloc_n(&b->lam, (size_t)G, s));
    CMG_TRY(dev_alloc_n(&b->res, (size_t)G, s));
    CMG_TRY(dev_alloc_n(&b->uf, (size_t)N, s));
    bytes += sizeof(int) * (G + L + 2 * (size_t)L * G) + sizeof(double) * ((size_t)L * G + 2 * G + N);
    if (o.schedule == CMG_SCHEDULE_REPLAY) {
        std::vector<int> rep((size_t)G * CMG_MAX_LEVELS);
        for (int q = 0; q < G; q++)
            for (int j = 0; j < CMG_MAX_LEVELS; j++) rep[(size_t)q * CMG_MAX_LEVELS + j] = o.replay_sweeps[j];
        CMG_TRY(dev_alloc_n(&b->replay, rep.size(), s));
        CMG_CUDA(cudaMemcpyAsync(b->replay, rep.data(), sizeof(int) * rep.size(), cudaMemcpyHostToDevice, s));
        bytes += sizeof(int) * rep.size();
    }
    b->bytes = bytes;
    CMG_TRY(build_lists(b, s));
    CMG_TRY(allow_max_dynamic_smem((const void *)k_order_level));
    b->ev_fork.assign(L, nullptr);
    b->ev_join.assign(L, nullptr);
    for (int j = 0; j < L; j++) {
        CMG_CUDA(cudaEventCreateWithFlags(&b->ev_fork[j], cudaEventDisableTiming));
        CMG_CUDA(cudaEventCreateWithFlags(&b->ev_join[j], cudaEventDisableTiming));
    }
    for (int j = 0; j < L; j++) {
        b->lv[j].shape = default_shape(b->lv[j]);
        CMG_TRY(level_workspace(b, j, s));
    }
    CMG_CUDA(cudaStreamSynchronize(s));
    return CMG_OK;
}

// Records the solve launches into a CUDA graph (library stream, then replayed
// on the caller's stream).
static cmg_status_t capture(cmg_batch_s *b) {
    drop_graph(b);
    const unsigned long long l0 = launches_issued();
    cudaStream_t cs = b->cap;
    CMG_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cmg_status_t st = enqueue_solve(b, -1, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (st != CMG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return from_cuda(e);
    b->graph = g;
    CMG_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    b->dirty = false;
    // captured launches run when the graph is replayed, and count there
    b->graph_kernels = launches_issued() - l0;
    add_launches(-(long long)b->graph_kernels);
    return CMG_OK;
}

// ================================================================== C-ABI
struct DeviceGuard {
    int prev = 0;
    int want = 0;
    bool switched = false;
    explicit DeviceGuard(int dev) : want(dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) switched = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (switched) cudaSetDevice(prev);
    }
};

extern "C" cmg_status_t cmg_setup_batch(int32_t num_graphs, const int64_t *graph_offsets,
                                        const int64_t *row_ptr, const int32_t *col, const double *w,
                                        int32_t mem, const cmg_options_t *opts, void *stream,
                                        cmg_batch_t *out) {
    if (!out) return CMG_ERR_INVALID_ARG;
    *out = nullptr;
    if (num_graphs < 1 || !graph_offsets || !row_ptr) return CMG_ERR_INVALID_ARG;
    if (mem != CMG_MEM_HOST && mem != CMG_MEM_DEVICE) return CMG_ERR_INVALID_ARG;
    if (graph_offsets[0] != 0) return CMG_ERR_INVALID_ARG;
    for (int q = 0; q < num_graphs; q++) {
        if (graph_offsets[q + 1] < graph_offsets[q]) return CMG_ERR_INVALID_ARG;
    }
    for (int q = 0; q < num_graphs; q++)
        if (graph_offsets[q + 1] - graph_offsets[q] < 2) return CMG_ERR_TOO_SMALL;
    if (graph_offsets[num_graphs] >= 2147483647ll) return CMG_ERR_TOO_LARGE;
    cmg_options_t o;
    cmg_options_default(&o);
    if (opts) o = *opts;
    CMG_TRY(check_options(o));
    cmg_batch_s *b = new cmg_batch_s();
    b->opts = o;
    b->G = num_graphs;
    b->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking) != cudaSuccess) {
        free_batch(b);
        return CMG_ERR_CUDA;
    }
    cmg_status_t st = build_batch(b, graph_offsets, row_ptr, col, w, mem);
    if (st != CMG_OK) {
        free_batch(b);
        return st;
    }
    *out = b;
    return CMG_OK;
}

extern "C" cmg_status_t cmg_fiedler_batch(cmg_batch_t b, double *u_out, int32_t u_mem,
                                          double *lambda2_out, double *residual_out,
                                          int32_t *status_out, void *stream) {
    if (!b) return CMG_ERR_INVALID_ARG;
    if (u_out && u_mem != CMG_MEM_HOST && u_mem != CMG_MEM_DEVICE) return CMG_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int G = b->G, L = (int)b->lv.size();
    if (b->opts.timing) {
        // eager launches with an event pair around each level
        std::vector<cudaEvent_t> ev(2 * L);
        for (auto &e : ev) CMG_CUDA(cudaEventCreate(&e));
        cmg_status_t st = from_cuda(cudaMemsetAsync(b->queue, 0, sizeof(int) * 2 * L, s));
        for (int j = L - 1; j >= 0 && st == CMG_OK; j--) {
            bool ordered = false;
            cudaEventRecord(ev[2 * j], s);
            st = order_level(b, j, s, &ordered);
            if (st == CMG_OK) st = launch_level(b, j, -1, s, ordered);
            cudaEventRecord(ev[2 * j + 1], s);
        }
        if (st == CMG_OK) st = from_cuda(cudaStreamSynchronize(s));
        b->level_ms.assign(L, 0.0);
        for (int j = 0; j < L && st == CMG_OK; j++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * j], ev[2 * j + 1]) == cudaSuccess) b->level_ms[j] = ms;
        }
        for (auto &e : ev) cudaEventDestroy(e);
        CMG_TRY(st);
    } else {
        if (b->dirty) CMG_TRY(capture(b));
        CMG_CUDA(cudaGraphLaunch(b->exec, s));
        add_launches((long long)b->graph_kernels);
    }
    b->h_sweeps.resize((size_t)L * G);
    b->h_flags.resize((size_t)L * G);
    b->h_cos.resize((size_t)L * G);
    b->h_lam.resize(G);
    b->h_res.resize(G);
    CMG_CUDA(cudaMemcpyAsync(b->h_sweeps.data(), b->sweeps, sizeof(int) * L * G, cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(b->h_flags.data(), b->flags, sizeof(int) * L * G, cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(b->h_cos.data(), b->cosv, sizeof(double) * L * G, cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(b->h_lam.data(), b->lam, sizeof(double) * G, cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(b->h_res.data(), b->res, sizeof(double) * G, cudaMemcpyDeviceToHost, s));
    if (u_out)
        CMG_CUDA(cudaMemcpyAsync(u_out, b->uf, sizeof(double) * (size_t)b->lv[0].n,
                                 u_mem == CMG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    b->solved = true;
    bool capped = false;
    for (int q = 0; q < G; q++) {
        bool cq = false;
        for (int j = 0; j <= b->J[q]; j++) cq = cq || (b->h_flags[(size_t)j * G + q] & 1);
        capped = capped || cq;
        if (status_out) status_out[q] = cq ? CMG_WARN_MAXITER : CMG_OK;
        if (lambda2_out) lambda2_out[q] = b->h_lam[q];
        if (residual_out) residual_out[q] = b->h_res[q];
    }
    return capped ? CMG_WARN_MAXITER : CMG_OK;
}

extern "C" cmg_status_t cmg_batch_info(cmg_batch_t b, int32_t *num_graphs, int32_t *union_levels,
                                       int32_t level, int64_t *n_level, int64_t *nnz_level) {
    if (!b) return CMG_ERR_INVALID_ARG;
    if (num_graphs) *num_graphs = b->G;
    if (union_levels) *union_levels = (int32_t)b->lv.size();
    if (level >= 0) {
        if (level >= (int)b->lv.size()) return CMG_ERR_INVALID_ARG;
        if (n_level) *n_level = b->lv[level].n;
        if (nnz_level) *nnz_level = b->lv[level].nnz;
    }
    return CMG_OK;
}

extern "C" cmg_status_t cmg_batch_stats(cmg_batch_t b, int32_t graph, cmg_stats_t *st) {
    if (!b || !st || graph < 0 || graph >= b->G) return CMG_ERR_INVALID_ARG;
    memset(st, 0, sizeof(*st));
    const int G = b->G, Jq = b->J[graph];
    st->levels = Jq + 1;
    for (int j = 0; j <= Jq; j++) {
        const BLevel &L = b->lv[j];
        st->n[j] = L.hvoff[graph + 1] - L.hvoff[graph];
        st->nnz[j] = L.heoff[graph + 1] - L.heoff[graph];
    }
    if (!b->solved) return CMG_OK;
    bool capped = false;
    for (int j = 0; j <= Jq; j++) {
        st->sweeps[j] = b->h_sweeps[(size_t)j * G + graph];
        st->cos_final[j] = b->h_cos[(size_t)j * G + graph];
        capped = capped || (b->h_flags[(size_t)j * G + graph] & 1);
    }
    st->lambda2 = b->h_lam[graph];
    st->residual = b->h_res[graph];
    st->status = capped ? CMG_WARN_MAXITER : CMG_OK;
    return CMG_OK;
}

extern "C" cmg_status_t cmg_batch_get_aggregates(cmg_batch_t b, int32_t graph, int32_t level,
                                                 int32_t *agg_out) {
    if (!b || !agg_out || graph < 0 || graph >= b->G) return CMG_ERR_INVALID_ARG;
    if (level < 0 || level >= b->J[graph]) return CMG_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    const BLevel &L = b->lv[level];
    const int v0 = L.hvoff[graph], n = L.hvoff[graph + 1] - v0;
    const int c0 = b->lv[level + 1].hvoff[graph];
    CMG_CUDA(cudaMemcpyAsync(agg_out, L.agg + v0, sizeof(int) * n, cudaMemcpyDeviceToHost, b->stream));
    CMG_CUDA(cudaStreamSynchronize(b->stream));
    for (int i = 0; i < n; i++) agg_out[i] -= c0;
    return CMG_OK;
}

extern "C" cmg_status_t cmg_batch_get_level_csr(cmg_batch_t b, int32_t graph, int32_t level,
                                                int64_t *row_ptr, int32_t *col, double *w,
                                                double *g_out) {
    if (!b || graph < 0 || graph >= b->G) return CMG_ERR_INVALID_ARG;
    if (level < 0 || level > b->J[graph]) return CMG_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    const BLevel &L = b->lv[level];
    const int v0 = L.hvoff[graph], n = L.hvoff[graph + 1] - v0;
    const int e0 = L.heoff[graph], m = L.heoff[graph + 1] - e0;
    cudaStream_t s = b->stream;
    std::vector<int> rp(n + 1);
    CMG_CUDA(cudaMemcpyAsync(rp.data(), L.rp + v0, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s));
    if (col && m > 0) CMG_CUDA(cudaMemcpyAsync(col, L.col + e0, sizeof(int) * m, cudaMemcpyDeviceToHost, s));
    if (w && m > 0) CMG_CUDA(cudaMemcpyAsync(w, L.w + e0, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if (row_ptr)
        for (int i = 0; i <= n; i++) row_ptr[i] = rp[i] - e0;
    if (col)
        for (int k = 0; k < m; k++) col[k] -= v0;
    if (g_out) *g_out = L.hg[graph];
    return CMG_OK;
}

extern "C" cmg_status_t cmg_batch_set_replay(cmg_batch_t b, const int32_t *sweeps) {
    if (!b) return CMG_ERR_INVALID_ARG;
    if (b->opts.schedule != CMG_SCHEDULE_REPLAY) return CMG_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    const size_t cnt = (size_t)b->G * CMG_MAX_LEVELS;
    std::vector<int> rep(cnt);
    for (size_t k = 0; k < cnt; k++)
        rep[k] = sweeps ? sweeps[k] : b->opts.replay_sweeps[k % CMG_MAX_LEVELS];
    for (int v : rep)
        if (v < 0) return CMG_ERR_INVALID_ARG;
    CMG_CUDA(cudaMemcpyAsync(b->replay, rep.data(), sizeof(int) * cnt, cudaMemcpyHostToDevice, b->stream));
    CMG_CUDA(cudaStreamSynchronize(b->stream));
    return CMG_OK;
}

extern "C" cmg_status_t cmg_batch_config(cmg_batch_t b, int32_t level, int32_t set,
                                         cmg_batch_shape_t *shape) {
    if (!b || !shape || level < 0 || level >= (int)b->lv.size()) return CMG_ERR_INVALID_ARG;
    if (!set) {
        *shape = b->lv[level].shape;
        return CMG_OK;
    }
    if (!shape_valid(*shape)) return CMG_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    const cmg_batch_shape_t old = b->lv[level].shape;
    b->lv[level].shape = *shape;
    cmg_status_t st = level_workspace(b, level, b->stream);
    if (st == CMG_OK) {
        // the shape must be launchable
        const int fp32 = level_fp32(b, level);
        int per_sm = 0;
        const cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, (const void *)batch_kernel(fp32, b->lv[level].lay.col16, shape->lanes_per_row), threads_for_gpc(*shape),
            (size_t)b->lv[level].smem_group * shape->graphs_per_cta);
        if (e != cudaSuccess || per_sm < 1) st = CMG_ERR_INVALID_ARG;
    }
    if (st != CMG_OK) {
        b->lv[level].shape = old;
        level_workspace(b, level, b->stream);
        return st;
    }
    drop_graph(b);
    return CMG_OK;
}

// Autotuning replays every graph's real sweep counts, scaled down by
// kTuneScale, so a candidate shape is timed on the level's real mix of long
// and short sweep chains (the slowest graphs decide a level's time).
constexpr int kTuneScale = 8;

extern "C" cmg_status_t cmg_batch_autotune(cmg_batch_t b, void *stream) {
    if (!b) return CMG_ERR_INVALID_ARG;
    DeviceGuard dg(b->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int L = (int)b->lv.size(), G = b->G;
    // 1. one solve with the current shapes gives the sweep counts
    CMG_CUDA(cudaMemsetAsync(b->queue, 0, sizeof(int) * 2 * L, s));
    for (int j = L - 1; j >= 0; j--) {
        bool ordered = false;
        CMG_TRY(order_level(b, j, s, &ordered));
        CMG_TRY(launch_level(b, j, -1, s, ordered));
    }
    std::vector<int> sw((size_t)L * G);
    CMG_CUDA(cudaMemcpyAsync(sw.data(), b->sweeps, sizeof(int) * sw.size(), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    std::vector<int> rep((size_t)G * CMG_MAX_LEVELS, 1);
    for (int q = 0; q < G; q++)
        for (int j = 0; j <= b->J[q] && j < CMG_MAX_LEVELS; j++)
            rep[(size_t)q * CMG_MAX_LEVELS + j] = std::max(1, (sw[(size_t)j * G + q] + kTuneScale - 1) / kTuneScale);
    CMG_TRY(dev_alloc_n(&b->tune_replay, rep.size(), s));
    CMG_CUDA(cudaMemcpyAsync(b->tune_replay, rep.data(), sizeof(int) * rep.size(), cudaMemcpyHostToDevice, s));
    cudaEvent_t e0, e1;
    CMG_CUDA(cudaEventCreate(&e0));
    CMG_CUDA(cudaEventCreate(&e1));
    cmg_status_t st = CMG_OK;
    // 2. per level, coarse to fine (a level's order uses the replayed counts
    // of the level below it), time the candidate shapes
    auto time_shape = [&](int j, const cmg_batch_shape_t &sh, float *ms) -> cmg_status_t {
        BLevel &V = b->lv[j];
        V.shape = sh;
        CMG_TRY(level_workspace(b, j, s));
        int per_sm = 0;
        CMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, (const void *)batch_kernel(level_fp32(b, j), V.lay.col16, sh.lanes_per_row), threads_for_gpc(sh),
            (size_t)V.smem_group * sh.graphs_per_cta));
        if (per_sm < 1) {
            *ms = 1e30f;
            return CMG_OK;
        }
        CMG_CUDA(cudaMemsetAsync(b->queue + 2 * j, 0, 2 * sizeof(int), s));
        CMG_CUDA(cudaEventRecord(e0, s));
        bool ordered = false;
        CMG_TRY(order_level(b, j, s, &ordered));
        CMG_TRY(launch_level(b, j, -1, s, ordered));
        CMG_CUDA(cudaEventRecord(e1, s));
        CMG_CUDA(cudaEventSynchronize(e1));
        CMG_CUDA(cudaEventElapsedTime(ms, e0, e1));
        return CMG_OK;
    };
    for (int j = L - 1; j >= 0 && st == CMG_OK; j--) {
        if (b->lv[j].count == 0) continue;
        cmg_batch_shape_t best = b->lv[j].shape;
        float best_ms = 1e30f;
        auto consider = [&](cmg_batch_shape_t sh) -> cmg_status_t {
            if (!shape_valid(sh)) return CMG_OK;
            float ms = 0.f;
            CMG_TRY(time_shape(j, sh, &ms));
            if (ms < best_ms) {
                best_ms = ms;
                best = sh;
            }
            return CMG_OK;
        };
        // threads per graph x graphs per CTA, then lanes per heavy row, then staging
        const int lanes0 = best.lanes_per_row;
        for (int tpg : {32, 64, 128, 256, 512})
            for (int cta : {256, 512, 1024}) {
                if (tpg > cta || st != CMG_OK) continue;
                st = consider(cmg_batch_shape_t{tpg, lanes0, std::max(1, cta / tpg), 1});
            }
        for (int lpr : {1, 4, 16, 32}) {
            if (st != CMG_OK) break;
            cmg_batch_shape_t sh = best;
            sh.lanes_per_row = lpr;
            st = consider(sh);
        }
        if (st == CMG_OK) {
            cmg_batch_shape_t sh = best;
            sh.stage_csr = 1 - sh.stage_csr;
            st = consider(sh);
        }
        b->lv[j].shape = best;
        if (st == CMG_OK) st = level_workspace(b, j, s);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    dev_free(b->tune_replay, s);
    b->tune_replay = nullptr;
    drop_graph(b);
    return st;
}

extern "C" cmg_status_t cmg_batch_level_ms(cmg_batch_t b, int32_t level, double *ms) {
    if (!b || !ms || level < 0 || level >= (int)b->lv.size()) return CMG_ERR_INVALID_ARG;
    *ms = level < (int)b->level_ms.size() ? b->level_ms[level] : 0.0;
    return CMG_OK;
}

extern "C" cmg_status_t cmg_batch_device_bytes(cmg_batch_t b, size_t *bytes) {
    if (!b || !bytes) return CMG_ERR_INVALID_ARG;
    *bytes = b->bytes;
    return CMG_OK;
}

extern "C" cmg_status_t cmg_batch_free(cmg_batch_t b) {
    if (!b) return CMG_ERR_INVALID_ARG;
    free_batch(b);
    return CMG_OK;
}
