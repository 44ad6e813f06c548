// hec.cu -- heavy edge coarsening (Alg. 2 of arXiv 1412.0565) as data-parallel
// kernels.
//
// Alg. 2 visits the vertices in the order p = randperm(n); an unmapped vertex
// v joins the aggregate of its heaviest neighbour m(v) or, if m(v) is still
// unmapped, opens a new aggregate {v, m(v)}.  The sequential loop is replaced
// by an exact characterisation that depends only on ranks r = p^{-1}:
//
//   active(v)  <=>  no active u with m(u) = v and r(u) < r(v)
//               (v is still unmapped when its turn comes; "passive" otherwise)
//   creator(u) <=>  active(u), r(m(u)) > r(u) and u is the lowest-ranked
//                   active vertex with m(.) = m(u)
//   label:  creators are numbered 0..c-1 in rank order; a passive vertex takes
//           the label of its lowest-ranked active in-neighbour (a creator); a
//           non-creator active u takes the label of m(u), found by walking
//           v -> m(v) through non-creator actives (ranks strictly decrease
//           along that walk, so it ends).
//
// active/passive is a fixed point resolved in rounds: a vertex decides once
// every lower-ranked in-neighbour has decided.  Each round decides at least
// the lowest-ranked undecided vertex, so at most n rounds are needed; random
// ranks make the count small (4-8 on the graphs measured).
#include <algorithm>

#include "internal.h"

namespace cmg {

// splitmix64: one output of the SplitMix64 generator (Steele, Lea, Flood 2014)
// from state x -- the state is advanced by the golden gamma and mixed.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Visit rank of vertex v: 4-round balanced Feistel network on k-bit words
// (k the smallest even number >= 2 with 2^k >= n), round t maps (L, R) to
// (R, L ^ F_t(R)) with F_t(R) = splitmix64(R ^ K_t) restricted to k/2 bits and
// K_t = splitmix64(seed ^ level * 0x9E3779B97F4A7C15 ^ t); values >= n are
// walked through the permutation again until they land in [0, n).
__device__ __forceinline__ uint32_t feistel_rank(uint32_t v, uint32_t n, int half,
                                                 const uint64_t (&key)[4]) {
    const uint64_t mask = (1ull << half) - 1ull;
    uint64_t x = v;
    do {
        uint64_t L = x >> half, R = x & mask;
#pragma unroll
        for (int t = 0; t < 4; t++) {
            uint64_t F = splitmix64(R ^ key[t]) & mask;
            uint64_t nr = L ^ F;
            L = R;
            R = nr;
        }
        x = (L << half) | R;
    } while (x >= n);
    return (uint32_t)x;
}

__global__ void k_ranks(int n, uint64_t seed, int level, uint32_t *__restrict__ r) {
    int k = 2;
    while ((1ll << k) < (long long)n) k += 2;
    uint64_t key[4];
#pragma unroll
    for (int t = 0; t < 4; t++)
        key[t] = splitmix64(seed ^ ((uint64_t)(int64_t)level * 0x9E3779B97F4A7C15ull) ^ (uint64_t)t);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        r[v] = feistel_rank((uint32_t)v, (uint32_t)n, k / 2, key);
}

// Ranks of a block-diagonal union of graphs (vertex offsets voff[0..G]):
// vertex v of graph q gets voff[q] + (its rank within graph q, level `level`).
// Rank space is then graph-major, so HEC on the union numbers each graph's
// aggregates contiguously and in that graph's own creator order.
__global__ void k_ranks_batch(int n, int G, const int *__restrict__ voff, uint64_t seed, int level,
                              uint32_t *__restrict__ r) {
    uint64_t key[4];
#pragma unroll
    for (int t = 0; t < 4; t++)
        key[t] = splitmix64(seed ^ ((uint64_t)(int64_t)level * 0x9E3779B97F4A7C15ull) ^ (uint64_t)t);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int lo = 0, hi = G - 1;   // last q with voff[q] <= v
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(voff + mid) <= v) lo = mid;
            else hi = mid - 1;
        }
        const int v0 = __ldg(voff + lo);
        const int ng = __ldg(voff + lo + 1) - v0;
        int k = 2;
        while ((1ll << k) < (long long)ng) k += 2;
        r[v] = (uint32_t)v0 + feistel_rank((uint32_t)(v - v0), (uint32_t)ng, k / 2, key);
    }
}

// Heaviest neighbour, G lanes per row: strict '>' on the weight, ties to the
// lowest column (Alg. 2's argmin of the column of L).  -1 for an empty row.
template <int G>
__global__ void k_heaviest(int n, const int *__restrict__ rp, const int *__restrict__ col,
                           const double *__restrict__ w, int *__restrict__ m) {
    const int lane = threadIdx.x & (G - 1);
    const int groups_per_grid = (gridDim.x * blockDim.x) / G;
    for (int base = (blockIdx.x * blockDim.x + threadIdx.x) / G;; base += groups_per_grid) {
        // all lanes of a warp iterate together so the shuffles stay converged
        int warp_first = __shfl_sync(0xffffffffu, base, 0);
        if (warp_first >= n) break;
        const int row = base;
        double bw = -1.0;
        int bj = 0x7fffffff;
        if (row < n) {
            const int e1 = __ldg(rp + row + 1);
            for (int e = __ldg(rp + row) + lane; e < e1; e += G) {
                const double x = __ldg(w + e);
                const int j = __ldg(col + e);
                if (x > bw || (x == bw && j < bj)) {
                    bw = x;
                    bj = j;
                }
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
            const double ow = __shfl_xor_sync(0xffffffffu, bw, o);
            const int oj = __shfl_xor_sync(0xffffffffu, bj, o);
            if (ow > bw || (ow == bw && oj < bj)) {
                bw = ow;
                bj = oj;
            }
        }
        if (row < n && lane == 0) m[row] = (bw < 0.0) ? -1 : bj;
    }
}

int lanes_for_avg(double avg) {
    if (avg <= 2.0) return 2;
    if (avg <= 6.0) return 4;
    if (avg <= 12.0) return 8;
    if (avg <= 24.0) return 16;
    return 32;
}

template <int G>
static cmg_status_t launch_heaviest_g(int n, const int *rp, const int *col, const double *w,
                                      int *m, cudaStream_t s) {
    const int threads = 256;
    const int blocks = grid_for((long long)n * G, threads);
    k_heaviest<G><<<blocks, threads, 0, s>>>(n, rp, col, w, m);
    return launch_status();
}

cmg_status_t launch_heaviest(int n, double avg, const int *rp, const int *col, const double *w,
                             int *m, cudaStream_t s) {
    if (n <= 0) return CMG_OK;
    switch (lanes_for_avg(avg)) {
        case 2: return launch_heaviest_g<2>(n, rp, col, w, m, s);
        case 4: return launch_heaviest_g<4>(n, rp, col, w, m, s);
        case 8: return launch_heaviest_g<8>(n, rp, col, w, m, s);
        case 16: return launch_heaviest_g<16>(n, rp, col, w, m, s);
        default: return launch_heaviest_g<32>(n, rp, col, w, m, s);
    }
}

cmg_status_t launch_ranks(int n, uint64_t seed, int level, uint32_t *r, cudaStream_t s) {
    if (n <= 0) return CMG_OK;
    const int threads = 256;
    k_ranks<<<grid_for(n, threads), threads, 0, s>>>(n, seed, level, r);
    return launch_status();
}

cmg_status_t launch_ranks_batch(int n, int G, const int *voff, uint64_t seed, int level, uint32_t *r,
                                cudaStream_t s) {
    if (n <= 0) return CMG_OK;
    const int threads = 256;
    k_ranks_batch<<<grid_for(n, threads), threads, 0, s>>>(n, G, voff, seed, level, r);
    return launch_status();
}

// ------------------------------------------------------------------ resolution
enum : unsigned char { kUndecided = 0, kActive = 1, kPassive = 2 };
constexpr uint32_t kInf = 0xffffffffu;

__device__ __forceinline__ int block_exclusive_scan(int v, int *sm, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = (lane < nw) ? sm[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sm[lane] = t;
    }
    __syncthreads();
    const int before = (warp > 0) ? sm[warp - 1] : 0;
    *total = sm[nw - 1];
    __syncthreads();
    return before + x - v;
}

struct HecArgs {
    int n;
    const int *m;
    const uint32_t *r;
    unsigned char *state;
    uint32_t *minA;
    uint32_t *minU;
    int *ids;           // int[n]: creator flags by rank, then their exclusive scan
    int *cta_tot;       // int[gridDim.x]
    int *undecided;     // int[3], a ring of per-round counters (zeroed)
    int max_rounds;
    int *agg;
    int *c_out;         // device int
    int *rounds_out;    // device int
};

__device__ __forceinline__ bool is_creator(const HecArgs &a, int u) {
    if (a.state[u] != kActive) return false;
    const int mu = a.m[u];
    if (mu < 0) return true;  // a vertex without neighbours is its own aggregate
    const uint32_t ru = a.r[u];
    return a.r[mu] > ru && a.minA[mu] == ru;
}

// One cooperative launch performs the whole resolution and labelling.
__global__ void k_hec_resolve(HecArgs a, GridSync *gs) {
    __shared__ int sm_scan[32];
    __shared__ int sm_red[32];
    const int n = a.n;
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nth = gridDim.x * blockDim.x;

    for (int v = tid; v < n; v += nth) {
        a.state[v] = kUndecided;
        a.minA[v] = kInf;
        a.minU[v] = kInf;
    }
    if (!grid_sync(gs)) return;

    int rounds = 0;
    for (int round = 0; round < a.max_rounds; round++) {
        rounds = round + 1;
        // the counter slot of the next round was last read two barriers ago
        if (tid == 0) a.undecided[(round + 1) % 3] = 0;
        // push: every active / undecided vertex reports its rank to m(v)
        for (int v = tid; v < n; v += nth) {
            const unsigned char s = a.state[v];
            const int mv = a.m[v];
            if (mv < 0) continue;
            if (s == kActive) atomicMin(&a.minA[mv], a.r[v]);
            else if (s == kUndecided) atomicMin(&a.minU[mv], a.r[v]);
        }
        if (!grid_sync(gs)) return;
        // decide
        int und = 0;
        for (int v = tid; v < n; v += nth) {
            const unsigned char s = a.state[v];
            const uint32_t mu = a.minU[v];
            a.minU[v] = kInf;
            if (s != kUndecided) continue;
            const uint32_t rv = a.r[v];
            if (a.minA[v] < rv) a.state[v] = kPassive;
            else if (mu > rv) a.state[v] = kActive;
            else und++;
        }
        und = warp_sum_int(und);
        if ((threadIdx.x & 31) == 0) sm_red[threadIdx.x >> 5] = und;
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int i = 0; i < (int)(blockDim.x + 31) / 32; i++) t += sm_red[i];
            if (t) atomicAdd(&a.undecided[round % 3], t);
        }
        if (!grid_sync(gs)) return;
        if (*((volatile int *)&a.undecided[round % 3]) == 0) break;
    }

    // minA over all active in-neighbours
    for (int v = tid; v < n; v += nth) a.minA[v] = kInf;
    if (!grid_sync(gs)) return;
    for (int v = tid; v < n; v += nth) {
        const int mv = a.m[v];
        if (mv >= 0 && a.state[v] == kActive) atomicMin(&a.minA[mv], a.r[v]);
    }
    if (!grid_sync(gs)) return;
    // creator flags, indexed by rank
    for (int v = tid; v < n; v += nth) a.ids[a.r[v]] = is_creator(a, v) ? 1 : 0;
    if (!grid_sync(gs)) return;

    // exclusive scan of the flags in rank order: contiguous chunk per CTA
    const int chunk = (n + gridDim.x - 1) / gridDim.x;
    const int lo = min(n, blockIdx.x * chunk), hi = min(n, lo + chunk);
    int cnt = 0;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) cnt += a.ids[i];
    cnt = warp_sum_int(cnt);
    if ((threadIdx.x & 31) == 0) sm_red[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < (int)(blockDim.x + 31) / 32; i++) t += sm_red[i];
        a.cta_tot[blockIdx.x] = t;
    }
    if (!grid_sync(gs)) return;
    __shared__ int s_base;
    if (threadIdx.x == 0) {
        int b = 0;
        for (int i = 0; i < (int)blockIdx.x; i++) b += a.cta_tot[i];
        s_base = b;
        if (blockIdx.x == gridDim.x - 1) {
            *a.c_out = b + a.cta_tot[blockIdx.x];
            *a.rounds_out = rounds;
        }
    }
    __syncthreads();
    int run = s_base;
    for (int t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int i = t0 + threadIdx.x;
        const int f = (i < hi) ? a.ids[i] : 0;
        int tot;
        const int ex = block_exclusive_scan(f, sm_scan, &tot);
        if (i < hi) a.ids[i] = run + ex;
        run += tot;
    }
    if (!grid_sync(gs)) return;

    // labels
    for (int v = tid; v < n; v += nth) {
        const unsigned char s = a.state[v];
        int lab;
        if (s == kPassive) {
            lab = a.ids[a.minA[v]];
        } else if (is_creator(a, v)) {
            lab = a.ids[a.r[v]];
        } else {
            int x = a.m[v];
            lab = -1;
            for (int step = 0; step < n; step++) {
                if (a.state[x] == kPassive) {
                    lab = a.ids[a.minA[x]];
                    break;
                }
                if (is_creator(a, x)) {
                    lab = a.ids[a.r[x]];
                    break;
                }
                x = a.m[x];
            }
        }
        a.agg[v] = lab;
    }
}

cmg_status_t hec_level_async(int n, long long nnz, const int *rp, const int *col, const double *w,
                             uint64_t seed, int level, const uint32_t *rank, int *agg_out,
                             int *c_dev, GridSync *gs, cudaStream_t s) {
    Scratch scr(s);
    int *m;
    uint32_t *r, *minA, *minU;
    unsigned char *state;
    int *ids, *cta_tot, *undecided, *rounds;
    // every round decides at least the lowest-ranked undecided vertex
    const int max_rounds = n + 1;
    CMG_TRY(scr.get(&m, n));
    CMG_TRY(scr.get(&minA, n));
    CMG_TRY(scr.get(&minU, n));
    CMG_TRY(scr.get(&state, n));
    CMG_TRY(scr.get(&ids, n));
    CMG_TRY(scr.get(&undecided, 3));
    CMG_TRY(scr.get(&rounds, 1));
    if (!rank) {
        CMG_TRY(scr.get(&r, n));
        CMG_TRY(launch_ranks(n, seed, level, r, s));
    } else {
        r = const_cast<uint32_t *>(rank);
    }
    CMG_TRY(launch_heaviest(n, (double)nnz / (double)n, rp, col, w, m, s));

    const int threads = 512;
    int maxb = 0;
    CMG_TRY(coop_max_blocks((const void *)k_hec_resolve, threads, 0, &maxb));
    DeviceInfo di;
    CMG_TRY(device_info(&di));
    int blocks = std::max(1, std::min(std::min(maxb, 2 * di.sms), div_up(n, threads * 2)));
    CMG_TRY(scr.get(&cta_tot, blocks));
    CMG_CUDA(cudaMemsetAsync(undecided, 0, sizeof(int) * 3, s));
    HecArgs a;
    a.n = n;
    a.m = m;
    a.r = r;
    a.state = state;
    a.minA = minA;
    a.minU = minU;
    a.ids = ids;
    a.cta_tot = cta_tot;
    a.undecided = undecided;
    a.max_rounds = max_rounds;
    a.agg = agg_out;
    a.c_out = c_dev;
    a.rounds_out = rounds;
    void *args[] = {&a, &gs};
    return coop_launch((const void *)k_hec_resolve, blocks, threads, 0, s, args, gs);
}

cmg_status_t hec_level(int n, long long nnz, const int *rp, const int *col, const double *w,
                       uint64_t seed, int level, const uint32_t *rank, int *agg_out, int *c_host,
                       cudaStream_t s) {
    Scratch scr(s);
    int *c_dev;
    GridSync *gs;
    CMG_TRY(scr.get(&c_dev, 1));
    CMG_TRY(scr.get(&gs, 1));
    CMG_TRY(gs_clear(gs, s));
    CMG_TRY(hec_level_async(n, nnz, rp, col, w, seed, level, rank, agg_out, c_dev, gs, s));
    int c = 0;
    GridSync hgs;
    CMG_CUDA(cudaMemcpyAsync(&c, c_dev, sizeof(int), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(&hgs, gs, sizeof(GridSync), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if (hgs.err) return CMG_ERR_DEVICE_TIMEOUT;
    *c_host = c;
    return CMG_OK;
}

}  // namespace cmg
