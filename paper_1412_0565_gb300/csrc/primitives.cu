// primitives.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Both are written for this library (no CUB/Thrust): the Galerkin product
// needs a stable key sort so that every coarse weight is summed in the fine
// (i, j) order, and several steps need an exclusive scan.
#include <algorithm>

#include "internal.h"

namespace cmg {

// ------------------------------------------------------------------ scan
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int block_scan_excl(int v, int *sm, int *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
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

__global__ void k_scan_reduce(const int *__restrict__ in, int n, int *__restrict__ part) {
    __shared__ int sm[32];
    const long long base = (long long)blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        long long i = base + (long long)threadIdx.x * kScanItems + k;
        if (i < n) s += in[i];
    }
    s = warp_sum_int(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < kScanThreads / 32; i++) t += sm[i];
        part[blockIdx.x] = t;
    }
}

// One CTA: exclusive scan of part[0..m) in place; part[m] = total.
__global__ void k_scan_partials(int *part, int m) {
    __shared__ int sm[32];
    int run = 0;
    for (int t0 = 0; t0 < m; t0 += blockDim.x) {
        const int i = t0 + threadIdx.x;
        const int v = (i < m) ? part[i] : 0;
        int tot;
        const int ex = block_scan_excl(v, sm, &tot);
        if (i < m) part[i] = run + ex;
        run += tot;
    }
    if (threadIdx.x == 0) part[m] = run;
}

__global__ void k_scan_down(const int *__restrict__ in, int *__restrict__ out, int n,
                            const int *__restrict__ part) {
    __shared__ int sm[32];
    const long long base = (long long)blockIdx.x * kScanTile;
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        long long i = base + (long long)threadIdx.x * kScanItems + k;
        v[k] = (i < n) ? in[i] : 0;
        s += v[k];
    }
    int tot;
    int run = block_scan_excl(s, sm, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
        long long i = base + (long long)threadIdx.x * kScanItems + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == blockDim.x - 1) out[n] = run;
}

// One CTA of 1024 threads, 8 consecutive items each: the whole scan of up to
// kScanSmall items in one launch (setup scans many short arrays, where the
// three launches of the tiled scan cost more than the work).
constexpr int kScanSmall = 8192;
__global__ void __launch_bounds__(1024) k_scan_small(const int *__restrict__ in, int *__restrict__ out, int n) {
    __shared__ int sm[32];
    int v[8];
    int t = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int i = threadIdx.x * 8 + k;
        v[k] = (i < n) ? in[i] : 0;
        t += v[k];
    }
    int tot;
    int run = block_scan_excl(t, sm, &tot);
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int i = threadIdx.x * 8 + k;
        if (i < n) out[i] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) out[n] = tot;
}

cmg_status_t exclusive_scan(const int *in, int *out, int n, Scratch &scr, cudaStream_t s) {
    if (n <= 0) {
        CMG_CUDA(cudaMemsetAsync(out, 0, sizeof(int), s));
        return CMG_OK;
    }
    if (n <= kScanSmall) {
        k_scan_small<<<1, 1024, 0, s>>>(in, out, n);
        return launch_status();
    }
    const int nb = div_up(n, kScanTile);
    int *part;
    CMG_TRY(scr.get(&part, (size_t)nb + 1));
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(in, n, part);
    CMG_TRY(launch_status());
    k_scan_partials<<<1, 1024, 0, s>>>(part, nb);
    CMG_TRY(launch_status());
    k_scan_down<<<nb, kScanThreads, 0, s>>>(in, out, n, part);
    return launch_status();
}

// ------------------------------------------------------------------ radix sort
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortRounds = 16;
constexpr int kSortTile = kSortThreads * kSortRounds;
constexpr int kSortWarps = kSortThreads / 32;

// Per-tile digit histogram, stored digit-major: hist[d * ntiles + tile].
// The item count is read from device memory (tiles past it count nothing).
__global__ void k_radix_hist(const uint64_t *__restrict__ keys, const int *__restrict__ count_dev,
                             int shift, int *__restrict__ hist) {
    const int count = *count_dev;
    __shared__ int h[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) h[d] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
    for (int k = 0; k < kSortRounds; k++) {
        const long long i = base + (long long)k * kSortThreads + threadIdx.x;
        if (i < count) atomicAdd(&h[(int)((keys[i] >> shift) & (kRadix - 1))], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x)
        hist[(long long)d * gridDim.x + blockIdx.x] = h[d];
}

// Stable scatter: items of a tile are ranked in (round, warp, lane) order,
// which is their input order.
__global__ void k_radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                                uint64_t *__restrict__ kout, uint32_t *__restrict__ vout,
                                const int *__restrict__ count_dev, int shift,
                                const int *__restrict__ offs) {
    const int count = *count_dev;
    __shared__ int running[kRadix];
    __shared__ int cnt[kSortWarps][kRadix];
    __shared__ int pre[kSortWarps][kRadix];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
        running[d] = offs[(long long)d * gridDim.x + blockIdx.x];
        for (int w = 0; w < kSortWarps; w++) cnt[w][d] = 0;
    }
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * kSortTile;
    for (int k = 0; k < kSortRounds; k++) {
        const long long i = base + (long long)k * kSortThreads + threadIdx.x;
        const bool valid = i < count;
        uint64_t key = 0;
        uint32_t val = 0;
        int digit = kRadix;  // sentinel for missing items
        if (valid) {
            key = kin[i];
            val = vin[i];
            digit = (int)((key >> shift) & (kRadix - 1));
        }
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const int rank = __popc(peers & lt_mask);
        if (valid && rank == 0) cnt[warp][digit] = __popc(peers);
        __syncthreads();
        for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
            int r = running[d];
            for (int w = 0; w < kSortWarps; w++) {
                const int c = cnt[w][d];
                pre[w][d] = r;
                r += c;
                cnt[w][d] = 0;
            }
            running[d] = r;
        }
        __syncthreads();
        if (valid) {
            const int pos = pre[warp][digit] + rank;
            kout[pos] = key;
            vout[pos] = val;
        }
    }
}

cmg_status_t radix_sort_pairs(uint64_t **keys, uint32_t **vals, uint64_t *keys_alt,
                              uint32_t *vals_alt, int cap, const int *count_dev, int bits,
                              Scratch &scr, cudaStream_t s) {
    if (cap <= 1 || bits <= 0) return CMG_OK;
    const int ntiles = div_up(cap, kSortTile);
    int *hist, *offs;
    CMG_TRY(scr.get(&hist, (size_t)kRadix * ntiles));
    CMG_TRY(scr.get(&offs, (size_t)kRadix * ntiles + 1));
    uint64_t *ka = *keys, *kb = keys_alt;
    uint32_t *va = *vals, *vb = vals_alt;
    for (int shift = 0; shift < bits; shift += kRadixBits) {
        k_radix_hist<<<ntiles, kSortThreads, 0, s>>>(ka, count_dev, shift, hist);
        CMG_TRY(launch_status());
        CMG_TRY(exclusive_scan(hist, offs, kRadix * ntiles, scr, s));
        k_radix_scatter<<<ntiles, kSortThreads, 0, s>>>(ka, va, kb, vb, count_dev, shift, offs);
        CMG_TRY(launch_status());
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    *keys = ka;
    *vals = va;
    return CMG_OK;
}

}  // namespace cmg
