// galerkin.cu -- Galerkin coarse Laplacian L^{i+1} = I L I^T (Sec. 2, Step 1 of
// arXiv 1412.0565) by key sort and segmented sum.
//
// For aggregates a != b the coarse weight is w_ab = sum of w_ij over fine
// pairs i in a, j in b; pairs inside one aggregate drop out, and the coarse
// diagonal (coarse degree) is the row sum, so coarse rows sum to zero
// exactly (Proposition 2.7).  Summation order (for bitwise reproducible and
// bitwise symmetric coarse weights): every fine entry (i, j) with
// agg(i) < agg(j) is visited in CSR order and emitted twice, as record
// (a, b) and as record (b, a), both carrying the fine entry index e.  The two
// record streams are laid out one after the other, each in e order, so a
// stable sort by key leaves every (a, b) group in ascending (i, j) order; each
// group is then summed left to right.  w_ab and w_ba are therefore the same
// sum of the same terms in the same order, and the sorted keys are already
// the coarse CSR (rows ascending, columns ascending).
#include <algorithm>

#include "internal.h"

namespace cmg {

// Every kernel below reads the sizes it depends on (aggregate count c,
// cross-entry count, coarse nnz) from device memory, so the product runs
// without host synchronisation; grids are sized by upper bounds (c <= n,
// records <= nnz).

__global__ void k_count_cross(int n, const int *__restrict__ rp, const int *__restrict__ col,
                              const int *__restrict__ agg, int *__restrict__ cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int a = agg[i];
        int c = 0;
        for (int e = __ldg(rp + i), e1 = __ldg(rp + i + 1); e < e1; e++) c += (a < agg[__ldg(col + e)]);
        cnt[i] = c;
    }
}

// off[n] holds the cross-entry count; records (a, b) go to [0, ncross),
// records (b, a) to [ncross, 2 ncross).
__global__ void k_emit(int n, const int *__restrict__ rp, const int *__restrict__ col,
                       const int *__restrict__ agg, const int *__restrict__ off, int bb,
                       uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
                       LevelCounts *__restrict__ cnt) {
    const long long ncross = off[n];
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt->m = (int)(2 * ncross);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t a = (uint64_t)agg[i];
        long long k = off[i];
        for (int e = __ldg(rp + i), e1 = __ldg(rp + i + 1); e < e1; e++) {
            const uint64_t b = (uint64_t)agg[__ldg(col + e)];
            if (a < b) {
                keys[k] = (a << bb) | b;
                vals[k] = (uint32_t)e;
                keys[ncross + k] = (b << bb) | a;
                vals[ncross + k] = (uint32_t)e;
                k++;
            }
        }
    }
}

// head[k] = 1 where a group of equal keys starts, 0 elsewhere (and past m).
__global__ void k_heads(long long cap, const uint64_t *__restrict__ keys,
                        const LevelCounts *__restrict__ cnt, int *__restrict__ head) {
    const long long m = cnt->m;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < cap;
         k += (long long)gridDim.x * blockDim.x)
        head[k] = (k < m && (k == 0 || keys[k] != keys[k - 1])) ? 1 : 0;
}

// One thread per segment (group of equal keys): left-to-right FP64 sum.
__global__ void k_segsum(long long cap, const uint64_t *__restrict__ keys,
                         const uint32_t *__restrict__ vals, const int *__restrict__ head,
                         const int *__restrict__ segid, const double *__restrict__ w, int bb,
                         const LevelCounts *__restrict__ cnt, int *__restrict__ col_c,
                         double *__restrict__ w_c, int *__restrict__ row_of) {
    const long long m = cnt->m;
    const uint64_t mask = (1ull << bb) - 1ull;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x) {
        if (!head[k]) continue;
        const uint64_t key = keys[k];
        double acc = 0.0;
        long long t = k;
        do {
            acc += __ldg(w + vals[t]);
            t++;
        } while (t < m && keys[t] == key);
        const int s = segid[k];
        col_c[s] = (int)(key & mask);
        w_c[s] = acc;
        row_of[s] = (int)(key >> bb);
    }
}

// Coarse row pointers from the (row-sorted) segment rows; segid[cap] holds
// the segment count, which is also recorded as the coarse nnz.
__global__ void k_rowptr(long long cap, const int *__restrict__ segid,
                         const int *__restrict__ row_of, LevelCounts *__restrict__ cnt,
                         int *__restrict__ rp_c) {
    const int nseg = segid[cap];
    const int c = cnt->c;
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt->nseg = nseg;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s <= nseg; s += gridDim.x * blockDim.x) {
        const int lo = (s == 0) ? -1 : row_of[s - 1];
        const int hi = (s == nseg) ? c : row_of[s];
        for (int r = lo + 1; r <= hi; r++) rp_c[r] = s;
    }
}

// g = max_i (d_i + d_i), d_i = sum_j w_ij left to right (Alg. 3, first line).
// The row count is n_dev[0] when n_dev is given, else n.
__global__ void k_gershgorin(int n, const int *__restrict__ n_dev, const int *__restrict__ rp,
                             const double *__restrict__ w, unsigned long long *__restrict__ gbits) {
    if (n_dev) n = *n_dev;
    double best = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int e = __ldg(rp + i), e1 = __ldg(rp + i + 1); e < e1; e++) d += __ldg(w + e);
        best = fmax(best, d + d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
    // non-negative doubles order like their bit patterns
    if ((threadIdx.x & 31) == 0) atomicMax(gbits, (unsigned long long)__double_as_longlong(best));
}

cmg_status_t launch_gershgorin(int n, const int *rp, const double *w, double *g_dev,
                               cudaStream_t s) {
    CMG_CUDA(cudaMemsetAsync(g_dev, 0, sizeof(double), s));
    const int threads = 256;
    k_gershgorin<<<grid_for(n, threads, 4), threads, 0, s>>>(
        n, nullptr, rp, w, reinterpret_cast<unsigned long long *>(g_dev));
    return launch_status();
}

cmg_status_t galerkin_async(int n, long long nnz, const int *rp, const int *col, const double *w,
                            const int *agg, int key_bits, LevelCounts *cnt, int *rp_c, int *col_c,
                            double *w_c, cudaStream_t s) {
    Scratch scr(s);
    const int threads = 256;
    // every cross pair {i, j} is stored twice in a symmetric CSR and counted
    // once (agg(i) < agg(j)), so the record count 2 ncross is at most nnz
    const long long cap = std::max<long long>(nnz, 1);
    int *ccount, *off;
    CMG_TRY(scr.get(&ccount, n));
    CMG_TRY(scr.get(&off, (size_t)n + 1));
    k_count_cross<<<grid_for(n, threads), threads, 0, s>>>(n, rp, col, agg, ccount);
    CMG_TRY(launch_status());
    CMG_TRY(exclusive_scan(ccount, off, n, scr, s));
    uint64_t *ka, *kb;
    uint32_t *va, *vb;
    CMG_TRY(scr.get(&ka, (size_t)cap));
    CMG_TRY(scr.get(&kb, (size_t)cap));
    CMG_TRY(scr.get(&va, (size_t)cap));
    CMG_TRY(scr.get(&vb, (size_t)cap));
    k_emit<<<grid_for(n, threads), threads, 0, s>>>(n, rp, col, agg, off, key_bits, ka, va, cnt);
    CMG_TRY(launch_status());
    CMG_TRY(radix_sort_pairs(&ka, &va, kb, vb, (int)cap, &cnt->m, 2 * key_bits, scr, s));
    int *head, *segid, *row_of;
    CMG_TRY(scr.get(&head, (size_t)cap));
    CMG_TRY(scr.get(&segid, (size_t)cap + 1));
    CMG_TRY(scr.get(&row_of, (size_t)cap));
    k_heads<<<grid_for(cap, threads), threads, 0, s>>>(cap, ka, cnt, head);
    CMG_TRY(launch_status());
    CMG_TRY(exclusive_scan(head, segid, (int)cap, scr, s));
    k_segsum<<<grid_for(cap, threads), threads, 0, s>>>(cap, ka, va, head, segid, w, key_bits, cnt,
                                                        col_c, w_c, row_of);
    CMG_TRY(launch_status());
    k_rowptr<<<grid_for(cap + 1, threads), threads, 0, s>>>(cap, segid, row_of, cnt, rp_c);
    CMG_TRY(launch_status());
    CMG_CUDA(cudaMemsetAsync(&cnt->gbits, 0, sizeof(cnt->gbits), s));
    k_gershgorin<<<grid_for(n, threads, 4), threads, 0, s>>>(n, &cnt->c, rp_c, w_c, &cnt->gbits);
    return launch_status();
}

}  // namespace cmg
