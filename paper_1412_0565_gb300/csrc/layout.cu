// layout.cu -- the sweep layout of a level (or of every graph of a union
// level), used by the power-iteration kernels that read slices.
//
// The layout itself is described with SweepLayout in internal.h.  It is
// built with one stable radix sort of the rows by (graph, decreasing degree),
// per-graph counts and scans, and one fill pass over the renumbered rows.
#include <algorithm>

#include "internal.h"

namespace cmg {

// ------------------------------------------------------------------ layout kernels
// largest row length of the level
__global__ void k_max_degree(int n, const int *__restrict__ rp, int *__restrict__ out) {
    int m = 0;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        m = max(m, rp[v + 1] - rp[v]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// keys (graph, decreasing degree) of every union vertex, for a stable sort;
// the degree field holds maxdeg - degree in db bits
__global__ void k_layout_keys(int n, int G, const int *__restrict__ voff, const int *__restrict__ rp,
                              int maxdeg, int db, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int lo = 0, hi = G - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (voff[mid] <= v) lo = mid;
            else hi = mid - 1;
        }
        const uint32_t deg = (uint32_t)(rp[v + 1] - rp[v]);
        keys[v] = ((uint64_t)lo << db) | (uint64_t)(maxdeg - deg);
        vals[v] = (uint32_t)v;
    }
}

__global__ void k_layout_inv(int n, const uint32_t *__restrict__ perm, int *__restrict__ inv) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x)
        inv[perm[p]] = p;
}

__device__ __forceinline__ int perm_deg(const int *rp, const uint32_t *perm, int p) {
    const int v = (int)perm[p];
    return rp[v + 1] - rp[v];
}

// Per graph (one thread): the heavy rows are a prefix of the renumbered rows
// (decreasing degree), found by binary search; mcnt = h + nsl + 1 meta words.
__global__ void k_layout_heavy(int G, const int *__restrict__ voff, const int *__restrict__ rp,
                               const uint32_t *__restrict__ perm, int *__restrict__ heavy,
                               int *__restrict__ mcnt) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < G; q += gridDim.x * blockDim.x) {
        const int v0 = voff[q], n = voff[q + 1] - v0;
        int lo = 0, hi = n;   // first position with degree <= kHeavy
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (perm_deg(rp, perm, v0 + mid) > kHeavy) lo = mid + 1;
            else hi = mid;
        }
        heavy[q] = lo;
        mcnt[q] = lo + ((n - lo + 31) >> 5) + 1;
    }
}

__device__ __forceinline__ int find_graph(const int *off, int G, int x) {
    int lo = 0, hi = G - 1;   // last q with off[q] <= x
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Item sizes (one thread per renumbered row): a heavy row's entries rounded
// up to a multiple of 8 (padding: weight 0, the row's own column), or for
// the first row of a slice the slice's 32 x its longest row; a final item of
// size 0 per graph.
__global__ void k_layout_items(int n, int G, const int *__restrict__ voff, const int *__restrict__ rp,
                               const uint32_t *__restrict__ perm, const int *__restrict__ heavy,
                               const int *__restrict__ moff, int *__restrict__ items) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int q = find_graph(voff, G, p);
        const int v0 = voff[q], ng = voff[q + 1] - v0, r = p - v0, h = heavy[q];
        int *it = items + moff[q];
        if (r < h) {
            it[r] = (perm_deg(rp, perm, p) + 7) & ~7;   // 8-entry aligned, for vector loads
        } else if (((r - h) & 31) == 0) {
            it[h + ((r - h) >> 5)] = 32 * perm_deg(rp, perm, p);
        }
        if (r == 0) it[h + ((ng - h + 31) >> 5)] = 0;
    }
}

// meta = item offsets local to each graph; eoff = each graph's first entry.
__global__ void k_layout_meta(int T, int G, const int *__restrict__ moff, const int *__restrict__ itemoff,
                              int *__restrict__ meta, int *__restrict__ eoff) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= T; t += gridDim.x * blockDim.x) {
        if (t == T) {
            eoff[G] = itemoff[T];
            continue;
        }
        const int q = find_graph(moff, G, t);
        const int base = itemoff[moff[q]];
        meta[t] = itemoff[t] - base;
        if (t == moff[q]) eoff[q] = base;
    }
}

// Entries of every renumbered row; the last slice's phantom rows (past n) and
// short rows are padded with weight 0 and a valid column.
template <typename T, typename IDX>
__global__ void k_layout_fill(int n, int G, const int *__restrict__ voff, const int *__restrict__ rp,
                              const int *__restrict__ col, const double *__restrict__ w,
                              const uint32_t *__restrict__ perm, const int *__restrict__ inv,
                              const int *__restrict__ heavy, const int *__restrict__ eoff,
                              const int *__restrict__ moff, const int *__restrict__ meta,
                              IDX *__restrict__ bcol, T *__restrict__ bw) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        int lo = 0, hi = G - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (voff[mid] <= p) lo = mid;
            else hi = mid - 1;
        }
        const int q = lo, v0 = voff[q], ng = voff[q + 1] - v0, r = p - v0, h = heavy[q];
        const int *m = meta + moff[q];
        const int v = (int)perm[p];
        const int e0 = rp[v], deg = rp[v + 1] - e0;
        IDX *gc = bcol + eoff[q];
        T *gw = bw + eoff[q];
        if (r < h) {
            const int d0 = m[r];
            for (int j = 0; j < deg; j++) {
                gc[d0 + j] = (IDX)(inv[col[e0 + j]] - v0);
                gw[d0 + j] = (T)w[e0 + j];
            }
            for (int j = deg; j < m[r + 1] - d0; j++) {   // padding to a multiple of 8
                gc[d0 + j] = (IDX)r;
                gw[d0 + j] = (T)0;
            }
            continue;
        }
        const int sl = (r - h) >> 5, l = (r - h) & 31;
        const int so = m[h + sl], wd = (m[h + sl + 1] - so) >> 5;
        for (int j = 0; j < wd; j++) {
            const int d = so + 32 * j + l;
            if (j < deg) {
                gc[d] = (IDX)(inv[col[e0 + j]] - v0);
                gw[d] = (T)w[e0 + j];
            } else {
                gc[d] = (IDX)r;
                gw[d] = (T)0;
            }
        }
        // the graph's last row also pads the phantom rows of its last slice
        if (r == ng - 1) {
            for (int l2 = l + 1; l2 < 32; l2++)
                for (int j = 0; j < wd; j++) {
                    gc[so + 32 * j + l2] = (IDX)0;
                    gw[so + 32 * j + l2] = (T)0;
                }
        }
    }
}


// chunk counts of the heavy rows of a one-graph layout
__global__ void k_layout_chunks(int h, const int *__restrict__ meta, int *__restrict__ cnt) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < h; r += gridDim.x * blockDim.x)
        cnt[r] = (meta[r + 1] - meta[r] + kHeavyChunk - 1) / kHeavyChunk;
}

// heavy row of every chunk
__global__ void k_layout_chunk_rows(int h, const int *__restrict__ hchunk, int *__restrict__ crow) {
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < h; r += gridDim.x * blockDim.x)
        for (int c = hchunk[r]; c < hchunk[r + 1]; c++) crow[c] = r;
}

cmg_status_t build_sweep_layout(int G, const int *voff, const std::vector<int> &hvoff, int N,
                                const int *rp, const int *col, const double *w, int fp32,
                                SweepLayout *L, size_t *bytes, cudaStream_t s, bool perm_only) {
    int maxn = 0;
    for (int q = 0; q < G; q++) maxn = std::max(maxn, hvoff[q + 1] - hvoff[q]);
    L->col16 = maxn <= 65536 ? 1 : 0;
    Scratch scr(s);
    uint64_t *ka, *kb;
    uint32_t *va, *vb;
    int *cnt_n, *mcnt;
    CMG_TRY(scr.get(&ka, (size_t)N));
    CMG_TRY(scr.get(&kb, (size_t)N));
    CMG_TRY(scr.get(&va, (size_t)N));
    CMG_TRY(scr.get(&vb, (size_t)N));
    CMG_TRY(scr.get(&cnt_n, 1));
    CMG_TRY(scr.get(&mcnt, (size_t)G));
    int *dmax;
    CMG_TRY(scr.get(&dmax, 1));
    CMG_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
    k_max_degree<<<grid_for(N, 256), 256, 0, s>>>(N, rp, dmax);
    CMG_TRY(launch_status());
    int maxdeg = 0;
    CMG_CUDA(cudaMemcpyAsync(&maxdeg, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(cnt_n, &N, sizeof(int), cudaMemcpyHostToDevice, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    const int db = bits_for(maxdeg + 1);
    const int kbits = db + (G > 1 ? bits_for(G) : 0);
    k_layout_keys<<<grid_for(N, 256), 256, 0, s>>>(N, G, voff, rp, maxdeg, db, ka, va);
    CMG_TRY(launch_status());
    CMG_TRY(radix_sort_pairs(&ka, &va, kb, vb, N, cnt_n, kbits, scr, s));
    CMG_TRY(dev_alloc_n(&L->perm, (size_t)N, s));
    CMG_TRY(dev_alloc_n(&L->inv, (size_t)N, s));
    CMG_CUDA(cudaMemcpyAsync(L->perm, va, sizeof(uint32_t) * N, cudaMemcpyDeviceToDevice, s));
    k_layout_inv<<<grid_for(N, 256), 256, 0, s>>>(N, L->perm, L->inv);
    CMG_TRY(launch_status());
    if (perm_only) {
        L->hheavy.assign(G, 0);
        L->hecnt.assign(G, 0);
        L->hmcnt.assign(G, 0);
        L->entries = 0;
        if (bytes) *bytes += (size_t)N * 8;
        return CMG_OK;
    }
    CMG_TRY(dev_alloc_n(&L->heavy, (size_t)G, s));
    CMG_TRY(dev_alloc_n(&L->eoff, (size_t)G + 1, s));
    CMG_TRY(dev_alloc_n(&L->moff, (size_t)G + 1, s));
    k_layout_heavy<<<grid_for(G, 256), 256, 0, s>>>(G, voff, rp, L->perm, L->heavy, mcnt);
    CMG_TRY(launch_status());
    CMG_TRY(exclusive_scan(mcnt, L->moff, G, scr, s));
    int nitems = 0;
    CMG_CUDA(cudaMemcpyAsync(&nitems, L->moff + G, sizeof(int), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    int *items, *itemoff;
    CMG_TRY(scr.get(&items, (size_t)nitems));
    CMG_TRY(scr.get(&itemoff, (size_t)nitems + 1));
    k_layout_items<<<grid_for(N, 256), 256, 0, s>>>(N, G, voff, rp, L->perm, L->heavy, L->moff, items);
    CMG_TRY(launch_status());
    CMG_TRY(exclusive_scan(items, itemoff, nitems, scr, s));
    CMG_TRY(dev_alloc_n(&L->meta, (size_t)std::max(nitems, 1), s));
    k_layout_meta<<<grid_for((long long)nitems + 1, 256), 256, 0, s>>>(nitems, G, L->moff, itemoff, L->meta,
                                                                        L->eoff);
    CMG_TRY(launch_status());
    std::vector<int> heo(G + 1);
    L->hmcnt.resize(G);
    L->hecnt.resize(G);
    L->hheavy.resize(G);
    CMG_CUDA(cudaMemcpyAsync(heo.data(), L->eoff, sizeof(int) * (G + 1), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(L->hmcnt.data(), mcnt, sizeof(int) * G, cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(L->hheavy.data(), L->heavy, sizeof(int) * G, cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    for (int q = 0; q < G; q++) L->hecnt[q] = heo[q + 1] - heo[q];
    const long long te = heo[G], tm = nitems;
    // the entry scan is 32-bit: refuse layouts beyond it
    if (te < 0 || (long long)heo[G] < (long long)heo[0]) return CMG_ERR_TOO_LARGE;
    L->entries = te;
    const size_t isz = L->col16 ? 2 : 4, esz = fp32 ? 4 : 8;
    CMG_TRY(dev_alloc(&L->bcol, isz * (size_t)std::max<long long>(te, 1), s));
    CMG_TRY(dev_alloc(&L->bw, esz * (size_t)std::max<long long>(te, 1), s));
    const int fb = grid_for(N, 256);
#define CMG_FILL(T, I)                                                                          \
    k_layout_fill<T, I><<<fb, 256, 0, s>>>(N, G, voff, rp, col, w, L->perm, L->inv, L->heavy,    \
                                           L->eoff, L->moff, L->meta, reinterpret_cast<I *>(L->bcol), \
                                           reinterpret_cast<T *>(L->bw))
    if (fp32 && L->col16) CMG_FILL(float, uint16_t);
    else if (fp32) CMG_FILL(float, int);
    else if (L->col16) CMG_FILL(double, uint16_t);
    else CMG_FILL(double, int);
#undef CMG_FILL
    CMG_TRY(launch_status());
    if (G == 1 && L->hheavy[0] > 0) {
        // heavy rows of a single graph are summed by several warps, a chunk each
        const int h = L->hheavy[0];
        int *cnt;
        CMG_TRY(scr.get(&cnt, (size_t)h));
        CMG_TRY(dev_alloc_n(&L->hchunk, (size_t)h + 1, s));
        CMG_TRY(dev_alloc_n(&L->hcount, (size_t)h, s));
        k_layout_chunks<<<grid_for(h, 256), 256, 0, s>>>(h, L->meta, cnt);
        CMG_TRY(launch_status());
        CMG_TRY(exclusive_scan(cnt, L->hchunk, h, scr, s));
        CMG_CUDA(cudaMemcpyAsync(&L->nchunks, L->hchunk + h, sizeof(int), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
        CMG_TRY(dev_alloc(&L->cpart, esz * (size_t)std::max(L->nchunks, 1), s));
        CMG_TRY(dev_alloc_n(&L->crow, (size_t)std::max(L->nchunks, 1), s));
        k_layout_chunk_rows<<<grid_for(h, 256), 256, 0, s>>>(h, L->hchunk, L->crow);
        CMG_TRY(launch_status());
        if (bytes) *bytes += (size_t)h * 8 + (esz + 4) * (size_t)L->nchunks;
    }
    if (bytes) *bytes += (size_t)N * 8 + (size_t)G * 12 + (size_t)tm * 4 + (size_t)te * (isz + esz);
    return CMG_OK;
}

// Layout entries (slice padding included: it is gathered too) whose column
// is below S, added to *out.
template <typename IDX>
__global__ void k_count_below(long long m, const IDX *__restrict__ bcol, int S,
                              unsigned long long *__restrict__ out) {
    unsigned long long c = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += (long long)gridDim.x * blockDim.x)
        c += ((int)bcol[k] < S) ? 1ull : 0ull;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

cmg_status_t layout_count_below(const SweepLayout &L, int S, unsigned long long *out, cudaStream_t s) {
    CMG_CUDA(cudaMemsetAsync(out, 0, sizeof(unsigned long long), s));
    if (L.entries <= 0) return CMG_OK;
    const int blocks = (int)std::min<long long>(4096, (L.entries + 255) / 256);
    if (L.col16)
        k_count_below<<<blocks, 256, 0, s>>>(L.entries, (const uint16_t *)L.bcol, S, out);
    else
        k_count_below<<<blocks, 256, 0, s>>>(L.entries, (const int *)L.bcol, S, out);
    return launch_status();
}

void free_sweep_layout(SweepLayout &L, cudaStream_t s) {
    dev_free(L.hchunk, s);
    dev_free(L.crow, s);
    dev_free(L.hcount, s);
    dev_free(L.cpart, s);
    dev_free(L.perm, s);
    dev_free(L.inv, s);
    dev_free(L.heavy, s);
    dev_free(L.eoff, s);
    dev_free(L.moff, s);
    dev_free(L.meta, s);
    dev_free(L.bcol, s);
    dev_free(L.bw, s);
    L = SweepLayout();
}

}  // namespace cmg
