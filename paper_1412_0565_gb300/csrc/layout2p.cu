// layout2p.cu -- the two-phase sweep layout of a large single-graph level
// (XLayout in internal.h describes what a sweep does with it).
//
// Construction, all on the device:
//   1. per row (sweep-layout order) its degree, scanned into entry offsets;
//   2. passes (balanced by entries), then per pass a multiple of P dest
//      blocks balanced by cost (entries + the pass's mean degree per row),
//      enough blocks that none holds more rows than the kernel's capacity;
//   3. one record per entry, keyed (dest block, source block), in row-major
//      order; a stable radix sort gives the list order (dest block, source
//      block, row, CSR position);
//   4. a stable sort of the list order by (pass, source block) gives the
//      phase-1 stream; the runs of one (dest block, source block) are the
//      cells, contiguous and identically ordered in both.
#include <algorithm>

#include "internal.h"

namespace cmg {

namespace {

// First i in [lo, hi] with a[i] >= x (hi when none); a non-decreasing.
__device__ __forceinline__ int lbound(const int *a, int lo, int hi, long long x) {
    while (lo < hi) {
        const int mid = lo + ((hi - lo) >> 1);
        if ((long long)a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ long long lbound64(const uint64_t *a, long long lo, long long hi, uint64_t x) {
    while (lo < hi) {
        const long long mid = lo + ((hi - lo) >> 1);
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_x2_deg(int n, const int *__restrict__ rp, const uint32_t *__restrict__ perm, int *__restrict__ deg) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int v = (int)perm[p];
        deg[p] = rp[v + 1] - rp[v];
    }
}

// pass row boundaries pr[0..T] (balanced by entries)
__global__ void k_x2_passes(int n, int T, const int *__restrict__ epos, int *__restrict__ pr) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > T) return;
    const long long nnz = epos[n];
    pr[t] = (t == T) ? n : lbound(epos, 0, n, nnz * t / T);
}

// Dest-block row boundaries: the ndb[t+1] - ndb[t] blocks of pass t split
// its rows by cost (entries + lam_t per row, lam_t the pass's mean degree);
// dbr[ndb[T]] = n.
__global__ void k_x2_dblocks(int n, int T, const int *__restrict__ epos, const int *__restrict__ pr,
                             const int *__restrict__ ndb, int *__restrict__ dbr) {
    const int nb = ndb[T];
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= nb; g += gridDim.x * blockDim.x) {
        if (g == nb) {
            dbr[g] = n;
            continue;
        }
        int t = 0;   // pass of block g: last t with ndb[t] <= g
        {
            int lo = 0, hi = T - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (ndb[mid] <= g) lo = mid;
                else hi = mid - 1;
            }
            t = lo;
        }
        const int k = g - ndb[t], m = ndb[t + 1] - ndb[t];
        const int r0 = pr[t], r1 = pr[t + 1];
        int b0 = r0;
        if (k > 0 && r1 > r0) {
            const double e0 = epos[r0], et = (double)epos[r1] - e0, rt = (double)(r1 - r0);
            const double lam = et / rt;
            const double target = (et + lam * rt) * k / m;
            int lo = r0, hi = r1;   // first row p with cost(r0..p) >= target
            while (lo < hi) {
                const int mid = lo + ((hi - lo) >> 1);
                if (((double)epos[mid] - e0) + lam * (mid - r0) < target) lo = mid + 1;
                else hi = mid;
            }
            b0 = lo;
        }
        dbr[g] = b0;
    }
}

// dest block of every row
__global__ void k_x2_rowblock(int nb, const int *__restrict__ dbr, int *__restrict__ rdb) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nb; g += gridDim.x * blockDim.x)
        for (int p = dbr[g]; p < dbr[g + 1]; p++) rdb[p] = g;
}

// one record per entry, in row-major layout order
__global__ void k_x2_entries(int n, const int *__restrict__ rp, const int *__restrict__ col,
                             const uint32_t *__restrict__ perm, const int *__restrict__ inv,
                             const int *__restrict__ epos, const int *__restrict__ rdb, int SB, int qb,
                             uint64_t *__restrict__ key, uint32_t *__restrict__ val, int *__restrict__ ecol,
                             int *__restrict__ erow, int *__restrict__ eorig) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int v0 = (int)perm[p], b = rp[v0], d = rp[v0 + 1] - b, e = epos[p];
        const uint64_t hi = (uint64_t)rdb[p] << qb;
        for (int k = 0; k < d; k++) {
            const int c = inv[col[b + k]];
            key[e + k] = hi | (uint64_t)(c / SB);
            val[e + k] = (uint32_t)(e + k);
            ecol[e + k] = c;
            erow[e + k] = p;
            eorig[e + k] = b + k;
        }
    }
}

// list-order arrays and the keys of the phase-1 order
template <typename T>
__global__ void k_x2_list(long long m, const uint64_t *__restrict__ ks, const uint32_t *__restrict__ vs,
                          const int *__restrict__ erow, const int *__restrict__ eorig, const double *__restrict__ w,
                          const int *__restrict__ dbr, const int *__restrict__ dbt, int qb,
                          uint16_t *__restrict__ dst, T *__restrict__ w2, uint64_t *__restrict__ key2,
                          uint32_t *__restrict__ val2) {
    const uint64_t qmask = (1ull << qb) - 1ull;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x) {
        const int e = (int)vs[i];
        const int g = (int)(ks[i] >> qb);
        const int q = (int)(ks[i] & qmask);
        dst[i] = (uint16_t)(erow[e] - dbr[g]);
        w2[i] = (T)w[eorig[e]];
        key2[i] = ((uint64_t)dbt[g] << qb) | (uint64_t)q;
        val2[i] = (uint32_t)i;
    }
}

// pass of every dest block
__global__ void k_x2_dbt(int T, const int *__restrict__ ndb, int *__restrict__ dbt) {
    const int t = blockIdx.x;
    if (t >= T) return;
    for (int g = ndb[t] + threadIdx.x; g < ndb[t + 1]; g += blockDim.x) dbt[g] = t;
}

// phase-1 stream (source offsets within the block; pass t's entries from
// sal[t] on, so that each pass starts at a multiple of 8) and the heads of
// its cells
__global__ void k_x2_src(long long m, int T, const uint64_t *__restrict__ k2s, const uint32_t *__restrict__ v2s,
                         const uint32_t *__restrict__ vs, const uint64_t *__restrict__ ks, const int *__restrict__ ecol,
                         const int *__restrict__ pass_s, const int *__restrict__ sal, int SB, int qb,
                         uint16_t *__restrict__ src, int *__restrict__ head) {
    const uint64_t qmask = (1ull << qb) - 1ull;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x) {
        const int i = (int)v2s[j];
        const int q = (int)(k2s[j] & qmask);
        const int t = (int)(k2s[j] >> qb);
        src[sal[t] + (j - pass_s[t])] = (uint16_t)(ecol[vs[i]] - q * SB);
        // a cell = one (dest block, source block) run: the list key of the entry
        head[j] = (j == 0 || ks[i] != ks[v2s[j - 1]]) ? 1 : 0;
    }
}

// per cell: list position - stream position of its entries
__global__ void k_x2_cells(long long m, const int *__restrict__ head, const int *__restrict__ cid,
                           const uint32_t *__restrict__ v2s, int *__restrict__ cdel) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m; j += (long long)gridDim.x * blockDim.x)
        if (head[j]) cdel[cid[j]] = (int)v2s[j] - (int)j;
}

// Per 32-entry chunk of each pass's stream (chunks aligned to the pass
// start): the cell holding its first entry, and bit l (1..31) set where
// entry l starts a cell.
__global__ void k_x2_chunks(int T, const int *__restrict__ pass_s, const int *__restrict__ choff,
                            const int *__restrict__ head, const int *__restrict__ cid, uint2 *__restrict__ chk) {
    const int nch = choff[T];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nch; k += gridDim.x * blockDim.x) {
        int lo = 0, hi = T - 1;   // pass of chunk k: last t with choff[t] <= k
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (choff[mid] <= k) lo = mid;
            else hi = mid - 1;
        }
        const int t = lo;
        const int j0 = pass_s[t] + 32 * (k - choff[t]), jend = pass_s[t + 1];
        unsigned mask = 0u;
        for (int l = 1; l < 32 && j0 + l < jend; l++)
            if (head[j0 + l]) mask |= 1u << l;
        chk[k] = make_uint2((unsigned)(cid[j0] + head[j0] - 1), mask);
    }
}

__global__ void k_x2_qoff(int T, int Q, long long m, int qb, const uint64_t *__restrict__ k2s,
                          const int *__restrict__ pass_s, int *__restrict__ qoff) {
    const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (k >= (long long)T * (Q + 1)) return;
    const int t = (int)(k / (Q + 1)), q = (int)(k % (Q + 1));
    const uint64_t key = (q == Q) ? ((uint64_t)(t + 1) << qb) : (((uint64_t)t << qb) | (uint64_t)q);
    qoff[k] = (int)(lbound64(k2s, 0, m, key) - pass_s[t]);
}

__global__ void k_x2_dbl(int nb, const int *__restrict__ epos, const int *__restrict__ dbr, int *__restrict__ dbl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= nb) dbl[k] = epos[dbr[k]];
}

}  // namespace

void free_xlayout(XLayout &X, cudaStream_t s) {
    dev_free(X.src, s);
    dev_free(X.dst, s);
    dev_free(X.w, s);
    dev_free(X.pass_s, s);
    dev_free(X.sal, s);
    dev_free(X.qoff, s);
    dev_free(X.ndb, s);
    dev_free(X.dbr, s);
    dev_free(X.dbl, s);
    dev_free(X.cdel, s);
    dev_free(X.choff, s);
    dev_free(X.chk, s);
    dev_free(X.pmax, s);
    dev_free(X.xbuf[0], s);
    dev_free(X.xbuf[1], s);
    X = XLayout();
}

cmg_status_t build_xlayout(int n, long long nnz, const int *rp, const int *col, const double *w, int fp32,
                           const uint32_t *perm, const int *inv, const XParams &prm, XLayout *X,
                           size_t *bytes, cudaStream_t s) {
    if (n < 1 || nnz < 1 || nnz >= (1ll << 31) - 1) return CMG_ERR_TOO_LARGE;
    DeviceInfo di;
    CMG_TRY(device_info(&di));
    const size_t esz = fp32 ? sizeof(float) : sizeof(double);
    XLayout &L = *X;
    L = XLayout();
    L.P = di.sms;
    L.smem = xsweep_smem(fp32);
    if (L.smem == 0) return CMG_ERR_TOO_LARGE;
    const int sb_cap = (int)std::min<size_t>(L.smem / esz, 65536);
    L.SB = prm.sb > 0 ? std::min(prm.sb, sb_cap) : sb_cap;
    // per row: a 64-bit accumulator and the row's iterate entry
    L.VMAX = (int)std::min<size_t>(L.smem / (8 + esz), 65536);
    L.Q = (int)((n + (long long)L.SB - 1) / L.SB);
    L.entries = nnz;
    const int qb = bits_for(L.Q);
    const long long xcap_bytes = prm.xcap_bytes > 0 ? prm.xcap_bytes : (32ll << 20);
    const int m = (int)nnz;
    Scratch scr(s);
    // ---- 1. rows
    int *deg, *epos, *nnz_dev;
    CMG_TRY(scr.get(&deg, (size_t)n));
    CMG_TRY(scr.get(&epos, (size_t)n + 1));
    CMG_TRY(scr.get(&nnz_dev, 1));
    k_x2_deg<<<grid_for(n, 256), 256, 0, s>>>(n, rp, perm, deg);
    CMG_TRY(launch_status());
    CMG_TRY(exclusive_scan(deg, epos, n, scr, s));
    // ---- 2. passes and dest blocks
    const int T = (int)std::max<long long>(1, (nnz * (long long)esz + xcap_bytes - 1) / xcap_bytes);
    if (T > 4096) return CMG_ERR_TOO_LARGE;
    L.T = T;
    int *pr;
    CMG_TRY(scr.get(&pr, (size_t)T + 1));
    k_x2_passes<<<grid_for(T + 1, 256), 256, 0, s>>>(n, T, epos, pr);
    CMG_TRY(launch_status());
    std::vector<int> hpr(T + 1), hep(T + 1);
    CMG_CUDA(cudaMemcpyAsync(hpr.data(), pr, sizeof(int) * (T + 1), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    for (int t = 0; t <= T; t++)
        CMG_CUDA(cudaMemcpyAsync(&hep[t], epos + hpr[t], sizeof(int), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if ((long long)hep[T] != nnz) return CMG_ERR_BAD_CSR;
    // blocks per pass: P times enough to keep 2 R_t / blocks under VMAX,
    // doubled for a pass whose largest block still holds too many rows
    std::vector<int> mult(T);
    for (int t = 0; t < T; t++) {
        const long long rt = hpr[t + 1] - hpr[t];
        mult[t] = (int)std::max<long long>(1, (2 * rt + (long long)L.P * L.VMAX - 1) / ((long long)L.P * L.VMAX));
    }
    int *ndb = nullptr, *dbr = nullptr;
    std::vector<int> hndb(T + 1);
    for (int attempt = 0;; attempt++) {
        if (attempt > 12) return CMG_ERR_TOO_LARGE;
        hndb[0] = 0;
        for (int t = 0; t < T; t++) hndb[t + 1] = hndb[t] + L.P * mult[t];
        const int nb = hndb[T];
        Scratch tmp(s);
        int *ndb_t, *dbr_t;
        CMG_TRY(tmp.get(&ndb_t, (size_t)T + 1));
        CMG_TRY(tmp.get(&dbr_t, (size_t)nb + 1));
        CMG_CUDA(cudaMemcpyAsync(ndb_t, hndb.data(), sizeof(int) * (T + 1), cudaMemcpyHostToDevice, s));
        k_x2_dblocks<<<grid_for(nb + 1, 256), 256, 0, s>>>(n, T, epos, pr, ndb_t, dbr_t);
        CMG_TRY(launch_status());
        // per pass: the largest block
        std::vector<int> hdbr(nb + 1);
        CMG_CUDA(cudaMemcpyAsync(hdbr.data(), dbr_t, sizeof(int) * (nb + 1), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
        bool ok = true;
        for (int t = 0; t < T; t++) {
            int mx = 0;
            for (int g = hndb[t]; g < hndb[t + 1]; g++) mx = std::max(mx, hdbr[g + 1] - hdbr[g]);
            if (mx > L.VMAX) {
                mult[t] *= 2;
                ok = false;
            }
        }
        if (!ok) continue;
        CMG_TRY(scr.get(&ndb, (size_t)T + 1));
        CMG_TRY(scr.get(&dbr, (size_t)nb + 1));
        CMG_CUDA(cudaMemcpyAsync(ndb, ndb_t, sizeof(int) * (T + 1), cudaMemcpyDeviceToDevice, s));
        CMG_CUDA(cudaMemcpyAsync(dbr, dbr_t, sizeof(int) * (nb + 1), cudaMemcpyDeviceToDevice, s));
        break;
    }
    const int nb = hndb[T];
    L.nblocks = nb;
    int *rdb, *dbt;
    CMG_TRY(scr.get(&rdb, (size_t)n));
    CMG_TRY(scr.get(&dbt, (size_t)nb));
    k_x2_rowblock<<<grid_for(nb, 256), 256, 0, s>>>(nb, dbr, rdb);
    CMG_TRY(launch_status());
    k_x2_dbt<<<T, 256, 0, s>>>(T, ndb, dbt);
    CMG_TRY(launch_status());
    // ---- 3. entry records, sorted into list order
    int hm = m;
    CMG_CUDA(cudaMemcpyAsync(nnz_dev, &hm, sizeof(int), cudaMemcpyHostToDevice, s));
    uint64_t *ka, *kb2;
    uint32_t *va, *vb;
    int *ecol, *erow, *eorig;
    CMG_TRY(scr.get(&ka, (size_t)m));
    CMG_TRY(scr.get(&kb2, (size_t)m));
    CMG_TRY(scr.get(&va, (size_t)m));
    CMG_TRY(scr.get(&vb, (size_t)m));
    CMG_TRY(scr.get(&ecol, (size_t)m));
    CMG_TRY(scr.get(&erow, (size_t)m));
    CMG_TRY(scr.get(&eorig, (size_t)m));
    k_x2_entries<<<grid_for(n, 256), 256, 0, s>>>(n, rp, col, perm, inv, epos, rdb, L.SB, qb, ka, va, ecol, erow,
                                                   eorig);
    CMG_TRY(launch_status());
    uint64_t *ks = ka;
    uint32_t *vs = va;
    CMG_TRY(radix_sort_pairs(&ks, &vs, kb2, vb, m, nnz_dev, bits_for(nb) + qb, scr, s));
    // ---- list-order arrays and the phase-1 keys
    // list arrays padded by 8: the kernel reads 8 aligned entries at a time
    CMG_TRY(dev_alloc_n(&L.dst, (size_t)m + 8, s));
    CMG_TRY(dev_alloc(&L.w, esz * ((size_t)m + 8), s));
    CMG_CUDA(cudaMemsetAsync(L.dst + m, 0, 8 * sizeof(uint16_t), s));
    CMG_CUDA(cudaMemsetAsync(reinterpret_cast<char *>(L.w) + esz * (size_t)m, 0, 8 * esz, s));
    uint64_t *k2a, *k2b;
    uint32_t *v2a, *v2b;
    int *head, *cid;
    CMG_TRY(scr.get(&k2a, (size_t)m));
    CMG_TRY(scr.get(&k2b, (size_t)m));
    CMG_TRY(scr.get(&v2a, (size_t)m));
    CMG_TRY(scr.get(&v2b, (size_t)m));
    CMG_TRY(scr.get(&head, (size_t)m));
    CMG_TRY(scr.get(&cid, (size_t)m + 1));
    const int gb = grid_for(m, 256);
    if (fp32)
        k_x2_list<float><<<gb, 256, 0, s>>>(m, ks, vs, erow, eorig, w, dbr, dbt, qb, L.dst,
                                            reinterpret_cast<float *>(L.w), k2a, v2a);
    else
        k_x2_list<double><<<gb, 256, 0, s>>>(m, ks, vs, erow, eorig, w, dbr, dbt, qb, L.dst,
                                             reinterpret_cast<double *>(L.w), k2a, v2a);
    CMG_TRY(launch_status());
    uint64_t *k2s = k2a;
    uint32_t *v2s = v2a;
    CMG_TRY(radix_sort_pairs(&k2s, &v2s, k2b, v2b, m, nnz_dev, bits_for(T) + qb, scr, s));
    // pass offsets: of the entries (both orders) and of the padded stream
    std::vector<int> hsal(T + 1);
    hsal[0] = 0;
    for (int t = 0; t < T; t++) hsal[t + 1] = hsal[t] + ((hep[t + 1] - hep[t] + 7) & ~7);
    CMG_TRY(dev_alloc_n(&L.pass_s, (size_t)T + 1, s));
    CMG_TRY(dev_alloc_n(&L.sal, (size_t)T + 1, s));
    CMG_CUDA(cudaMemcpyAsync(L.pass_s, hep.data(), sizeof(int) * (T + 1), cudaMemcpyHostToDevice, s));
    CMG_CUDA(cudaMemcpyAsync(L.sal, hsal.data(), sizeof(int) * (T + 1), cudaMemcpyHostToDevice, s));
    CMG_TRY(dev_alloc_n(&L.src, (size_t)hsal[T] + 8, s));
    CMG_CUDA(cudaMemsetAsync(L.src, 0, sizeof(uint16_t) * ((size_t)hsal[T] + 8), s));
    k_x2_src<<<gb, 256, 0, s>>>(m, T, k2s, v2s, vs, ks, ecol, L.pass_s, L.sal, L.SB, qb, L.src, head);
    CMG_TRY(launch_status());
    // ---- cells, chunks, pass and block tables
    CMG_TRY(exclusive_scan(head, cid, m, scr, s));
    CMG_CUDA(cudaMemcpyAsync(&L.ncells, cid + m, sizeof(int), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    CMG_TRY(dev_alloc_n(&L.cdel, (size_t)std::max(L.ncells, 1), s));
    k_x2_cells<<<gb, 256, 0, s>>>(m, head, cid, v2s, L.cdel);
    CMG_TRY(launch_status());
    CMG_TRY(dev_alloc_n(&L.dbl, (size_t)nb + 1, s));
    k_x2_dbl<<<grid_for(nb + 1, 256), 256, 0, s>>>(nb, epos, dbr, L.dbl);
    CMG_TRY(launch_status());
    std::vector<int> hch(T + 1);
    hch[0] = 0;
    for (int t = 0; t < T; t++) hch[t + 1] = hch[t] + (hep[t + 1] - hep[t] + 31) / 32;
    L.nchunks = hch[T];
    CMG_TRY(dev_alloc_n(&L.choff, (size_t)T + 1, s));
    CMG_CUDA(cudaMemcpyAsync(L.choff, hch.data(), sizeof(int) * (T + 1), cudaMemcpyHostToDevice, s));
    CMG_TRY(dev_alloc_n(&L.chk, (size_t)std::max(L.nchunks, 1), s));
    k_x2_chunks<<<grid_for(std::max(L.nchunks, 1), 256), 256, 0, s>>>(T, L.pass_s, L.choff, head, cid, L.chk);
    CMG_TRY(launch_status());
    CMG_TRY(dev_alloc_n(&L.qoff, (size_t)T * (L.Q + 1), s));
    k_x2_qoff<<<grid_for((long long)T * (L.Q + 1), 256), 256, 0, s>>>(T, L.Q, m, qb, k2s, L.pass_s, L.qoff);
    CMG_TRY(launch_status());
    CMG_TRY(dev_alloc_n(&L.ndb, (size_t)T + 1, s));
    CMG_CUDA(cudaMemcpyAsync(L.ndb, ndb, sizeof(int) * (T + 1), cudaMemcpyDeviceToDevice, s));
    CMG_TRY(dev_alloc_n(&L.dbr, (size_t)nb + 1, s));
    CMG_CUDA(cudaMemcpyAsync(L.dbr, dbr, sizeof(int) * ((size_t)nb + 1), cudaMemcpyDeviceToDevice, s));
    CMG_TRY(dev_alloc_n(&L.pmax, (size_t)2 * L.P, s));
    long long emax = 1;
    for (int t = 0; t < T; t++) emax = std::max<long long>(emax, (long long)hep[t + 1] - hep[t]);
    // a pass's list positions sit in xbuf from (pass start & ~7) on, and the
    // kernel reads 8 aligned entries at a time: 16 elements of slack
    L.xcap = emax + 16;
    CMG_TRY(dev_alloc(&L.xbuf[0], esz * (size_t)L.xcap, s));
    CMG_TRY(dev_alloc(&L.xbuf[1], esz * (size_t)L.xcap, s));
    CMG_CUDA(cudaMemsetAsync(L.xbuf[0], 0, esz * (size_t)L.xcap, s));
    CMG_CUDA(cudaMemsetAsync(L.xbuf[1], 0, esz * (size_t)L.xcap, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if (bytes)
        *bytes += (size_t)(m + 8) * (2 + esz) + ((size_t)hsal[T] + 8) * 2 + (size_t)L.ncells * 4 + (size_t)L.nchunks * 8 + (size_t)(T + 1) * 12 +
                  (size_t)T * (L.Q + 1) * 4 + ((size_t)nb + 1) * 8 + (size_t)2 * L.P * 8 + 2 * esz * (size_t)L.xcap;
    return CMG_OK;
}

}  // namespace cmg
