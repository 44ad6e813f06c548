// api.cu -- the C-ABI of libcmg (include/cmg.h): input validation, the
// resident hierarchy of Alg. 1 Step 1, and the solve of Alg. 1 Steps 2-3.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"

using namespace cmg;

// ------------------------------------------------------------------ validation
enum : unsigned {
    kBadCsr = 1u,
    kSelfLoop = 2u,
    kBadWeight = 4u,
    kNotSym = 8u,
    kIsolated = 16u,
};

__global__ void k_check_rowptr(int n, const int64_t *__restrict__ rp64, int64_t nnz,
                               int *__restrict__ rp32, unsigned *__restrict__ flags) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i <= n;
         i += (long long)gridDim.x * blockDim.x) {
        const int64_t v = rp64[i];
        unsigned f = 0;
        if (i == 0 && v != 0) f |= kBadCsr;
        if (v < 0 || v > nnz) f |= kBadCsr;
        if (i < n) {
            const int64_t nx = rp64[i + 1];
            if (nx < v) f |= kBadCsr;
            else if (nx == v) f |= kIsolated;
        }
        rp32[i] = (int)(v < 0 ? 0 : (v > nnz ? nnz : v));
        if (f) atomicOr(flags, f);
    }
}

__global__ void k_check_entries(int n, const int *__restrict__ rp, const int *__restrict__ col,
                                const double *__restrict__ w, unsigned *__restrict__ flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned f = 0;
        const int e0 = rp[i], e1 = rp[i + 1];
        for (int e = e0; e < e1; e++) {
            const int j = col[e];
            if (j < 0 || j >= n) {
                f |= kBadCsr;
                continue;
            }
            if (e > e0 && col[e - 1] >= j) f |= kBadCsr;
            if (j == i) f |= kSelfLoop;
            const double x = w[e];
            if (!(x > 0.0) || isinf(x)) f |= kBadWeight;
            // mirrored entry (j, i) with a bitwise equal weight
            int lo = rp[j], hi = rp[j + 1] - 1;
            bool found = false;
            while (lo <= hi) {
                const int mid = (lo + hi) >> 1;
                const int c = col[mid];
                if (c == i) {
                    found = __double_as_longlong(w[mid]) == __double_as_longlong(x);
                    break;
                }
                if (c < i) lo = mid + 1;
                else hi = mid - 1;
            }
            if (!found) f |= kNotSym;
        }
        if (f) atomicOr(flags, f);
    }
}

__global__ void k_to_float(long long m, const double *__restrict__ w, float *__restrict__ w32) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < m;
         k += (long long)gridDim.x * blockDim.x)
        w32[k] = (float)w[k];
}

// ------------------------------------------------------------------ hierarchy
struct LevelData {
    int n = 0;
    long long nnz = 0;
    int *rp = nullptr;
    int *col = nullptr;
    double *w = nullptr;
    float *w32 = nullptr;
    int *agg = nullptr;  // onto the next level
    int *tiles = nullptr;
    int ntiles = 0;
    long long sell_nnz = 0;
    double g = 0.0;
    bool has_lay = false;   // large level: sweeps read the sweep layout
    SweepLayout lay;
    bool has_xl = false;    // ... or its two-phase layout (lay then holds only the row order)
    XLayout xl;
    int cl_ctas = 0, cl_threads = 0, cl_emax = 0;   // FP64 sweeps in one cluster (cluster_plan)
    size_t cl_smem = 0;
    int fp32 = 0;           // this level's sweeps run in FP32
};

struct cmg_hierarchy_s {
    int device = 0;
    cudaStream_t stream = nullptr;
    cmg_options_t opts;
    std::vector<LevelData> lv;
    // solve workspace
    std::vector<void *> bufs;  // 3 per level (iterate ring)
    std::vector<double *> gd;  // FP64 form: g - d_i per level
    PiResult *res = nullptr;   // one per level
    GridSync *gs = nullptr;
    double *out2 = nullptr;
    double *u_dev = nullptr;
    size_t bytes = 0;
};

static void free_level(LevelData &L, cudaStream_t s) {
    dev_free(L.rp, s);
    dev_free(L.col, s);
    dev_free(L.w, s);
    dev_free(L.w32, s);
    dev_free(L.agg, s);
    dev_free(L.tiles, s);
    free_sweep_layout(L.lay, s);
    free_xlayout(L.xl, s);
    L = LevelData();
}

static void free_hierarchy(cmg_hierarchy_s *h) {
    if (!h) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    for (auto &L : h->lv) free_level(L, h->stream);
    for (void *p : h->bufs) dev_free(p, h->stream);
    for (double *p : h->gd) dev_free(p, h->stream);
    dev_free(h->res, h->stream);
    dev_free(h->gs, h->stream);
    dev_free(h->out2, h->stream);
    dev_free(h->u_dev, h->stream);
    cudaStreamSynchronize(h->stream);
    cudaSetDevice(prev);
    delete h;
}

cmg_status_t cmg::check_options(const cmg_options_t &o) {
    if (!(o.tol >= 0.0) || !(o.tol < 1.0)) return CMG_ERR_INVALID_ARG;
    if (o.coarse_size < 1 || o.max_levels < 1 || o.max_levels > CMG_MAX_LEVELS)
        return CMG_ERR_INVALID_ARG;
    if (o.precision != CMG_PRECISION_FP64 && o.precision != CMG_PRECISION_FP32_SWEEP)
        return CMG_ERR_INVALID_ARG;
    if (o.schedule < CMG_SCHEDULE_TOL || o.schedule > CMG_SCHEDULE_REPLAY) return CMG_ERR_INVALID_ARG;
    if (o.schedule == CMG_SCHEDULE_FIXED && (o.k0 < 0 || !(o.beta > 0.0))) return CMG_ERR_INVALID_ARG;
    if (o.max_sweeps < 1 || o.max_sweeps_coarsest < 1) return CMG_ERR_INVALID_ARG;
    if (o.reserved != 0) return CMG_ERR_INVALID_ARG;
    return CMG_OK;
}

static cmg_status_t map_flags(unsigned f) {
    if (f & kBadCsr) return CMG_ERR_BAD_CSR;
    if (f & kSelfLoop) return CMG_ERR_SELF_LOOP;
    if (f & kBadWeight) return CMG_ERR_BAD_WEIGHT;
    if (f & kNotSym) return CMG_ERR_NOT_SYMMETRIC;
    if (f & kIsolated) return CMG_ERR_ISOLATED_VERTEX;
    return CMG_OK;
}

cmg_status_t cmg::load_level0(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                              int32_t mem, int validate, int **rp_out, int **col_out,
                              double **w_out, long long *nnz_out, cudaStream_t s) {
    // ---- nnz and size limits
    int64_t nnz = 0;
    if (mem == CMG_MEM_HOST) {
        nnz = row_ptr[n];
    } else {
        CMG_CUDA(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
    }
    if (nnz < 0) return CMG_ERR_BAD_CSR;
    if (nnz >= 2147483647ll) return CMG_ERR_TOO_LARGE;
    *nnz_out = nnz;
    // ---- copy in (int64 row pointers converted on the device); the caller
    // owns the three arrays once they are allocated, also on error
    CMG_TRY(dev_alloc_n(rp_out, (size_t)n + 1, s));
    CMG_TRY(dev_alloc_n(col_out, (size_t)std::max<int64_t>(nnz, 1), s));
    CMG_TRY(dev_alloc_n(w_out, (size_t)std::max<int64_t>(nnz, 1), s));
    Scratch scr(s);
    int64_t *rp64;
    unsigned *flags;
    CMG_TRY(scr.get(&flags, 1));
    CMG_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned), s));
    const cudaMemcpyKind kind = (mem == CMG_MEM_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (mem == CMG_MEM_HOST) {
        CMG_TRY(scr.get(&rp64, (size_t)n + 1));
        CMG_CUDA(cudaMemcpyAsync(rp64, row_ptr, sizeof(int64_t) * ((size_t)n + 1), kind, s));
    } else {
        rp64 = const_cast<int64_t *>(row_ptr);
    }
    if (nnz > 0) {
        CMG_CUDA(cudaMemcpyAsync(*col_out, col, sizeof(int32_t) * (size_t)nnz, kind, s));
        CMG_CUDA(cudaMemcpyAsync(*w_out, w, sizeof(double) * (size_t)nnz, kind, s));
    }
    const int threads = 256;
    k_check_rowptr<<<grid_for(n + 1, threads), threads, 0, s>>>((int)n, rp64, nnz, *rp_out, flags);
    CMG_TRY(launch_status());
    if (validate) {
        unsigned hf = 0;
        CMG_CUDA(cudaMemcpyAsync(&hf, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
        if (hf & kBadCsr) return CMG_ERR_BAD_CSR;
        k_check_entries<<<grid_for(n, threads), threads, 0, s>>>((int)n, *rp_out, *col_out, *w_out, flags);
        CMG_TRY(launch_status());
        CMG_CUDA(cudaMemcpyAsync(&hf, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
        CMG_TRY(map_flags(hf));
    }
    return CMG_OK;
}

cmg_status_t cmg::launch_to_float(long long m, const double *w, float *w32, cudaStream_t s) {
    if (m <= 0) return CMG_OK;
    k_to_float<<<grid_for(m, 256), 256, 0, s>>>(m, w, w32);
    return launch_status();
}

// Fewest stored entries of a level that sweeps in FP32 in the FP32 form
// (2^20 entries: at least 8 MB of FP32 sweep stream).
constexpr long long kFp32MinEntries = 1ll << 20;

static PiLevel level_view(const LevelData &L) {
    PiLevel v = {};
    v.n = L.n;
    v.nnz = L.nnz;
    v.rp = L.rp;
    v.col = L.col;
    v.w = L.w;
    v.w32 = L.w32;
    v.g = L.g;
    v.agg = L.agg;
    v.tile_row = L.tiles;
    v.ntiles = L.ntiles;
    v.sell_nnz = L.sell_nnz;
    v.lay = L.has_lay ? &L.lay : nullptr;
    v.xl = L.has_xl ? &L.xl : nullptr;
    v.cl_ctas = L.cl_ctas;
    v.cl_threads = L.cl_threads;
    v.cl_emax = L.cl_emax;
    v.cl_smem = L.cl_smem;
    return v;
}

// Levels swept through the two-phase layout: only on request (CMG_2P=1,
// read at setup: every level with a sweep layout).  Measured on the
// 4.19M-vertex Chung-Lu graph's levels 0-2 it is about twice as slow as the
// slice kernel (it writes and reads back every gathered value through L2 and
// restages source blocks each pass), so no level takes it by default.
static cmg_status_t wants_two_phase(const LevelData &, bool *out, cudaStream_t) {
    const char *env = getenv("CMG_2P");
    *out = env && env[0] == '1';
    return CMG_OK;
}

// Test knobs of the two-phase layout: CMG_2P_SB (source block vertices),
// CMG_2P_XCAP (bytes per pass buffer).
static XParams two_phase_params() {
    XParams p;
    if (const char *e = getenv("CMG_2P_SB")) p.sb = atoi(e);
    if (const char *e = getenv("CMG_2P_XCAP")) p.xcap_bytes = atoll(e);
    return p;
}

static cmg_status_t build_hierarchy(cmg_hierarchy_s *h, int64_t n, const int64_t *row_ptr,
                                    const int32_t *col, const double *w, int32_t mem) {
    cudaStream_t s = h->stream;
    const cmg_options_t &o = h->opts;
    // ---- level 0: copy in, validate
    LevelData L0;
    L0.n = (int)n;
    h->lv.push_back(L0);
    LevelData &Z = h->lv.back();
    CMG_TRY(load_level0(n, row_ptr, col, w, mem, o.validate, &Z.rp, &Z.col, &Z.w, &Z.nnz, s));
    Scratch scr(s);
    {
        double *gd;
        CMG_TRY(scr.get(&gd, 1));
        CMG_TRY(launch_gershgorin((int)n, Z.rp, Z.w, gd, s));
        CMG_CUDA(cudaMemcpyAsync(&Z.g, gd, sizeof(double), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
    }
    // ---- Alg. 1 Step 1: coarsen while n_i > coarse_size.  Each level runs
    // HEC, the Galerkin product and the SELL-32 sizing on the device into
    // buffers sized by upper bounds, then reads its sizes back with one
    // host synchronisation and moves the coarse CSR into exact allocations.
    LevelCounts *cnt_dev;
    CMG_TRY(scr.get(&cnt_dev, 1));
    int level = 0;
    while (h->lv.back().n > o.coarse_size && (int)h->lv.size() < o.max_levels) {
        const LevelData F = h->lv.back();
        int *agg = nullptr, *rp_t = nullptr, *col_t = nullptr;
        double *w_t = nullptr;
        LevelCounts hc;
        auto release = [&]() {
            dev_free(agg, s);
            dev_free(rp_t, s);
            dev_free(col_t, s);
            dev_free(w_t, s);
        };
        cmg_status_t st = CMG_OK;
        do {
            const size_t cap = (size_t)std::max<long long>(F.nnz, 1);
            if ((st = dev_alloc_n(&agg, (size_t)F.n, s)) != CMG_OK) break;
            if ((st = dev_alloc_n(&rp_t, (size_t)F.n + 1, s)) != CMG_OK) break;
            if ((st = dev_alloc_n(&col_t, cap, s)) != CMG_OK) break;
            if ((st = dev_alloc_n(&w_t, cap, s)) != CMG_OK) break;
            if ((st = from_cuda(cudaMemsetAsync(cnt_dev, 0, sizeof(LevelCounts), s))) != CMG_OK) break;
            st = hec_level_async(F.n, F.nnz, F.rp, F.col, F.w, o.seed, level, nullptr, agg,
                                 &cnt_dev->c, &cnt_dev->gs, s);
            if (st != CMG_OK) break;
            st = galerkin_async(F.n, F.nnz, F.rp, F.col, F.w, agg, bits_for(F.n), cnt_dev, rp_t,
                                col_t, w_t, s);
            if (st != CMG_OK) break;
            if ((st = sell_size_async(&cnt_dev->c, F.n, rp_t, &cnt_dev->sell, s)) != CMG_OK) break;
            st = from_cuda(cudaMemcpyAsync(&hc, cnt_dev, sizeof(hc), cudaMemcpyDeviceToHost, s));
            if (st != CMG_OK) break;
            if ((st = from_cuda(cudaStreamSynchronize(s))) != CMG_OK) break;
            if (hc.gs.err) st = CMG_ERR_DEVICE_TIMEOUT;
        } while (0);
        if (st != CMG_OK || hc.c < 2) {  // c < 2: HEC collapsed the level, it is the coarsest
            release();
            if (st != CMG_OK) return st;
            break;
        }
        LevelData C;
        C.n = hc.c;
        C.nnz = hc.nseg;
        memcpy(&C.g, &hc.gbits, sizeof(double));
        C.sell_nnz = (C.n <= 65536) ? (long long)hc.sell : 0;
        st = dev_alloc_n(&C.rp, (size_t)C.n + 1, s);
        if (st == CMG_OK) st = dev_alloc_n(&C.col, (size_t)std::max<long long>(C.nnz, 1), s);
        if (st == CMG_OK) st = dev_alloc_n(&C.w, (size_t)std::max<long long>(C.nnz, 1), s);
        if (st == CMG_OK)
            st = from_cuda(cudaMemcpyAsync(C.rp, rp_t, sizeof(int) * ((size_t)C.n + 1),
                                           cudaMemcpyDeviceToDevice, s));
        if (st == CMG_OK && C.nnz > 0)
            st = from_cuda(cudaMemcpyAsync(C.col, col_t, sizeof(int) * (size_t)C.nnz,
                                           cudaMemcpyDeviceToDevice, s));
        if (st == CMG_OK && C.nnz > 0)
            st = from_cuda(cudaMemcpyAsync(C.w, w_t, sizeof(double) * (size_t)C.nnz,
                                           cudaMemcpyDeviceToDevice, s));
        h->lv.back().agg = agg;
        agg = nullptr;
        release();
        h->lv.push_back(C);  // freed with the hierarchy, also on error
        if (st != CMG_OK) return st;
        level++;
    }
    // ---- sweep precision per level.  In the FP32 form only levels with at
    // least kFp32MinEntries stored entries sweep in FP32: those carry the
    // bytes that FP32 halves.  Smaller levels keep FP64 sweeps: their sweeps
    // are latency-bound
    // (FP32 saves little there), and they run the longest sweep chains
    // (thousands of sweeps on the coarse levels), along which FP32 rounding
    // accumulates in slowly converging components that the finer levels
    // inherit (measured: up to 3e-6 relative in lambda2 on preferential-
    // attachment graphs whose coarse levels ran in FP32).
    const int form32 = o.precision == CMG_PRECISION_FP32_SWEEP;
    const int nlev = (int)h->lv.size();
    {
        unsigned long long *cnt;
        CMG_TRY(scr.get(&cnt, 1));
        for (int k = 0; k < nlev; k++) {
            LevelData &L = h->lv[k];
            if (k == 0 && L.n <= 65536) CMG_TRY(sell_size(L.n, L.rp, cnt, &L.sell_nnz, s));
            L.fp32 = (form32 && L.nnz >= kFp32MinEntries) ? 1 : 0;
        }
    }
    for (auto &L : h->lv) {
        if (!L.fp32) continue;
        CMG_TRY(dev_alloc_n(&L.w32, (size_t)std::max<long long>(L.nnz, 1), s));
        CMG_TRY(launch_to_float(L.nnz, L.w, L.w32, s));
    }
    // ---- FP64 levels of 512 to a few thousand rows: sweeps in one thread-
    // block cluster (every CTA holds the iterate; rows split over the SMs)
    // (CMG_CLUSTER=0: never; CMG_CLUSTER=<rows>: from that many rows on)
    const char *cl_env = getenv("CMG_CLUSTER");
    if (!cl_env || cl_env[0] != '0') {
        const int cl_min = cl_env ? std::max(128, atoi(cl_env)) : 512;
        std::vector<int> rph;
        for (auto &L : h->lv) {
            if (L.fp32 || L.n < cl_min || !cluster_may_hold(L.n)) continue;
            rph.resize((size_t)L.n + 1);
            CMG_CUDA(cudaMemcpyAsync(rph.data(), L.rp, sizeof(int) * ((size_t)L.n + 1), cudaMemcpyDeviceToHost, s));
            CMG_CUDA(cudaStreamSynchronize(s));
            PiLevel v = level_view(L);
            cluster_plan(&v, rph.data());
            L.cl_ctas = v.cl_ctas;
            L.cl_threads = v.cl_threads;
            L.cl_emax = v.cl_emax;
            L.cl_smem = v.cl_smem;
        }
    }
    // ---- sweep layouts for the levels the shared-memory kernels cannot hold
    size_t lay_bytes = 0;
    std::vector<int> stage_try(nlev, 0), partial_try(nlev, 0);
    std::vector<unsigned long long> below(2 * (size_t)nlev, 0);
    unsigned long long *below_dev = nullptr;
    {
        int *voff1;
        CMG_TRY(scr.get(&voff1, 2));
        CMG_TRY(scr.get(&below_dev, 2 * (size_t)nlev));
        for (int k = 0; k < nlev; k++) {
            LevelData &L = h->lv[k];
            if (L.cl_ctas > 0 || small_level_fits(level_view(L), L.fp32)) continue;
            const int hv[2] = {0, L.n};
            CMG_CUDA(cudaMemcpyAsync(voff1, hv, sizeof(hv), cudaMemcpyHostToDevice, s));
            bool x2 = false;
            CMG_TRY(wants_two_phase(L, &x2, s));
            if (x2) {
                CMG_TRY(build_sweep_layout(1, voff1, std::vector<int>{0, L.n}, L.n, L.rp, L.col, L.w, L.fp32,
                                           &L.lay, &lay_bytes, s, true));
                size_t xb = 0;
                const cmg_status_t st = build_xlayout(L.n, L.nnz, L.rp, L.col, L.w, L.fp32, L.lay.perm, L.lay.inv,
                                                      two_phase_params(), &L.xl, &xb, s);
                if (st == CMG_OK) {
                    L.has_xl = true;
                    L.has_lay = true;
                    lay_bytes += xb;
                    continue;
                }
                // beyond the two-phase layout's limits: the slice layout
                free_xlayout(L.xl, s);
                free_sweep_layout(L.lay, s);
                if (st != CMG_ERR_TOO_LARGE) return st;
            }
            CMG_TRY(build_sweep_layout(1, voff1, std::vector<int>{0, L.n}, L.n, L.rp, L.col, L.w, L.fp32,
                                       &L.lay, &lay_bytes, s));
            L.has_lay = true;
            // gathers that a staged prefix of the iterate would serve
            stage_try[k] = std::min(L.n, stage_capacity(L.fp32));
            if (stage_try[k] > 0) CMG_TRY(layout_count_below(L.lay, stage_try[k], below_dev + k, s));
            if (L.fp32 && stage_try[k] > kPartialStage) {
                partial_try[k] = kPartialStage;
                CMG_TRY(layout_count_below(L.lay, kPartialStage, below_dev + nlev + k, s));
            }
        }
    }
    // ---- solve workspace: an iterate ring per level, results, barrier state
    for (auto &L : h->lv) {
        const size_t esz = L.fp32 ? sizeof(float) : sizeof(double);
        for (int k = 0; k < 3; k++) {
            void *p = nullptr;
            CMG_TRY(dev_alloc(&p, esz * (size_t)L.n, s));
            h->bufs.push_back(p);
        }
        double *gdp = nullptr;
        if (!L.fp32) CMG_TRY(dev_alloc_n(&gdp, (size_t)L.n, s));
        h->gd.push_back(gdp);
    }
    CMG_TRY(dev_alloc_n(&h->res, h->lv.size(), s));
    CMG_TRY(dev_alloc_n(&h->gs, 1, s));
    CMG_TRY(dev_alloc_n(&h->out2, 2, s));
    CMG_TRY(dev_alloc_n(&h->u_dev, (size_t)n, s));
    // ---- bytes held
    size_t bytes = 0;
    for (auto &L : h->lv) {
        bytes += sizeof(int) * ((size_t)L.n + 1) + (sizeof(int) + sizeof(double)) * (size_t)L.nnz;
        if (L.w32) bytes += sizeof(float) * (size_t)L.nnz;
        if (L.agg) bytes += sizeof(int) * (size_t)L.n;
        bytes += 3 * (L.fp32 ? sizeof(float) : sizeof(double)) * (size_t)L.n;
        if (!L.fp32) bytes += sizeof(double) * (size_t)L.n;
    }
    bytes += sizeof(double) * (size_t)n;
    h->bytes = bytes + lay_bytes;
    bool any_stage = false;
    for (int k = 0; k < nlev; k++) any_stage = any_stage || stage_try[k] > 0;
    if (any_stage)
        CMG_CUDA(cudaMemcpyAsync(below.data(), below_dev, sizeof(unsigned long long) * 2 * (size_t)nlev,
                                 cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if (any_stage) {
        // CMG_STAGE=0: never stage the iterate; CMG_STAGE=1: stage it on every
        // level with a sweep layout; otherwise where stage_pays() says so, or
        // a short prefix where partial_stage_pays() does (FP32 sweeps)
        const char *env = getenv("CMG_STAGE");
        const int mode = (env && env[0] == '0') ? 0 : ((env && env[0] == '1') ? 1 : 2);
        DeviceInfo di;
        CMG_TRY(device_info(&di));
        for (int k = 0; k < nlev; k++) {
            const LevelData &L = h->lv[k];
            if (stage_try[k] > 0 && (mode == 1 || (mode == 2 && stage_pays(below[k], L.lay.entries, di.sms))))
                h->lv[k].lay.stage_n = stage_try[k];
            else if (mode == 2 && partial_try[k] > 0 &&
                     partial_stage_pays(below[nlev + k], L.lay.entries, L.n, di.sms))
                h->lv[k].lay.stage_n = partial_try[k];
        }
    }
    return CMG_OK;
}

cmg_status_t cmg::hierarchy_view(cmg_hierarchy_t h, HierarchyView *out) {
    if (!h || !out) return CMG_ERR_INVALID_ARG;
    out->lv.clear();
    for (const auto &L : h->lv) {
        PiLevel v = level_view(L);
        v.w32 = nullptr;
        v.lay = nullptr;
        v.xl = nullptr;
        v.cl_ctas = 0;
        out->lv.push_back(v);
    }
    out->device = h->device;
    out->seed = h->opts.seed;
    out->opts = h->opts;
    out->gs = h->gs;
    return CMG_OK;
}

// ------------------------------------------------------------------ C-ABI
extern "C" {

cmg_status_t cmg_options_default(cmg_options_t *o) {
    if (!o) return CMG_ERR_INVALID_ARG;
    memset(o, 0, sizeof(*o));
    o->tol = 1e-8;
    o->beta = 4.0;
    o->seed = 1412;
    o->coarse_size = 25;
    o->max_levels = CMG_MAX_LEVELS;
    o->precision = CMG_PRECISION_FP64;
    o->schedule = CMG_SCHEDULE_TOL;
    o->k0 = 1;
    o->max_sweeps = 20000;
    o->max_sweeps_coarsest = 100000;
    o->validate = 1;
    return CMG_OK;
}

const char *cmg_status_string(cmg_status_t s) {
    switch (s) {
        case CMG_OK: return "ok";
        case CMG_WARN_MAXITER: return "a sweep cap was reached (result usable)";
        case CMG_ERR_INVALID_ARG: return "invalid argument";
        case CMG_ERR_NOT_SYMMETRIC: return "adjacency matrix not symmetric";
        case CMG_ERR_SELF_LOOP: return "self-loop in the graph";
        case CMG_ERR_BAD_WEIGHT: return "edge weight not finite and positive";
        case CMG_ERR_ISOLATED_VERTEX: return "vertex without neighbours";
        case CMG_ERR_TOO_SMALL: return "graph has fewer than 2 vertices";
        case CMG_ERR_OOM: return "device memory allocation failed";
        case CMG_ERR_CUDA: return "CUDA runtime error";
        case CMG_ERR_DEVICE_TIMEOUT: return "device-side wait timed out";
        case CMG_ERR_BAD_CSR: return "malformed CSR (row pointers, column range or order)";
        case CMG_ERR_TOO_LARGE: return "graph too large";
        case CMG_ERR_TIMEOUT: return "host-side wait timed out";
    }
    return "unknown status";
}

const char *cmg_version(void) { return "cmg-gb300 1.0 sm_103a"; }

cmg_status_t cmg_setup(int64_t n, const int64_t *row_ptr, const int32_t *col, const double *w,
                       int32_t mem, const cmg_options_t *opts, void *stream, cmg_hierarchy_t *out) {
    if (!out) return CMG_ERR_INVALID_ARG;
    *out = nullptr;
    if (!row_ptr || (mem != CMG_MEM_HOST && mem != CMG_MEM_DEVICE)) return CMG_ERR_INVALID_ARG;
    if (n < 2) return CMG_ERR_TOO_SMALL;
    if (n >= 2147483647ll) return CMG_ERR_TOO_LARGE;
    cmg_options_t o;
    if (opts) o = *opts;
    else cmg_options_default(&o);
    CMG_TRY(check_options(o));
    if (!col || !w) return CMG_ERR_INVALID_ARG;
    cmg_hierarchy_s *h = new cmg_hierarchy_s();
    h->opts = o;
    h->stream = (cudaStream_t)stream;
    cudaGetDevice(&h->device);
    cmg_status_t st = build_hierarchy(h, n, row_ptr, col, w, mem);
    if (st != CMG_OK) {
        free_hierarchy(h);
        return st;
    }
    *out = h;
    return CMG_OK;
}


// Alg. 1 Steps 2-3 on a resident hierarchy.  seed keys the Gaussian start of
// Step 2; x0 (device, nullable) replaces the cascade above level x0_level by
// a given start vector on that level (levels above it are not visited).
static cmg_status_t fiedler_impl(cmg_hierarchy_t h, uint64_t seed, const double *x0, int x0_level,
                                 double *u_out, int32_t u_mem, double *lambda2_out,
                                 cmg_stats_t *stats_out, cudaStream_t s) {
    const cmg_options_t &o = h->opts;
    const int J = (int)h->lv.size() - 1;
    const int top = x0 ? x0_level : J;
    std::vector<PiLevel> views(J + 1);
    for (int j = 0; j <= J; j++) views[j] = level_view(h->lv[j]);
    // one error flag for every launch of this call (a timeout in any of them
    // must reach the status)
    cmg_status_t st = gs_clear(h->gs, s);
    const bool timing = o.timing != 0;
    std::vector<cudaEvent_t> ev;
    if (timing) {
        ev.resize(2 * (J + 2));
        for (auto &e : ev)
            if (cudaEventCreate(&e) != cudaSuccess) st = CMG_ERR_CUDA;
    }
    for (int j = top; j >= 0 && st == CMG_OK; j--) {
        PiRun r = {};
        r.lv = &views[j];
        r.fp32 = h->lv[j].fp32;
        r.tol = o.tol;
        r.seed = seed;
        r.max_sweeps = (j == J) ? o.max_sweeps_coarsest : o.max_sweeps;
        r.mode = 0;
        if (o.schedule == CMG_SCHEDULE_FIXED && j < J) {
            r.mode = 1;
            r.k_fixed = (int)ceil((double)o.k0 * pow(o.beta, (double)j));
        } else if (o.schedule == CMG_SCHEDULE_REPLAY) {
            r.mode = 1;
            r.k_fixed = o.replay_sweeps[j];
        }
        if (j == top && x0) {
            r.x_init = x0;
        } else if (j < J) {
            for (int k = 0; k < 3; k++) r.coarse_bufs[k] = h->bufs[3 * (j + 1) + k];
            r.coarse_fp64 = h->lv[j + 1].fp32 ? 0 : 1;
            r.coarse_res = h->res + (j + 1);
            r.coarse_agg = h->lv[j].agg;
            r.coarse_inv = h->lv[j + 1].has_lay ? h->lv[j + 1].lay.inv : nullptr;
        }
        for (int k = 0; k < 3; k++) r.bufs[k] = h->bufs[3 * j + k];
        r.gd = h->gd[j];
        r.res = h->res + j;
        if (timing) cudaEventRecord(ev[2 * j], s);
        st = power_iteration(r, h->gs, s);
        if (timing) cudaEventRecord(ev[2 * j + 1], s);
    }
    double *u_dev = (u_out && u_mem == CMG_MEM_DEVICE) ? u_out : h->u_dev;
    if (timing && st == CMG_OK) cudaEventRecord(ev[2 * (J + 1)], s);
    if (st == CMG_OK)
        st = finalize(views[0], h->lv[0].fp32, &h->bufs[0], h->res, u_dev, 1, 0, h->out2, h->gs, s);
    if (timing && st == CMG_OK) cudaEventRecord(ev[2 * (J + 1) + 1], s);
    std::vector<PiResult> hr(J + 1);
    double out2[2] = {0.0, 0.0};
    GridSync hgs = {};
    if (st == CMG_OK) {
        cudaError_t e = cudaMemcpyAsync(hr.data(), h->res, sizeof(PiResult) * (J + 1),
                                        cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out2, h->out2, sizeof(out2), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hgs, h->gs, sizeof(hgs), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && u_out && u_mem == CMG_MEM_HOST)
            e = cudaMemcpyAsync(u_out, u_dev, sizeof(double) * (size_t)h->lv[0].n,
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = from_cuda(e);
    }
    if (st == CMG_OK && hgs.err) st = CMG_ERR_DEVICE_TIMEOUT;
    std::vector<double> level_ms(J + 2, 0.0);
    if (timing) {
        for (int j = 0; j <= J + 1 && st == CMG_OK; j++) {
            if (j <= J && j > top) continue;
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[2 * j], ev[2 * j + 1]) == cudaSuccess) level_ms[j] = ms;
        }
        for (auto &e : ev) cudaEventDestroy(e);
    }
    if (st != CMG_OK) return st;
    // levels above the start level were not visited in this solve
    for (int j = top + 1; j <= J; j++) hr[j] = PiResult{};
    int capped = 0;
    for (int j = 0; j <= top; j++) capped |= hr[j].capped;
    if (lambda2_out) *lambda2_out = out2[0];
    if (stats_out) {
        memset(stats_out, 0, sizeof(*stats_out));
        stats_out->lambda2 = out2[0];
        stats_out->residual = out2[1];
        stats_out->levels = J + 1;
        stats_out->status = capped ? CMG_WARN_MAXITER : CMG_OK;
        for (int j = 0; j <= J; j++) {
            stats_out->n[j] = h->lv[j].n;
            stats_out->nnz[j] = h->lv[j].nnz;
            stats_out->sweeps[j] = hr[j].sweeps;
            stats_out->cos_final[j] = hr[j].cos;
            stats_out->level_ms[j] = level_ms[j];
        }
        stats_out->finalize_ms = level_ms[J + 1];
    }
    return capped ? CMG_WARN_MAXITER : CMG_OK;
}

cmg_status_t cmg_fiedler(cmg_hierarchy_t h, double *u_out, int32_t u_mem, double *lambda2_out,
                         cmg_stats_t *stats_out, void *stream) {
    if (!h) return CMG_ERR_INVALID_ARG;
    cmg_solve_options_t so;
    cmg_solve_options_default(h, &so);
    return cmg_fiedler_ex(h, &so, u_out, u_mem, lambda2_out, stats_out, stream);
}

cmg_status_t cmg_solve_options_default(cmg_hierarchy_t h, cmg_solve_options_t *so) {
    if (!so) return CMG_ERR_INVALID_ARG;
    memset(so, 0, sizeof(*so));
    so->seed = h ? h->opts.seed : 1412;
    so->x0_mem = CMG_MEM_HOST;
    return CMG_OK;
}

cmg_status_t cmg_fiedler_ex(cmg_hierarchy_t h, const cmg_solve_options_t *so, double *u_out,
                            int32_t u_mem, double *lambda2_out, cmg_stats_t *stats_out,
                            void *stream) {
    if (!h || !so) return CMG_ERR_INVALID_ARG;
    if (u_out && u_mem != CMG_MEM_HOST && u_mem != CMG_MEM_DEVICE) return CMG_ERR_INVALID_ARG;
    for (int k = 0; k < 4; k++)
        if (so->reserved[k] != 0) return CMG_ERR_INVALID_ARG;
    const int J = (int)h->lv.size() - 1;
    if (so->x0 && (so->x0_level < 0 || so->x0_level > J ||
                   (so->x0_mem != CMG_MEM_HOST && so->x0_mem != CMG_MEM_DEVICE)))
        return CMG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int prev = 0;
    CMG_CUDA(cudaGetDevice(&prev));
    if (prev != h->device) CMG_CUDA(cudaSetDevice(h->device));
    const double *x0 = so->x0;
    cmg_status_t st = CMG_OK;
    if (x0 && so->x0_mem == CMG_MEM_HOST) {
        // staged in the final-vector buffer (n_0 >= n of any level), which the
        // solve writes only after the start level's power iteration has read it
        const size_t nb = sizeof(double) * (size_t)h->lv[so->x0_level].n;
        st = from_cuda(cudaMemcpyAsync(h->u_dev, x0, nb, cudaMemcpyHostToDevice, s));
        x0 = h->u_dev;
    }
    if (st == CMG_OK)
        st = fiedler_impl(h, so->seed, x0, so->x0_level, u_out, u_mem, lambda2_out, stats_out, s);
    if (prev != h->device) cudaSetDevice(prev);
    return st;
}

cmg_status_t cmg_hierarchy_info(cmg_hierarchy_t h, int32_t *levels, int64_t *n_per_level,
                                int64_t *nnz_per_level) {
    if (!h) return CMG_ERR_INVALID_ARG;
    if (levels) *levels = (int32_t)h->lv.size();
    for (size_t j = 0; j < h->lv.size(); j++) {
        if (n_per_level) n_per_level[j] = h->lv[j].n;
        if (nnz_per_level) nnz_per_level[j] = h->lv[j].nnz;
    }
    return CMG_OK;
}

cmg_status_t cmg_level_kernels(cmg_hierarchy_t h, int32_t *kind_out, int32_t *staged_out) {
    if (!h) return CMG_ERR_INVALID_ARG;
    for (size_t j = 0; j < h->lv.size(); j++) {
        const LevelData &L = h->lv[j];
        const int staged = L.has_lay ? L.lay.stage_n : 0;
        int kind = 0;
        if (L.cl_ctas > 0) kind = 5;
        else if (L.has_xl) kind = 4;
        else if (L.has_lay) kind = staged > 0 ? 2 : 1;
        else if (!small_level_fits(level_view(L), L.fp32)) kind = 3;
        if (kind_out) kind_out[j] = kind;
        if (staged_out) staged_out[j] = staged;
    }
    return CMG_OK;
}

cmg_status_t cmg_level_precision(cmg_hierarchy_t h, int32_t *prec_out) {
    if (!h || !prec_out) return CMG_ERR_INVALID_ARG;
    for (size_t j = 0; j < h->lv.size(); j++)
        prec_out[j] = h->lv[j].fp32 ? CMG_PRECISION_FP32_SWEEP : CMG_PRECISION_FP64;
    return CMG_OK;
}

cmg_status_t cmg_hierarchy_device_bytes(cmg_hierarchy_t h, size_t *bytes) {
    if (!h || !bytes) return CMG_ERR_INVALID_ARG;
    *bytes = h->bytes;
    return CMG_OK;
}

cmg_status_t cmg_estimate_device_bytes(int64_t n, int64_t nnz, int32_t precision, size_t *bytes) {
    if (!bytes || n < 0 || nnz < 0) return CMG_ERR_INVALID_ARG;
    // levels: the input plus coarse levels (at most n/2 vertices and nnz
    // entries per level, geometric in practice: budget 2x level 0), the
    // solve buffers, and the transient setup scratch of level 0
    // (sort keys/values double-buffered: 4 * 12 B per entry).
    const double wb = (precision == CMG_PRECISION_FP32_SWEEP) ? 16.0 : 12.0;
    const double vb = (precision == CMG_PRECISION_FP32_SWEEP) ? 8.0 : 16.0;
    double b = 2.0 * (wb * (double)nnz + (4.0 + 4.0 + vb) * (double)n) + 8.0 * (double)n;
    b += 48.0 * (double)nnz + 32.0 * (double)n + (1 << 20);
    *bytes = (size_t)b;
    return CMG_OK;
}

cmg_status_t cmg_get_aggregates(cmg_hierarchy_t h, int32_t level, int32_t *agg_out) {
    if (!h || !agg_out || level < 0 || level >= (int)h->lv.size() - 1) return CMG_ERR_INVALID_ARG;
    const LevelData &L = h->lv[level];
    CMG_CUDA(cudaMemcpyAsync(agg_out, L.agg, sizeof(int) * (size_t)L.n, cudaMemcpyDeviceToHost,
                             h->stream));
    CMG_CUDA(cudaStreamSynchronize(h->stream));
    return CMG_OK;
}

cmg_status_t cmg_get_level_csr(cmg_hierarchy_t h, int32_t level, int64_t *row_ptr, int32_t *col,
                               double *w, double *g_out) {
    if (!h || level < 0 || level >= (int)h->lv.size()) return CMG_ERR_INVALID_ARG;
    const LevelData &L = h->lv[level];
    cudaStream_t s = h->stream;
    if (row_ptr) {
        std::vector<int> tmp((size_t)L.n + 1);
        CMG_CUDA(cudaMemcpyAsync(tmp.data(), L.rp, sizeof(int) * tmp.size(), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
        for (size_t i = 0; i < tmp.size(); i++) row_ptr[i] = tmp[i];
    }
    if (col && L.nnz)
        CMG_CUDA(cudaMemcpyAsync(col, L.col, sizeof(int) * (size_t)L.nnz, cudaMemcpyDeviceToHost, s));
    if (w && L.nnz)
        CMG_CUDA(cudaMemcpyAsync(w, L.w, sizeof(double) * (size_t)L.nnz, cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if (g_out) *g_out = L.g;
    return CMG_OK;
}

cmg_status_t cmg_free(cmg_hierarchy_t h) {
    if (!h) return CMG_ERR_INVALID_ARG;
    free_hierarchy(h);
    return CMG_OK;
}

// ------------------------------------------------------------------ step entry points
static cmg_status_t read_nnz(const int32_t *rp, int32_t n, cudaStream_t s, long long *nnz) {
    int v = 0;
    CMG_CUDA(cudaMemcpyAsync(&v, rp + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    *nnz = v;
    return CMG_OK;
}

cmg_status_t cmg_heaviest_neighbour(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                    const double *w, int32_t *m_out, void *stream) {
    if (n < 0 || (n > 0 && (!row_ptr || !col || !w || !m_out))) return CMG_ERR_INVALID_ARG;
    if (n == 0) return CMG_OK;
    cudaStream_t s = (cudaStream_t)stream;
    long long nnz;
    CMG_TRY(read_nnz(row_ptr, n, s, &nnz));
    return launch_heaviest(n, (double)nnz / (double)n, row_ptr, col, w, m_out, s);
}

cmg_status_t cmg_visit_ranks(int32_t n, uint64_t seed, int32_t level, uint32_t *rank_out,
                             void *stream) {
    if (n < 0 || (n > 0 && !rank_out)) return CMG_ERR_INVALID_ARG;
    return launch_ranks(n, seed, level, rank_out, (cudaStream_t)stream);
}

cmg_status_t cmg_hec_aggregate(int32_t n, const int32_t *row_ptr, const int32_t *col,
                               const double *w, const uint32_t *rank, int32_t *agg_out,
                               int64_t *c_out, void *stream) {
    if (n < 1 || !row_ptr || !col || !w || !rank || !agg_out) return CMG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    long long nnz;
    CMG_TRY(read_nnz(row_ptr, n, s, &nnz));
    int c = 0;
    CMG_TRY(hec_level(n, nnz, row_ptr, col, w, 0, 0, rank, agg_out, &c, s));
    if (c_out) *c_out = c;
    return CMG_OK;
}

cmg_status_t cmg_power_sweeps(int32_t n, const int32_t *row_ptr, const int32_t *col,
                              const double *w, double g, const double *x_in, int32_t k,
                              double *u_out, double *cos_out, void *stream) {
    if (n < 2 || !row_ptr || !col || !w || !x_in || !u_out || k < 0) return CMG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    long long nnz;
    CMG_TRY(read_nnz(row_ptr, n, s, &nnz));
    Scratch scr(s);
    if (!(g > 0.0)) {
        double *gd;
        CMG_TRY(scr.get(&gd, 1));
        CMG_TRY(launch_gershgorin(n, row_ptr, w, gd, s));
        CMG_CUDA(cudaMemcpyAsync(&g, gd, sizeof(double), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
    }
    PiLevel lv = {};
    lv.n = n;
    lv.nnz = nnz;
    lv.rp = row_ptr;
    lv.col = col;
    lv.w = w;
    lv.g = g;
    double *b[3], *gd, *out2;
    PiResult *res;
    GridSync *gs;
    for (int q = 0; q < 3; q++) CMG_TRY(scr.get(&b[q], n));
    CMG_TRY(scr.get(&gd, n));
    CMG_TRY(scr.get(&res, 1));
    CMG_TRY(scr.get(&gs, 1));
    CMG_TRY(scr.get(&out2, 2));
    CMG_TRY(gs_clear(gs, s));
    PiRun r = {};
    r.lv = &lv;
    r.mode = 1;
    r.k_fixed = k;
    r.max_sweeps = k;
    r.x_init = x_in;
    for (int q = 0; q < 3; q++) r.bufs[q] = b[q];
    r.gd = gd;
    r.res = res;
    void *bv[3] = {b[0], b[1], b[2]};
    CMG_TRY(power_iteration(r, gs, s));
    CMG_TRY(finalize(lv, 0, bv, res, u_out, 0, 0, out2, gs, s));
    PiResult hr;
    GridSync hgs;
    CMG_CUDA(cudaMemcpyAsync(&hr, res, sizeof(hr), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(&hgs, gs, sizeof(hgs), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if (hgs.err) return CMG_ERR_DEVICE_TIMEOUT;
    if (cos_out) *cos_out = hr.cos;
    return CMG_OK;
}

cmg_status_t cmg_rayleigh_residual(int32_t n, const int32_t *row_ptr, const int32_t *col,
                                   const double *w, const double *u, double *lambda_out,
                                   double *residual_out, void *stream) {
    if (n < 1 || !row_ptr || !col || !w || !u) return CMG_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    long long nnz;
    CMG_TRY(read_nnz(row_ptr, n, s, &nnz));
    PiLevel lv = {};
    lv.n = n;
    lv.nnz = nnz;
    lv.rp = row_ptr;
    lv.col = col;
    lv.w = w;
    Scratch scr(s);
    double *out2;
    GridSync *gs;
    CMG_TRY(scr.get(&out2, 2));
    CMG_TRY(scr.get(&gs, 1));
    CMG_TRY(gs_clear(gs, s));
    CMG_TRY(finalize(lv, 0, nullptr, nullptr, const_cast<double *>(u), 0, 1, out2, gs, s));
    double h2[2];
    GridSync hgs;
    CMG_CUDA(cudaMemcpyAsync(h2, out2, sizeof(h2), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(&hgs, gs, sizeof(hgs), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if (hgs.err) return CMG_ERR_DEVICE_TIMEOUT;
    if (lambda_out) *lambda_out = h2[0];
    if (residual_out) *residual_out = h2[1];
    return CMG_OK;
}

cmg_status_t cmg_kernel_launches(uint64_t *count) {
    if (!count) return CMG_ERR_INVALID_ARG;
    *count = launches_issued();
    return CMG_OK;
}

cmg_status_t cmg_debug_fail_alloc_after(int64_t k) {
    debug_fail_alloc_after(k);
    return CMG_OK;
}

cmg_status_t cmg_debug_stall_barrier(int64_t launch, int32_t barrier) {
    if (launch >= 0 && (barrier < 0 || barrier > 254)) return CMG_ERR_INVALID_ARG;
    debug_stall_barrier(launch, barrier);
    return CMG_OK;
}

}  // extern "C"
