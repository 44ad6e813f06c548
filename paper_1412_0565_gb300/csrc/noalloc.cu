// noalloc.cu -- cmg_power_sweeps_noalloc: the fixed-count power sweeps of
// cmg_power_sweeps without any device allocation.
//
// Its scratch (three iterate vectors, g - d_i, row tiles, partial sums, the result
// record, barrier state and the shift) lives in one file-scope __device__
// array.  Host code must not use the array's name as a device address: each
// call looks the address up with cudaGetSymbolAddress on the current device
// (the first lookup on a device loads the module there).  Every call on a device
// shares the array, so calls whose work overlaps on the GPU race; everything
// that must start from zero is cleared by the call itself.
#include "internal.h"

namespace {

constexpr int kMaxN = CMG_NOALLOC_MAX_N;
constexpr long long kMaxNnz = CMG_NOALLOC_MAX_NNZ;
constexpr int kTileCap = 2048;             // >= (kMaxNnz + 4 kMaxN) / 3840 + 2
constexpr int kPartCap = 2 * 1024 * 5;     // sweep partial sums, up to 1024 CTAs
constexpr int kFinCap = 12 * 1024;         // final-pass partial sums, up to 1024 CTAs

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kVec = align256(sizeof(double) * kMaxN);
constexpr size_t kOffB0 = 0;                 // iterate ring: 3 vectors
constexpr size_t kOffGd = kOffB0 + 3 * kVec; // g - d_i
constexpr size_t kOffTiles = kOffGd + kVec;
constexpr size_t kOffPart = kOffTiles + align256(sizeof(int) * kTileCap);
constexpr size_t kOffFin = kOffPart + align256(sizeof(double) * kPartCap);
constexpr size_t kOffRes = kOffFin + align256(sizeof(double) * kFinCap);
constexpr size_t kOffSync = kOffRes + align256(sizeof(cmg::PiResult));
constexpr size_t kOffOut = kOffSync + align256(sizeof(cmg::GridSync));
constexpr size_t kOffG = kOffOut + align256(2 * sizeof(double));
constexpr size_t kBytes = kOffG + align256(sizeof(double));

// The scratch of every cmg_power_sweeps_noalloc call on this device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kBytes];

// Device address of the scratch array on the current device.  Looked up on
// every call (cudaGetSymbolAddress allocates nothing): a cached address
// would go stale if the context were destroyed and the module loaded again.
cmg_status_t scratch_base(unsigned char **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cmg::from_cuda(e != cudaSuccess ? e : cudaErrorUnknown);
    *out = static_cast<unsigned char *>(p);
    return CMG_OK;
}

}  // namespace

extern "C" cmg_status_t cmg_power_sweeps_noalloc(int32_t n, const int32_t *row_ptr,
                                                 const int32_t *col, const double *w, double g,
                                                 const double *x_in, int32_t k, double *u_out,
                                                 double *cos_out, void *stream) {
    using namespace cmg;
    if (n < 2 || !row_ptr || !col || !w || !x_in || !u_out || k < 0) return CMG_ERR_INVALID_ARG;
    if (n > kMaxN) return CMG_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    CMG_TRY(scratch_base(&base));
    int nnz_i = 0;
    CMG_CUDA(cudaMemcpyAsync(&nnz_i, row_ptr + n, sizeof(int), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    const long long nnz = nnz_i;
    if (nnz < 0) return CMG_ERR_INVALID_ARG;
    if (nnz > kMaxNnz) return CMG_ERR_TOO_LARGE;
    void *ring[3];
    for (int q = 0; q < 3; q++) ring[q] = base + kOffB0 + q * kVec;
    double *gdv = reinterpret_cast<double *>(base + kOffGd);
    PiResult *res = reinterpret_cast<PiResult *>(base + kOffRes);
    GridSync *gs = reinterpret_cast<GridSync *>(base + kOffSync);
    double *out2 = reinterpret_cast<double *>(base + kOffOut);
    double *gdev = reinterpret_cast<double *>(base + kOffG);
    CMG_TRY(gs_clear(gs, s));
    if (!(g > 0.0)) {
        CMG_TRY(launch_gershgorin(n, row_ptr, w, gdev, s));
        CMG_CUDA(cudaMemcpyAsync(&g, gdev, sizeof(double), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
    }
    PiLevel lv = {};
    lv.n = n;
    lv.nnz = nnz;
    lv.rp = row_ptr;
    lv.col = col;
    lv.w = w;
    lv.g = g;
    PiWorkspace ws;
    ws.tile_row = reinterpret_cast<int *>(base + kOffTiles);
    ws.tile_cap = kTileCap;
    ws.partials = reinterpret_cast<double *>(base + kOffPart);
    ws.partials_cap = kPartCap;
    ws.fin_part = reinterpret_cast<double *>(base + kOffFin);
    ws.fin_part_cap = kFinCap;
    PiRun r = {};
    r.lv = &lv;
    r.mode = 1;
    r.k_fixed = k;
    r.max_sweeps = k;
    r.x_init = x_in;
    for (int q = 0; q < 3; q++) r.bufs[q] = ring[q];
    r.gd = gdv;
    r.res = res;
    CMG_TRY(power_iteration(r, gs, s, &ws));
    CMG_TRY(finalize(lv, 0, ring, res, u_out, 0, 0, out2, gs, s, &ws));
    PiResult hr;
    GridSync hgs;
    CMG_CUDA(cudaMemcpyAsync(&hr, res, sizeof(hr), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(&hgs, gs, sizeof(hgs), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if (hgs.err) return CMG_ERR_DEVICE_TIMEOUT;
    if (cos_out) *cos_out = hr.cos;
    return CMG_OK;
}
