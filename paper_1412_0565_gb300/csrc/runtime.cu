// runtime.cu -- error mapping, the library's device memory pool, device
// properties and cooperative-launch helpers.
#include <stddef.h>
#include <stdio.h>
#include <stdlib.h>

#include <atomic>
#include <mutex>

#include "internal.h"

namespace cmg {

cmg_status_t from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return CMG_OK;
    cudaGetLastError();  // clear a non-sticky error so the context stays usable
    if (e == cudaErrorMemoryAllocation) return CMG_ERR_OOM;
    return CMG_ERR_CUDA;
}

cmg_status_t from_cuda_at(cudaError_t e, const char *file, int line) {
    if (e != cudaSuccess) {
        static const bool report = getenv("CMG_DEBUG_ERRORS") != nullptr;
        if (report) fprintf(stderr, "cmg: %s at %s:%d\n", cudaGetErrorName(e), file, line);
    }
    return from_cuda(e);
}

namespace {
std::atomic<unsigned long long> g_launches{0};
}

cmg_status_t launch_status() {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return from_cuda_at(cudaGetLastError(), "kernel launch", 0);
}

unsigned long long launches_issued() { return g_launches.load(std::memory_order_relaxed); }

void add_launches(long long k) { g_launches.fetch_add((unsigned long long)k, std::memory_order_relaxed); }

// ----------------------------------------------------------------- memory pool
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[kMaxDevices] = {};
DeviceInfo g_info[kMaxDevices] = {};
bool g_info_ok[kMaxDevices] = {};
// test hook: the k-th next allocation fails (-1 = never)
std::atomic<long long> g_fail_after{-1};

cmg_status_t pool_for(int dev, cudaMemPool_t *out) {
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    if (dev < 0 || dev >= kMaxDevices) return CMG_ERR_CUDA;
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        CMG_CUDA(cudaMemPoolCreate(&p, &props));
        // keep freed blocks cached in the pool between calls
        uint64_t thr = ~0ull;
        CMG_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr));
        g_pool[dev] = p;
    }
    *out = g_pool[dev];
    return CMG_OK;
}
}  // namespace

cmg_status_t dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    long long f = g_fail_after.load();
    if (f >= 0) {
        if (f == 0) {
            g_fail_after.store(-1);
            return CMG_ERR_OOM;
        }
        g_fail_after.store(f - 1);
    }
    int dev = 0;
    CMG_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    CMG_TRY(pool_for(dev, &pool));
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
    if (e != cudaSuccess) {
        *p = nullptr;
        return from_cuda(e);
    }
    return CMG_OK;
}

void dev_free(void *p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

void debug_fail_alloc_after(long long k) { g_fail_after.store(k); }

cmg_status_t pool_used_high(size_t *high, int reset) {
    int dev = 0;
    CMG_CUDA(cudaGetDevice(&dev));
    cudaMemPool_t pool;
    CMG_TRY(pool_for(dev, &pool));
    if (reset) {
        uint64_t zero = 0;
        CMG_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    }
    uint64_t v = 0;
    CMG_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &v));
    if (high) *high = (size_t)v;
    return CMG_OK;
}

cmg_status_t device_info(DeviceInfo *out) {
    int dev = 0;
    CMG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return CMG_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lk(g_pool_mutex);
        if (g_info_ok[dev]) {
            *out = g_info[dev];
            return CMG_OK;
        }
    }
    DeviceInfo d;
    d.device = dev;
    CMG_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
    CMG_CUDA(cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    CMG_CUDA(cudaDeviceGetAttribute(&d.l2_bytes, cudaDevAttrL2CacheSize, dev));
    std::lock_guard<std::mutex> lk(g_pool_mutex);
    g_info[dev] = d;
    g_info_ok[dev] = true;
    *out = d;
    return CMG_OK;
}

int grid_for(long long work, int per_cta, int waves) {
    DeviceInfo d;
    int sms = 148;
    if (device_info(&d) == CMG_OK) sms = d.sms;
    long long b = (work + per_cta - 1) / per_cta;
    const long long cap = (long long)sms * 8 * waves;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (int)b;
}

cmg_status_t allow_max_dynamic_smem(const void *kernel) {
    DeviceInfo d;
    CMG_TRY(device_info(&d));
    // static plus dynamic shared memory may not exceed the opt-in maximum
    cudaFuncAttributes fa;
    CMG_CUDA(cudaFuncGetAttributes(&fa, kernel));
    const int dyn = d.max_smem_optin - (int)fa.sharedSizeBytes;
    CMG_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    return CMG_OK;
}

cmg_status_t coop_max_blocks(const void *kernel, int threads, size_t smem, int *out) {
    DeviceInfo d;
    CMG_TRY(device_info(&d));
    int per_sm = 0;
    CMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
    if (per_sm < 1) return CMG_ERR_CUDA;
    *out = per_sm * d.sms;
    return CMG_OK;
}

namespace {
// stall hook: multi-CTA cooperative launches still to pass before the held
// one (-1: off), and the barrier it holds
std::atomic<long long> g_stall_launch{-1};
std::atomic<int> g_stall_barrier{0};
}  // namespace

void debug_stall_barrier(long long launch, int barrier) {
    g_stall_barrier.store(barrier);
    g_stall_launch.store(launch);
}

cmg_status_t gs_clear(GridSync *gs, cudaStream_t s) {
    CMG_CUDA(cudaMemsetAsync(gs, 0, sizeof(GridSync), s));
    return CMG_OK;
}

cmg_status_t coop_launch(const void *kernel, int blocks, int threads, size_t smem,
                         cudaStream_t s, void **args, GridSync *gs) {
    // count, gen and stall lie before err, which this leaves alone
    static_assert(offsetof(GridSync, err) == 3 * sizeof(unsigned int), "GridSync layout");
    int hold = 0;
    if (blocks > 1) {
        long long k = g_stall_launch.load();
        while (k >= 0 && !g_stall_launch.compare_exchange_weak(k, k - 1)) {
        }
        if (k == 0) {
            const int b = g_stall_barrier.load();
            hold = 1 + (b < 0 ? 0 : (b > 254 ? 254 : b));
        }
    }
    if (hold == 0) {
        CMG_CUDA(cudaMemsetAsync(gs, 0, 3 * sizeof(unsigned int), s));
    } else {
        CMG_CUDA(cudaMemsetAsync(gs, 0, 2 * sizeof(unsigned int), s));
        // every byte of the stall word is 1 + the barrier index; the barrier
        // reads the low one
        CMG_CUDA(cudaMemsetAsync(&gs->stall, hold, sizeof(unsigned int), s));
    }
    CMG_CUDA(cudaLaunchCooperativeKernel(kernel, dim3(blocks), dim3(threads), args, smem, s));
    return launch_status();
}

}  // namespace cmg
