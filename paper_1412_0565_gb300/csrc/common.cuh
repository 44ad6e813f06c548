// common.cuh -- internal helpers of libcmg (not part of the C-ABI).
//
// Error mapping, the library's stream-ordered device memory pool, a bounded
// grid-wide barrier for cooperative persistent kernels, and warp/block
// reductions with a fixed combination order (results are bitwise
// reproducible from run to run).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/cmg.h"

namespace cmg {

// ----------------------------------------------------------------- errors
cmg_status_t from_cuda(cudaError_t e);
// from_cuda for the call at file:line; with CMG_DEBUG_ERRORS set in the
// environment the failing call is reported on stderr.
cmg_status_t from_cuda_at(cudaError_t e, const char *file, int line);

#define CMG_TRY(expr)                                                        \
    do {                                                                     \
        cmg_status_t _st = (expr);                                           \
        if (_st != CMG_OK && _st != CMG_WARN_MAXITER) return _st;            \
    } while (0)

#define CMG_CUDA(expr)                                                       \
    do {                                                                     \
        cudaError_t _ce = (expr);                                            \
        if (_ce != cudaSuccess) return ::cmg::from_cuda_at(_ce, __FILE__, __LINE__); \
    } while (0)

// Status of the last kernel launch (launch-configuration errors only); also
// counts the launch.  Every kernel launch of the library is followed by it.
cmg_status_t launch_status();
unsigned long long launches_issued();
// Adjusts the launch count (kernels replayed from a CUDA graph count when replayed).
void add_launches(long long k);

// ----------------------------------------------------------------- memory
// Stream-ordered allocations from a library-owned pool on the current device.
cmg_status_t dev_alloc(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);
// Test hook: make the k-th next allocation fail with CMG_ERR_OOM (k < 0: off).
void debug_fail_alloc_after(long long k);
// Most bytes of the current device's pool in use at once since the last
// reset (a measurement of the driver's, not the library's bookkeeping);
// reset != 0 restarts it from the bytes in use now.
cmg_status_t pool_used_high(size_t *high, int reset);

template <typename T>
cmg_status_t dev_alloc_n(T **p, size_t count, cudaStream_t s) {
    return dev_alloc(reinterpret_cast<void **>(p), count * sizeof(T), s);
}

// Frees every registered pointer (stream-ordered) when it goes out of scope.
struct Scratch {
    cudaStream_t stream;
    std::vector<void *> ptrs;
    explicit Scratch(cudaStream_t s) : stream(s) {}
    ~Scratch() {
        for (void *p : ptrs) dev_free(p, stream);
    }
    template <typename T>
    cmg_status_t get(T **p, size_t count) {
        cmg_status_t st = dev_alloc_n(p, count ? count : 1, stream);
        if (st == CMG_OK) ptrs.push_back(*p);
        return st;
    }
    Scratch(const Scratch &) = delete;
    Scratch &operator=(const Scratch &) = delete;
};

// Device properties of the current device (cached).
struct DeviceInfo {
    int device;
    int sms;
    int max_smem_optin;
    int l2_bytes;
};
cmg_status_t device_info(DeviceInfo *out);

// ----------------------------------------------------------------- grid barrier
// State of one cooperative launch.  `count` and `gen` implement a sense-free
// generation barrier and are cleared before every launch; `err` records a
// barrier wait that ran out of time and is cleared once per API call, so a
// timeout in any launch of a call reaches the host (every later launch of
// the call returns at its first barrier).  `stall` is a test hook: when its
// low byte is b > 0, barrier number b - 1 of the launch is never released,
// so its waits run out (after kStallTimeoutNs); 0 in normal operation.
struct GridSync {
    unsigned int count;
    unsigned int gen;
    unsigned int stall;
    unsigned int err;
};

// Nanoseconds since an arbitrary origin (device global timer).
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// A barrier wait gives up after this long and sets GridSync::err.
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;
// The same for a launch with the stall hook armed (keeps its test short).
constexpr unsigned long long kStallTimeoutNs = 20000000ull;

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int ld_relaxed_gpu(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__device__ __forceinline__ void st_relaxed_gpu(unsigned int *p, unsigned int v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void red_add_release_gpu(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" :: "l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  Every
// thread of every CTA must call it.  Arrival is an acq_rel atomic on a
// counter (releasing the CTA's writes, ordered before it by __syncthreads);
// the last arriver resets the counter and releases a generation number that
// the others poll with acquire loads.  A wait gives up after
// kBarrierTimeoutNs and sets GridSync::err; a wait also ends as soon as err
// is seen set.  Returns false (in every thread of the CTA) when this or an
// earlier barrier of the call timed out; callers then return.
__device__ __forceinline__ bool grid_sync(GridSync *gs) {
    __shared__ int s_ok;
    __syncthreads();
    if (gridDim.x == 1) return true;
    if (threadIdx.x == 0) {
        // the hook word is read beside the arrival, off its critical path
        const unsigned int stall = ld_relaxed_gpu(&gs->stall) & 0xffu;
        const unsigned int g0 = ld_relaxed_gpu(&gs->gen);
        const unsigned int arrived = atom_add_acq_rel_gpu(&gs->count, 1u);
        const bool held = stall != 0u && stall == g0 + 1u;
        const unsigned long long limit = stall ? kStallTimeoutNs : kBarrierTimeoutNs;
        int ok = 1;
        if (arrived == gridDim.x - 1 && !held) {
            st_relaxed_gpu(&gs->count, 0u);
            red_add_release_gpu(&gs->gen, 1u);
        } else {
            unsigned long long t0 = 0;
            for (unsigned int spin = 0;; spin++) {
                if (ld_acquire_gpu(&gs->gen) != g0) break;
                if ((spin & 1023u) == 1023u) {
                    const unsigned long long t = global_ns();
                    if (t0 == 0) {
                        t0 = t;
                    } else if (t - t0 > limit) {
                        atomicExch(&gs->err, 1u);
                        ok = 0;
                        break;
                    }
                    if (ld_relaxed_gpu(&gs->err)) {
                        ok = 0;
                        break;
                    }
                }
            }
        }
        if (ld_relaxed_gpu(&gs->err)) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ----------------------------------------------------------------- reductions
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum over aligned groups of G lanes (G a power of two <= 32); every lane of
// the warp must call it; all lanes of a group receive the group's sum.
template <int G, typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of K doubles per thread into out[0..K-1] of thread 0
// (fixed order: lanes by xor-tree, then warps in index order).  `sm` must
// hold 32*K doubles.  Contains __syncthreads.
template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double *sm, double (&out)[K]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = warp_sum(v[k]);
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) sm[warp * K + k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = 0.0;
            for (int i = 0; i < nw; i++) s += sm[i * K + k];
            out[k] = s;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int warp_sum_int(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ----------------------------------------------------------------- launch helpers
inline int div_up(long long a, long long b) { return (int)((a + b - 1) / b); }

// Grid size for a plain grid-stride kernel: enough CTAs to cover `work`
// items at `per_cta` items each, at most `waves` full waves of the GPU.
int grid_for(long long work, int per_cta, int waves = 8);

// Lets `kernel` take up to the device's opt-in maximum of dynamic shared
// memory.  Every caller sets the same value, so threads launching the kernel
// concurrently with different shared-memory sizes never lower the limit
// under one another.
cmg_status_t allow_max_dynamic_smem(const void *kernel);

// Largest co-resident grid for a cooperative launch of `kernel`.
cmg_status_t coop_max_blocks(const void *kernel, int threads, size_t smem, int *out);

// Launches `kernel` cooperatively after clearing the barrier counters of
// `gs` (count, gen; the stall hook is set when armed); `err` is kept, so
// clear it with gs_clear once at the start of each API call.
cmg_status_t coop_launch(const void *kernel, int blocks, int threads, size_t smem,
                         cudaStream_t s, void **args, GridSync *gs);
// Clears all of `gs` (stream-ordered).
cmg_status_t gs_clear(GridSync *gs, cudaStream_t s);
// Test hook: the `launch`-th next cooperative launch with more than one CTA
// (0: the next) holds its barrier number `barrier`; launch < 0 disarms.
void debug_stall_barrier(long long launch, int barrier);

}  // namespace cmg
