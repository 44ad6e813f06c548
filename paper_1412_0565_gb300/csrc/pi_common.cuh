// pi_common.cuh -- device pieces shared by the power-iteration kernels of
// the single-graph form (refine.cu) and the batched form (batch.cu): the
// Gaussian start of Alg. 1 Step 2, float-float partial sums of one sweep, and
// power-of-two rescaling helpers.
#pragma once

#include <math.h>
#include <stdint.h>

#include "common.cuh"
#include "ffloat.cuh"

namespace cmg {

constexpr float kZeroTol2_64 = 2.0194839e-28f;  // (64 eps_64)^2
constexpr float kZeroTol2_32 = 5.8207661e-11f;  // (64 eps_32)^2

__device__ __forceinline__ uint64_t sm64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Alg. 1 Step 2's randn: Box-Muller on two splitmix64 uniforms in (0, 1]:
// a = splitmix64(seed ^ 0xC0A45E ^ 2i), b = splitmix64(seed ^ 0xC0A45E ^ (2i+1)).
__device__ __forceinline__ double gaussian_entry(uint64_t seed, long long i) {
    const uint64_t a = sm64(seed ^ 0xC0A45Eull ^ (uint64_t)(2 * i));
    const uint64_t b = sm64(seed ^ 0xC0A45Eull ^ (uint64_t)(2 * i + 1));
    const double u1 = (double)((a >> 11) + 1) * (1.0 / 9007199254740992.0);
    const double u2 = (double)((b >> 11) + 1) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925286766559 * u2);
}

// ------------------------------------------------------------------ partial sums
// A = sum y (the mean must be removed to rounding level relative to |y|, so
// it needs float-float like B = sum y^2 and C = sum y y_prev, which decide
// the stopping cosine).
struct Part {
    ff A, B, C;
};

__device__ __forceinline__ Part part_zero() {
    Part p;
    p.A = p.B = p.C = ff_zero();
    return p;
}

__device__ __forceinline__ Part part_add(Part x, Part y) {
    Part r;
    r.A = ff_add_lazy(x.A, y.A);
    r.B = ff_add_lazy(x.B, y.B);
    r.C = ff_add_lazy(x.C, y.C);
    return r;
}

// Sum over lanes 0, lo, 2 lo, ... (lo a power of two; lanes between hold
// nothing), taking the xor tree from stride 16 down to lo in a fixed order.
// The sum ends in lane 0 (and every lane of its residue class), renormalised.
__device__ __forceinline__ Part warp_sum_part(Part p, int lo = 1, int width = 32) {
    for (int o = width >> 1; o >= lo; o >>= 1) {
        Part q;
        q.A = shfl_xor_ff(p.A, o);
        q.B = shfl_xor_ff(p.B, o);
        q.C = shfl_xor_ff(p.C, o);
        p = part_add(p, q);
    }
    p.A = ff_norm(p.A);
    p.B = ff_norm(p.B);
    p.C = ff_norm(p.C);
    return p;
}

__device__ __forceinline__ int pow2_at_least(int v) {
    int w = 1;
    while (w < v) w <<= 1;
    return w;
}

// Per-thread accumulation of (sum y, sum y^2, sum y x) for one sweep.
template <typename T>
struct Acc;

template <>
struct Acc<float> {
    ff A, B, C;
    __device__ __forceinline__ void reset() { A = B = C = ff_zero(); }
    __device__ __forceinline__ void add(float y, float x) {
        A = ff_add_lazy(A, ff_make(y, 0.f));
        B = ff_add_lazy(B, two_prod(y, y));
        C = ff_add_lazy(C, two_prod(y, x));
    }
    __device__ __forceinline__ Part get() const {
        Part p;
        p.A = ff_norm(A);
        p.B = ff_norm(B);
        p.C = ff_norm(C);
        return p;
    }
};

template <>
struct Acc<double> {
    double A, B, C;
    __device__ __forceinline__ void reset() { A = B = C = 0.0; }
    __device__ __forceinline__ void add(double y, double x) {
        A += y;
        B = fma(y, y, B);
        C = fma(y, x, C);
    }
    __device__ __forceinline__ Part get() const {
        Part p;
        p.A = ff_from_double(A);
        p.B = ff_from_double(B);
        p.C = ff_from_double(C);
        return p;
    }
};

__device__ __forceinline__ double to_d(ff a) { return ff_to_double(a); }

__device__ __forceinline__ int start_exponent(double ss0) {
    // 2^e0 ~ 1 / ||proj y_0||
    if (!(ss0 > 0.0)) return 0;
    return -(int)floor(0.5 * log2(ss0) + 0.5);
}

// x * 2^e for a normal float x and a small e (exponent arithmetic, exact).
__device__ __forceinline__ float scale2f(float x, int e) { return __int_as_float(__float_as_int(x) + (e << 23)); }

// Sum over the entries f = f0, f0 + stride, ... < f1 of a row: FP32 edge form
// sum w (x_i - x_j), FP64 degree form sum w x_j.  Entries are taken in
// groups of 8 -- all column loads, then all gathers -- so a long row costs
// one round trip to memory per 8 entries, not per entry.  `ld` loads x.
template <typename T, typename IDX, typename LD>
__device__ __forceinline__ T row_sum_grouped(const IDX *C, const T *W, int f0, int f1, int stride, T xi,
                                             LD ld, bool stream = false) {
    T a0 = (T)0, a1 = (T)0;
    for (int f = f0; f < f1; f += 8 * stride) {
        int cc[8];
        T ww[8];
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const int g = f + u * stride;
            const bool ok = g < f1;
            if (stream) {
                // global streams read once per sweep: evict-first, so the
                // gathered iterate keeps its place in L2
                cc[u] = ok ? (int)__ldcs(C + g) : -1;
                ww[u] = ok ? __ldcs(W + g) : (T)0;
            } else {
                cc[u] = ok ? (int)C[g] : -1;
                ww[u] = ok ? W[g] : (T)0;
            }
        }
        T xx[8];
#pragma unroll
        for (int u = 0; u < 8; u++) xx[u] = (cc[u] >= 0) ? ld(cc[u]) : xi;
#pragma unroll
        for (int u = 0; u < 8; u++) {
            if (sizeof(T) == 8) {
                if (u & 1) a1 = fma(ww[u], xx[u], a1);
                else a0 = fma(ww[u], xx[u], a0);
            } else {
                if (u & 1) a1 += ww[u] * (xi - xx[u]);
                else a0 += ww[u] * (xi - xx[u]);
            }
        }
    }
    return a0 + a1;
}

// Eight consecutive layout entries from an index that is a multiple of 8
// (16-byte aligned vectors); stream: evict-first loads.
__device__ __forceinline__ void load_cols8(const uint16_t *C, int f, int (&cc)[8], bool stream) {
    const uint4 *p = reinterpret_cast<const uint4 *>(C + f);
    const uint4 v = stream ? __ldcs(p) : *p;
    const unsigned u[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; k++) {
        cc[2 * k] = (int)(u[k] & 0xffffu);
        cc[2 * k + 1] = (int)(u[k] >> 16);
    }
}
__device__ __forceinline__ void load_cols8(const int *C, int f, int (&cc)[8], bool stream) {
    const int4 *p = reinterpret_cast<const int4 *>(C + f);
    const int4 a = stream ? __ldcs(p) : p[0];
    const int4 b = stream ? __ldcs(p + 1) : p[1];
    cc[0] = a.x; cc[1] = a.y; cc[2] = a.z; cc[3] = a.w;
    cc[4] = b.x; cc[5] = b.y; cc[6] = b.z; cc[7] = b.w;
}
__device__ __forceinline__ void load_w8(const float *W, int f, float (&ww)[8], bool stream) {
    const float4 *p = reinterpret_cast<const float4 *>(W + f);
    const float4 a = stream ? __ldcs(p) : p[0];
    const float4 b = stream ? __ldcs(p + 1) : p[1];
    ww[0] = a.x; ww[1] = a.y; ww[2] = a.z; ww[3] = a.w;
    ww[4] = b.x; ww[5] = b.y; ww[6] = b.z; ww[7] = b.w;
}
__device__ __forceinline__ void load_w8(const double *W, int f, double (&ww)[8], bool stream) {
    const double2 *p = reinterpret_cast<const double2 *>(W + f);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const double2 v = stream ? __ldcs(p + k) : p[k];
        ww[2 * k] = v.x;
        ww[2 * k + 1] = v.y;
    }
}

// The sum of row_sum_grouped over a run of whole octets (8 entries from a
// multiple of 8): octets o0, o0 + 32, ... < o1 belong to this lane, which
// loads each with vector loads and takes OCT octets per round trip.
template <typename T, typename IDX, int OCT, typename LD>
__device__ __forceinline__ T row_sum_octets(const IDX *C, const T *W, int o0, int o1, T xi, LD ld,
                                            bool stream) {
    T a0 = (T)0, a1 = (T)0;
    for (int o = o0; o < o1; o += 32 * OCT) {
        int cc[OCT][8];
        T ww[OCT][8];
#pragma unroll
        for (int v = 0; v < OCT; v++) {
            if (o + 32 * v < o1) {
                load_cols8(C, 8 * (o + 32 * v), cc[v], stream);
                load_w8(W, 8 * (o + 32 * v), ww[v], stream);
            } else {
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    cc[v][u] = -1;
                    ww[v][u] = (T)0;
                }
            }
        }
        T xx[OCT][8];
#pragma unroll
        for (int v = 0; v < OCT; v++)
#pragma unroll
            for (int u = 0; u < 8; u++) xx[v][u] = (cc[v][u] >= 0) ? ld(cc[v][u]) : xi;
#pragma unroll
        for (int v = 0; v < OCT; v++)
#pragma unroll
            for (int u = 0; u < 8; u++) {
                if (sizeof(T) == 8) {
                    if (u & 1) a1 = fma(ww[v][u], xx[v][u], a1);
                    else a0 = fma(ww[v][u], xx[v][u], a0);
                } else {
                    if (u & 1) a1 += ww[v][u] * (xi - xx[v][u]);
                    else a0 += ww[v][u] * (xi - xx[v][u]);
                }
            }
    }
    return a0 + a1;
}

}  // namespace cmg
