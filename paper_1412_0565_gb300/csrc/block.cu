// block.cu -- k eigenpairs by the cascade (the Remark after Alg. 4):
// cmg_eigenpairs.
//
// The cascade of Alg. 1 carries k vectors.  On every level the power
// iteration multiplies all k by B_g = g I - L in one pass over the matrix
// (the k values of a row are stored together, so one gather fetches a
// neighbour's k values), then orthonormalises them: Gram-Schmidt against 1
// and against the earlier vectors, done here as a Cholesky QR of the mean-free
// block -- with Y the raw block, mu its column means and R the Cholesky
// factor of (Y - 1 mu^T)^T (Y - 1 mu^T), X = (Y - 1 mu^T) R^{-1} is exactly
// the Gram-Schmidt result (the same vectors in exact arithmetic).
//
// The orthonormalisation is folded into the next sweep: B_g X = (B_g Y -
// g 1 mu^T) R^{-1}, so each sweep reads the raw block Y_t, and a row of
// Y_{t+1} = (B_g Y_t - g 1 mu_t^T) R_t^{-1} / g needs only mu_t and R_t, which
// come from sums over Y_t accumulated by the previous sweep.  One grid
// barrier per sweep: every CTA reduces the CTA partial sums of Y_t in the same
// order (so all hold the same mu_t, R_t and stop decision), then computes its
// rows of Y_{t+1} and their partial sums (column sums, the Gram matrix, and
// the products with the normalised current rows X_t that give the cosines of
// the stop rule for sweep t + 1).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "pi_common.cuh"

namespace cmg {

constexpr int kBlkThreads = 256;

struct BlockArgs {
    int n, k;
    const int *rp;
    const int *col;
    const double *w;
    double g;
    int start;              // 0 Gaussian (vector i keyed by seed + i), 1 prolongation
    uint64_t seed;
    const double *xc;       // start = 1: the coarse level's normalised block (row-major)
    const int *agg;         // this level -> the coarse level
    double *Y0, *Y1;        // raw blocks (row-major n x k), parity by sweep
    double *xout;           // the level's normalised result (row-major n x k)
    double *part;           // [2][gridDim][P] CTA partial sums, P = k + 2 k^2
    int mode, k_fixed, max_sweeps;
    double tol;
    int *info;              // [0] sweeps, [1] capped, [2] degenerate block
    double *cos_out;        // [k] cosines of the last sweep
};

// Partial-sum record of a block of rows: m[k] (column sums), G[k][k] (Gram
// matrix, row-major), C[k][k] with C[j][i] = sum_r y_rj x_ri (x the current
// normalised rows).
__host__ __device__ constexpr int blk_parts(int k) { return k + 2 * k * k; }

// Cholesky factor R (upper triangular, R^T R = A) and R^{-1} of a k x k SPD
// matrix, in place in shared memory; returns false when a pivot is not
// positive (the block has lost rank).
__device__ bool chol_inv(int k, double *A, double *Ri) {
    for (int j = 0; j < k; j++) {
        double s = A[j * k + j];
        for (int p = 0; p < j; p++) s -= A[p * k + j] * A[p * k + j];
        if (!(s > 0.0)) return false;
        const double r = sqrt(s);
        A[j * k + j] = r;
        for (int i = j + 1; i < k; i++) {
            double t = A[j * k + i];
            for (int p = 0; p < j; p++) t -= A[p * k + j] * A[p * k + i];
            A[j * k + i] = t / r;
        }
    }
    // R^{-1} (upper triangular) by back substitution, column by column
    for (int i = 0; i < k; i++)
        for (int j = 0; j < k; j++) Ri[j * k + i] = 0.0;
    for (int c = 0; c < k; c++) {
        Ri[c * k + c] = 1.0 / A[c * k + c];
        for (int r = c - 1; r >= 0; r--) {
            double t = 0.0;
            for (int p = r + 1; p <= c; p++) t += A[r * k + p] * Ri[p * k + c];
            Ri[r * k + c] = -t / A[r * k + r];
        }
    }
    return true;
}

template <int KM>
__global__ void __launch_bounds__(kBlkThreads) k_block_pi(BlockArgs a, GridSync *gs) {
    const int n = a.n, k = a.k, P = blk_parts(a.k);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kBlkThreads / 32;
    constexpr int PMAX = KM + 2 * KM * KM;
    constexpr int PL = (PMAX + 31) / 32;          // partial sums per lane
    __shared__ double s_sum[PMAX];                // reduced sums of the current block
    __shared__ double s_A[KM * KM], s_Ri[KM * KM], s_mu[KM];
    __shared__ int s_flag[2];
    // dynamic: per warp the y_new and x_cur of 32 rows ([NW][32][2k]), then
    // the per-warp partial sums ([NW][P])
    extern __shared__ __align__(16) double s_dyn[];
    double *const my_tile = s_dyn + (size_t)warp * 32 * 2 * k;
    double *const s_wp = s_dyn + (size_t)NW * 32 * 2 * k;
    const int r0 = (int)((long long)n * blockIdx.x / gridDim.x);
    const int r1 = (int)((long long)n * (blockIdx.x + 1) / gridDim.x);

    // ---- start block Y_0 and its partial sums (C unused: no previous iterate)
    double acc[PL];
#pragma unroll
    for (int q = 0; q < PL; q++) acc[q] = 0.0;
    for (int base = r0 + warp * 32; base < r1; base += NW * 32) {
        const int r = base + lane;
        double y[KM];
#pragma unroll
        for (int i = 0; i < KM; i++) y[i] = 0.0;
        if (r < r1) {
            for (int i = 0; i < k; i++) {
                y[i] = a.start == 0 ? gaussian_entry(a.seed + (uint64_t)i, r)
                                    : a.xc[(size_t)a.agg[r] * k + i];
                a.Y0[(size_t)r * k + i] = y[i];
            }
        }
        for (int i = 0; i < k; i++) {
            my_tile[lane * 2 * k + i] = y[i];
            my_tile[lane * 2 * k + k + i] = 0.0;
        }
        __syncwarp();
        const int rows = min(32, r1 - base);
        for (int q = 0; q < PL; q++) {
            const int p = lane + 32 * q;
            if (p >= P) break;
            double s = 0.0;
            for (int l = 0; l < rows; l++) {
                const double *t = my_tile + l * 2 * k;
                if (p < k) s += t[p];
                else if (p < k + k * k) s += t[(p - k) / k] * t[(p - k) % k];
                else s += t[(p - k - k * k) / k] * t[k + (p - k - k * k) % k];
            }
            acc[q] += s;
        }
        __syncwarp();
    }
    auto publish = [&](int parity) {
        for (int q = 0; q < PL; q++) {
            const int p = lane + 32 * q;
            if (p < P) s_wp[warp * P + p] = acc[q];
        }
        __syncthreads();
        for (int p = tid; p < P; p += kBlkThreads) {
            double s = 0.0;
            for (int ww = 0; ww < NW; ww++) s += s_wp[ww * P + p];
            a.part[((size_t)parity * gridDim.x + blockIdx.x) * P + p] = s;
        }
    };
    publish(0);
    if (!grid_sync(gs)) return;

    for (int t = 0;; t++) {
        // ---- sums of Y_t over all CTAs (same order in every CTA)
        const double *src = a.part + (size_t)(t & 1) * gridDim.x * P;
        for (int p = tid; p < P; p += kBlkThreads) {
            double s = 0.0;
            for (int b = 0; b < (int)gridDim.x; b++) s += __ldcg(src + (size_t)b * P + p);
            s_sum[p] = s;
        }
        __syncthreads();
        if (tid == 0) {
            // mu, the mean-free Gram matrix, its Cholesky factor and inverse
            for (int i = 0; i < k; i++) s_mu[i] = s_sum[i] / (double)n;
            for (int i = 0; i < k; i++)
                for (int j = 0; j < k; j++)
                    s_A[i * k + j] = s_sum[k + i * k + j] - (double)n * s_mu[i] * s_mu[j];
            const bool ok = chol_inv(k, s_A, s_Ri);
            int stop = 0, capped = 0;
            double cmin = 1.0;
            if (ok && t >= 1) {
                // cos_i = x_{t,i} . x_{t-1,i} = sum_{j <= i} Ri[j][i] C[j][i]
                for (int i = 0; i < k; i++) {
                    double c = 0.0;
                    for (int j = 0; j <= i; j++) c += s_Ri[j * k + i] * s_sum[k + k * k + j * k + i];
                    if (blockIdx.x == 0) a.cos_out[i] = c;
                    cmin = fmin(cmin, c);
                }
            }
            if (!ok) stop = 2;
            else if (a.mode == 1) stop = t >= a.k_fixed;
            else if (t >= 1 && cmin >= 1.0 - a.tol) stop = 1;
            else if (t >= a.max_sweeps) stop = capped = 1;
            s_flag[0] = stop;
            s_flag[1] = capped;
        }
        __syncthreads();
        const int stop = s_flag[0];
        if (stop == 2) {
            // a block that lost rank: keep the previous result (xout), report it
            if (blockIdx.x == 0 && tid == 0) {
                a.info[0] = t;
                a.info[1] = 0;
                a.info[2] = 1;
            }
            return;
        }
        const double *Yt = (t & 1) ? a.Y1 : a.Y0;
        double *Yn = (t & 1) ? a.Y0 : a.Y1;
        if (stop) {
            // the level's result: X_t = (Y_t - 1 mu^T) R^{-1}
            for (int r = r0 + tid; r < r1; r += kBlkThreads)
                for (int i = 0; i < k; i++) {
                    double x = 0.0;
                    for (int j = 0; j <= i; j++) x += (Yt[(size_t)r * k + j] - s_mu[j]) * s_Ri[j * k + i];
                    a.xout[(size_t)r * k + i] = x;
                }
            if (blockIdx.x == 0 && tid == 0) {
                a.info[0] = t;
                a.info[1] = s_flag[1];
                a.info[2] = 0;
            }
            return;
        }
        // ---- rows of Y_{t+1} = (B_g Y_t - g 1 mu_t^T) R_t^{-1} / g and their sums
#pragma unroll
        for (int q = 0; q < PL; q++) acc[q] = 0.0;
        const double inv_g = 1.0 / a.g;
        for (int base = r0 + warp * 32; base < r1; base += NW * 32) {
            const int r = base + lane;
            double z[KM], yn[KM], xcur[KM];
#pragma unroll
            for (int i = 0; i < KM; i++) z[i] = yn[i] = xcur[i] = 0.0;
            if (r < r1) {
                // B_g y_r = (g - d_r) y_r + sum_e w_e y_col(e)
                double d = 0.0;
                const int e0 = a.rp[r], e1 = a.rp[r + 1];
                for (int e = e0; e < e1; e++) {
                    const double we = a.w[e];
                    const double *yc = Yt + (size_t)a.col[e] * k;
                    d += we;
#pragma unroll
                    for (int i = 0; i < KM; i++)
                        if (i < k) z[i] = fma(we, __ldcg(yc + i), z[i]);
                }
                const double gd = a.g - d;
#pragma unroll
                for (int i = 0; i < KM; i++)
                    if (i < k) {
                        const double yi = __ldcg(Yt + (size_t)r * k + i);
                        z[i] = fma(gd, yi, z[i]) - a.g * s_mu[i];
                        xcur[i] = yi - s_mu[i];
                    }
                // apply R^{-1} (upper triangular): column i mixes rows j <= i
#pragma unroll
                for (int i = KM - 1; i >= 0; i--) {
                    if (i >= k) continue;
                    double s = 0.0, c = 0.0;
                    for (int j = 0; j <= i; j++) {
                        s += z[j] * s_Ri[j * k + i];
                        c += xcur[j] * s_Ri[j * k + i];
                    }
                    yn[i] = s * inv_g;
                    xcur[i] = c;
                }
                for (int i = 0; i < k; i++) Yn[(size_t)r * k + i] = yn[i];
            }
            for (int i = 0; i < k; i++) {
                my_tile[lane * 2 * k + i] = yn[i];
                my_tile[lane * 2 * k + k + i] = xcur[i];
            }
            __syncwarp();
            const int rows = min(32, r1 - base);
            for (int q = 0; q < PL; q++) {
                const int p = lane + 32 * q;
                if (p >= P) break;
                double s = 0.0;
                for (int l = 0; l < rows; l++) {
                    const double *tt = my_tile + l * 2 * k;
                    if (p < k) s += tt[p];
                    else if (p < k + k * k) s += tt[(p - k) / k] * tt[(p - k) % k];
                    else s += tt[(p - k - k * k) / k] * tt[k + (p - k - k * k) % k];
                }
                acc[q] += s;
            }
            __syncwarp();
        }
        __syncthreads();
        publish((t + 1) & 1);
        if (!grid_sync(gs)) return;
    }
}

// Column-major U (vector i at U + i n) from the row-major block.
__global__ void k_block_columns(int n, int k, const double *__restrict__ X, double *__restrict__ U) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * k;
         e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / k, i = e % k;
        U[i * n + r] = X[e];
    }
}

template <int KM>
static cmg_status_t launch_block(BlockArgs &a, GridSync *gs, cudaStream_t s) {
    const void *kern = (const void *)k_block_pi<KM>;
    DeviceInfo di;
    CMG_TRY(device_info(&di));
    const size_t smem = sizeof(double) * ((size_t)(kBlkThreads / 32) * (32 * 2 * a.k + blk_parts(a.k)));
    CMG_TRY(allow_max_dynamic_smem(kern));
    int maxb = 0;
    CMG_TRY(coop_max_blocks(kern, kBlkThreads, smem, &maxb));
    // one CTA per SM at most: every CTA reduces all CTAs' partial sums
    const int blocks = std::max(1, std::min({maxb, di.sms, (a.n + 63) / 64}));
    Scratch scr(s);
    CMG_TRY(scr.get(&a.part, (size_t)2 * blocks * blk_parts(a.k)));
    void *args[] = {&a, &gs};
    return coop_launch(kern, blocks, kBlkThreads, smem, s, args, gs);
}

}  // namespace cmg

using namespace cmg;

extern "C" cmg_status_t cmg_eigenpairs(cmg_hierarchy_t h, int32_t k, const cmg_solve_options_t *so,
                                       double *U_out, int32_t u_mem, double *lambda_out,
                                       double *residual_out, cmg_stats_t *stats_out, void *stream) {
    if (!h || k < 1 || k > CMG_MAX_EIGENPAIRS) return CMG_ERR_INVALID_ARG;
    if (U_out && u_mem != CMG_MEM_HOST && u_mem != CMG_MEM_DEVICE) return CMG_ERR_INVALID_ARG;
    if (so && (so->x0 || so->reserved[0] || so->reserved[1] || so->reserved[2] || so->reserved[3]))
        return CMG_ERR_INVALID_ARG;
    HierarchyView hv;
    CMG_TRY(hierarchy_view(h, &hv));
    const int J = (int)hv.lv.size() - 1;
    if (k > hv.lv[J].n - 1) return CMG_ERR_INVALID_ARG;
    const uint64_t seed = so ? so->seed : hv.seed;
    const cmg_options_t &o = hv.opts;
    cudaStream_t s = (cudaStream_t)stream;
    int prev = 0;
    CMG_CUDA(cudaGetDevice(&prev));
    if (prev != hv.device) CMG_CUDA(cudaSetDevice(hv.device));
    cmg_status_t st = CMG_OK;
    std::vector<int> sweeps(J + 1, 0), capped(J + 1, 0);
    std::vector<double> lam(k, 0.0), res(k, 0.0);
    {
        Scratch scr(s);
        int *info = nullptr;
        double *cosv = nullptr, *out2 = nullptr, *U = nullptr;
        if (st == CMG_OK) st = scr.get(&info, 3 * (size_t)(J + 1));
        if (st == CMG_OK) st = scr.get(&cosv, (size_t)k);
        if (st == CMG_OK) st = scr.get(&out2, 2 * (size_t)k);
        if (st == CMG_OK) st = gs_clear(hv.gs, s);
        const double *xc = nullptr;
        double *x0 = nullptr;
        for (int j = J; j >= 0 && st == CMG_OK; j--) {
            const PiLevel &L = hv.lv[j];
            BlockArgs a = {};
            double *Y0, *Y1, *xo;
            if ((st = scr.get(&Y0, (size_t)L.n * k)) != CMG_OK) break;
            if ((st = scr.get(&Y1, (size_t)L.n * k)) != CMG_OK) break;
            if ((st = scr.get(&xo, (size_t)L.n * k)) != CMG_OK) break;
            a.n = L.n;
            a.k = k;
            a.rp = L.rp;
            a.col = L.col;
            a.w = L.w;
            a.g = L.g;
            a.start = (j == J) ? 0 : 1;
            a.seed = seed;
            a.xc = xc;
            a.agg = L.agg;
            a.Y0 = Y0;
            a.Y1 = Y1;
            a.xout = xo;
            // the hierarchy's schedule and stop rule, as cmg_fiedler
            a.mode = 0;
            a.k_fixed = 0;
            if (o.schedule == CMG_SCHEDULE_FIXED && j < J) {
                a.mode = 1;
                a.k_fixed = (int)ceil((double)o.k0 * pow(o.beta, (double)j));
            } else if (o.schedule == CMG_SCHEDULE_REPLAY) {
                a.mode = 1;
                a.k_fixed = o.replay_sweeps[j];
            }
            a.max_sweeps = (j == J) ? o.max_sweeps_coarsest : o.max_sweeps;
            a.tol = o.tol;
            a.info = info + 3 * j;
            a.cos_out = cosv;
            st = (k <= 4) ? launch_block<4>(a, hv.gs, s)
                          : (k <= 8 ? launch_block<8>(a, hv.gs, s) : launch_block<16>(a, hv.gs, s));
            xc = xo;
            x0 = xo;
        }
        if (st == CMG_OK) st = scr.get(&U, (size_t)hv.lv[0].n * k);
        if (st == CMG_OK) {
            const int n0 = hv.lv[0].n;
            k_block_columns<<<grid_for((long long)n0 * k, 256), 256, 0, s>>>(n0, k, x0, U);
            st = launch_status();
            // per vector: sign rule, Rayleigh quotient and residual
            for (int i = 0; i < k && st == CMG_OK; i++)
                st = finalize(hv.lv[0], 0, nullptr, nullptr, U + (size_t)i * n0, 1, 1, out2 + 2 * i, hv.gs, s);
        }
        std::vector<int> hinfo(3 * (J + 1), 0);
        std::vector<double> h2(2 * k, 0.0);
        GridSync hgs = {};
        if (st == CMG_OK) {
            cudaError_t e = cudaMemcpyAsync(hinfo.data(), info, sizeof(int) * hinfo.size(), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h2.data(), out2, sizeof(double) * h2.size(), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hgs, hv.gs, sizeof(hgs), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && U_out)
                e = cudaMemcpyAsync(U_out, U, sizeof(double) * (size_t)hv.lv[0].n * k,
                                    u_mem == CMG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = from_cuda(e);
        }
        if (st == CMG_OK && hgs.err) st = CMG_ERR_DEVICE_TIMEOUT;
        if (st == CMG_OK) {
            for (int j = 0; j <= J; j++) {
                sweeps[j] = hinfo[3 * j];
                capped[j] = hinfo[3 * j + 1];
                if (hinfo[3 * j + 2]) st = CMG_ERR_TOO_SMALL;   // the block lost rank
            }
            for (int i = 0; i < k; i++) {
                lam[i] = h2[2 * i];
                res[i] = h2[2 * i + 1];
            }
        }
    }
    if (prev != hv.device) cudaSetDevice(prev);
    if (st != CMG_OK) return st;
    int any_cap = 0;
    for (int j = 0; j <= J; j++) any_cap |= capped[j];
    for (int i = 0; i < k; i++) {
        if (lambda_out) lambda_out[i] = lam[i];
        if (residual_out) residual_out[i] = res[i];
    }
    if (stats_out) {
        memset(stats_out, 0, sizeof(*stats_out));
        stats_out->lambda2 = lam[0];
        stats_out->residual = res[0];
        stats_out->levels = J + 1;
        stats_out->status = any_cap ? CMG_WARN_MAXITER : CMG_OK;
        for (int j = 0; j <= J; j++) {
            stats_out->n[j] = hv.lv[j].n;
            stats_out->nnz[j] = hv.lv[j].nnz;
            stats_out->sweeps[j] = sweeps[j];
        }
    }
    return any_cap ? CMG_WARN_MAXITER : CMG_OK;
}
