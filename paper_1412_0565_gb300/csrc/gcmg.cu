// gcmg.cu -- geometric cascadic multigrid (Alg. 4, Sec. 3) on structured
// grids: cmg_gcmg_grid.
//
// The grid is the unit-weight grid graph on N^dim vertices (dim 2: 5-point,
// dim 3: 7-point; vertex (x, y, z) has id (z N + y) N + x), coarsened
// geometrically by keeping every other vertex: level j has
// N_j = (N - 1) / 2^j + 1 vertices per side, and coarse vertex I sits at fine
// vertex 2I.  A_j is level j's graph Laplacian.  Per level:
//   - the start: on the coarsest level its exact eigenvector for lambda_2
//     that varies along x, cos(pi (x + 1/2) / N_J) (the separable grid
//     spectrum); on the others the multilinear interpolant of the coarser
//     result (a fine vertex between coarse ones averages its 2, 4 or 8 coarse
//     neighbours);
//   - Gram-Schmidt against 1 and normalisation, then the Rayleigh quotient
//     r_0 of that start;
//   - k_j = ceil(k0 beta^j) smoothing steps u <- (I - omega_j A_j) u with
//     omega_j = 1 / ||A_j||_inf, each followed by Gram-Schmidt against 1 and
//     normalisation -- the power-iteration sweep of Alg. 3 with the shift
//     g = ||A_j||_inf, so the sweeps run in the library's power-iteration
//     kernels -- and the Rayleigh quotient r_k of the result.
// Grids, starts and interpolation are built on the device; nothing is read
// back before the end except what the kernels' launch sizes need.
#include <math.h>

#include <vector>

#include "internal.h"

namespace cmg {

// Coordinates of vertex v of an N^dim grid.
__device__ __forceinline__ void grid_coords(int dim, int N, long long v, int &x, int &y, int &z) {
    x = (int)(v % N);
    y = (int)((v / N) % N);
    z = dim == 3 ? (int)(v / ((long long)N * N)) : 0;
}

__global__ void k_grid_degree(int dim, int N, int n, int *__restrict__ deg) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        grid_coords(dim, N, v, x, y, z);
        int d = (x > 0) + (x < N - 1) + (y > 0) + (y < N - 1);
        if (dim == 3) d += (z > 0) + (z < N - 1);
        deg[v] = d;
    }
}

// Columns in ascending id order (-z, -y, -x, +x, +y, +z), unit weights.
__global__ void k_grid_fill(int dim, int N, int n, const int *__restrict__ rp, int *__restrict__ col,
                            double *__restrict__ w) {
    const long long NN = (long long)N * N;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        int x, y, z;
        grid_coords(dim, N, v, x, y, z);
        int e = rp[v];
        if (dim == 3 && z > 0) col[e++] = (int)(v - NN);
        if (y > 0) col[e++] = (int)(v - N);
        if (x > 0) col[e++] = (int)(v - 1);
        if (x < N - 1) col[e++] = (int)(v + 1);
        if (y < N - 1) col[e++] = (int)(v + N);
        if (dim == 3 && z < N - 1) col[e++] = (int)(v + NN);
        for (int k = rp[v]; k < e; k++) w[k] = 1.0;
    }
}

// The coarsest level's eigenvector for lambda_2 = 2 - 2 cos(pi / N) along x.
__global__ void k_grid_coarsest(int dim, int N, int n, double *__restrict__ x0) {
    const double pi = 3.14159265358979323846264338327950288;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x)
        x0[v] = cos(pi * ((double)(v % N) + 0.5) / (double)N);
}

// Multilinear interpolation from the Nc-grid to the (2 Nc - 1)-grid: along
// each axis a fine index c lies on coarse index c/2 (c even) or between c/2
// and c/2 + 1 (c odd); the fine value is the mean of the 1, 2, 4 or 8 coarse
// values at the corners so selected.
__global__ void k_grid_prolong(int dim, int Nc, const double *__restrict__ yc, double *__restrict__ yf) {
    const int Nf = 2 * Nc - 1;
    const long long nf = dim == 3 ? (long long)Nf * Nf * Nf : (long long)Nf * Nf;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < nf;
         v += (long long)gridDim.x * blockDim.x) {
        int c[3];
        grid_coords(dim, Nf, v, c[0], c[1], c[2]);
        int lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = c[a] >> 1;
            hi[a] = (c[a] & 1) ? lo[a] + 1 : lo[a];
        }
        double s = 0.0;
        int cnt = 0;
        for (int iz = 0; iz < (dim == 3 ? 2 : 1); iz++)
            for (int iy = 0; iy < 2; iy++)
                for (int ix = 0; ix < 2; ix++) {
                    const int X = ix ? hi[0] : lo[0], Y = iy ? hi[1] : lo[1];
                    const int Z = dim == 3 ? (iz ? hi[2] : lo[2]) : 0;
                    s += yc[((long long)Z * Nc + Y) * Nc + X];
                    cnt++;
                }
        yf[v] = s / (double)cnt;
    }
}

}  // namespace cmg

using namespace cmg;

extern "C" cmg_status_t cmg_gcmg_grid(int32_t dim, int32_t N, int32_t J, double beta, int32_t k0,
                                      double *u_out, int32_t u_mem, double *r0_out, double *rk_out,
                                      int32_t *k_out, void *stream) {
    if ((dim != 2 && dim != 3) || J < 0 || J > 30 || N < 3 || k0 < 0 || !(beta > 0.0))
        return CMG_ERR_INVALID_ARG;
    if (u_out && u_mem != CMG_MEM_HOST && u_mem != CMG_MEM_DEVICE) return CMG_ERR_INVALID_ARG;
    if (((long long)(N - 1) % (1ll << J)) != 0 || (N - 1) >> J < 1) return CMG_ERR_INVALID_ARG;
    const long long n0 = dim == 3 ? (long long)N * N * N : (long long)N * N;
    if (2ll * dim * n0 >= 2147483647ll) return CMG_ERR_TOO_LARGE;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch scr(s);
    GridSync *gs;
    PiResult *res;
    double *out4;   // [4 (J + 1)]: per level (r_0, its residual, r_k, its residual)
    CMG_TRY(scr.get(&gs, 1));
    CMG_TRY(scr.get(&res, 1));
    CMG_TRY(scr.get(&out4, 4 * (size_t)(J + 1)));
    CMG_TRY(gs_clear(gs, s));
    std::vector<int> ks(J + 1, 0);
    double *yc = nullptr;   // the coarser level's result
    int Nj = (N - 1) / (1 << J) + 1;
    for (int j = J; j >= 0; j--) {
        const long long nl = dim == 3 ? (long long)Nj * Nj * Nj : (long long)Nj * Nj;
        const int n = (int)nl;
        // ---- the level's grid graph (CSR with int32 row pointers)
        int *deg, *rp, *col;
        double *w;
        CMG_TRY(scr.get(&deg, (size_t)n));
        CMG_TRY(scr.get(&rp, (size_t)n + 1));
        k_grid_degree<<<grid_for(n, 256), 256, 0, s>>>(dim, Nj, n, deg);
        CMG_TRY(launch_status());
        CMG_TRY(exclusive_scan(deg, rp, n, scr, s));
        // stored entries: every vertex pair at distance 1 along an axis, both ways
        const long long nnz = 2ll * dim * (long long)(Nj - 1) * (nl / Nj);
        CMG_TRY(scr.get(&col, (size_t)nnz));
        CMG_TRY(scr.get(&w, (size_t)nnz));
        k_grid_fill<<<grid_for(n, 256), 256, 0, s>>>(dim, Nj, n, rp, col, w);
        CMG_TRY(launch_status());
        // ---- start vector
        double *xin;
        CMG_TRY(scr.get(&xin, (size_t)n));
        if (j == J) {
            k_grid_coarsest<<<grid_for(n, 256), 256, 0, s>>>(dim, Nj, n, xin);
        } else {
            k_grid_prolong<<<grid_for(n, 256), 256, 0, s>>>(dim, (Nj + 1) / 2, yc, xin);
        }
        CMG_TRY(launch_status());
        PiLevel lv = {};
        lv.n = n;
        lv.nnz = nnz;
        lv.rp = rp;
        lv.col = col;
        lv.w = w;
        lv.g = 2.0 * (Nj >= 3 ? 2 * dim : dim);   // ||A_j||_inf = 2 max degree
        double *b[3], *gd, *u;
        for (int q = 0; q < 3; q++) CMG_TRY(scr.get(&b[q], (size_t)n));
        CMG_TRY(scr.get(&gd, (size_t)n));
        CMG_TRY(scr.get(&u, (size_t)n));
        void *bv[3] = {b[0], b[1], b[2]};
        const int k = (j == J) ? 0 : (int)ceil((double)k0 * pow(beta, (double)j));
        ks[j] = k;
        // Gram-Schmidt and normalisation of the start (no sweep), its Rayleigh
        // quotient, then the k smoothing steps and the result's quotient
        for (int pass = 0; pass < (k > 0 ? 2 : 1); pass++) {
            PiRun r = {};
            r.lv = &lv;
            r.mode = 1;
            r.k_fixed = pass == 0 ? 0 : k;
            r.max_sweeps = r.k_fixed;
            r.x_init = pass == 0 ? xin : u;
            for (int q = 0; q < 3; q++) r.bufs[q] = b[q];
            r.gd = gd;
            r.res = res;
            CMG_TRY(power_iteration(r, gs, s));
            // the final pass writes the Rayleigh quotient and the residual
            CMG_TRY(finalize(lv, 0, bv, res, u, 0, 0, out4 + 4 * j + 2 * pass, gs, s));
        }
        if (k == 0)
            CMG_CUDA(cudaMemcpyAsync(out4 + 4 * j + 2, out4 + 4 * j, 2 * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
        yc = u;
        if (j > 0) Nj = 2 * Nj - 1;
    }
    std::vector<double> h4(4 * (size_t)(J + 1));
    GridSync hgs;
    CMG_CUDA(cudaMemcpyAsync(h4.data(), out4, sizeof(double) * h4.size(), cudaMemcpyDeviceToHost, s));
    CMG_CUDA(cudaMemcpyAsync(&hgs, gs, sizeof(hgs), cudaMemcpyDeviceToHost, s));
    if (u_out)
        CMG_CUDA(cudaMemcpyAsync(u_out, yc, sizeof(double) * (size_t)n0,
                                 u_mem == CMG_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    CMG_CUDA(cudaStreamSynchronize(s));
    if (hgs.err) return CMG_ERR_DEVICE_TIMEOUT;
    for (int j = 0; j <= J; j++) {
        if (r0_out) r0_out[j] = h4[4 * j];
        if (rk_out) rk_out[j] = h4[4 * j + 2];
        if (k_out) k_out[j] = ks[j];
    }
    return CMG_OK;
}
