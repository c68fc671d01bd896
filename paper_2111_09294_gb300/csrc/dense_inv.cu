// Batched in-place inversion of symmetric positive definite matrices in FP64
// by blocked symmetric sweeps (set-up only): the explicit inverses of the
// coarse matrix E = Z^T K Z (Section 3.2) and of the dense diagonal blocks of
// a block-Jacobi preconditioner (Section 3.4, Eqs. block_jacobi,
// block_jacobi_enr).
//
// The sweep on a pivot set P maps a symmetric A to B with
//   B_PP = -A_PP^-1,  B_QP = A_QP A_PP^-1,  B_PQ = A_PP^-1 A_PQ,
//   B_QQ = A_QQ - A_QP A_PP^-1 A_PQ,
// and after every index has been swept once the array holds -A^-1.  Pivot
// blocks of kNB indices are swept in order; each step is four launches over
// all matrices at once: the pivot block's own sweep (one CTA per matrix,
// pivots checked against a threshold), the column panel C = A_QP A_PP^-1,
// the trailing update A_QQ -= C A_PQ on the upper tiles (mirrored), and the
// write-back of the panel.  The trailing update carries the n^3 work as
// 64 x 64 x 64 FP64 tile products spread over every SM.
#include <climits>

#include "internal.h"

namespace xdcg {

constexpr int kNB = 64;                 // pivot block and tile edge
constexpr int kInvThreads = 256;        // 16 x 16 threads, 4 x 4 outputs each
constexpr int kLd = kNB + 1;            // padded shared-memory row

// tile index -> (matrix, tile row I, tile column J >= I) of the upper tiles
__device__ __forceinline__ int find_matrix(const int *prefix, int nMat, int t) {
    int lo = 0, hi = nMat - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= t)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// row-major element (i, j) of matrix m
__device__ __forceinline__ double *mat_at(const DenseBatch &B, int m, int i, int j) {
    return B.A + B.off[m] + (long long)i * B.dim[m] + j;
}

// out (64 x 64, registers 4 x 4 per thread) = X (64 x nb) * Y (nb x 64), both
// in shared memory with row stride kLd
__device__ __forceinline__ void tile_mm(const double *X, const double *Y, int nb,
                                        double (&acc)[4][4]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int kk = 0; kk < nb; ++kk) {
        double xa[4], yb[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) xa[a] = X[(ty + 16 * a) * kLd + kk];
#pragma unroll
        for (int b = 0; b < 4; ++b) yb[b] = Y[kk * kLd + tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fma(xa[a], yb[b], acc[a][b]);
    }
}

// ---- step 0: pivot thresholds relative to each matrix's largest diagonal ----

__global__ void k_inv_thresholds(DenseBatch B, double rel) {
    const int m = blockIdx.x;
    const int n = B.dim[m];
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, *mat_at(B, m, i, i));
    __shared__ double red[kInvThreads];
    red[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) B.thr[m] = rel * red[0];
}

// ---- step k, launch 1: sweep the pivot block (nb x nb) of every matrix -----

__global__ void __launch_bounds__(kInvThreads)
k_inv_pivot(DenseBatch B, int k) {
    const int m = blockIdx.x;
    const int n = B.dim[m], k0 = k * kNB;
    if (k0 >= n) return;
    const int nb = min(kNB, n - k0);
    __shared__ double S[kNB * kLd];
    __shared__ double col[kNB], row[kNB];
    __shared__ int failed;
    if (threadIdx.x == 0) failed = -1;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e - i * nb;
        S[i * kLd + j] = *mat_at(B, m, k0 + i, k0 + j);
    }
    __syncthreads();
    const double thr = B.thr[m];
    for (int j = 0; j < nb; ++j) {
        const double p = S[j * kLd + j];
        const bool ok = p > thr && isfinite(p);
        if (!ok && threadIdx.x == 0 && failed < 0) failed = k0 + j;
        // a failed pivot still sweeps (with a harmless value) so the kernel
        // finishes; the failure is reported and the result not used
        const double inv = ok ? 1.0 / p : 0.0;
        for (int i = threadIdx.x; i < nb; i += blockDim.x) {
            col[i] = S[i * kLd + j];
            row[i] = S[j * kLd + i];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            const int i = e / nb, l = e - i * nb;
            double v;
            if (i == j && l == j)
                v = -inv;
            else if (i == j)
                v = row[l] * inv;
            else if (l == j)
                v = col[i] * inv;
            else
                v = S[i * kLd + l] - col[i] * row[l] * inv;
            S[i * kLd + l] = v;
        }
        __syncthreads();
    }
    // the swept block, -A_PP^-1, for the panel and write-back launches
    double *D = B.D + (long long)m * kNB * kNB;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
        const int i = e / nb, j = e - i * nb;
        D[i * kNB + j] = S[i * kLd + j];
    }
    if (threadIdx.x == 0 && failed >= 0) atomicMin(B.bad, B.badByMatrix ? m : failed);
}

// ---- step k, launch 2: column panel C = A_QP A_PP^-1 = -A_QP D -------------

__global__ void __launch_bounds__(kInvThreads)
k_inv_panel(DenseBatch B, int k) {
    const int t = blockIdx.x;
    const int m = find_matrix(B.rowTileOff, B.nMat, t);
    const int I = t - B.rowTileOff[m];
    const int n = B.dim[m], k0 = k * kNB;
    if (k0 >= n || I == k) return;
    const int nb = min(kNB, n - k0);
    extern __shared__ double sm[];
    double *X = sm, *Y = sm + kNB * kLd;
    const int r0 = I * kNB;
    const double *D = B.D + (long long)m * kNB * kNB;
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
        const int i = e / kNB, j = e - i * kNB;
        X[i * kLd + j] = (r0 + i < n && j < nb) ? *mat_at(B, m, r0 + i, k0 + j) : 0.0;
        Y[i * kLd + j] = (i < nb && j < nb) ? -D[i * kNB + j] : 0.0;
    }
    __syncthreads();
    double acc[4][4] = {};
    tile_mm(X, Y, nb, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double *C = B.C + B.cOff[m];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = r0 + ty + 16 * a, j = tx + 16 * b;
            if (i < n && j < nb) C[(long long)i * kNB + j] = acc[a][b];
        }
}

// ---- step k, launch 3: A_IJ -= C_I A_kJ on upper tiles J >= I (I, J != k),
// mirrored into A_JI ------------------------------------------------------------

__global__ void __launch_bounds__(kInvThreads)
k_inv_update(DenseBatch B, int k) {
    const int t = blockIdx.x;
    const int m = find_matrix(B.tileOff, B.nMat, t);
    const int n = B.dim[m], k0 = k * kNB;
    if (k0 >= n) return;
    const int T = (n + kNB - 1) / kNB;
    // upper tile number u -> (I, J >= I), row by row
    int u = t - B.tileOff[m], I = 0;
    while (u >= T - I) {
        u -= T - I;
        ++I;
    }
    const int J = I + u;
    if (I == k || J == k) return;
    const int nb = min(kNB, n - k0);
    extern __shared__ double sm[];
    double *X = sm, *Y = sm + kNB * kLd;
    const int r0 = I * kNB, c0 = J * kNB;
    const double *C = B.C + B.cOff[m];
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
        const int i = e / kNB, j = e - i * kNB;
        X[i * kLd + j] = (r0 + i < n && j < nb) ? C[(long long)(r0 + i) * kNB + j] : 0.0;
        Y[i * kLd + j] = (i < nb && c0 + j < n) ? *mat_at(B, m, k0 + i, c0 + j) : 0.0;
    }
    __syncthreads();
    double acc[4][4] = {};
    tile_mm(X, Y, nb, acc);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = r0 + ty + 16 * a, j = c0 + tx + 16 * b;
            if (i < n && j < n) *mat_at(B, m, i, j) -= acc[a][b];
        }
    if (I == J) return;
    // the mirrored tile A_JI = A_IJ^T: new values through shared memory so
    // that both stores are row-wise
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) X[(ty + 16 * a) * kLd + tx + 16 * b] = acc[a][b];
    __syncthreads();
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
        const int jj = e / kNB, ii = e - jj * kNB;   // A(c0 + jj, r0 + ii) -= acc(ii, jj)
        if (c0 + jj < n && r0 + ii < n) *mat_at(B, m, c0 + jj, r0 + ii) -= X[ii * kLd + jj];
    }
}

// ---- step k, launch 4: A_Ik = C_I, A_kI = C_I^T, A_kk = -A_kk^-1 -------------

__global__ void __launch_bounds__(kInvThreads)
k_inv_writeback(DenseBatch B, int k) {
    const int t = blockIdx.x;
    const int m = find_matrix(B.rowTileOff, B.nMat, t);
    const int I = t - B.rowTileOff[m];
    const int n = B.dim[m], k0 = k * kNB;
    if (k0 >= n) return;
    const int nb = min(kNB, n - k0);
    const int r0 = I * kNB;
    if (I == k) {
        const double *D = B.D + (long long)m * kNB * kNB;
        for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
            const int i = e / nb, j = e - i * nb;
            *mat_at(B, m, k0 + i, k0 + j) = D[i * kNB + j];
        }
        return;
    }
    const double *C = B.C + B.cOff[m];
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
        const int i = e / kNB, j = e - i * kNB;
        if (r0 + i < n && j < nb) *mat_at(B, m, r0 + i, k0 + j) = C[(long long)(r0 + i) * kNB + j];
    }
    for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
        const int j = e / kNB, i = e - j * kNB;        // row k0 + j, column r0 + i
        if (r0 + i < n && j < nb) *mat_at(B, m, k0 + j, r0 + i) = C[(long long)(r0 + i) * kNB + j];
    }
}

__global__ void k_inv_negate(double *A, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        A[i] = -A[i];
}

size_t dense_inv_panel_doubles(int dim) { return (size_t)dim * kNB; }
size_t dense_inv_pivot_doubles() { return (size_t)kNB * kNB; }
int dense_inv_tiles(int dim) { return (dim + kNB - 1) / kNB; }

cudaError_t launch_dense_inverse(const DenseBatch &B, int maxDim, long long nEntries, double rel,
                                 cudaStream_t st) {
    if (B.nMat == 0) return cudaSuccess;
    const int smem = 2 * kNB * kLd * (int)sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(k_inv_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_inv_update, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_inv_thresholds<<<B.nMat, kInvThreads, 0, st>>>(B, rel);
    const int steps = (maxDim + kNB - 1) / kNB;
    for (int k = 0; k < steps; ++k) {
        k_inv_pivot<<<B.nMat, kInvThreads, 0, st>>>(B, k);
        k_inv_panel<<<B.nRowTiles, kInvThreads, smem, st>>>(B, k);
        k_inv_update<<<B.nTiles, kInvThreads, smem, st>>>(B, k);
        k_inv_writeback<<<B.nRowTiles, kInvThreads, 0, st>>>(B, k);
    }
    const long long g = (nEntries + 255) / 256;
    k_inv_negate<<<(int)(g < 8LL * device_sm_count() ? (g > 0 ? g : 1) : 8LL * device_sm_count()),
                   256, 0, st>>>(B.A, nEntries);
    return cudaGetLastError();
}

}  // namespace xdcg
