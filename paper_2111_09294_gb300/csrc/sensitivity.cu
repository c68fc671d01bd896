// Sensitivity of a solve to each element's Young's modulus: with
// K = sum_e E_e Khat_e (Khat_e the element stiffness for E = 1 at fixed
// Poisson ratio) and u = K^-1 f, a loss J(u) has
//     dJ/dE_e = -lam_e^T Khat_e u_e,   K lam = dJ/du
// (the adjoint of the solve; lam comes from a second solve on the same
// context, K being symmetric).  Not part of the paper's method: it serves
// differentiable use of the solver.
//
// One warp per element.  The element's u and lam entries are gathered into
// shared memory; lane j forms s_j = sum_i lam_i Khat_ij for its columns
// j = lane, lane + 32, ... (row-major Khat_e: consecutive lanes read
// consecutive entries of row i) and adds u_j s_j; the lane sums are added by
// a fixed butterfly.  Elements without enriched nodes may share one matrix,
// which then stays in L1.
#include <cmath>
#include <cstdint>

#include "internal.h"

namespace xdcg {

constexpr int kSensWarps = 8;

__global__ void __launch_bounds__(kSensWarps * 32)
k_element_sensitivity(long long nEl, long long n, const int64_t *__restrict__ dofPtr,
                      const int32_t *__restrict__ dofs, const int64_t *__restrict__ matOff,
                      long long matLen, const double *__restrict__ mats,
                      const double *__restrict__ u, const double *__restrict__ lam,
                      double *__restrict__ out, int *bad) {
    __shared__ double su[kSensWarps][kSensMaxDofs], sl[kSensWarps][kSensMaxDofs];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long e = (long long)blockIdx.x * kSensWarps + warp;
    if (e >= nEl) return;
    const long long d0 = dofPtr[e], de64 = dofPtr[e + 1] - d0, m0 = matOff[e];
    if (de64 < 0 || de64 > kSensMaxDofs || m0 < 0 || m0 + de64 * de64 > matLen) {
        if (lane == 0) {
            out[e] = NAN;
            atomicExch(bad, 1);
        }
        return;
    }
    const int de = (int)de64;
    bool ok = true;
    for (int i = lane; i < de; i += 32) {
        const int d = dofs[d0 + i];
        ok = ok && d < n;
        const bool live = d >= 0 && d < n;
        su[warp][i] = live ? u[d] : 0.0;
        sl[warp][i] = live ? lam[d] : 0.0;
    }
    if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) {
            out[e] = NAN;
            atomicExch(bad, 1);
        }
        return;
    }
    __syncwarp();
    const double *Kh = mats + m0;
    double acc = 0.0;
    for (int j = lane; j < de; j += 32) {
        double s = 0.0;
        for (int i = 0; i < de; ++i) s = fma(sl[warp][i], Kh[(size_t)i * de + j], s);
        acc = fma(su[warp][j], s, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) out[e] = -acc;
}

void launch_element_sensitivity(long long nEl, long long n, const int64_t *dofPtr,
                                const int32_t *dofs, const int64_t *matOff, long long matLen,
                                const double *mats, const double *u, const double *lam,
                                double *out, int *bad, cudaStream_t st) {
    if (nEl <= 0) return;
    const long long grid = (nEl + kSensWarps - 1) / kSensWarps;
    k_element_sensitivity<<<(unsigned)grid, kSensWarps * 32, 0, st>>>(
        nEl, n, dofPtr, dofs, matOff, matLen, mats, u, lam, out, bad);
}

// dJ/dK sampled on K's stored pattern: for the stored block p = (I, J),
// entry (a, b) of the block receives -lam[dofStart[I] + a] * u[dofStart[J] + b],
// the outer product -lam u^T (the gradient of J(u), u = K^-1 f, with respect
// to K's entries, K lam = dJ/du) at the positions K stores.  One thread per
// stored block; its row I by binary search in rowPtr.  A structural entry out
// of range (column, value range, dof) sets *bad and leaves that block
// unwritten.
__global__ void k_stiffness_gradient(int nNodes, long long nnzb, long long n, long long nval,
                                     const int32_t *__restrict__ dofStart,
                                     const int32_t *__restrict__ rowPtr,
                                     const int32_t *__restrict__ col,
                                     const int64_t *__restrict__ valPtr,
                                     const double *__restrict__ lam,
                                     const double *__restrict__ u, double *__restrict__ out,
                                     int *bad) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= nnzb) return;
    int lo = 0, hi = nNodes - 1;   // last row I with rowPtr[I] <= p
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (rowPtr[mid] <= p)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int I = lo, J = col[p];
    if (J < 0 || J >= nNodes) {
        atomicExch(bad, 1);
        return;
    }
    const long long dI = dofStart[I], dJ = dofStart[J];
    const int bI = dofStart[I + 1] - dofStart[I], bJ = dofStart[J + 1] - dofStart[J];
    const long long v0 = valPtr[p];
    if (bI < 1 || bJ < 1 || dI + bI > n || dJ + bJ > n || v0 < 0 || valPtr[p + 1] != v0 + bI * bJ ||
        v0 + bI * bJ > nval) {
        atomicExch(bad, 1);
        return;
    }
    for (int a = 0; a < bI; ++a) {
        const double la = -lam[dI + a];
        for (int b = 0; b < bJ; ++b) out[v0 + a * bJ + b] = la * u[dJ + b];
    }
}

void launch_stiffness_gradient(int nNodes, long long nnzb, long long n, long long nval,
                               const int32_t *dofStart, const int32_t *rowPtr, const int32_t *col,
                               const int64_t *valPtr, const double *lam, const double *u,
                               double *out, int *bad, cudaStream_t st) {
    if (nnzb <= 0) return;
    k_stiffness_gradient<<<(unsigned)((nnzb + 255) / 256), 256, 0, st>>>(
        nNodes, nnzb, n, nval, dofStart, rowPtr, col, valPtr, lam, u, out, bad);
}

}  // namespace xdcg
