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

}  // namespace xdcg
