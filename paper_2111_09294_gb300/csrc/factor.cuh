// Packed node-block Cholesky factors (FacDev): entry access and the two
// triangular solves, shared by the FP64 <-> FP32 transforms of the mixed path.
#pragma once

#include "internal.h"

namespace xdcg {

__host__ __device__ constexpr int tri2(int i, int j) { return i * (i + 1) / 2 + j; }

// entry (i, j), j <= i, of node I's factor; the diagonal is stored inverted
__device__ __forceinline__ double Lent(const FacDev &F, int l, int t, int i, int j) {
    return F.L[l][(size_t)tri2(i, j) * F.cnt[l] + t];
}

// x := L^-1 x (forward substitution) in place, x[k * stride] for k < b
template <typename P>
__device__ __forceinline__ void fwd_solve(const FacDev &F, int l, int t, int b, P x, int stride) {
    for (int i = 0; i < b; ++i) {
        double s = x[i * stride];
        for (int j = 0; j < i; ++j) s -= Lent(F, l, t, i, j) * x[j * stride];
        x[i * stride] = s * Lent(F, l, t, i, i);
    }
}

// x := L^-T x (backward substitution) in place
template <typename P>
__device__ __forceinline__ void bwd_solve(const FacDev &F, int l, int t, int b, P x, int stride) {
    for (int i = b - 1; i >= 0; --i) {
        double s = x[i * stride];
        for (int j = i + 1; j < b; ++j) s -= Lent(F, l, t, j, i) * x[j * stride];
        x[i * stride] = s * Lent(F, l, t, i, i);
    }
}

// the same for node I, unit stride
__device__ __forceinline__ void fwd_solve_node(const FacDev &F, int I, int b, double *x) {
    fwd_solve(F, F.nodeList[I], F.nodeIdx[I], b, x, 1);
}

__device__ __forceinline__ void bwd_solve_node(const FacDev &F, int I, int b, double *x) {
    bwd_solve(F, F.nodeList[I], F.nodeIdx[I], b, x, 1);
}

}  // namespace xdcg
