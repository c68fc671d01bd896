// Packed node-block Cholesky factors (FacDev): entry access and the two
// triangular solves, shared by the FP64 <-> FP32 transforms of the mixed path.
#pragma once

#include <type_traits>

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

// The same with the block size B a compile-time constant, so that x stays in
// registers (a runtime-sized x lives in local memory).  The factor list of a
// B-dof node is fixed by B (3, 6, 15 -> 0, 1, 2), so it is not indexed at
// run time either; t is the node's index within that list.
template <int B>
__device__ __forceinline__ void fwd_solve_fixed(const FacDev &F, int t, double (&x)[B]) {
    constexpr int l = B == 3 ? 0 : (B == 6 ? 1 : 2);
    const double *L = F.L[l];
    const size_t cnt = (size_t)F.cnt[l];
#pragma unroll
    for (int i = 0; i < B; ++i) {
        double s = x[i];
#pragma unroll
        for (int j = 0; j < i; ++j) s -= L[tri2(i, j) * cnt + t] * x[j];
        x[i] = s * L[tri2(i, i) * cnt + t];
    }
}

template <int B>
__device__ __forceinline__ void bwd_solve_fixed(const FacDev &F, int t, double (&x)[B]) {
    constexpr int l = B == 3 ? 0 : (B == 6 ? 1 : 2);
    const double *L = F.L[l];
    const size_t cnt = (size_t)F.cnt[l];
#pragma unroll
    for (int i = B - 1; i >= 0; --i) {
        double s = x[i];
#pragma unroll
        for (int j = i + 1; j < B; ++j) s -= L[tri2(j, i) * cnt + t] * x[j];
        x[i] = s * L[tri2(i, i) * cnt + t];
    }
}

// Calls f(std::integral_constant<int, b>) for a node of b dofs: 3, 6 or 15,
// the only node sizes set-up accepts.
template <typename Fn>
__device__ __forceinline__ void with_node_size(int b, Fn &&f) {
    if (b == 3)
        f(std::integral_constant<int, 3>());
    else if (b == 6)
        f(std::integral_constant<int, 6>());
    else
        f(std::integral_constant<int, 15>());
}

}  // namespace xdcg
