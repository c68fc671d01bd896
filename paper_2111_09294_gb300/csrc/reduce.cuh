// Deterministic warp / block / grid reductions.  Every block stores its
// partial sums; the last block to finish (ticket counter) adds them in a
// fixed order, so results do not depend on block scheduling.
//
// The accumulator type A is the kernel's own precision: FP32 kernels keep
// their per-thread, warp and block sums in FP32 (FP64 arithmetic runs at
// 1/64 of the FP32 rate on this GPU), and only the per-block partials are
// combined in FP64 by the last block.
#pragma once

#include "internal.h"
#include "pdl.cuh"

namespace xdcg {

template <typename A, int NV>
__device__ __forceinline__ void warp_sum(A (&v)[NV]) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    }
}

// Sum over the block; the result is valid in thread 0.
template <typename A, int NV>
__device__ __forceinline__ void block_sum(A (&v)[NV]) {
    __shared__ A sm[NV][32];
    warp_sum<A, NV>(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    __syncthreads();
    if (l == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) sm[i][w] = v[i];
    }
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = (l < nw) ? sm[i][l] : A(0);
        warp_sum<A, NV>(v);
    }
}

// The last block's share of a grid-wide sum: value i of the nblk blocks'
// partials (partials[i * nblk + b]) added by one warp, its lanes striding
// over the blocks with four accumulators each, then across the lanes (a fixed
// order, and FP64 work spread over the warps: FP64 arithmetic is slow here).
// Thread 0 gets the totals and resets the ticket.
template <int NV>
__device__ __forceinline__ void sum_partials(const double *partials, unsigned int *ticket,
                                             double (&tot)[NV], int nblk) {
    __shared__ double fin[NV];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = w; i < NV; i += nw) {
        const double *p = partials + (size_t)i * nblk;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int b = l;
        for (; b + 96 < nblk; b += 128) {
            s0 += __ldcg(p + b);
            s1 += __ldcg(p + b + 32);
            s2 += __ldcg(p + b + 64);
            s3 += __ldcg(p + b + 96);
        }
        for (; b < nblk; b += 32) s0 += __ldcg(p + b);
        double s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (l == 0) fin[i] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) tot[i] = fin[i];
        *ticket = 0u;
    }
}

// Grid-wide sum of NV <= 32 values whose block totals lanes 0 .. NV - 1 of
// warp 0 already hold (one per lane, in v): as grid_sum_of without the block
// reduction.  Every thread of the block calls it.
template <int NV>
__device__ __forceinline__ bool grid_sum_lanes(double v, double *partials, unsigned int *ticket,
                                               double (&tot)[NV], int blk, int nblk) {
    __shared__ bool last;
    if (threadIdx.x < 32) {
        if ((int)threadIdx.x < NV) partials[(size_t)threadIdx.x * nblk + blk] = v;
        __threadfence();
        __syncwarp();
        if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == (unsigned int)nblk - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    sum_partials<NV>(partials, ticket, tot, nblk);
    return true;
}

// Sum over the blocks blk = 0 .. nblk - 1 of one reduction (the launch's
// blocks, or one system's share of a launch over several systems).  Returns
// true in exactly one of them (the last to finish), where thread 0 then holds
// the FP64 totals in tot.  partials: NV * nblk doubles.
template <typename A, int NV>
__device__ __forceinline__ bool grid_sum_of(A (&v)[NV], double *partials, unsigned int *ticket,
                                            double (&tot)[NV], int blk, int nblk) {
    __shared__ bool last;
    block_sum<A, NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) partials[(size_t)i * nblk + blk] = (double)v[i];
        __threadfence();
        unsigned int t = atomicAdd(ticket, 1u);
        last = (t == (unsigned int)nblk - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    sum_partials<NV>(partials, ticket, tot, nblk);
    return true;
}

// Double-float arithmetic: a value as an unevaluated sum hi + lo of two
// floats (about 48 significant bits), added with FP32 operations only
// (Knuth's two-sum, then renormalisation).  Used where many blocks each add
// the same few hundred partial sums: FP64 runs at about 1/64 of the FP32
// rate on this part.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    const float e = (a.x - (s - bb)) + (b.x - bb);
    const float t = (e + a.y) + b.y;
    const float hi = s + t;
    return make_float2(hi, t - (hi - s));
}
__device__ __forceinline__ float2 df_of(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// The total of n block partials (double-float) a previous kernel stored
// (kFinDefer and the FP32 iteration's deferred sums): every thread loads its
// share at once (one round trip), the shares are added in a fixed order
// within each thread, by a tree over the lanes and over the warps, so every
// block of the consuming kernel gets the same bits; valid in every thread.
// Replaces the producer's ticketed last-block reduction (fence, atomic, the
// last block's tail).
__device__ __forceinline__ double block_read_total(const float2 *partials, int n) {
    constexpr int kLoads = 8;
    __shared__ float2 wsum[32];
    __shared__ double total;
    const int t = threadIdx.x, nt = blockDim.x;
    float2 v[kLoads];
#pragma unroll
    for (int q = 0; q < kLoads; ++q) {
        const int i = t + q * nt;
        v[q] = i < n ? __ldcg(partials + i) : make_float2(0.f, 0.f);
    }
    float2 acc = v[0];
#pragma unroll
    for (int q = 1; q < kLoads; ++q) acc = df_add(acc, v[q]);
    for (int i = t + kLoads * nt; i < n; i += nt) acc = df_add(acc, __ldcg(partials + i));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float2 other;
        other.x = __shfl_xor_sync(0xffffffffu, acc.x, o);
        other.y = __shfl_xor_sync(0xffffffffu, acc.y, o);
        acc = df_add(acc, other);
    }
    if ((t & 31) == 0) wsum[t >> 5] = acc;
    __syncthreads();
    if (t == 0) {
        float2 s = wsum[0];
        for (int w = 1; w < (nt >> 5); ++w) s = df_add(s, wsum[w]);
        total = (double)s.x + (double)s.y;
    }
    __syncthreads();
    return total;
}

// Grid-wide sum over the launch's blocks (see grid_sum_of).
template <typename A, int NV>
__device__ __forceinline__ bool grid_sum(A (&v)[NV], double *partials, unsigned int *ticket,
                                         double (&tot)[NV]) {
    return grid_sum_of<A, NV>(v, partials, ticket, tot, (int)blockIdx.x, (int)gridDim.x);
}

// Grid-wide sum of one value already reduced to thread 0 of each block:
// returns true in the last block to finish, where thread 0 holds the FP64
// total (block partials added in block order).
__device__ __forceinline__ bool grid_sum_t0(double v, double *partials, unsigned int *ticket,
                                            double &tot) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = v;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double s[1] = {0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) s[0] += __ldcg(partials + b);
    block_sum<double, 1>(s);
    if (threadIdx.x == 0) {
        tot = s[0];
        *ticket = 0u;
    }
    return true;
}

// Shared last-block actions on the scalar block.
__device__ __forceinline__ void finalize(Scalars *sc, int fin, int slot, double val) {
    if (fin == kFinAlpha) {
        sc->pq = val;
        sc->its += 1;
        if (!(val > 0.0) || !isfinite(val)) {
            sc->done = kBreakdown;
        } else {
            sc->alpha = sc->rho / val;
        }
    } else if (fin == kFinRR) {
        sc->rr = val;
        if (sc->hist && sc->histCap > 0) sc->hist[0] = val;
        if (val <= sc->tol2ff) sc->done = kConverged;
    } else {
        sc->scratch[slot] = val;
    }
}

}  // namespace xdcg
