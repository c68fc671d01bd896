// Node-level kernels of the A-DEF2 iteration: the update u += alpha p,
// r -= alpha q (Algorithm 1) fused with y = M^-1 r through the node-block
// Cholesky factors (Algorithm 3, first step; blocks of Eqs. block_jacobi /
// block_jacobi_enr) and the partial sums ||r||^2, r^T y; and the set-up
// factorisation of the node blocks.
#include "reduce.cuh"

namespace xdcg {

// ---- update + block-Jacobi apply ----------------------------------------

__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

template <typename T, int B>
__device__ __forceinline__ void update_node(const T *__restrict__ L, int cnt, int t,
                                            long long d0, T *u, T *r, const T *p, const T *q,
                                            T *y, int mode, T alpha, double &rr, double &ry) {
    T w[B];
#pragma unroll
    for (int i = 0; i < B; ++i) w[i] = r[d0 + i];
    if (mode == 0) {
#pragma unroll
        for (int i = 0; i < B; ++i) {
            u[d0 + i] = fma(alpha, p[d0 + i], u[d0 + i]);
            w[i] = fma(-alpha, q[d0 + i], w[i]);
            r[d0 + i] = w[i];
        }
    }
    T rv[B];
#pragma unroll
    for (int i = 0; i < B; ++i) rv[i] = w[i];
    // L w = r (forward), then L^T y = w (backward); diagonal stored inverted
#pragma unroll
    for (int i = 0; i < B; ++i) {
        T s = w[i];
#pragma unroll
        for (int j = 0; j < i; ++j) s = fma(-L[(size_t)tri(i, j) * cnt + t], w[j], s);
        w[i] = s * L[(size_t)tri(i, i) * cnt + t];
    }
#pragma unroll
    for (int i = B - 1; i >= 0; --i) {
        T s = w[i];
#pragma unroll
        for (int j = i + 1; j < B; ++j) s = fma(-L[(size_t)tri(j, i) * cnt + t], w[j], s);
        w[i] = s * L[(size_t)tri(i, i) * cnt + t];
    }
#pragma unroll
    for (int i = 0; i < B; ++i) {
        y[d0 + i] = w[i];
        rr += (double)rv[i] * (double)rv[i];
        ry += (double)rv[i] * (double)w[i];
    }
}

// Branch-enriched node (15 dofs): one warp per node, lane i holds dof i;
// each solved entry of the forward and backward substitutions is broadcast
// by a shuffle, so no thread keeps the whole block in registers.
template <typename T>
__device__ __forceinline__ void update_tip_warp(const T *__restrict__ L, int cnt, int t,
                                                long long d0, T *u, T *r, const T *p,
                                                const T *q, T *y, int mode, T alpha, double &rr,
                                                double &ry) {
    constexpr int B = 15;
    const int lane = threadIdx.x & 31;
    const bool act = lane < B;
    T ri = T(0);
    if (act) {
        ri = r[d0 + lane];
        if (mode == 0) {
            u[d0 + lane] = fma(alpha, p[d0 + lane], u[d0 + lane]);
            ri = fma(-alpha, q[d0 + lane], ri);
            r[d0 + lane] = ri;
        }
    }
    const T dinv = act ? L[(size_t)tri(lane, lane) * cnt + t] : T(0);
    T acc = T(0), w = T(0);
#pragma unroll
    for (int j = 0; j < B; ++j) {
        const T wj = __shfl_sync(0xffffffffu, (ri - acc) * dinv, j);
        if (lane == j) w = wj;
        if (act && lane > j) acc = fma(L[(size_t)tri(lane, j) * cnt + t], wj, acc);
    }
    T yv = T(0);
    T acc2 = T(0);
#pragma unroll
    for (int i = B - 1; i >= 0; --i) {
        const T yi = __shfl_sync(0xffffffffu, (w - acc2) * dinv, i);
        if (lane == i) yv = yi;
        if (act && lane < i) acc2 = fma(L[(size_t)tri(i, lane) * cnt + t], yi, acc2);
    }
    if (act) {
        y[d0 + lane] = yv;
        rr += (double)ri * (double)ri;
        ry += (double)ri * (double)yv;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_update(NodeDev<T> N, T *u, T *r, const T *p, const T *q, T *y, int mode, int nb3, int nb6,
         double *partials, Scalars *sc) {
    pdl_wait();
    if (sc->done != kRunning) return;
    const T alpha = (T)sc->alpha;
    double v[2] = {0.0, 0.0};
    const int bid = blockIdx.x;
    if (bid < nb3) {
        const int t = bid * kThreads + threadIdx.x;
        if (t < N.nStd)
            update_node<T, 3>(N.Lstd, N.nStd, t, N.dofStart[N.stdNodes[t]], u, r, p, q, y, mode,
                              alpha, v[0], v[1]);
    } else if (bid < nb3 + nb6) {
        const int t = (bid - nb3) * kThreads + threadIdx.x;
        if (t < N.nH)
            update_node<T, 6>(N.Lh, N.nH, t, N.dofStart[N.hNodes[t]], u, r, p, q, y, mode,
                              alpha, v[0], v[1]);
    } else {
        const int t = (bid - nb3 - nb6) * kWarps + (threadIdx.x >> 5);
        if (t < N.nT)
            update_tip_warp<T>(N.Lt, N.nT, t, N.dofStart[N.tNodes[t]], u, r, p, q, y, mode,
                               alpha, v[0], v[1]);
    }
    double tot[2];
    if (grid_sum<double, 2>(v, partials, &sc->ticket[2], tot) && threadIdx.x == 0) {
        sc->ry = tot[1];
        sc->rr = tot[0];
        if (sc->hist && sc->its < sc->histCap) sc->hist[sc->its] = tot[0];
        if (tot[0] <= sc->tol2ff)
            sc->done = kConverged;
        else if (sc->its >= sc->max_it)
            sc->done = kMaxIter;
        else if (!isfinite(tot[0]) || !isfinite(tot[1]))
            sc->done = kBreakdown;
    }
}

static inline int cdiv(long long a, int b) { return (int)((a + b - 1) / b); }

template <typename T>
void launch_update(const NodeDev<T> &N, T *u, T *r, const T *p, const T *q, T *y, int mode,
                   double *partials, Scalars *sc, cudaStream_t st) {
    const int nb3 = cdiv(N.nStd, kThreads), nb6 = cdiv(N.nH, kThreads),
              nb15 = cdiv(N.nT, kWarps);
    int grid = nb3 + nb6 + nb15;
    if (grid == 0) grid = 1;
    launch_pdl(k_update<T>, grid, kThreads, 0, st, N, u, r, p, q, y, mode, nb3, nb6, partials, sc);
}
template void launch_update<double>(const NodeDev<double> &, double *, double *, const double *,
                                    const double *, double *, int, double *, Scalars *,
                                    cudaStream_t);
template void launch_update<float>(const NodeDev<float> &, float *, float *, const float *,
                                   const float *, float *, int, double *, Scalars *, cudaStream_t);

// ---- set-up: node-block Cholesky (FP64) ------------------------------------

// Node t of the list (count nodes) factored into position pos[t] of a list
// of total entries (pos == nullptr: t itself, total = count).
template <int B>
__global__ void k_block_cholesky(int count, const int *nodes, const double *__restrict__ D,
                                 double *L64, float *L32, int *bad, const int *pos, int total) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const int w = pos ? pos[t] : t;
    double a[B * (B + 1) / 2];
    double dmax = 0.0;
#pragma unroll
    for (int i = 0; i < B; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) a[tri(i, j)] = D[(size_t)(i * B + j) * count + t];
        dmax = fmax(dmax, a[tri(i, i)]);
    }
    bool ok = dmax > 0.0;
#pragma unroll
    for (int j = 0; j < B; ++j) {
        double s = a[tri(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= a[tri(j, k)] * a[tri(j, k)];
        if (!(s > 1e-14 * dmax)) ok = false;
        const double ljj = sqrt(fmax(s, 1e-300));
        a[tri(j, j)] = ljj;
#pragma unroll
        for (int i = j + 1; i < B; ++i) {
            double v = a[tri(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= a[tri(i, k)] * a[tri(j, k)];
            a[tri(i, j)] = v / ljj;
        }
    }
    if (!ok) atomicMin(bad, nodes[t]);
#pragma unroll
    for (int i = 0; i < B; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            const double v = (i == j) ? 1.0 / a[tri(i, i)] : a[tri(i, j)];
            L64[(size_t)tri(i, j) * total + w] = v;
            if (L32) L32[(size_t)tri(i, j) * total + w] = (float)v;
        }
    }
}

int launch_block_cholesky(int B, int count, const int *nodes, const double *Dsoa, double *L64,
                          float *L32, int *bad, cudaStream_t st, const int *pos, int total) {
    if (count == 0) return 0;
    if (!pos) total = count;
    const int th = 128, grid = cdiv(count, th);
    switch (B) {
        case 3:
            k_block_cholesky<3><<<grid, th, 0, st>>>(count, nodes, Dsoa, L64, L32, bad, pos, total);
            break;
        case 6:
            k_block_cholesky<6><<<grid, th, 0, st>>>(count, nodes, Dsoa, L64, L32, bad, pos, total);
            break;
        case 15:
            k_block_cholesky<15><<<grid, th, 0, st>>>(count, nodes, Dsoa, L64, L32, bad, pos, total);
            break;
        default: return -1;
    }
    return 0;
}

// Factors carried over from an earlier context: entry e of position dst[i]
// (list of total entries) = entry e of position src[i] of the earlier list
// (prevTotal entries); ents = B (B + 1) / 2 entries per node.
__global__ void k_copy_factors(int count, int ents, const int *src, const int *dst,
                               const double *prev, int prevTotal, double *L, int total) {
    const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (idx >= (long long)count * ents) return;
    const int i = (int)(idx % count), e = (int)(idx / count);
    L[(size_t)e * total + dst[i]] = prev[(size_t)e * prevTotal + src[i]];
}

void launch_copy_factors(int count, int ents, const int *src, const int *dst, const double *prev,
                         int prevTotal, double *L, int total, cudaStream_t st) {
    if (count == 0) return;
    const long long n = (long long)count * ents;
    k_copy_factors<<<(int)((n + 255) / 256), 256, 0, st>>>(count, ents, src, dst, prev, prevTotal, L,
                                                          total);
}

// *differ = 1 if a and b (n doubles) differ anywhere (bitwise)
__global__ void k_differ(const double *a, const double *b, long long n, int *differ) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (__double_as_longlong(a[i]) != __double_as_longlong(b[i])) {
            *differ = 1;
            return;
        }
}

void launch_differ(const double *a, const double *b, long long n, int *differ, cudaStream_t st) {
    if (n <= 0) return;
    const long long g = (n + 255) / 256;
    k_differ<<<(int)(g < 4LL * device_sm_count() ? g : 4LL * device_sm_count()), 256, 0, st>>>(
        a, b, n, differ);
}

__global__ void k_xrel(int n, const double *coords, const double *centre, const int *sub,
                       double *x64, float *x32) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= n) return;
    const int s = sub[I];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double v = coords[3 * I + d] - centre[3 * s + d];
        x64[3 * I + d] = v;
        if (x32) x32[3 * I + d] = (float)v;
    }
}

void launch_xrel(int nNodes, const double *coords, const double *centre, const int *sub,
                 double *x64, float *x32, cudaStream_t st) {
    k_xrel<<<cdiv(nNodes, kThreads), kThreads, 0, st>>>(nNodes, coords, centre, sub, x64, x32);
}

}  // namespace xdcg
