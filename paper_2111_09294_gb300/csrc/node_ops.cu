// Node- and box-level kernels of the A-DEF2 iteration:
//   update   u += alpha p, r -= alpha q (Algorithm 1), y = M^-1 r with the
//            node-block Cholesky factors (Algorithm 3, first step; blocks of
//            Eqs. block_jacobi / block_jacobi_enr), partial ||r||^2, r^T y;
//   restrict g = Z^T r - W^T y per box (Algorithm 3, right-hand sides of
//            both coarse solves merged: lambda - mu = E^-1 (Z^T r - W^T y));
//   prolong  p = y + Z nu + beta p (Algorithm 3 last step fused with the
//            direction update of Algorithm 1), or u = Z nu (Algorithm 2).
// Z is never stored: its rows are rebuilt from the node position relative
// to the box centre (Eqs. dcg_deflation_space, dcg_deflation_space_enr_std,
// dcg_deflation_space_enr_enr).
#include "reduce.cuh"

namespace xdcg {

// ---- rigid-body block R(x) of the deflation space -------------------------

// R^T a for a 3-vector a: the 6 coarse entries a node's 3 dofs feed.
template <typename T>
__device__ __forceinline__ void rigid_t(double a0, double a1, double a2, T X, T Y, T Z,
                                        double (&o)[6]) {
    o[0] = a0;
    o[1] = a1;
    o[2] = a2;
    o[3] = -(double)Z * a1 + (double)Y * a2;
    o[4] = (double)Z * a0 - (double)X * a2;
    o[5] = -(double)Y * a0 + (double)X * a1;
}

// R nu for 6 coarse values: the displacement the rigid modes give the node.
template <typename T>
__device__ __forceinline__ void rigid(const T (&n)[6], T X, T Y, T Z, T (&v)[3]) {
    v[0] = n[0] + Z * n[4] - Y * n[5];
    v[1] = n[1] - Z * n[3] + X * n[5];
    v[2] = n[2] + Y * n[3] - X * n[4];
}

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
    if (grid_sum<2>(v, partials, &sc->ticket[2], tot) && threadIdx.x == 0) {
        sc->ry = tot[1];
        sc->rr = tot[0];
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
    k_update<T><<<grid, kThreads, 0, st>>>(N, u, r, p, q, y, mode, nb3, nb6, partials, sc);
}
template void launch_update<double>(const NodeDev<double> &, double *, double *, const double *,
                                    const double *, double *, int, double *, Scalars *,
                                    cudaStream_t);
template void launch_update<float>(const NodeDev<float> &, float *, float *, const float *,
                                   const float *, float *, int, double *, Scalars *, cudaStream_t);

// ---- restriction g = Z^T a - W^T b -----------------------------------------

constexpr int kBoxThreads = 128;

template <typename T, int M>
__device__ __forceinline__ void restrict_box(const NodeDev<T> &N, const BoxDev<T> &B, int s,
                                             const T *a, const T *b, int withW, double *g,
                                             double *zr) {
    double acc[2 * M];
#pragma unroll
    for (int c = 0; c < 2 * M; ++c) acc[c] = 0.0;
    const int o1 = B.ownPtr[s + 1];
    for (int t = B.ownPtr[s] + threadIdx.x; t < o1; t += blockDim.x) {
        const int I = B.ownNodes[t];
        const long long d0 = N.dofStart[I];
        const T X = N.xrel[3 * I], Y = N.xrel[3 * I + 1], Z = N.xrel[3 * I + 2];
        double z[6];
        rigid_t<T>((double)a[d0], (double)a[d0 + 1], (double)a[d0 + 2], X, Y, Z, z);
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] += z[c];
        if (M == 12) {
            const double H = (double)N.hsign[I];
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[6 + c] += H * z[c];
            if (N.dofStart[I + 1] - d0 == 6) {
                rigid_t<T>((double)a[d0 + 3], (double)a[d0 + 4], (double)a[d0 + 5], X, Y, Z, z);
#pragma unroll
                for (int c = 0; c < 6; ++c) acc[6 + c] += z[c];
            }
        }
    }
    if (withW) {
        const int e1 = B.extPtr[s + 1];
        for (int e = B.extPtr[s] + threadIdx.x; e < e1; e += blockDim.x) {
            const int I = B.extNode[e];
            const long long d0 = N.dofStart[I];
            const int bI = N.dofStart[I + 1] - (int)d0;
            const T *Wb = B.W + B.wOff[e];
            for (int i = 0; i < bI; ++i) {
                const double bv = (double)b[d0 + i];
#pragma unroll
                for (int c = 0; c < M; ++c) acc[M + c] += (double)Wb[i * M + c] * bv;
            }
        }
    }
    block_sum<2 * M>(acc);
    if (threadIdx.x == 0) {
        const int c0 = N.col0[s];
#pragma unroll
        for (int c = 0; c < M; ++c) {
            g[c0 + c] = acc[c] - acc[M + c];
            if (zr) zr[c0 + c] = acc[c];
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kBoxThreads)
k_restrict(NodeDev<T> N, BoxDev<T> B, const T *a, const T *b, int withW, double *g, double *zr,
           const Scalars *sc) {
    if (sc && sc->done != kRunning) return;
    const int s = blockIdx.x;
    if (N.menr[s])
        restrict_box<T, 12>(N, B, s, a, b, withW, g, zr);
    else
        restrict_box<T, 6>(N, B, s, a, b, withW, g, zr);
}

template <typename T>
void launch_restrict(const NodeDev<T> &N, const BoxDev<T> &B, const T *a, const T *b, int withW,
                     double *g, double *zr, cudaStream_t st, const Scalars *sc) {
    k_restrict<T><<<B.nBox, kBoxThreads, 0, st>>>(N, B, a, b, withW, g, zr, sc);
}
template void launch_restrict<double>(const NodeDev<double> &, const BoxDev<double> &,
                                      const double *, const double *, int, double *, double *,
                                      cudaStream_t, const Scalars *);
template void launch_restrict<float>(const NodeDev<float> &, const BoxDev<float> &, const float *,
                                     const float *, int, double *, double *, cudaStream_t,
                                     const Scalars *);

// ---- prolongation ----------------------------------------------------------

// mode 0: p = y + Z nu + beta p;  mode 1: p = Z nu;  mode 2: p = y + Z nu
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_prolong(NodeDev<T> N, const double *__restrict__ nu, const T *__restrict__ y, T *p, int mode,
          Scalars *sc) {
    if (sc->done != kRunning) return;
    const int I = blockIdx.x * kThreads + threadIdx.x;
    if (I >= N.nNodes) return;
    const long long d0 = N.dofStart[I];
    const int bI = N.dofStart[I + 1] - (int)d0;
    const int s = N.sub[I];
    const int c0 = N.col0[s];
    const int menr = N.menr[s];
    const T X = N.xrel[3 * I], Y = N.xrel[3 * I + 1], Z = N.xrel[3 * I + 2];
    T n6[6], v[3], ve[3] = {T(0), T(0), T(0)};
#pragma unroll
    for (int c = 0; c < 6; ++c) n6[c] = (T)nu[c0 + c];
    rigid<T>(n6, X, Y, Z, v);
    if (menr) {
#pragma unroll
        for (int c = 0; c < 6; ++c) n6[c] = (T)nu[c0 + 6 + c];
        rigid<T>(n6, X, Y, Z, ve);
        const T H = (T)N.hsign[I];
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c] += H * ve[c];
    }
    const T beta = (T)sc->beta;
    for (int i = 0; i < bI; ++i) {
        T zv;
        if (i < 3)
            zv = v[i];
        else if (bI == 6 && menr)
            zv = ve[i - 3];
        else
            zv = T(0);
        const long long d = d0 + i;
        if (mode == 0)
            p[d] = y[d] + zv + beta * p[d];
        else if (mode == 1)
            p[d] = zv;
        else
            p[d] = y[d] + zv;
    }
}

template <typename T>
void launch_prolong(const NodeDev<T> &N, const double *nu, const T *y, T *p, int mode,
                    Scalars *sc, cudaStream_t st) {
    k_prolong<T><<<cdiv(N.nNodes, kThreads), kThreads, 0, st>>>(N, nu, y, p, mode, sc);
}
template void launch_prolong<double>(const NodeDev<double> &, const double *, const double *,
                                     double *, int, Scalars *, cudaStream_t);
template void launch_prolong<float>(const NodeDev<float> &, const double *, const float *,
                                    float *, int, Scalars *, cudaStream_t);

// ---- set-up: node-block Cholesky (FP64) ------------------------------------

template <int B>
__global__ void k_block_cholesky(int count, const int *nodes, const double *__restrict__ D,
                                 double *L64, float *L32, int *bad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
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
            L64[(size_t)tri(i, j) * count + t] = v;
            if (L32) L32[(size_t)tri(i, j) * count + t] = (float)v;
        }
    }
}

int launch_block_cholesky(int B, int count, const int *nodes, const double *Dsoa, double *L64,
                          float *L32, int *bad, cudaStream_t st) {
    if (count == 0) return 0;
    const int th = 128, grid = cdiv(count, th);
    switch (B) {
        case 3: k_block_cholesky<3><<<grid, th, 0, st>>>(count, nodes, Dsoa, L64, L32, bad); break;
        case 6: k_block_cholesky<6><<<grid, th, 0, st>>>(count, nodes, Dsoa, L64, L32, bad); break;
        case 15: k_block_cholesky<15><<<grid, th, 0, st>>>(count, nodes, Dsoa, L64, L32, bad); break;
        default: return -1;
    }
    return 0;
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
