// Box-level kernels of Algorithm 3: the restriction g = Z^T r - W^T y
// (right-hand sides of both coarse solves, merged) and the prolongation
// p = y + Z nu (+ beta p), one CTA per box subdomain.
//
// Work split: the lanes of a warp form 32 / M groups of M lanes (M = 6 or 12
// coarse columns of the box); lane (group, column c) accumulates column c
// over its share of the box's nodes, so every lane keeps two running sums
// and the only cross-lane step is a short, fixed-order sum in shared memory.
// Node data are stored in box order (slots), so a box's nodes are contiguous.
//
// Z is applied matrix-free from the node position relative to the box
// centre (Eqs. dcg_deflation_space, dcg_deflation_space_enr_std,
// dcg_deflation_space_enr_enr) in the FP64 path, and from the explicit
// scaled basis Z~ = L^T Z in the FP32 block-scaled path.
#include "cache.cuh"
#include "reduce.cuh"

namespace xdcg {

constexpr int kBoxThreads = 128;   // small CTAs: all boxes of an 8^3 split resident at once

// column c (0..5) of R(x)^T a, R the rigid block of Eq. dcg_deflation_space
template <typename A>
__device__ __forceinline__ A rigid_col(int c, A a0, A a1, A a2, A X, A Y, A Z) {
    switch (c) {
        case 0: return a0;
        case 1: return a1;
        case 2: return a2;
        case 3: return -Z * a1 + Y * a2;
        case 4: return Z * a0 - X * a2;
        default: return -Y * a0 + X * a1;
    }
}

// Sum over rows i of one node block: acc += blk[i * M + c] * v[d0 + i].  The
// three standard rows are loaded straight-line so that four entries' loads
// are in flight together; enriched rows (i >= 3) follow in a loop.
template <typename T, typename A, int M, int U>
__device__ __forceinline__ void block_col_dot(const T *base, const long long (&off)[U],
                                              const int (&d0)[U], const int (&bI)[U],
                                              const T *v, int c, A &acc) {
    A w[U][3], x[U][3];
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            w[u][i] = bI[u] ? (A)base[off[u] + i * M + c] : A(0);
            x[u][i] = bI[u] ? (A)v[d0[u] + i] : A(0);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
        for (int i = 0; i < 3; ++i) acc = fma(w[u][i], x[u][i], acc);
        if (bI[u] > 3) {
            // enriched rows (3 jump or 12 branch dofs): all loads first
            A we[12], xe[12];
#pragma unroll
            for (int i = 0; i < 12; ++i) {
                const bool ok = 3 + i < bI[u];
                we[i] = ok ? (A)base[off[u] + (3 + i) * M + c] : A(0);
                xe[i] = ok ? (A)v[d0[u] + 3 + i] : A(0);
            }
#pragma unroll
            for (int i = 0; i < 12; ++i) acc = fma(we[i], xe[i], acc);
        }
    }
}

template <typename T, typename A, int M, bool EXPL>
__device__ __forceinline__ void restrict_box(const BoxDev<T> &B, int s, const T *a, const T *b,
                                             int withW, double *g, double *zr) {
    constexpr int G = 32 / M;
    constexpr int kSlots = (kBoxThreads / 32) * G;
    constexpr int U = 4;
    __shared__ double red[2][kSlots * M];
    __shared__ double tot[2][M];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / M, c = lane - grp * M;
    const bool act = grp < G;
    const int slot = warp * G + grp;
    A za = A(0), wb = A(0);
    if (act) {
        const int o0 = B.ownPtr[s], o1 = B.ownPtr[s + 1];
        if (EXPL) {
            for (int t = o0 + slot; t < o1; t += U * kSlots) {
                long long off[U];
                int d0[U], bI[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int tt = t + u * kSlots;
                    const bool ok = tt < o1;
                    off[u] = ok ? B.ownZ[tt] : 0;
                    d0[u] = ok ? B.ownDof[tt] : 0;
                    bI[u] = ok ? B.ownB[tt] : 0;
                }
                block_col_dot<T, A, M, U>(B.Zt, off, d0, bI, a, c, za);
            }
        } else {
            const int c6 = (M == 12 && c >= 6) ? c - 6 : c;
            for (int t = o0 + slot; t < o1; t += kSlots) {
                const int d0 = B.ownDof[t];
                const A X = B.ownX[3 * t], Y = B.ownX[3 * t + 1], Z = B.ownX[3 * t + 2];
                A v = rigid_col<A>(c6, a[d0], a[d0 + 1], a[d0 + 2], X, Y, Z);
                if (M == 12 && c >= 6) {
                    v *= (A)B.ownH[t];
                    if (B.ownB[t] == 6)
                        v += rigid_col<A>(c6, a[d0 + 3], a[d0 + 4], a[d0 + 5], X, Y, Z);
                }
                za += v;
            }
        }
        if (withW) {
            const int e1 = B.extPtr[s + 1];
            for (int e = B.extPtr[s] + slot; e < e1; e += U * kSlots) {
                long long off[U];
                int d0[U], bI[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int ee = e + u * kSlots;
                    const bool ok = ee < e1;
                    off[u] = ok ? B.wOff[ee] : 0;
                    d0[u] = ok ? B.extDof[ee] : 0;
                    bI[u] = ok ? B.extB[ee] : 0;
                }
                block_col_dot<T, A, M, U>(B.W, off, d0, bI, b, c, wb);
            }
        }
        red[0][slot * M + c] = (double)za;
        red[1][slot * M + c] = (double)wb;
    }
    __syncthreads();
    if (threadIdx.x < 2 * M) {
        const int which = threadIdx.x / M, cc = threadIdx.x - which * M;
        double sum = 0.0;
        for (int q = 0; q < kSlots; ++q) sum += red[which][q * M + cc];
        tot[which][cc] = sum;
    }
    __syncthreads();
    if (threadIdx.x < M) {
        const int c0 = B.col0[s];
        g[c0 + threadIdx.x] = tot[0][threadIdx.x] - tot[1][threadIdx.x];
        if (zr) zr[c0 + threadIdx.x] = tot[0][threadIdx.x];
    }
}

template <typename T, typename A, bool EXPL>
__global__ void __launch_bounds__(kBoxThreads, 4)
k_restrict(BoxDev<T> B, const T *a, const T *b, int withW, double *g, double *zr,
           const Scalars *sc) {
    pdl_wait();
    if (sc && sc->done != kRunning) return;
    const int s = blockIdx.x;
    if (B.menr[s])
        restrict_box<T, A, 12, EXPL>(B, s, a, b, withW, g, zr);
    else
        restrict_box<T, A, 6, EXPL>(B, s, a, b, withW, g, zr);
}

void launch_restrict(const BoxDev<double> &B, const double *a, const double *b, int withW,
                     double *g, double *zr, const Scalars *sc, cudaStream_t st) {
    // Z by value (B.Zt) or from the geometry
    launch_pdl(B.Zt ? k_restrict<double, double, true> : k_restrict<double, double, false>, B.nBox,
               kBoxThreads, 0, st, B, a, b, withW, g, zr, sc);
}


// ---- prolongation ----------------------------------------------------------

// mode 0: p = y + Z nu + beta p;  mode 1: p = Z nu;  mode 2: p = y + Z nu
template <typename T>
__device__ __forceinline__ void emit(T *p, const T *y, int d, T zv, int mode, T beta) {
    if (mode == 0)
        p[d] = y[d] + zv + beta * p[d];
    else if (mode == 1)
        p[d] = zv;
    else
        p[d] = y[d] + zv;
}

template <typename T, int M, bool EXPL>
__device__ __forceinline__ void prolong_box(const BoxDev<T> &B, int s, const T *nu, const T *y,
                                            T *p, int mode, T beta) {
    const int c0 = B.col0[s];
    T n[M];
#pragma unroll
    for (int c = 0; c < M; ++c) n[c] = nu[c0 + c];
    const int o1 = B.ownPtr[s + 1];
    for (int t = B.ownPtr[s] + threadIdx.x; t < o1; t += blockDim.x) {
        const int d0 = B.ownDof[t], bI = B.ownB[t];
        if (EXPL) {
            const T *Zb = B.Zt + B.ownZ[t];
            T z[3][M];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
#pragma unroll
                for (int c = 0; c < M; ++c) z[i][c] = Zb[i * M + c];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                T zv = T(0);
#pragma unroll
                for (int c = 0; c < M; ++c) zv = fma(z[i][c], n[c], zv);
                emit(p, y, d0 + i, zv, mode, beta);
            }
            for (int i0 = 3; i0 < bI; i0 += 3) {
                // enriched rows three at a time, loads first
                T ze[3][M];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
#pragma unroll
                    for (int c = 0; c < M; ++c) ze[i][c] = Zb[(i0 + i) * M + c];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    T zv = T(0);
#pragma unroll
                    for (int c = 0; c < M; ++c) zv = fma(ze[i][c], n[c], zv);
                    emit(p, y, d0 + i0 + i, zv, mode, beta);
                }
            }
        } else {
            const T X = B.ownX[3 * t], Y = B.ownX[3 * t + 1], Z = B.ownX[3 * t + 2];
            T v[3], ve[3] = {T(0), T(0), T(0)};
            v[0] = n[0] + Z * n[4] - Y * n[5];
            v[1] = n[1] - Z * n[3] + X * n[5];
            v[2] = n[2] + Y * n[3] - X * n[4];
            if (M == 12) {
                ve[0] = n[6] + Z * n[10] - Y * n[11];
                ve[1] = n[7] - Z * n[9] + X * n[11];
                ve[2] = n[8] + Y * n[9] - X * n[10];
                const T H = (T)B.ownH[t];
#pragma unroll
                for (int i = 0; i < 3; ++i) v[i] += H * ve[i];
            }
#pragma unroll
            for (int i = 0; i < 3; ++i) emit(p, y, d0 + i, v[i], mode, beta);
            if (bI == 6) {
#pragma unroll
                for (int i = 0; i < 3; ++i) emit(p, y, d0 + 3 + i, M == 12 ? ve[i] : T(0), mode, beta);
            } else {
                for (int i = 3; i < bI; ++i) emit(p, y, d0 + i, T(0), mode, beta);
            }
        }
    }
}

template <typename T, bool EXPL>
__global__ void __launch_bounds__(kBoxThreads, 4)
k_prolong(BoxDev<T> B, const T *nu, const T *y, T *p, int mode, Scalars *sc) {
    pdl_wait();
    if (sc->done != kRunning) return;
    const int s = blockIdx.x;
    const T beta = (T)sc->beta;
    if (B.menr[s])
        prolong_box<T, 12, EXPL>(B, s, nu, y, p, mode, beta);
    else
        prolong_box<T, 6, EXPL>(B, s, nu, y, p, mode, beta);
}

void launch_prolong(const BoxDev<double> &B, const double *nu, const double *y, double *p,
                    int mode, Scalars *sc, cudaStream_t st) {
    launch_pdl(B.Zt ? k_prolong<double, true> : k_prolong<double, false>, B.nBox, kBoxThreads, 0,
               st, B, nu, y, p, mode, sc);
}


// ---- row-parallel box kernels of the block-scaled FP32 path -----------------

constexpr int kRowThreads = 256;

// A unit covers own rows [ownBegin, ownEnd) and coupled rows [extBegin,
// extEnd) of one box (most boxes are one unit).  acc[0..M): Z~^T r over its
// own rows, acc[M..2M): W~^T r over its coupled rows, acc[2M]: ||r||^2;
// returns (in thread 0) the unit's ||r||^2 after one block reduction.
// YV (caller blocks, mode 3): the coupled rows take W~^T of y = M~^-1 r
template <int M, bool YV>
__device__ __forceinline__ float restrict_update_unit(const RowBoxDev &B, int unit, float *u,
                                                      const float *r_cur, float *r_next,
                                                      const float *p, const float *q,
                                                      const float *yv, int mode, float alpha,
                                                      double *g, double *zr) {
    const int s = B.unitBox[unit];
    float acc[2 * M + 1];
#pragma unroll
    for (int c = 0; c <= 2 * M; ++c) acc[c] = 0.0f;
    const uint64_t keep = l2_keep_policy();
    {
        const int r0 = B.ownRowPtr[s], R = B.ownRowPtr[s + 1] - r0;
        const float *Z = B.Z + B.zBase[s];
        const int re = B.unitOwnEnd[unit];
#pragma unroll 4
        for (int r = B.unitOwnBegin[unit] + threadIdx.x; r < re; r += blockDim.x) {
            float rn = r_cur[r];
            if (mode == 0) {
                rn = fmaf(-alpha, q[r], rn);
                r_next[r] = rn;
                u[r] = fmaf(alpha, p[r], u[r]);
            }
            acc[2 * M] = fmaf(rn, rn, acc[2 * M]);
            const int rl = r - r0;
#pragma unroll
            for (int c = 0; c < M; ++c)
                acc[c] = fmaf(ld_keep(Z + (size_t)c * R + rl, keep), rn, acc[c]);
        }
    }
    if (mode != 2) {
        const int r0 = B.extRowPtr[s], R = B.extRowPtr[s + 1] - r0;
        const float *W = B.W + B.wBase[s];
        const int re = B.unitExtEnd[unit];
#pragma unroll 4
        for (int r = B.unitExtBegin[unit] + threadIdx.x; r < re; r += blockDim.x) {
            const int d = ld_keep(B.extRowDof + r, keep);
            const float rn = YV ? yv[d] : ((mode == 0) ? fmaf(-alpha, q[d], r_cur[d]) : r_cur[d]);
            const int rl = r - r0;
#pragma unroll
            for (int c = 0; c < M; ++c)
                acc[M + c] = fmaf(ld_keep(W + (size_t)c * R + rl, keep), rn, acc[M + c]);
        }
    }
    block_sum<float, 2 * M + 1>(acc);
    const int u0 = B.boxUnit[s], nu = B.boxUnit[s + 1] - u0;
    const int c0 = B.col0[s];
    __shared__ float red[2 * 12];
    if (nu == 1) {
        // the whole box in this block: no cross-block combination
        if (threadIdx.x == 0) {
#pragma unroll
            for (int c = 0; c < 2 * M; ++c) red[c] = acc[c];
        }
        __syncthreads();
        if (threadIdx.x < M) {
            const int c = threadIdx.x;
            const double zs = red[c], ws = red[M + c];
            g[c0 + c] = zs - ws;
            B.g32[c0 + c] = (float)(zs - ws);
            if (zr) zr[c0 + c] = zs;
        }
        return acc[2 * M];
    }
    __shared__ bool lastUnit;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < 2 * M; ++c) B.unitPart[(size_t)unit * 24 + c] = (double)acc[c];
        __threadfence();
        lastUnit = atomicAdd(&B.boxTicket[s], 1u) == (unsigned int)nu - 1;
    }
    __syncthreads();
    if (lastUnit) {
        __threadfence();
        if (threadIdx.x < M) {
            const int c = threadIdx.x;
            double zs = 0.0, ws = 0.0;
            for (int v = u0; v < u0 + nu; ++v) {
                zs += __ldcg(B.unitPart + (size_t)v * 24 + c);
                ws += __ldcg(B.unitPart + (size_t)v * 24 + M + c);
            }
            g[c0 + c] = zs - ws;
            B.g32[c0 + c] = (float)(zs - ws);
            if (zr) zr[c0 + c] = zs;
        }
        if (threadIdx.x == 0) B.boxTicket[s] = 0u;
    }
    return acc[2 * M];
}

// Deferred form (deferred != 0, mode 0 of an iteration of the FP32 iteration): the
// product left its blocks' sums of p^T q in pqPart instead of reducing them
// itself; every block adds them (block_read_total), takes alpha = rho / pq,
// and block 0 records pq, alpha and counts the iteration (its += 1: the
// launch's arguments do not depend on the iteration, so a captured batch of
// iterations can be replayed), or the breakdown (or a failed wait of the
// product).
template <bool YV>
__global__ void __launch_bounds__(kRowThreads)
k_restrict_update(RowBoxDev B, float *u, const float *r_cur, float *r_next, const float *p,
                  const float *q, const float *yv, int mode, double *g, double *zr,
                  double *partials, Scalars *sc, int deferred, const float2 *pqPart, int pqN) {
    pdl_wait();
    if (sc->done != kRunning) return;
    const int unit = blockIdx.x;
    float alpha = (mode == 0) ? (float)sc->alpha : 0.0f;
    if (deferred) {
        const bool fault = sc->fault != 0;
        const double pq = block_read_total(pqPart, pqN);
        const double rho = sc->rho;
        const bool broken = !(pq > 0.0) || !isfinite(pq);
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (fault) {
                sc->done = kFault;
            } else {
                sc->pq = pq;
                sc->its += 1;
                if (broken)
                    sc->done = kBreakdown;
                else
                    sc->alpha = rho / pq;
            }
        }
        if (fault || broken) return;
        alpha = (float)(rho / pq);
    }
    float rr;
    if (B.menr[B.unitBox[unit]])
        rr = restrict_update_unit<12, YV>(B, unit, u, r_cur, r_next, p, q, yv, mode, alpha, g, zr);
    else
        rr = restrict_update_unit<6, YV>(B, unit, u, r_cur, r_next, p, q, yv, mode, alpha, g, zr);
    if (mode >= 2) return;
    double tot;
    if (grid_sum_t0((double)rr, partials, &sc->ticket[2], tot) && threadIdx.x == 0) {
        sc->rr = tot;
        sc->ry = tot;
        if (tot <= sc->tol2ff)
            sc->done = kConverged;
        else if (sc->its >= sc->max_it)
            sc->done = kMaxIter;
        else if (!isfinite(tot))
            sc->done = kBreakdown;
    }
}

void launch_restrict_update(const RowBoxDev &B, float *u, const float *r_cur, float *r_next,
                            const float *p, const float *q, int mode, double *g, double *zr,
                            double *partials, Scalars *sc, cudaStream_t st, const float *y) {
    launch_pdl(mode == 3 ? k_restrict_update<true> : k_restrict_update<false>, B.nUnits,
               kRowThreads, 0, st, B, u, r_cur, r_next, p, q, y, mode, g, zr, partials, sc, 0,
               (const float2 *)nullptr, 0);
}

void launch_restrict_update_deferred(const RowBoxDev &B, float *u, const float *r_cur,
                                     float *r_next, const float *p, const float *q, double *g,
                                     double *zr, double *partials, Scalars *sc,
                                     const float2 *pqPart, int pqN, cudaStream_t st) {
    launch_pdl(k_restrict_update<false>, B.nUnits, kRowThreads, 0, st, B, u, r_cur, r_next, p, q,
               (const float *)nullptr, 0, g, zr, partials, sc, 1, pqPart, pqN);
}

template <int M>
__device__ __forceinline__ void prolong_rows_unit(const RowBoxDev &B, int unit,
                                                  const float *nu32, const float *y, float *p,
                                                  int mode, float beta) {
    const int s = B.pUnitBox[unit];
    const int c0 = B.col0[s];
    float n[M];
#pragma unroll
    for (int c = 0; c < M; ++c) n[c] = nu32[c0 + c];
    const int r0 = B.ownRowPtr[s], R = B.ownRowPtr[s + 1] - r0;
    const float *Z = B.Z + B.zBase[s];
    const int re = B.pUnitEnd[unit];
    const uint64_t keep = l2_keep_policy();
#pragma unroll 2
    for (int r = B.pUnitBegin[unit] + threadIdx.x; r < re; r += blockDim.x) {
        const int rl = r - r0;
        float zv = 0.0f;
#pragma unroll
        for (int c = 0; c < M; ++c) zv = fmaf(ld_keep(Z + (size_t)c * R + rl, keep), n[c], zv);
        emit(p, y, r, zv, mode, beta);
    }
}

__global__ void __launch_bounds__(kRowThreads)
k_prolong_rows(RowBoxDev B, const float *nu32, const float *y, float *p, int mode, Scalars *sc) {
    pdl_wait();
    if (sc->done != kRunning) return;
    const int unit = blockIdx.x;
    const float beta = (float)sc->beta;
    if (B.menr[B.pUnitBox[unit]])
        prolong_rows_unit<12>(B, unit, nu32, y, p, mode, beta);
    else
        prolong_rows_unit<6>(B, unit, nu32, y, p, mode, beta);
}

void launch_prolong_rows(const RowBoxDev &B, const float *nu32, const float *y, float *p,
                         int mode, Scalars *sc, cudaStream_t st) {
    launch_pdl(k_prolong_rows, B.nPUnits, kRowThreads, 0, st, B, nu32, y, p, mode, sc);
}

// set-up: row-major per-item blocks (b x M at srcOff) to the per-box
// column-major layout
__global__ void k_to_colmajor(int nItems, const int *itemBox, const int *rowStart,
                              const unsigned char *itemB, const long long *srcOff,
                              const int *boxRowPtr, const long long *boxBase, const int *menr,
                              const float *src, float *dst) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nItems) return;
    const int s = itemBox[t], M = menr[s] ? 12 : 6, b = itemB[t];
    const int R = boxRowPtr[s + 1] - boxRowPtr[s];
    const int rl0 = rowStart[t] - boxRowPtr[s];
    for (int i = 0; i < b; ++i)
        for (int c = 0; c < M; ++c)
            dst[boxBase[s] + (long long)c * R + rl0 + i] = src[srcOff[t] + i * M + c];
}

void launch_to_colmajor(int nItems, const int *itemBox, const int *rowStart,
                        const unsigned char *itemB, const long long *srcOff,
                        const int *boxRowPtr, const long long *boxBase, const int *menr,
                        const float *src, float *dst, cudaStream_t st) {
    if (nItems == 0) return;
    k_to_colmajor<<<(nItems + 127) / 128, 128, 0, st>>>(nItems, itemBox, rowStart, itemB, srcOff,
                                                        boxRowPtr, boxBase, menr, src, dst);
}

}  // namespace xdcg
