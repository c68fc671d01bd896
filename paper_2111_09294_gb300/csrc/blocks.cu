// Block Jacobi with caller-given blocks (Section 3.4, Eqs. block_jacobi and
// block_jacobi_enr; the paper's blocks are whole subdomains, enriched dofs
// included): set-up gathers each block's diagonal part of K as a dense FP64
// matrix and inverts it (dense_inv.cu); every iteration applies y = M^-1 r as
// one dense product per block.  The FP32 path applies the inverse of the
// block-scaled system's blocks, L_b^T (K_bb)^-1 L_b (L the node-block Cholesky
// factors that scale K~ = L^-1 K L^-T), rounded to FP32.
#include "factor.cuh"
#include "reduce.cuh"

namespace xdcg {

// ---- set-up ------------------------------------------------------------------

// K's entries coupling two nodes of one block, copied into that block's dense
// matrix (row-major, positions = dofs of K's numbering minus the block's first
// dof).  One thread per stored node block (I, J).
__global__ void k_gather_blocks(KinDev K, long long nnzb, const int *blockRow,
                                const int *blockOfNode, const int *bStart, const int *bDim,
                                const long long *aOff, double *A) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= nnzb) return;
    const int I = blockRow[p], J = K.col[p];
    const int b = blockOfNode[I];
    if (blockOfNode[J] != b) return;
    const int nb = bDim[b], d0 = bStart[b];
    const int rI = K.dofStart[I] - d0, cJ = K.dofStart[J] - d0;
    const int bI = K.dofStart[I + 1] - K.dofStart[I], bJ = K.dofStart[J + 1] - K.dofStart[J];
    const double *src = K.val + K.valPtr[p];
    double *dst = A + aOff[b];
    for (int i = 0; i < bI; ++i)
        for (int j = 0; j < bJ; ++j) dst[(long long)(rI + i) * nb + cJ + j] = src[i * bJ + j];
}

void launch_gather_blocks(const KinDev &K, long long nnzb, const int *blockRow,
                          const int *blockOfNode, const int *bStart, const int *bDim,
                          const long long *aOff, double *A, cudaStream_t st) {
    if (nnzb == 0) return;
    k_gather_blocks<<<(int)((nnzb + 255) / 256), 256, 0, st>>>(K, nnzb, blockRow, blockOfNode,
                                                               bStart, bDim, aOff, A);
}

// Y = X L_b (X = (K_bb)^-1 in FP64): thread per block row; for every node J
// of the block, the row's b_J entries times J's lower Cholesky factor.
__global__ void k_scale_inverse_right(int n, const int *rowBlock, const int *bStart,
                                      const int *bDim, const int *bNode0, const int *bNode1,
                                      const long long *aOff, const int *dofStart,
                                      FacDev F, const double *X, double *Y) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n) return;
    const int b = rowBlock[d];
    const int nb = bDim[b], i = d - bStart[b];
    const double *xr = X + aOff[b] + (long long)i * nb;
    double *yr = Y + aOff[b] + (long long)i * nb;
    for (int J = bNode0[b]; J < bNode1[b]; ++J) {
        const int c0 = dofStart[J] - bStart[b], bJ = dofStart[J + 1] - dofStart[J];
        const int l = F.nodeList[J], t = F.nodeIdx[J];
        // (x L)_c = sum_{k >= c} x_k L_kc; the stored diagonal is 1 / L_cc
        for (int cc = 0; cc < bJ; ++cc) {
            double s = xr[c0 + cc] / Lent(F, l, t, cc, cc);
            for (int k = cc + 1; k < bJ; ++k) s = fma(xr[c0 + k], Lent(F, l, t, k, cc), s);
            yr[c0 + cc] = s;
        }
    }
}

// Z = L_b^T Y rounded to FP32: thread per (block, column) pair, i.e. per
// position d of K's numbering acting as a column of its block.
__global__ void k_scale_inverse_left(int n, const int *rowBlock, const int *bStart,
                                     const int *bDim, const int *bNode0, const int *bNode1,
                                     const long long *aOff, const int *dofStart, FacDev F,
                                     const double *Y, float *Z) {
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= n) return;
    const int b = rowBlock[d];
    const int nb = bDim[b], j = d - bStart[b];
    const double *yc = Y + aOff[b] + j;
    float *zc = Z + aOff[b] + j;
    for (int I = bNode0[b]; I < bNode1[b]; ++I) {
        const int r0 = dofStart[I] - bStart[b], bI = dofStart[I + 1] - dofStart[I];
        const int l = F.nodeList[I], t = F.nodeIdx[I];
        // (L^T y)_r = sum_{k >= r} L_kr y_k
        for (int rr = 0; rr < bI; ++rr) {
            double s = yc[(long long)(r0 + rr) * nb] / Lent(F, l, t, rr, rr);
            for (int k = rr + 1; k < bI; ++k)
                s = fma(Lent(F, l, t, k, rr), yc[(long long)(r0 + k) * nb], s);
            zc[(long long)(r0 + rr) * nb] = (float)s;
        }
    }
}

void launch_scale_block_inverse(int n, const int *rowBlock, const int *bStart, const int *bDim,
                                const int *bNode0, const int *bNode1, const long long *aOff,
                                const int *dofStart, const FacDev &F, const double *X, double *Y,
                                float *Z, cudaStream_t st) {
    if (n == 0) return;
    const int g = (n + 127) / 128;
    k_scale_inverse_right<<<g, 128, 0, st>>>(n, rowBlock, bStart, bDim, bNode0, bNode1, aOff,
                                             dofStart, F, X, Y);
    k_scale_inverse_left<<<g, 128, 0, st>>>(n, rowBlock, bStart, bDim, bNode0, bNode1, aOff,
                                            dofStart, F, Y, Z);
}

// ---- per iteration ---------------------------------------------------------------

// y = M^-1 r block by block: unit u covers rows [unitRow0[u], unitRow1[u]) of
// block unitBlk[u]; the CTA stages the block's whole r in shared memory (a
// gather through idx), and each warp forms whole rows of the dense product
// (lanes along the row, coalesced), summing in a fixed order.  The grid also
// reduces r^T y into sc->ry (deterministic, last block).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_block_apply(BlkDev<T> B, const T *__restrict__ r, T *__restrict__ y, double *partials,
              Scalars *sc) {
    __shared__ T rs[XDCG_MAX_BLOCK_DOFS];
    pdl_wait();
    if (sc->done != kRunning) return;
    const int u = blockIdx.x;
    const int b = B.unitBlk[u];
    const int p0 = B.bPos[b], nb = B.bPos[b + 1] - p0;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) rs[j] = r[B.idx[p0 + j]];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T *Ab = B.A + B.aOff[b];
    T part[1] = {T(0)};
    for (int i = B.unitRow0[u] + warp; i < B.unitRow1[u]; i += kWarps) {
        const T *row = Ab + (long long)i * nb;
        T s0 = T(0), s1 = T(0), s2 = T(0), s3 = T(0);
        int j = lane;
        for (; j + 96 < nb; j += 128) {
            s0 = fma(__ldcs(row + j), rs[j], s0);
            s1 = fma(__ldcs(row + j + 32), rs[j + 32], s1);
            s2 = fma(__ldcs(row + j + 64), rs[j + 64], s2);
            s3 = fma(__ldcs(row + j + 96), rs[j + 96], s3);
        }
        for (; j < nb; j += 32) s0 = fma(__ldcs(row + j), rs[j], s0);
        T s = (s0 + s1) + (s2 + s3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) {
            y[B.idx[p0 + i]] = s;
            part[0] = fma(rs[i], s, part[0]);
        }
    }
    double tot[1];
    if (grid_sum<T, 1>(part, partials, &sc->ticket[1], tot) && threadIdx.x == 0) sc->ry = tot[0];
}

template <typename T>
void launch_block_apply(const BlkDev<T> &B, const T *r, T *y, double *partials, Scalars *sc,
                        cudaStream_t st) {
    launch_pdl(k_block_apply<T>, B.nUnits, kThreads, 0, st, B, r, y, partials, sc);
}
template void launch_block_apply<double>(const BlkDev<double> &, const double *, double *,
                                         double *, Scalars *, cudaStream_t);
template void launch_block_apply<float>(const BlkDev<float> &, const float *, float *, double *,
                                        Scalars *, cudaStream_t);

// u += alpha p, r -= alpha q (mode 0; mode 1: r as it is) and ||r||^2 with the
// stopping tests, when M^-1 is applied by a separate launch (caller blocks).
template <typename T>
__global__ void __launch_bounds__(kThreads)
k_update_plain(T *u, T *r, const T *p, const T *q, long long n, int mode, double *partials,
               Scalars *sc) {
    pdl_wait();
    if (sc->done != kRunning) return;
    const T alpha = (T)sc->alpha;
    T v[1] = {T(0)};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        T ri = r[i];
        if (mode == 0) {
            u[i] = fma(alpha, p[i], u[i]);
            ri = fma(-alpha, q[i], ri);
            r[i] = ri;
        }
        v[0] = fma(ri, ri, v[0]);
    }
    double tot[1];
    if (grid_sum<T, 1>(v, partials, &sc->ticket[2], tot) && threadIdx.x == 0) {
        sc->rr = tot[0];
        if (sc->hist && sc->its < sc->histCap) sc->hist[sc->its] = tot[0];
        if (tot[0] <= sc->tol2ff)
            sc->done = kConverged;
        else if (sc->its >= sc->max_it)
            sc->done = kMaxIter;
        else if (!isfinite(tot[0]))
            sc->done = kBreakdown;
    }
}

template <typename T>
void launch_update_plain(T *u, T *r, const T *p, const T *q, long long n, int mode,
                         double *partials, Scalars *sc, cudaStream_t st) {
    const long long g = (n + kThreads - 1) / kThreads, cap = 2LL * device_sm_count();
    launch_pdl(k_update_plain<T>, (int)(g < cap ? (g > 0 ? g : 1) : cap), kThreads, 0, st, u, r,
               p, q, n, mode, partials, sc);
}
template void launch_update_plain<double>(double *, double *, const double *, const double *,
                                          long long, int, double *, Scalars *, cudaStream_t);
template void launch_update_plain<float>(float *, float *, const float *, const float *,
                                         long long, int, double *, Scalars *, cudaStream_t);

}  // namespace xdcg
