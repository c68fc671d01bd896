// Batched FP32 iteration of the mixed path: MB right-hand sides of one
// system advance together (the multi-load-case solves of a propagation step:
// the same K, several load cases).  Every kernel reads the matrix data once
// per iteration for all columns, so the bytes per right-hand side fall by up
// to MB.  Vectors are interleaved by column: entry (dof d, column j) at
// d * MB + j, so a chunk gathered by the product is one run of 3 * MB floats
// and a row of the box kernels is one run of MB floats.  Columns that have
// converged (or are padding) are inactive: their alpha and beta are 0 and
// their vectors stay as they are.
#include "cache.cuh"
#include "factor.cuh"
#include "reduce.cuh"
#include "spmv_cfg.cuh"
#include "tma.cuh"

namespace xdcg {

// ---- per-column scalar updates ----------------------------------------------

// fin 0 (iteration): pq_j, its, alpha_j (0 for inactive columns); a column
// whose p^T K p is not positive is marked broken and a replacement requested.
// fin 1 (start): rr_j.
__device__ __forceinline__ void batch_finalize(BatchScalars *bs, int m, int fin,
                                               const double *tot) {
    if (fin == 0) {
        bs->its += 1;
        bool request = false;
        for (int j = 0; j < m; ++j) {
            bs->pq[j] = tot[j];
            if (!bs->active[j]) {
                bs->alpha[j] = 0.0;
            } else if (!(tot[j] > 0.0) || !isfinite(tot[j])) {
                bs->alpha[j] = 0.0;
                bs->broken[j] = 1;
                request = true;
            } else {
                bs->alpha[j] = bs->rho[j] / tot[j];
            }
        }
        if (request) bs->done = kConverged;
    } else {
        for (int j = 0; j < m; ++j) bs->rr[j] = tot[j];
    }
}

// ---- batched product Y = K~ X (+ x_j^T y_j, or ||y_j||^2 with y = b - K~ x) --

template <int MB, bool RES>
__global__ void __launch_bounds__(kSpmvThreads)
k_spmm(SpmvDev<float> A, int m, const float *__restrict__ x, float *__restrict__ y,
       const float *__restrict__ b, double *partials, BatchScalars *bs, int fin) {
    constexpr int C = SpmvCfg<float, 0>::C, NS = SpmvCfg<float, 0>::NS, SB = stage_bytes<float, 0>();
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *ring = smem + (size_t)warp * NS * SB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)kSpmvWarps * NS * SB) + warp * NS;
    int *meta = reinterpret_cast<int *>(smem + (size_t)kSpmvWarps * NS * (SB + 8)) + warp * NS * 3;
    const int nS = A.S.nSlices;
    const int gw = blockIdx.x * kSpmvWarps + warp;
    const int sEnd = A.warpSlice[gw + 1];
    if (lane == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bars + s, 1);
        mbar_init_fence();
    }
    __syncwarp();
    const uint64_t stream = l2_stream_policy();
    const unsigned long long deadline = global_ns() + A.waitNs;
    int issued = 0, more = 1, pSlice = A.warpSlice[gw] - 1, pStep = 0, pSteps = 0;
    long long pBase = 0;
    const int *pCol = nullptr;
    const float *pVal = nullptr;
    auto issue = [&]() {
        if (pStep >= pSteps) {
            if (++pSlice >= sEnd) {
                more = 0;
                return;
            }
            const bool isS = pSlice < nS;
            const SellDev<float> &P = isS ? A.S : A.X;
            const int sl = isS ? pSlice : pSlice - nS;
            pBase = P.slicePtr[sl];
            pSteps = (int)((P.slicePtr[sl + 1] - pBase) >> 5);
            pStep = 0;
            pCol = P.col;
            pVal = P.val;
        }
        const int st = issued % NS;
        const int n = min(C, pSteps - pStep);
        meta[st * 3] = pSlice;
        meta[st * 3 + 1] = pStep;
        meta[st * 3 + 2] = n;
        unsigned char *dst = ring + st * SB;
        const uint32_t cb = (uint32_t)n * 128u, vb = (uint32_t)n * 288u * 4u;
        const long long off = pBase + 32LL * pStep;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bars + st, cb + vb);
        bulk_g2s(dst, pCol + off, cb, bars + st, stream);
        bulk_g2s(dst + C * 128, pVal + 9 * off, vb, bars + st, stream);
        pStep += n;
        ++issued;
    };
    // prologue copies before the wait unless the run has visibly stopped
    // (an L2 read that may be stale; the read after the wait decides)
    const bool early = __ldcg(&bs->done) == kRunning;
    if (lane == 0 && early)
        while (more && issued < NS) issue();
    issued = __shfl_sync(0xffffffffu, issued, 0);
    pdl_wait();
    if (bs->done != kRunning) {
        const unsigned long long drain = global_ns() + kDrainNs;
        for (int k = 0; k < issued; ++k) mbar_wait(bars + k % NS, (uint32_t)(k / NS) & 1u, drain);
        __syncwarp();
        return;
    }
    if (!early) {
        if (lane == 0)
            while (more && issued < NS) issue();
        issued = __shfl_sync(0xffffffffu, issued, 0);
    }

    float part[MB];
#pragma unroll
    for (int j = 0; j < MB; ++j) part[j] = 0.0f;
    int cur = -1, rpw = 16, rl = 0, h = 0;
    bool valid = false, isS = true;
    float a[3][MB];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < MB; ++j) a[i][j] = 0.0f;
    auto finish = [&]() {
        for (int o = rpw; o < 32; o <<= 1) {
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < MB; ++j) a[i][j] += __shfl_xor_sync(0xffffffffu, a[i][j], o);
        }
        if (valid && h == 0) {
            const long long r3 = 3 * (long long)(isS ? A.S.row[rl] : A.X.row[rl]);
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                float4 *yr = reinterpret_cast<float4 *>(y + (r3 + i) * MB);
                const float4 *src = reinterpret_cast<const float4 *>(RES ? b : x) + (r3 + i) * (MB / 4);
#pragma unroll
                for (int q = 0; q < MB / 4; ++q) {
                    const float4 s4 = src[q];
                    float4 o4;
                    if (RES) {
                        o4 = make_float4(s4.x - a[i][4 * q], s4.y - a[i][4 * q + 1],
                                         s4.z - a[i][4 * q + 2], s4.w - a[i][4 * q + 3]);
                        part[4 * q] = fmaf(o4.x, o4.x, part[4 * q]);
                        part[4 * q + 1] = fmaf(o4.y, o4.y, part[4 * q + 1]);
                        part[4 * q + 2] = fmaf(o4.z, o4.z, part[4 * q + 2]);
                        part[4 * q + 3] = fmaf(o4.w, o4.w, part[4 * q + 3]);
                    } else {
                        o4 = make_float4(a[i][4 * q], a[i][4 * q + 1], a[i][4 * q + 2],
                                         a[i][4 * q + 3]);
                        part[4 * q] = fmaf(s4.x, o4.x, part[4 * q]);
                        part[4 * q + 1] = fmaf(s4.y, o4.y, part[4 * q + 1]);
                        part[4 * q + 2] = fmaf(s4.z, o4.z, part[4 * q + 2]);
                        part[4 * q + 3] = fmaf(s4.w, o4.w, part[4 * q + 3]);
                    }
                    yr[q] = o4;
                }
            }
        }
    };
    int k = 0;
    bool ok = true;
    for (; k < issued; ++k) {
        const int st = k % NS;
        ok = __all_sync(0xffffffffu, mbar_wait(bars + st, (uint32_t)(k / NS) & 1u, deadline));
        if (!ok) break;
        const int sl = meta[st * 3], n = meta[st * 3 + 2];
        if (sl != cur) {
            if (cur >= 0) finish();
            cur = sl;
            isS = sl < nS;
            rpw = isS ? 32 / kTprS : 32 / kTprX;
            rl = (isS ? sl : sl - nS) * rpw + (lane % rpw);
            h = lane / rpw;
            valid = rl < (isS ? A.S.nRows : A.X.nRows);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < MB; ++j) a[i][j] = 0.0f;
        }
        const int *cs = reinterpret_cast<const int *>(ring + st * SB);
        const float *vs = reinterpret_cast<const float *>(ring + st * SB + C * 128);
#pragma unroll
        for (int t = 0; t < C; ++t) {
            if (t < n) {
                const int c = cs[t * 32 + lane];
                const float4 *xc = reinterpret_cast<const float4 *>(x) + (size_t)c * (3 * MB / 4);
                float xv[3][MB];
#pragma unroll
                for (int jc = 0; jc < 3; ++jc)
#pragma unroll
                    for (int q = 0; q < MB / 4; ++q) {
                        const float4 v4 = __ldg(xc + jc * (MB / 4) + q);
                        xv[jc][4 * q] = v4.x;
                        xv[jc][4 * q + 1] = v4.y;
                        xv[jc][4 * q + 2] = v4.z;
                        xv[jc][4 * q + 3] = v4.w;
                    }
                const float *v = vs + t * 288 + lane;
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int jc = 0; jc < 3; ++jc) {
                        const float kv = v[(3 * i + jc) * 32];
#pragma unroll
                        for (int j = 0; j < MB; ++j) a[i][j] = fmaf(kv, xv[jc][j], a[i][j]);
                    }
            }
        }
        __syncwarp();
        if (lane == 0 && more) issue();
        issued = __shfl_sync(0xffffffffu, issued, 0);
    }
    if (ok) {
        if (cur >= 0) finish();
    } else {
        if (lane == 0) atomicExch(&bs->fault, 1);
        const unsigned long long drain = global_ns() + kDrainNs;
        for (; k < issued; ++k) mbar_wait(bars + k % NS, (uint32_t)(k / NS) & 1u, drain);
        __syncwarp();
    }
    double tot[MB];
    if (grid_sum<float, MB>(part, partials, &bs->ticket[0], tot) && threadIdx.x == 0) {
        if (bs->fault)
            bs->done = kFault;
        else
            batch_finalize(bs, m, fin, tot);
    }
}

template <int MB>
void launch_spmm(const SpmvDev<float> &A, int m, const float *x, float *y, const float *b,
                 int residual_mode, double *partials, BatchScalars *bs, int fin,
                 cudaStream_t st) {
    const int smem = spmv_smem_bytes<float, 0>();
    launch_pdl(residual_mode ? k_spmm<MB, true> : k_spmm<MB, false>, A.grid, kSpmvThreads, smem,
               st, A, m, x, y, b, partials, bs, fin);
}

bool spmm_prepare() {
    const int smem = spmv_smem_bytes<float, 0>();
    return cudaFuncSetAttribute(k_spmm<4, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem) == cudaSuccess &&
           cudaFuncSetAttribute(k_spmm<4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem) == cudaSuccess &&
           cudaFuncSetAttribute(k_spmm<8, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem) == cudaSuccess &&
           cudaFuncSetAttribute(k_spmm<8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                smem) == cudaSuccess;
}

// ---- batched restriction + update ---------------------------------------------

// Sums v over the block's threads that share t % MB; thread t = j * NV + c
// (t < MB * NV) receives the total of value c for column j, added warp by
// warp in warp order.
template <int MB, int NV>
__device__ __forceinline__ float block_sum_by_column(float (&v)[NV]) {
    __shared__ float wred[kThreads / 32][MB][NV];
#pragma unroll
    for (int o = MB; o < 32; o <<= 1)
#pragma unroll
        for (int c = 0; c < NV; ++c) v[c] += __shfl_xor_sync(0xffffffffu, v[c], o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l < MB)
#pragma unroll
        for (int c = 0; c < NV; ++c) wred[w][l][c] = v[c];
    __syncthreads();
    float s = 0.0f;
    if ((int)threadIdx.x < MB * NV) {
        const int j = threadIdx.x / NV, c = threadIdx.x % NV;
        for (int ww = 0; ww < (int)(blockDim.x >> 5); ++ww) s += wred[ww][j][c];
    }
    __syncthreads();
    return s;
}

// One unit (own rows, then coupled rows, of one box); thread t handles column
// j = t % MB of rows t / MB, t / MB + 256 / MB, ...  acc: Z~^T r (M), W~^T r (M),
// ||r||^2 of its column.
template <int MB, int M>
__device__ __forceinline__ void restrict_b_unit(const RowBoxDev &B, int unit, int m, float *u,
                                                const float *r_cur, float *r_next, const float *p,
                                                const float *q, int mode, const BatchScalars *bs,
                                                double *G, float *G32, double *ZR,
                                                double *unitPart, float (&rr)[MB]) {
    const int s = B.unitBox[unit];
    const int j = threadIdx.x % MB, row0 = threadIdx.x / MB;
    constexpr int kRowStep = kThreads / MB;
    const float alpha = (mode == 0 && j < m) ? (float)bs->alpha[j] : 0.0f;
    float acc[2 * M + 1];
#pragma unroll
    for (int c = 0; c <= 2 * M; ++c) acc[c] = 0.0f;
    const uint64_t keep = l2_keep_policy();
    {
        const int r0 = B.ownRowPtr[s], R = B.ownRowPtr[s + 1] - r0;
        const float *Z = B.Z + B.zBase[s];
        const int re = B.unitOwnEnd[unit];
#pragma unroll 2
        for (int r = B.unitOwnBegin[unit] + row0; r < re; r += kRowStep) {
            const size_t e = (size_t)r * MB + j;
            float rn = r_cur[e];
            if (mode == 0) {
                rn = fmaf(-alpha, q[e], rn);
                r_next[e] = rn;
                u[e] = fmaf(alpha, p[e], u[e]);
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
#pragma unroll 2
        for (int r = B.unitExtBegin[unit] + row0; r < re; r += kRowStep) {
            const size_t e = (size_t)ld_keep(B.extRowDof + r, keep) * MB + j;
            const float rn = (mode == 0) ? fmaf(-alpha, q[e], r_cur[e]) : r_cur[e];
            const int rl = r - r0;
#pragma unroll
            for (int c = 0; c < M; ++c)
                acc[M + c] = fmaf(ld_keep(W + (size_t)c * R + rl, keep), rn, acc[M + c]);
        }
    }
    const float tsum = block_sum_by_column<MB, 2 * M + 1>(acc);
    // thread t < MB * (2M + 1): column tj = t / (2M + 1), value tc = t % (2M + 1)
    const int tj = threadIdx.x / (2 * M + 1), tc = threadIdx.x % (2 * M + 1);
    const bool holder = (int)threadIdx.x < MB * (2 * M + 1);
    __shared__ float rrs[MB];
    if (holder && tc == 2 * M) rrs[tj] = tsum;
    const int u0 = B.boxUnit[s], nu = B.boxUnit[s + 1] - u0;
    const int c0 = B.col0[s];
    __shared__ float red[MB][2 * 12];
    __shared__ bool lastUnit;
    if (nu == 1) {
        if (holder && tc < 2 * M) red[tj][tc] = tsum;
        __syncthreads();
        if ((int)threadIdx.x < MB * M) {
            const int jj = threadIdx.x / M, c = threadIdx.x % M;
            const double zs = red[jj][c], ws = red[jj][M + c];
            G[(size_t)(c0 + c) * MB + jj] = zs - ws;
            G32[(size_t)(c0 + c) * MB + jj] = (float)(zs - ws);
            if (ZR) ZR[(size_t)(c0 + c) * MB + jj] = zs;
        }
    } else {
        if (holder && tc < 2 * M)
            unitPart[((size_t)unit * MB + tj) * 24 + tc] = (double)tsum;
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0)
            lastUnit = atomicAdd(&B.boxTicket[s], 1u) == (unsigned int)nu - 1;
        __syncthreads();
        if (lastUnit) {
            __threadfence();
            if ((int)threadIdx.x < MB * M) {
                const int jj = threadIdx.x / M, c = threadIdx.x % M;
                double zs = 0.0, ws = 0.0;
                for (int v = u0; v < u0 + nu; ++v) {
                    zs += __ldcg(unitPart + ((size_t)v * MB + jj) * 24 + c);
                    ws += __ldcg(unitPart + ((size_t)v * MB + jj) * 24 + M + c);
                }
                G[(size_t)(c0 + c) * MB + jj] = zs - ws;
                G32[(size_t)(c0 + c) * MB + jj] = (float)(zs - ws);
                if (ZR) ZR[(size_t)(c0 + c) * MB + jj] = zs;
            }
            if (threadIdx.x == 0) B.boxTicket[s] = 0u;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int jj = 0; jj < MB; ++jj) rr[jj] = rrs[jj];
}

// mode 0: r' = r - alpha_j q, u += alpha_j p, G from r'; mode 1: G from r;
// mode 2: G = Z~^T f only, no ||r||^2.  The last block sets rr_j and asks for
// a replacement once an active column reaches its trigger.
template <int MB>
__global__ void __launch_bounds__(kThreads)
k_restrict_b(RowBoxDev B, int m, float *u, const float *r_cur, float *r_next, const float *p,
             const float *q, int mode, double *G, float *G32, double *ZR, double *unitPart,
             double *partials, BatchScalars *bs) {
    pdl_wait();
    if (bs->done != kRunning) return;
    const int unit = blockIdx.x;
    float rr[MB];
#pragma unroll
    for (int j = 0; j < MB; ++j) rr[j] = 0.0f;
    if (B.menr[B.unitBox[unit]])
        restrict_b_unit<MB, 12>(B, unit, m, u, r_cur, r_next, p, q, mode, bs, G, G32, ZR,
                                unitPart, rr);
    else
        restrict_b_unit<MB, 6>(B, unit, m, u, r_cur, r_next, p, q, mode, bs, G, G32, ZR,
                               unitPart, rr);
    if (mode == 2) return;
    // rr holds the block's totals in thread 0 (zeros elsewhere)
    if (threadIdx.x != 0)
#pragma unroll
        for (int j = 0; j < MB; ++j) rr[j] = 0.0f;
    double tot[MB];
    if (grid_sum<float, MB>(rr, partials, &bs->ticket[2], tot) && threadIdx.x == 0) {
        bool request = false;
        for (int j = 0; j < m; ++j) {
            bs->rr[j] = tot[j];
            if (bs->active[j] && (tot[j] <= bs->trig[j] || !isfinite(tot[j]))) request = true;
        }
        if (request)
            bs->done = kConverged;
        else if (bs->its >= bs->max_it)
            bs->done = kMaxIter;
    }
}

template <int MB>
void launch_restrict_b(const RowBoxDev &B, int m, float *u, const float *r_cur, float *r_next,
                       const float *p, const float *q, int mode, double *G, float *G32,
                       double *ZR, double *unitPart, double *partials, BatchScalars *bs,
                       cudaStream_t st) {
    launch_pdl(k_restrict_b<MB>, B.nUnits, kThreads, 0, st, B, m, u, r_cur, r_next, p, q, mode, G,
               G32, ZR, unitPart, partials, bs);
}

// ---- batched coarse solve NU = E^-1 G -----------------------------------------

constexpr int kCoarseChunkB = 1024;
constexpr int kCoarsePadB = kCoarseChunkB + 4;   // row pitch of the transposed G chunk

// mode 0: nothing else; mode 1: rho_j = rr_j + nu_j^T zr_j, beta_j = 0; mode 2:
// the same rho_new, beta_j = rho_new / rho_j; mode 3 (after a replacement): as
// 2, with beta_j = 0 for a replaced column whose residual the replacement
// lengthened by more than 2x or that broke down (the other columns finish the
// iteration the trigger interrupted, as in mode 2).  Inactive columns get
// beta = 0.  One warp per row of E^-1 (16-byte loads when k is a multiple of
// 4); G staged in shared memory chunk by chunk, transposed (one padded row
// per column), so a lane's four consecutive entries of a column are one
// conflict-free 16-byte load.
template <int MB, int V>
__global__ void __launch_bounds__(kThreads)
k_coarse_b(const float *__restrict__ Einv, int k, int m, const float *__restrict__ G32,
           const double *__restrict__ ZR, double *NU, float *NU32, int mode, double *partials,
           BatchScalars *bs) {
    pdl_wait();
    if (bs->done != kRunning) return;
    __shared__ __align__(16) float gs[MB * kCoarsePadB];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kWarps + warp;
    const float *row = Einv + (size_t)(i < k ? i : 0) * k;
    const uint64_t keep = l2_keep_policy();
    float acc[MB];
#pragma unroll
    for (int j = 0; j < MB; ++j) acc[j] = 0.0f;
    for (int l0 = 0; l0 < k; l0 += kCoarseChunkB) {
        const int len = min(kCoarseChunkB, k - l0);
        __syncthreads();
        for (int e = threadIdx.x; e < len * MB; e += blockDim.x)
            gs[(e % MB) * kCoarsePadB + e / MB] = G32[(size_t)l0 * MB + e];
        __syncthreads();
        if (i >= k) continue;
        if (V == 4) {
            const float4 *r4 = reinterpret_cast<const float4 *>(row + l0);
#pragma unroll 4
            for (int l4 = lane; 4 * l4 < len; l4 += 32) {
                const float4 ev = ld_keep(r4 + l4, keep);
#pragma unroll
                for (int j = 0; j < MB; ++j) {
                    const float4 g = *reinterpret_cast<const float4 *>(gs + j * kCoarsePadB + 4 * l4);
                    float a = fmaf(ev.x, g.x, acc[j]);
                    a = fmaf(ev.y, g.y, a);
                    a = fmaf(ev.z, g.z, a);
                    acc[j] = fmaf(ev.w, g.w, a);
                }
            }
        } else {
#pragma unroll 4
            for (int l = lane; l < len; l += 32) {
                const float ev = ld_keep(row + l0 + l, keep);
#pragma unroll
                for (int j = 0; j < MB; ++j) acc[j] = fmaf(ev, gs[j * kCoarsePadB + l], acc[j]);
            }
        }
    }
    warp_sum<float, MB>(acc);
    double part[MB];
#pragma unroll
    for (int j = 0; j < MB; ++j) part[j] = 0.0;
    if (i < k && lane == 0) {
#pragma unroll
        for (int j = 0; j < MB; ++j) {
            NU[(size_t)i * MB + j] = (double)acc[j];
            NU32[(size_t)i * MB + j] = acc[j];
            if (mode != 0) part[j] = (double)acc[j] * ZR[(size_t)i * MB + j];
        }
    }
    double tot[MB];
    if (grid_sum<double, MB>(part, partials, &bs->ticket[3], tot) && threadIdx.x == 0 &&
        mode != 0) {
        for (int j = 0; j < m; ++j) {
            // a column not being replaced finishes its interrupted iteration as in mode 2
            const bool rep = mode == 1 || (mode == 3 && bs->repl[j]);
            const double rho_new = bs->rr[j] + tot[j];
            if (!bs->active[j]) {
                bs->beta[j] = 0.0;
            } else if (mode == 1 || (rep && (bs->broken[j] || bs->rr[j] > 4.0 * bs->rrRep[j]))) {
                bs->beta[j] = 0.0;
            } else {
                bs->beta[j] = rho_new / bs->rho[j];
            }
            bs->rho[j] = rho_new;
            if (rep) bs->broken[j] = 0;
        }
    }
}

template <int MB>
void launch_coarse_b(const float *Einv, int k, int m, const float *G32, const double *ZR,
                     double *NU, float *NU32, int mode, double *partials, BatchScalars *bs,
                     cudaStream_t st) {
    const int grid = (k + kWarps - 1) / kWarps;
    launch_pdl(k % 4 == 0 ? k_coarse_b<MB, 4> : k_coarse_b<MB, 1>, grid > 0 ? grid : 1, kThreads,
               0, st, Einv, k, m, G32, ZR, NU, NU32, mode, partials, bs);
}

// ---- batched prolongation -----------------------------------------------------

// mode 0: p = y + Z~ nu + beta_j p; mode 1: p = Z~ nu; mode 2: p = y + Z~ nu
template <int MB, int M>
__device__ __forceinline__ void prolong_b_unit(const RowBoxDev &B, int unit, const float *NU32,
                                               const float *y, float *p, int mode, float beta) {
    const int s = B.pUnitBox[unit];
    const int j = threadIdx.x % MB, row0 = threadIdx.x / MB;
    constexpr int kRowStep = kThreads / MB;
    const int c0 = B.col0[s];
    float nv[M];
#pragma unroll
    for (int c = 0; c < M; ++c) nv[c] = NU32[(size_t)(c0 + c) * MB + j];
    const int r0 = B.ownRowPtr[s], R = B.ownRowPtr[s + 1] - r0;
    const float *Z = B.Z + B.zBase[s];
    const int re = B.pUnitEnd[unit];
    const uint64_t keep = l2_keep_policy();
#pragma unroll 2
    for (int r = B.pUnitBegin[unit] + row0; r < re; r += kRowStep) {
        const int rl = r - r0;
        float zv = 0.0f;
#pragma unroll
        for (int c = 0; c < M; ++c) zv = fmaf(ld_keep(Z + (size_t)c * R + rl, keep), nv[c], zv);
        const size_t e = (size_t)r * MB + j;
        if (mode == 0)
            p[e] = y[e] + zv + beta * p[e];
        else if (mode == 1)
            p[e] = zv;
        else
            p[e] = y[e] + zv;
    }
}

template <int MB>
__global__ void __launch_bounds__(kThreads)
k_prolong_b(RowBoxDev B, int m, const float *NU32, const float *y, float *p, int mode,
            const BatchScalars *bs) {
    pdl_wait();
    if (bs->done != kRunning) return;
    const int unit = blockIdx.x;
    const int j = threadIdx.x % MB;
    const float beta = (mode == 0 && j < m) ? (float)bs->beta[j] : 0.0f;
    if (B.menr[B.pUnitBox[unit]])
        prolong_b_unit<MB, 12>(B, unit, NU32, y, p, mode, beta);
    else
        prolong_b_unit<MB, 6>(B, unit, NU32, y, p, mode, beta);
}

template <int MB>
void launch_prolong_b(const RowBoxDev &B, int m, const float *NU32, const float *y, float *p,
                      int mode, const BatchScalars *bs, cudaStream_t st) {
    launch_pdl(k_prolong_b<MB>, B.nPUnits, kThreads, 0, st, B, m, NU32, y, p, mode, bs);
}

// ---- FP64 <-> FP32 transforms of several columns --------------------------------

// out[(ot[I] + i) * MB + j] = scale_j (L^-1 r_j)_i for the active columns being
// replaced (repl_j); r_j = r + j * ldr in the caller's numbering (nat).
// Inactive columns get 0; active columns not being replaced are left as they
// are.  One thread per (node, column).
template <int MB>
__global__ void k_fwd_scale_b(int nNodes, int m, const int *nat, const int *ot, FacDev F,
                              const double *r, long long ldr, const BatchScalars *bs,
                              float *out) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nNodes * MB) return;
    const int I = (int)(t / MB), j = (int)(t % MB);
    const int b = nat[I + 1] - nat[I], d0 = nat[I], o0 = ot[I];
    const bool on = j < m && bs->active[j];
    if (on && !bs->repl[j]) return;
    const double sj = on ? bs->scale[j] : 0.0;
    const int q = F.nodeIdx[I];
    with_node_size(b, [&](auto Bc) {
        constexpr int B = decltype(Bc)::value;
        double x[B];
#pragma unroll
        for (int i = 0; i < B; ++i) x[i] = on ? r[j * ldr + d0 + i] : 0.0;
        if (on) fwd_solve_fixed<B>(F, q, x);
#pragma unroll
        for (int i = 0; i < B; ++i) out[(size_t)(o0 + i) * MB + j] = (float)(sj * x[i]);
    });
}

// u_j += (L^-T ut_j)_i / scale_j for active columns j < m; one thread per
// (node, column)
template <int MB>
__global__ void k_bwd_accum_b(int nNodes, int m, const int *nat, const int *in, FacDev F,
                              const float *ut, const BatchScalars *bs, double *u, long long ldu) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nNodes * MB) return;
    const int I = (int)(t / MB), j = (int)(t % MB);
    if (j >= m || !bs->active[j]) return;
    const int b = nat[I + 1] - nat[I], d0 = in[I], o0 = nat[I];
    const double inv = 1.0 / bs->scale[j];
    const int q = F.nodeIdx[I];
    with_node_size(b, [&](auto Bc) {
        constexpr int B = decltype(Bc)::value;
        double x[B];
#pragma unroll
        for (int i = 0; i < B; ++i) x[i] = (double)ut[(size_t)(d0 + i) * MB + j];
        bwd_solve_fixed<B>(F, q, x);
#pragma unroll
        for (int i = 0; i < B; ++i) u[j * ldu + o0 + i] += inv * x[i];
    });
}

template <int MB>
void launch_fwd_scale_b(int nNodes, int m, const int *nat, const int *ot, const FacDev &F,
                        const double *r, long long ldr, const BatchScalars *bs, float *out,
                        cudaStream_t st) {
    const long long nt = (long long)nNodes * MB;
    k_fwd_scale_b<MB><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(nNodes, m, nat, ot, F, r, ldr,
                                                                     bs, out);
}

template <int MB>
void launch_bwd_accum_b(int nNodes, int m, const int *nat, const int *in, const FacDev &F,
                        const float *ut, const BatchScalars *bs, double *u, long long ldu,
                        cudaStream_t st) {
    const long long nt = (long long)nNodes * MB;
    k_bwd_accum_b<MB><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(nNodes, m, nat, in, F, ut, bs,
                                                                     u, ldu);
}

#define XDCG_BATCH_INST(MB)                                                                    \
    template void launch_spmm<MB>(const SpmvDev<float> &, int, const float *, float *,          \
                                  const float *, int, double *, BatchScalars *, int,           \
                                  cudaStream_t);                                               \
    template void launch_restrict_b<MB>(const RowBoxDev &, int, float *, const float *,        \
                                        float *, const float *, const float *, int, double *,  \
                                        float *, double *, double *, double *, BatchScalars *, \
                                        cudaStream_t);                                         \
    template void launch_coarse_b<MB>(const float *, int, int, const float *, const double *,  \
                                      double *, float *, int, double *, BatchScalars *,        \
                                      cudaStream_t);                                           \
    template void launch_prolong_b<MB>(const RowBoxDev &, int, const float *, const float *,   \
                                       float *, int, const BatchScalars *, cudaStream_t);      \
    template void launch_fwd_scale_b<MB>(int, int, const int *, const int *, const FacDev &,   \
                                         const double *, long long, const BatchScalars *,      \
                                         float *, cudaStream_t);                               \
    template void launch_bwd_accum_b<MB>(int, int, const int *, const int *, const FacDev &,   \
                                         const float *, const BatchScalars *, double *,        \
                                         long long, cudaStream_t);
XDCG_BATCH_INST(4)
XDCG_BATCH_INST(8)
#undef XDCG_BATCH_INST

}  // namespace xdcg
