// Batched FP32 iteration of the mixed path: MB right-hand sides of one
// system advance together (the multi-load-case solves of a propagation step:
// the same K, several load cases).  Every kernel reads the matrix data once
// per iteration for all columns, so the bytes per right-hand side fall by up
// to MB.  Vectors are interleaved by column: entry (dof d, column j) at
// d * MB + j, so a chunk gathered by the product is one run of 3 * MB floats
// and a row of the box kernels is one run of MB floats.
//
// Columns advance independently (BatchScalars): an iteration updates the
// running columns (active and not held); a held column's residual is copied
// into the next buffer and its other vectors stay as they are, and a column
// that has left keeps zero vectors.  A replacement (open, FP64 residuals,
// judge, transforms, restriction / coarse / prolongation in their
// replacement modes, arm) touches only the columns it replaces.
//
// Every kernel body takes its block index and block count within its own
// system, so the same body runs as a launch for one system or as one launch
// over several systems (BatchSysTab): a column's result is the same bits
// either way.
#include <algorithm>
#include <climits>

#include "cache.cuh"
#include "factor.cuh"
#include "reduce.cuh"
#include "spmv_cfg.cuh"
#include "tma.cuh"

namespace xdcg {

__device__ __forceinline__ bool col_runs(const BatchScalars *bs, int j, int m) {
    return j < m && bs->active[j] && !bs->pend[j];
}

// whether a kernel of the system runs: an iteration's kernels also need the
// gate's go (a launch over several systems skips a system held for its
// replacement); the start and replacement kernels only need the run state
__device__ __forceinline__ bool batch_runs(const BatchScalars *bs, bool iteration) {
    return bs->done == kRunning && (!iteration || bs->go);
}

// the block's system in a launch over several systems: the largest s with
// off[s] <= b
__device__ __forceinline__ int sys_of(const int *__restrict__ off, int nSys, int b) {
    int lo = 0, hi = nSys - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---- per-column scalar updates ----------------------------------------------

// fin 0 (iteration): pq_j, alpha_j for the running columns (0 for the
// others); a running column whose p^T K p is not positive is held as broken.
// The iteration counts (its, its_j) advance when a column still runs;
// otherwise the system stops until the host's next replacement.
// fin 1 (start): rr_j.
__device__ __forceinline__ void batch_finalize(BatchScalars *bs, int m, int fin,
                                               const double *tot) {
    if (fin == 0) {
        bool any = false;
        for (int j = 0; j < m; ++j) {
            bs->pq[j] = tot[j];
            if (!col_runs(bs, j, m)) {
                bs->alpha[j] = 0.0;
                continue;
            }
            bs->itsc[j] += 1;
            if (!(tot[j] > 0.0) || !isfinite(tot[j])) {
                bs->alpha[j] = 0.0;
                bs->broken[j] = 1;
                bs->pend[j] = 1;
            } else {
                bs->alpha[j] = bs->rho[j] / tot[j];
                any = true;
            }
        }
        if (any)
            bs->its += 1;
        else
            bs->done = kConverged;
    } else {
        for (int j = 0; j < m; ++j) bs->rr[j] = tot[j];
    }
}

// ---- batched product Y = K~ X (+ x_j^T y_j, or ||y_j||^2 with y = b - K~ x) --

template <int MB, bool RES>
__device__ __forceinline__ void spmm_body(const SpmmArgs &args, int blk, int nblk,
                                          unsigned char *smem) {
    constexpr int C = SpmvCfg<float, 0>::C, NS = SpmvCfg<float, 0>::NS, SB = stage_bytes<float, 0>();
    const SpmvDev<float> &A = args.A;
    const int m = args.m, fin = args.fin;
    const float *__restrict__ x = args.x;
    const float *__restrict__ b = args.b;
    float *__restrict__ y = args.y;
    BatchScalars *bs = args.bs;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *ring = smem + (size_t)warp * NS * SB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)kSpmvWarps * NS * SB) + warp * NS;
    int *meta = reinterpret_cast<int *>(smem + (size_t)kSpmvWarps * NS * (SB + 8)) + warp * NS * 3;
    const int nS = A.S.nSlices;
    const int gw = blk * kSpmvWarps + warp;
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
    const bool early = __ldcg(&bs->done) == kRunning && (fin != 0 || __ldcg(&bs->go));
    if (lane == 0 && early)
        while (more && issued < NS) issue();
    issued = __shfl_sync(0xffffffffu, issued, 0);
    pdl_wait();
    if (!batch_runs(bs, fin == 0)) {
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
    if (grid_sum_of<float, MB>(part, args.partials, &bs->ticket[0], tot, blk, nblk) &&
        threadIdx.x == 0) {
        if (bs->fault)
            bs->done = kFault;
        else
            batch_finalize(bs, m, fin, tot);
    }
}

template <int MB, bool RES>
__global__ void __launch_bounds__(kSpmvThreads, 3) k_spmm(SpmmArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    spmm_body<MB, RES>(a, (int)blockIdx.x, (int)gridDim.x, smem);
}

template <int MB>
__global__ void __launch_bounds__(kSpmvThreads, 3)
k_spmm_sys(const SpmmArgs *__restrict__ tab, const int *__restrict__ off, int nSys) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int s = sys_of(off, nSys, (int)blockIdx.x);
    const int b0 = __ldg(off + s);
    spmm_body<MB, false>(tab[s], (int)blockIdx.x - b0, __ldg(off + s + 1) - b0, smem);
}

template <int MB>
void launch_spmm(const SpmmArgs &a, cudaStream_t st) {
    const int smem = spmv_smem_bytes<float, 0>();
    launch_pdl(a.fin ? k_spmm<MB, true> : k_spmm<MB, false>, a.A.grid, kSpmvThreads, smem, st, a);
}

template <typename K>
static bool set_smem(K k, int smem) {
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) ==
           cudaSuccess;
}

int spmm_persistent_grid(int MB, int nSlicesTotal) {
    if (!spmm_prepare()) return -1;
    int dev = 0, sms = device_sm_count(), nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || sms < 1) return -1;
    const int smem = spmv_smem_bytes<float, 0>();
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &nb, MB == 4 ? k_spmm<4, false> : k_spmm<8, false>, kSpmvThreads, smem) !=
            cudaSuccess ||
        nb < 1)
        return -1;
    const int need = (nSlicesTotal + kSpmvWarps - 1) / kSpmvWarps;
    return std::max(1, std::min(nb * sms, need));
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
// ||r||^2 of its column.  Mode 0 updates the running columns (r' = r -
// alpha_j q, u += alpha_j p) and copies the residual of the others.
template <int MB, int M>
__device__ __forceinline__ void restrict_b_unit(const RestrictBArgs &a, int unit,
                                                const float *r_cur, float *r_next,
                                                float (&rr)[MB]) {
    const RowBoxDev &B = a.B;
    const BatchScalars *bs = a.bs;
    const int mode = a.mode;
    float *u = a.u;
    const float *p = a.p, *q = a.q;
    const int s = B.unitBox[unit];
    const int j = threadIdx.x % MB, row0 = threadIdx.x / MB;
    constexpr int kRowStep = kThreads / MB;
    const bool run = mode == 0 && col_runs(bs, j, a.m);
    const float alpha = run ? (float)bs->alpha[j] : 0.0f;
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
                if (run) {
                    rn = fmaf(-alpha, q[e], rn);
                    u[e] = fmaf(alpha, p[e], u[e]);
                }
                r_next[e] = rn;
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
            const float rn = run ? fmaf(-alpha, q[e], r_cur[e]) : r_cur[e];
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
    double *G = a.G, *ZR = a.ZR, *unitPart = a.unitPart;
    float *G32 = a.G32;
    __shared__ float red[MB][2 * 12];
    __shared__ bool lastUnit;
    if (nu == 1) {
        if (holder && tc < 2 * M) red[tj][tc] = tsum;
        __syncthreads();
        if ((int)threadIdx.x < MB * M) {
            const int jj = threadIdx.x / M, c = threadIdx.x % M;
            const double zs = red[jj][c], ws = red[jj][M + c];
            G[(size_t)(c0 + c) * MB + jj] = zs - ws;
            G32[(size_t)jj * a.gld + c0 + c] = (float)(zs - ws);
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
                G32[(size_t)jj * a.gld + c0 + c] = (float)(zs - ws);
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

// mode 0 (iteration): r' = r - alpha_j q, u += alpha_j p for the running
// columns, G from r'; the last block sets rr_j of the running columns and
// holds those at their trigger or at the iteration limit.  mode 1: G and
// rr_j of the columns being replaced from the current residual.  mode 2:
// G = Z~^T f only.
template <int MB>
__device__ __forceinline__ void restrict_b_body(const RestrictBArgs &a, int blk, int nblk) {
    pdl_wait();
    BatchScalars *bs = a.bs;
    if (!batch_runs(bs, a.mode == 0)) return;
    const int its = bs->its, m = a.m, mode = a.mode;
    // iteration: the product advanced its, so buffer (its - 1) & 1 is read
    const float *r_cur = mode == 2 ? a.f : (((its & 1) != (mode == 0)) ? a.rB : a.rA);
    float *r_next = mode == 0 ? ((its & 1) ? a.rB : a.rA) : nullptr;
    const int unit = blk;
    float rr[MB];
#pragma unroll
    for (int j = 0; j < MB; ++j) rr[j] = 0.0f;
    if (a.B.menr[a.B.unitBox[unit]])
        restrict_b_unit<MB, 12>(a, unit, r_cur, r_next, rr);
    else
        restrict_b_unit<MB, 6>(a, unit, r_cur, r_next, rr);
    if (mode == 2) return;
    // rr holds the block's totals in thread 0 (zeros elsewhere)
    if (threadIdx.x != 0)
#pragma unroll
        for (int j = 0; j < MB; ++j) rr[j] = 0.0f;
    double tot[MB];
    if (grid_sum_of<float, MB>(rr, a.partials, &bs->ticket[2], tot, blk, nblk) &&
        threadIdx.x == 0) {
        if (mode == 1) {
            for (int j = 0; j < m; ++j)
                if (bs->repl[j]) bs->rr[j] = tot[j];
            return;
        }
        bool any = false;
        for (int j = 0; j < m; ++j) {
            if (!col_runs(bs, j, m)) continue;
            bs->rr[j] = tot[j];
            if (tot[j] <= bs->trig[j] || !isfinite(tot[j])) bs->pend[j] = 1;
            if (bs->itsc[j] >= bs->max_it) {
                bs->pend[j] = 1;
                bs->last[j] = 1;
            }
            any |= !bs->pend[j];
        }
        if (!any) bs->done = kConverged;
    }
}

template <int MB>
__global__ void __launch_bounds__(kThreads) k_restrict_b(RestrictBArgs a) {
    restrict_b_body<MB>(a, (int)blockIdx.x, (int)gridDim.x);
}

template <int MB>
__global__ void __launch_bounds__(kThreads)
k_restrict_b_sys(const RestrictBArgs *__restrict__ tab, const int *__restrict__ off, int nSys) {
    const int s = sys_of(off, nSys, (int)blockIdx.x);
    const int b0 = __ldg(off + s);
    restrict_b_body<MB>(tab[s], (int)blockIdx.x - b0, __ldg(off + s + 1) - b0);
}

template <int MB>
void launch_restrict_b(const RestrictBArgs &a, cudaStream_t st) {
    launch_pdl(k_restrict_b<MB>, a.B.nUnits, kThreads, 0, st, a);
}

// ---- batched coarse solve NU = E^-1 G -----------------------------------------

// Sums NV values over the warp's lanes by halving exchanges (fixed tree):
// afterwards lane L holds in v[0 .. NV / 32) the totals of values
// (NV / 32) L + i.
template <int NV>
__device__ __forceinline__ void lane_reduce_scatter(float (&v)[NV], int lane) {
    static_assert(NV >= 32 && NV % 32 == 0, "NV: a multiple of 32");
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int o = 16 >> st, half = (NV >> st) >> 1;
        const bool hi = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; ++i) {
            const float send = hi ? v[i] : v[i + half];
            const float keep = hi ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
}

// rows of E^-1 per block of the batched coarse solve (RB * MB = 32 partial
// sums per lane)
template <int MB>
__host__ __device__ constexpr int coarse_rows_b() { return 32 / MB; }
constexpr int kCoarseChunkB = 128;   // columns of G per staged chunk (4 per lane)
template <int MB>
constexpr int coarse_smem_b() {
    return kWarps * 2 * MB * kCoarseChunkB * (int)sizeof(float) +
           kWarps * 2 * (int)sizeof(uint64_t);
}

// One chunk's entries of E^-1 for a lane: 4 consecutive columns (one 16-byte
// load per row, V = 4) or 4 columns 32 apart (V = 1) of each of the RB rows.
template <int RB, int V>
__device__ __forceinline__ void coarse_load_e(const float *Eb, int k, int rLast, int lc, int clen,
                                              int lane, uint64_t keep, float (&e)[RB][4]) {
#pragma unroll
    for (int r = 0; r < RB; ++r) {
        const float *row = Eb + (size_t)min(r, rLast) * k + lc;
        if (V == 4) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (4 * lane < clen) v = ld_keep(reinterpret_cast<const float4 *>(row + 4 * lane), keep);
            e[r][0] = v.x;
            e[r][1] = v.y;
            e[r][2] = v.z;
            e[r][3] = v.w;
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                e[r][q] = lane + 32 * q < clen ? ld_keep(row + lane + 32 * q, keep) : 0.0f;
        }
    }
}

// NU = E^-1 G for the MB columns, then the scalars.  mode 0: nu only; mode 1
// (start, every column): rho_j = rr_j + nu_j^T zr_j, beta_j = 0; mode 2
// (iteration, running columns): the same rho_new, beta_j = rho_new / rho_j;
// mode 3 (replacement, the replaced columns): as 2, with beta_j = 0 for a
// column that leaves, that broke down or whose residual the replacement
// lengthened by more than 2x.  A block takes 32 / MB consecutive rows of
// E^-1 and its warps split the columns into segments (multiples of 4).  Each
// warp walks its segment in chunks of kCoarseChunkB columns: the chunk's
// part of G (stored column by column) is staged in shared memory by bulk
// copies, double-buffered (the next chunk's copy is in flight while this one
// is used), and the lane's entries of E^-1 are loaded before the wait for
// the chunk's copy (the first chunk's before the wait for the previous
// kernel: E^-1 does not depend on it), so a chunk costs one memory round
// trip.  The partial sums are reduced over the lanes, then over the warps in
// order.
template <int MB, int V>
__device__ __forceinline__ void coarse_b_body(const CoarseBArgs &a, int blk, int nblk,
                                              unsigned char *smem) {
    constexpr int RB = coarse_rows_b<MB>(), NV = RB * MB, P = NV / 32, CH = kCoarseChunkB;
    __shared__ float red[kWarps][NV];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *gs = reinterpret_cast<float *>(smem) + (size_t)warp * 2 * MB * CH;   // [2][MB][CH]
    uint64_t *bar =
        reinterpret_cast<uint64_t *>(smem + (size_t)kWarps * 2 * MB * CH * sizeof(float)) +
        2 * warp;
    if (lane == 0) {
        mbar_init(bar, 1);
        mbar_init(bar + 1, 1);
        mbar_init_fence();
    }
    __syncwarp();
    const int k = a.k;
    const int i0 = blk * RB;
    const int seg = (k + 4 * kWarps - 1) / (4 * kWarps) * 4;
    const int l0 = warp * seg, l1 = min(k, l0 + seg);
    const int nch = l1 > l0 ? (l1 - l0 + CH - 1) / CH : 0;
    const uint64_t keep = l2_keep_policy();
    const float *Eb = a.Einv + (size_t)i0 * k;
    const int rLast = k - 1 - i0;
    float e[RB][4];
    if (nch > 0) coarse_load_e<RB, V>(Eb, k, rLast, l0, min(CH, l1 - l0), lane, keep, e);
    pdl_wait();
    BatchScalars *bs = a.bs;
    if (!batch_runs(bs, a.mode == 2)) return;
    const int m = a.m, mode = a.mode;
    const unsigned long long deadline = global_ns() + a.waitNs;
    auto issue = [&](int c) {   // lane 0: chunk c of G into buffer c & 1
        const int lc = l0 + c * CH, cpad = (min(CH, l1 - lc) + 3) & ~3;
        float *dst = gs + (c & 1) * MB * CH;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar + (c & 1), (uint32_t)(MB * cpad * sizeof(float)));
#pragma unroll
        for (int j = 0; j < MB; ++j)
            bulk_g2s(dst + j * CH, a.G32 + (size_t)j * a.gld + lc, (uint32_t)(cpad * sizeof(float)),
                     bar + (c & 1), keep);
    };
    float acc[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) acc[t] = 0.0f;
    if (lane == 0 && nch > 0) issue(0);
    int c = 0;
    bool ok = true;
    for (; c < nch; ++c) {
        if (lane == 0 && c + 1 < nch) issue(c + 1);
        const int lc = l0 + c * CH, clen = min(CH, l1 - lc);
        if (c > 0) coarse_load_e<RB, V>(Eb, k, rLast, lc, clen, lane, keep, e);
        ok = __all_sync(0xffffffffu, mbar_wait(bar + (c & 1), (uint32_t)(c >> 1) & 1u, deadline));
        if (!ok) break;
        const float *g0 = gs + (c & 1) * MB * CH;
#pragma unroll
        for (int j = 0; j < MB; ++j) {
            float g[4];
            // entries past the chunk are never read (shared memory there may
            // hold anything, and 0 * NaN is NaN)
            if (V == 4) {
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (4 * lane < clen) v = *reinterpret_cast<const float4 *>(g0 + j * CH + 4 * lane);
                g[0] = v.x;
                g[1] = v.y;
                g[2] = v.z;
                g[3] = v.w;
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    g[q] = lane + 32 * q < clen ? g0[j * CH + lane + 32 * q] : 0.0f;
            }
#pragma unroll
            for (int r = 0; r < RB; ++r) {
                float t = fmaf(e[r][0], g[0], acc[r * MB + j]);
                t = fmaf(e[r][1], g[1], t);
                t = fmaf(e[r][2], g[2], t);
                acc[r * MB + j] = fmaf(e[r][3], g[3], t);
            }
        }
        __syncwarp();   // the buffer is read before a later copy overwrites it
    }
    if (!ok) {
        // copies in flight (chunks c and c + 1) land before the block leaves
        const unsigned long long drain = global_ns() + kDrainNs;
        for (int d = c; d < min(nch, c + 2); ++d) mbar_wait(bar + (d & 1), (uint32_t)(d >> 1) & 1u, drain);
        __syncwarp();
        if (lane == 0) atomicExch(&bs->fault, 1);
    }
    lane_reduce_scatter<NV>(acc, lane);
#pragma unroll
    for (int i = 0; i < P; ++i) red[warp][P * lane + i] = acc[i];
    __syncthreads();
    // warp 0 (lane = r * MB + j): nu_i for row i = i0 + r, column j, and its
    // share of nu_j^T zr_j, summed over the block's rows
    static_assert(NV == 32, "one lane per (row, column) of the block");
    double pj = 0.0;
    if (warp == 0) {
        float sum = 0.0f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) sum += red[w][lane];
        const int r = lane / MB, j = lane % MB, i = i0 + r;
        if (i < k) {
            a.NU[(size_t)i * MB + j] = (double)sum;
            a.NU32[(size_t)i * MB + j] = sum;
            if (mode != 0) pj = (double)sum * a.ZR[(size_t)i * MB + j];
        }
#pragma unroll
        for (int o = MB; o < 32; o <<= 1) pj += __shfl_xor_sync(0xffffffffu, pj, o);
    }
    double tot[MB];
    if (grid_sum_lanes<MB>(pj, a.partials, &bs->ticket[3], tot, blk, nblk) && threadIdx.x == 0) {
        if (bs->fault) {
            bs->done = kFault;
        } else if (mode != 0) {
            for (int j = 0; j < m; ++j) {
                const bool upd = mode == 2 ? col_runs(bs, j, m) : (mode == 1 || bs->repl[j]);
                if (!upd) continue;
                const double rho_new = bs->rr[j] + tot[j];
                if (mode == 1 || !bs->active[j] ||
                    (mode == 3 && (bs->broken[j] || bs->rr[j] > 4.0 * bs->rrRep[j])))
                    bs->beta[j] = 0.0;
                else
                    bs->beta[j] = rho_new / bs->rho[j];
                bs->rho[j] = rho_new;
                if (mode == 3) bs->broken[j] = 0;
            }
        }
    }
}

template <int MB, int V>
__global__ void __launch_bounds__(kThreads, MB == 8 ? 3 : 2) k_coarse_b(CoarseBArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    coarse_b_body<MB, V>(a, (int)blockIdx.x, (int)gridDim.x, smem);
}

template <int MB>
__global__ void __launch_bounds__(kThreads, MB == 8 ? 3 : 2)
k_coarse_b_sys(const CoarseBArgs *__restrict__ tab, const int *__restrict__ off, int nSys) {
    extern __shared__ __align__(128) unsigned char smem[];
    const int s = sys_of(off, nSys, (int)blockIdx.x);
    const int b0 = __ldg(off + s), nb = __ldg(off + s + 1) - b0;
    const CoarseBArgs &a = tab[s];
    if ((a.k & 3) == 0)
        coarse_b_body<MB, 4>(a, (int)blockIdx.x - b0, nb, smem);
    else
        coarse_b_body<MB, 1>(a, (int)blockIdx.x - b0, nb, smem);
}

int coarse_b_blocks(int k, int MB) {
    const int rb = MB == 4 ? coarse_rows_b<4>() : coarse_rows_b<8>();
    const int grid = (k + rb - 1) / rb;
    return grid > 0 ? grid : 1;
}

template <int MB>
void launch_coarse_b(const CoarseBArgs &a, cudaStream_t st) {
    launch_pdl(a.k % 4 == 0 ? k_coarse_b<MB, 4> : k_coarse_b<MB, 1>, coarse_b_blocks(a.k, MB),
               kThreads, coarse_smem_b<MB>(), st, a);
}

// ---- batched prolongation -----------------------------------------------------

// mode 0 (iteration, running columns) and mode 3 (replacement, the replaced
// columns): p = y + Z~ nu + beta_j p, 0 for a replaced column that leaves;
// mode 1 (start): p = Z~ nu; mode 2 (start): p = y + Z~ nu.  y is the current
// residual buffer.
template <int MB, int M>
__device__ __forceinline__ void prolong_b_unit(const RowBoxDev &B, int unit, const float *NU32,
                                               const float *y, float *p, int mode, float beta,
                                               bool leaves) {
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
        if (mode == 0 || mode == 3)
            p[e] = leaves ? 0.0f : y[e] + zv + beta * p[e];
        else if (mode == 1)
            p[e] = zv;
        else
            p[e] = y[e] + zv;
    }
}

template <int MB>
__device__ __forceinline__ void prolong_b_body(const ProlongBArgs &a, int blk) {
    pdl_wait();
    const BatchScalars *bs = a.bs;
    if (!batch_runs(bs, a.mode == 0)) return;
    const int unit = blk, mode = a.mode;
    const int j = threadIdx.x % MB;
    bool wr = true, leaves = false;
    if (mode == 0) {
        wr = col_runs(bs, j, a.m);
    } else if (mode == 3) {
        wr = j < a.m && bs->repl[j];
        leaves = wr && !bs->active[j];
    }
    if (!wr) return;   // no block-wide step follows
    const float beta = (mode == 0 || mode == 3) && !leaves ? (float)bs->beta[j] : 0.0f;
    const float *y = (bs->its & 1) ? a.rB : a.rA;
    if (a.B.menr[a.B.pUnitBox[unit]])
        prolong_b_unit<MB, 12>(a.B, unit, a.NU32, y, a.p, mode, beta, leaves);
    else
        prolong_b_unit<MB, 6>(a.B, unit, a.NU32, y, a.p, mode, beta, leaves);
}

template <int MB>
__global__ void __launch_bounds__(kThreads) k_prolong_b(ProlongBArgs a) {
    prolong_b_body<MB>(a, (int)blockIdx.x);
}

template <int MB>
__global__ void __launch_bounds__(kThreads)
k_prolong_b_sys(const ProlongBArgs *__restrict__ tab, const int *__restrict__ off, int nSys) {
    const int s = sys_of(off, nSys, (int)blockIdx.x);
    prolong_b_body<MB>(tab[s], (int)blockIdx.x - __ldg(off + s));
}

template <int MB>
void launch_prolong_b(const ProlongBArgs &a, cudaStream_t st) {
    launch_pdl(k_prolong_b<MB>, a.B.nPUnits, kThreads, 0, st, a);
}

// Before each iteration over several systems: whether it runs each system
// (running and not held), read once so that every block of the iteration's
// four kernels agrees.  A replacement's last kernel releases the hold after
// its other writes (k_batch_arm), so a gate that sees the release sees them.
__global__ void k_batch_gate(const SpmmArgs *__restrict__ tab, int nSys) {
    for (int s = threadIdx.x; s < nSys; s += blockDim.x) {
        BatchScalars *bs = tab[s].bs;
        const int held = *reinterpret_cast<volatile const int *>(&bs->hold);
        __threadfence();
        const int done = *reinterpret_cast<volatile const int *>(&bs->done);
        bs->go = done == kRunning && !held;
    }
}

// one FP32 iteration of every system of the table: the gate, then four launches
template <int MB>
void launch_iteration_sys(const BatchSysTab &t, cudaStream_t st) {
    k_batch_gate<<<1, 128, 0, st>>>(t.spmm, t.nSys);
    const int smem = spmv_smem_bytes<float, 0>();
    launch_pdl(k_spmm_sys<MB>, t.blocks[0], kSpmvThreads, smem, st, t.spmm, t.off[0], t.nSys);
    launch_pdl(k_restrict_b_sys<MB>, t.blocks[1], kThreads, 0, st, t.rst, t.off[1], t.nSys);
    launch_pdl(k_coarse_b_sys<MB>, t.blocks[2], kThreads, coarse_smem_b<MB>(), st, t.crs, t.off[2],
               t.nSys);
    launch_pdl(k_prolong_b_sys<MB>, t.blocks[3], kThreads, 0, st, t.pro, t.off[3], t.nSys);
}

// ---- column scalars -------------------------------------------------------------

__device__ __forceinline__ void fresh_slot(Scalars *sc) {
    Scalars z{};
    z.tol2ff = -1.0;
    z.max_it = INT_MAX;
    *sc = z;
}

__global__ void k_batch_slots(Scalars *slots, unsigned mask) {
    const int j = threadIdx.x;
    if (j < kMaxBatch && ((mask >> j) & 1u)) fresh_slot(slots + j);
}

// repl_j = column j is in mask, fresh reduction slots for them; the
// replacement's kernels run (done = kRunning) unless a wait has failed
__global__ void k_batch_open(BatchScalars *bs, Scalars *slots, unsigned mask) {
    const int j = threadIdx.x;
    if (j < kMaxBatch) {
        const int r = (mask >> j) & 1u;
        bs->repl[j] = r;
        if (r) fresh_slot(slots + j);
    }
    if (j == 0 && bs->done != kFault) bs->done = kRunning;
}

// the replaced columns' FP64 residuals ||f_j - K u_j||^2 (slot j, scratch 0):
// a column leaves converged (<= tol^2 ||f_j||^2), not finite, or at its last
// cycle (iteration limit or max_outer replacements)
__global__ void k_batch_judge(BatchScalars *bs, const Scalars *slots, int m) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int j = 0; j < m; ++j) {
        if (!bs->repl[j]) continue;
        if (slots[j].done == kFault) {
            bs->fault = 1;
            bs->done = kFault;
        }
        const double rn2 = slots[j].scratch[0];
        bs->rn2[j] = rn2;
        bs->cycles[j] += 1;
        bs->rrRep[j] = bs->rr[j];
        if (!isfinite(rn2)) {
            bs->active[j] = 0;
            bs->outcome[j] = kColBad;
        } else if (rn2 <= bs->tol * bs->tol * bs->ff[j]) {
            bs->active[j] = 0;
        } else if (bs->last[j] || bs->cycles[j] >= bs->max_outer) {
            bs->active[j] = 0;
            bs->outcome[j] = kColLimit;
        }
    }
}

// Triggers of the columns being replaced (first: every column, after the
// start): the next replacement of column j once its recursive residual has
// dropped by delta (squared: delta2), or to the floor below which the FP32
// recursion no longer tracks the true residual (a quarter of the target
// relative to the last replacement's ratio of recursive to true residual),
// but at least by kMinGroupDrop2; then release them.
__global__ void k_batch_arm(BatchScalars *bs, int m, int first) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    bool any = false;
    for (int j = 0; j < m; ++j) {
        if (first || bs->repl[j]) {
            if (!bs->active[j]) {
                bs->trig[j] = -1.0;
            } else if (first) {
                bs->trig[j] = bs->delta2 * bs->rr[j];
            } else {
                const double sj = bs->scale[j], rr = bs->rr[j], tol = bs->tol;
                const double gamma2 = rr / (sj * sj * bs->rn2[j]);
                const double f1 = 0.25 * tol * tol * bs->ff[j] * sj * sj * gamma2;
                const double f2 = kMinGroupDrop2 * rr;
                const double floor2 = f2 < f1 ? f2 : f1;
                const double t = bs->delta2 * rr;
                bs->trig[j] = floor2 > t ? floor2 : t;
            }
            bs->pend[j] = 0;
            bs->last[j] = 0;
            bs->repl[j] = 0;
        }
        any |= bs->active[j] && !bs->pend[j];
    }
    if (bs->done != kFault) bs->done = any ? kRunning : kConverged;
    __threadfence();   // every write of the replacement before the release
    *reinterpret_cast<volatile int *>(&bs->hold) = 0;
}

__global__ void k_batch_hold(BatchScalars *bs) {
    if (threadIdx.x == 0 && blockIdx.x == 0) bs->hold = 1;
}

void launch_batch_slots(Scalars *slots, unsigned mask, cudaStream_t st) {
    k_batch_slots<<<1, 32, 0, st>>>(slots, mask);
}
void launch_batch_open(BatchScalars *bs, Scalars *slots, unsigned mask, cudaStream_t st) {
    k_batch_open<<<1, 32, 0, st>>>(bs, slots, mask);
}
void launch_batch_judge(BatchScalars *bs, const Scalars *slots, int m, cudaStream_t st) {
    k_batch_judge<<<1, 32, 0, st>>>(bs, slots, m);
}
void launch_batch_arm(BatchScalars *bs, int m, int first, cudaStream_t st) {
    k_batch_arm<<<1, 32, 0, st>>>(bs, m, first);
}
void launch_batch_hold(BatchScalars *bs, cudaStream_t st) { k_batch_hold<<<1, 32, 0, st>>>(bs); }

// ---- FP64 <-> FP32 transforms of several columns --------------------------------

// out[(ot[I] + i) * MB + j] = scale_j (L^-1 r_j)_i for the columns being
// replaced (repl_j; every column at the start), 0 for those that leave and
// for padding columns; r_j = r + j * ldr in the caller's numbering (nat).
// out is the current residual buffer (outA, or outB when its is odd).  One
// thread per (node, column).
template <int MB>
__global__ void k_fwd_scale_b(int nNodes, int m, const int *nat, const int *ot, FacDev F,
                              const double *r, long long ldr, const BatchScalars *bs,
                              float *outA, float *outB) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nNodes * MB) return;
    const int I = (int)(t / MB), j = (int)(t % MB);
    if (j < m && !bs->repl[j]) return;
    float *out = (bs->its & 1) ? outB : outA;
    const int b = nat[I + 1] - nat[I], d0 = nat[I], o0 = ot[I];
    const bool on = j < m && bs->active[j];
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

// u_j += (L^-T ut_j)_i / scale_j, then ut_j = 0, for the columns being
// replaced; one thread per (node, column)
template <int MB>
__global__ void k_bwd_accum_b(int nNodes, int m, const int *nat, const int *in, FacDev F,
                              float *ut, const BatchScalars *bs, double *u, long long ldu) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t >= (long long)nNodes * MB) return;
    const int I = (int)(t / MB), j = (int)(t % MB);
    if (j >= m || !bs->repl[j]) return;
    const int b = nat[I + 1] - nat[I], d0 = in[I], o0 = nat[I];
    const double inv = 1.0 / bs->scale[j];
    const int q = F.nodeIdx[I];
    with_node_size(b, [&](auto Bc) {
        constexpr int B = decltype(Bc)::value;
        double x[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            float *e = ut + (size_t)(d0 + i) * MB + j;
            x[i] = (double)*e;
            *e = 0.0f;
        }
        bwd_solve_fixed<B>(F, q, x);
#pragma unroll
        for (int i = 0; i < B; ++i) u[j * ldu + o0 + i] += inv * x[i];
    });
}

template <int MB>
void launch_fwd_scale_b(int nNodes, int m, const int *nat, const int *ot, const FacDev &F,
                        const double *r, long long ldr, const BatchScalars *bs, float *outA,
                        float *outB, cudaStream_t st) {
    const long long nt = (long long)nNodes * MB;
    k_fwd_scale_b<MB><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(nNodes, m, nat, ot, F, r, ldr,
                                                                     bs, outA, outB);
}

template <int MB>
void launch_bwd_accum_b(int nNodes, int m, const int *nat, const int *in, const FacDev &F,
                        float *ut, const BatchScalars *bs, double *u, long long ldu,
                        cudaStream_t st) {
    const long long nt = (long long)nNodes * MB;
    k_bwd_accum_b<MB><<<(unsigned)((nt + 127) / 128), 128, 0, st>>>(nNodes, m, nat, in, F, ut, bs,
                                                                     u, ldu);
}

// dynamic shared memory limits of the batched kernels (once per process)
bool spmm_prepare() {
    const int smem = spmv_smem_bytes<float, 0>();
    return set_smem(k_spmm<4, false>, smem) && set_smem(k_spmm<4, true>, smem) &&
           set_smem(k_spmm<8, false>, smem) && set_smem(k_spmm<8, true>, smem) &&
           set_smem(k_spmm_sys<4>, smem) && set_smem(k_spmm_sys<8>, smem) &&
           set_smem(k_coarse_b<4, 4>, coarse_smem_b<4>()) &&
           set_smem(k_coarse_b<4, 1>, coarse_smem_b<4>()) &&
           set_smem(k_coarse_b<8, 4>, coarse_smem_b<8>()) &&
           set_smem(k_coarse_b<8, 1>, coarse_smem_b<8>()) &&
           set_smem(k_coarse_b_sys<4>, coarse_smem_b<4>()) &&
           set_smem(k_coarse_b_sys<8>, coarse_smem_b<8>());
}

#define XDCG_BATCH_INST(MB)                                                                    \
    template void launch_spmm<MB>(const SpmmArgs &, cudaStream_t);                             \
    template void launch_restrict_b<MB>(const RestrictBArgs &, cudaStream_t);                  \
    template void launch_coarse_b<MB>(const CoarseBArgs &, cudaStream_t);                      \
    template void launch_prolong_b<MB>(const ProlongBArgs &, cudaStream_t);                    \
    template void launch_iteration_sys<MB>(const BatchSysTab &, cudaStream_t);                 \
    template void launch_fwd_scale_b<MB>(int, int, const int *, const int *, const FacDev &,   \
                                         const double *, long long, const BatchScalars *,      \
                                         float *, float *, cudaStream_t);                      \
    template void launch_bwd_accum_b<MB>(int, int, const int *, const int *, const FacDev &,   \
                                         float *, const BatchScalars *, double *, long long,    \
                                         cudaStream_t);
XDCG_BATCH_INST(4)
XDCG_BATCH_INST(8)
#undef XDCG_BATCH_INST

}  // namespace xdcg
