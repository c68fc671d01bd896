// Chunked node-blocked SpMV q = K p (Algorithm 1, the product K p_i) with
// the fused partial of p^T q, plus the plain vector kernels of the solve.
//
// K is stored as 3x3 blocks between "chunks" (3 consecutive dofs: the
// standard dofs of a node, its jump dofs, or one branch function's 3 dofs),
// so standard and enriched couplings of Eq. linear_system stream through the
// same code.  Values and column indices are read once per product with
// evict-first loads; the gathered x chunks stay in L1/L2.
#include <algorithm>

#include "reduce.cuh"
#include "spmv_cfg.cuh"
#include "tma.cuh"

namespace xdcg {

// Persistent warps over the slices of both parts (S slices first, then X);
// warp w owns the slices [warpSlice[w], warpSlice[w + 1]), ranges balanced
// by steps at set-up.  Each warp streams its slices' column indices and
// values through its own ring of NS shared-memory stages with bulk copies
// (lane 0 issues, all lanes consume), so the HBM stream takes no per-lane
// load instructions and no registers in flight.  The x chunks of the next
// stage are gathered (from L1/L2) before the current stage is computed, and
// the first stages are in flight before the wait for the kernel that wrote
// x.  Padding slots hold zero values and a valid column, so every slot can
// be computed (unless GUARD).  The fused dot (x^T y, or y^T y in residual
// mode) is summed per warp over a fixed slice range, then by the
// deterministic grid reduction.
//
// No dependent global load sits on a warp's path from one slice to the
// next: the first 32 slices' extents are read into shared memory at kernel
// start (one slice per lane), and a slice's row indices are loaded when the
// slice begins, its x (or b) entries one stage later, for use when it ends.
template <typename T, bool RES, int SHAPE>
__global__ void __launch_bounds__(kSpmvThreads, SpmvCfg<T, SHAPE>::MINB)
k_spmv(SpmvDev<T> A, const T *__restrict__ x, T *__restrict__ y, const T *__restrict__ b,
       double *partials, Scalars *sc, int fin, int slot) {
    using Cfg = SpmvCfg<T, SHAPE>;
    constexpr int C = Cfg::C, NS = Cfg::NS, SB = stage_bytes<T, SHAPE>();
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *ring = smem + (size_t)warp * NS * SB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)kSpmvWarps * NS * SB) + warp * NS;
    int *meta = reinterpret_cast<int *>(smem + (size_t)kSpmvWarps * NS * (SB + 8)) + warp * NS * 3;
    const int nS = A.S.nSlices;
    const int gw = blockIdx.x * kSpmvWarps + warp;
    const int sFirst = A.warpSlice[gw], sEnd = A.warpSlice[gw + 1];
    // extents of the warp's first 32 slices (set-up data)
    __shared__ long long tBase[kSpmvWarps][32];
    __shared__ int tSteps[kSpmvWarps][32];
    if (sFirst + lane < sEnd) {
        const int g = sFirst + lane;
        const SellDev<T> &P = g < nS ? A.S : A.X;
        const int sl = g < nS ? g : g - nS;
        const long long b0 = P.slicePtr[sl];
        tBase[warp][lane] = b0;
        tSteps[warp][lane] = (int)((P.slicePtr[sl + 1] - b0) >> 5);
    }
    if (lane == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bars + s, 1);
        mbar_init_fence();
    }
    __syncwarp();
    const uint64_t stream = l2_stream_policy();
    const unsigned long long deadline = global_ns() + A.waitNs;

    // producer state, meaningful in lane 0
    int issued = 0, more = 1, pSlice = sFirst - 1, pStep = 0, pSteps = 0;
    long long pBase = 0;
    const int *pCol = nullptr;
    const T *pVal = nullptr;
    auto issue = [&]() {
        if (pStep >= pSteps) {
            if (++pSlice >= sEnd) {
                more = 0;
                return;
            }
            const bool isS = pSlice < nS;
            const SellDev<T> &P = isS ? A.S : A.X;
            const int sl = isS ? pSlice : pSlice - nS;
            if (pSlice - sFirst < 32) {
                pBase = tBase[warp][pSlice - sFirst];
                pSteps = tSteps[warp][pSlice - sFirst];
            } else {
                pBase = P.slicePtr[sl];
                pSteps = (int)((P.slicePtr[sl + 1] - pBase) >> 5);
            }
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
        const uint32_t cb = (uint32_t)n * 128u, vb = (uint32_t)n * 288u * (uint32_t)sizeof(T);
        const long long off = pBase + 32LL * pStep;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bars + st, cb + vb);
        bulk_g2s(dst, pCol + off, cb, bars + st, stream);
        bulk_g2s(dst + C * 128, pVal + 9 * off, vb, bars + st, stream);
        pStep += n;
        ++issued;
    };
    // the first stages stream set-up data only: issue them before waiting
    // for the kernel that produced x, unless the run has visibly stopped
    // already (launches queued past a stop).  That early read of the flag
    // bypasses L1 and may be stale; the flag read after the wait decides.
    const bool early = __ldcg(&sc->done) == kRunning;
    if (lane == 0 && early)
        while (more && issued < NS) issue();
    issued = __shfl_sync(0xffffffffu, issued, 0);
    pdl_wait();
    if (sc->done != kRunning) {
        // nothing to do: let the copies in flight land before leaving
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

    T part[1] = {T(0)};
    int cur = -1, rpw = 16, rl = 0, h = 0, tpr = 2, len = 0;
    bool valid = false, isS = true, own = false, pend = false;
    long long r3 = 0;            // first dof of the lane's row (own lanes)
    T e0 = T(0), e1 = T(0), e2 = T(0);   // its x (or b) entries
    T a0 = T(0), a1 = T(0), a2 = T(0);
    const T *ev = RES ? b : x;
    auto fetch_row_entries = [&]() {
        pend = false;
        if (own) {
            e0 = ev[r3];
            e1 = ev[r3 + 1];
            e2 = ev[r3 + 2];
        }
    };
    auto finish = [&]() {
        for (int o = rpw; o < 32; o <<= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (pend) fetch_row_entries();
        if (own) {
            if (RES) {
                a0 = e0 - a0;
                a1 = e1 - a1;
                a2 = e2 - a2;
                part[0] += a0 * a0 + a1 * a1 + a2 * a2;
            } else {
                part[0] += e0 * a0 + e1 * a1 + e2 * a2;
            }
            y[r3] = a0;
            y[r3 + 1] = a1;
            y[r3 + 2] = a2;
        }
    };
    // x chunks of a landed stage, gathered ahead of its computation
    auto gather = [&](int st, int n, T (&xv)[C][3]) {
        const int *cs = reinterpret_cast<const int *>(ring + st * SB);
#pragma unroll
        for (int t = 0; t < C; ++t) {
            if (t < n) {
                const int c = cs[t * 32 + lane];
                xv[t][0] = __ldg(x + 3 * c);
                xv[t][1] = __ldg(x + 3 * c + 1);
                xv[t][2] = __ldg(x + 3 * c + 2);
            }
        }
    };
    T xa[C][3], xb[C][3];
    int na = 0;
    bool ok = true;
    int k = 0;
    if (issued > 0) {
        ok = __all_sync(0xffffffffu, mbar_wait(bars, 0u, deadline));
        if (ok) {
            na = meta[2];
            gather(0, na, xa);
        }
    }
    for (; ok && k < issued; ++k) {
        const int st = k % NS;
        // land and gather the next stage first
        int nb = 0;
        if (k + 1 < issued) {
            const int s1 = (k + 1) % NS;
            ok = __all_sync(0xffffffffu, mbar_wait(bars + s1, (uint32_t)((k + 1) / NS) & 1u, deadline));
            if (!ok) break;
            nb = meta[s1 * 3 + 2];
            gather(s1, nb, xb);
        }
        const int sl = meta[st * 3];
        if (sl != cur) {
            if (cur >= 0) finish();
            cur = sl;
            isS = sl < nS;
            tpr = isS ? kTprS : kTprX;
            rpw = 32 / tpr;
            rl = (isS ? sl : sl - nS) * rpw + (lane % rpw);
            h = lane / rpw;
            valid = rl < (isS ? A.S.nRows : A.X.nRows);
            if (Cfg::GUARD) len = valid ? (isS ? A.S.len[rl] : A.X.len[rl]) : 0;
            own = valid && h == 0;
            // consumed when the slice ends; the row's x (or b) entries are
            // loaded after this stage, once the index has arrived
            r3 = own ? 3 * (long long)(isS ? A.S.row[rl] : A.X.row[rl]) : 0;
            pend = true;
            a0 = a1 = a2 = T(0);
        }
        const int s0 = meta[st * 3 + 1];
        const T *vs = reinterpret_cast<const T *>(ring + st * SB + C * 128);
#pragma unroll
        for (int t = 0; t < C; ++t) {
            if (t < na && (!Cfg::GUARD || (s0 + t) * tpr + h < len)) {
                const T *v = vs + t * 288 + lane;
                a0 = fma(v[0], xa[t][0], a0);
                a0 = fma(v[32], xa[t][1], a0);
                a0 = fma(v[64], xa[t][2], a0);
                a1 = fma(v[96], xa[t][0], a1);
                a1 = fma(v[128], xa[t][1], a1);
                a1 = fma(v[160], xa[t][2], a1);
                a2 = fma(v[192], xa[t][0], a2);
                a2 = fma(v[224], xa[t][1], a2);
                a2 = fma(v[256], xa[t][2], a2);
            }
        }
        __syncwarp();
        if (lane == 0 && more) issue();
        issued = __shfl_sync(0xffffffffu, issued, 0);
        if (pend) fetch_row_entries();
#pragma unroll
        for (int t = 0; t < C; ++t) {
            xa[t][0] = xb[t][0];
            xa[t][1] = xb[t][1];
            xa[t][2] = xb[t][2];
        }
        na = nb;
    }
    if (ok) {
        if (cur >= 0) finish();
    } else {
        // a copy did not land in time: flag it, give the copies still in
        // flight a bounded chance to land, and leave the shared memory
        if (lane == 0) atomicExch(&sc->fault, 1);
        const unsigned long long drain = global_ns() + kDrainNs;
        for (; k < issued; ++k) mbar_wait(bars + k % NS, (uint32_t)(k / NS) & 1u, drain);
        __syncwarp();
    }
    if (fin == kFinDefer) {
        // the next kernel adds the blocks' sums (block_read_total); a failed
        // wait is in sc->fault, which it reads too
        block_sum<T, 1>(part);
        if (threadIdx.x == 0)
            reinterpret_cast<float2 *>(partials)[blockIdx.x] = df_of((double)part[0]);
        return;
    }
    double tot[1];
    if (grid_sum<T, 1>(part, partials, &sc->ticket[0], tot) && threadIdx.x == 0) {
        if (sc->fault)
            sc->done = kFault;
        else
            finalize(sc, fin, slot, tot[0]);
    }
}

// The warp's copy schedule: its S slices, then its X slices, each part one
// contiguous run of steps (a step = 32 slots: 32 column indices and 9 planes
// of 32 values), cut into stages of at most C steps that may run across
// slice boundaries but not across the two parts (separate arrays).  Every
// lane walks the same schedule (uniform values), so no per-stage record is
// kept: the producer's walk runs NS stages ahead of the consumer's.
struct LeanWalk {
    long long pos, end, xPos, xEnd;
    int isS;
    __device__ __forceinline__ bool next(int C, int &sS, long long &p, int &n) {
        if (pos == end) {
            if (!isS || xPos == xEnd) return false;
            isS = 0;
            pos = xPos;
            end = xEnd;
        }
        sS = isS;
        p = pos;
        n = (int)min((long long)C, end - pos);
        pos += n;
        return true;
    }
};

// Same product as k_spmv (same layout, same per-row order of the 3x3 block
// terms and of the row reduction, same dot order), with less bookkeeping per
// step: the ring slot and its parity advance by increments, the row switch is
// a count of the steps left in the current slice, and the x gathers of the
// next stage go to the register set the current stage does not use (the
// stage loop is unrolled by two).
template <bool RES, int SHAPE>
__global__ void __launch_bounds__(kSpmvThreads, SpmvCfg<float, SHAPE>::MINB)
k_spmv_lean(SpmvDev<float> A, const float *__restrict__ x, float *__restrict__ y,
            const float *__restrict__ b, double *partials, Scalars *sc, int fin, int slot) {
    using Cfg = SpmvCfg<float, SHAPE>;
    constexpr int C = Cfg::C, NS = Cfg::NS, SB = stage_bytes<float, SHAPE>();
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *ring = smem + (size_t)warp * NS * SB;
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)kSpmvWarps * NS * SB) + warp * NS;
    const int nS = A.S.nSlices;
    const int gw = blockIdx.x * kSpmvWarps + warp;
    const int sFirst = A.warpSlice[gw], sEnd = A.warpSlice[gw + 1];
    // step counts of the warp's first 32 slices (set-up data)
    __shared__ int tSteps[kSpmvWarps][32];
    if (sFirst + lane < sEnd) {
        const int g = sFirst + lane;
        const SellDev<float> &P = g < nS ? A.S : A.X;
        const int sl = g < nS ? g : g - nS;
        tSteps[warp][lane] = (int)((P.slicePtr[sl + 1] - P.slicePtr[sl]) >> 5);
    }
    if (lane == 0) {
        for (int s = 0; s < NS; ++s) mbar_init(bars + s, 1);
        mbar_init_fence();
    }
    // the two parts' step runs: S slices [sFirst, sA), X slices [xa0, xa1)
    const int sA = min(sEnd, nS);
    const int xa0 = max(sFirst, nS) - nS, xa1 = sEnd - nS;
    LeanWalk init;
    init.xPos = xa0 < xa1 ? (A.X.slicePtr[xa0] >> 5) : 0;
    init.xEnd = xa0 < xa1 ? (A.X.slicePtr[xa1] >> 5) : 0;
    if (sFirst < sA) {
        init.isS = 1;
        init.pos = A.S.slicePtr[sFirst] >> 5;
        init.end = A.S.slicePtr[sA] >> 5;
    } else {
        init.isS = 0;
        init.pos = init.xPos;
        init.end = init.xEnd;
    }
    __syncwarp();
    const uint64_t stream = l2_stream_policy();
    const unsigned long long deadline = global_ns() + A.waitNs;

    // producer: every lane walks the schedule, lane 0 issues the copies
    LeanWalk pw = init;
    int issued = 0, pslot = 0;
    bool pmore = true;
    auto issue = [&]() {
        int sS, n;
        long long p;
        if (!pw.next(C, sS, p, n)) {
            pmore = false;
            return;
        }
        if (lane == 0) {
            const SellDev<float> &P = sS ? A.S : A.X;
            unsigned char *dst = ring + pslot * SB;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bars + pslot, (uint32_t)n * 1280u);
            bulk_g2s(dst, P.col + 32 * p, (uint32_t)n * 128u, bars + pslot, stream);
            bulk_g2s(dst + C * 128, P.val + 288 * p, (uint32_t)n * 1152u, bars + pslot, stream);
        }
        ++issued;
        pslot = pslot + 1 == NS ? 0 : pslot + 1;
    };
    // the first stages stream set-up data only: issue them before waiting
    // for the kernel that produced x, unless the run has visibly stopped
    // already (lane 0's early read decides for the warp; the flag read after
    // the wait decides for the launch)
    const bool early = __shfl_sync(0xffffffffu, __ldcg(&sc->done) == kRunning ? 1 : 0, 0) != 0;
    if (early)
        while (pmore && issued < NS) issue();
    pdl_wait();
    if (sc->done != kRunning) {
        const unsigned long long drain = global_ns() + kDrainNs;
        for (int k = 0; k < issued; ++k) mbar_wait(bars + k % NS, (uint32_t)(k / NS) & 1u, drain);
        __syncwarp();
        return;
    }
    if (!early)
        while (pmore && issued < NS) issue();

    // consumer
    float part[1] = {0.0f};
    int sl = sFirst - 1, remS = 0, rpw = 16, h = 0;
    bool own = false, pend = false;
    long long r3 = 0;
    float e0 = 0.0f, e1 = 0.0f, e2 = 0.0f;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
    const float *ev = RES ? b : x;
    auto fetch_row_entries = [&]() {
        pend = false;
        if (own) {
            e0 = ev[r3];
            e1 = ev[r3 + 1];
            e2 = ev[r3 + 2];
        }
    };
    auto finish = [&]() {
        for (int o = rpw; o < 32; o <<= 1) {
            a0 += __shfl_xor_sync(0xffffffffu, a0, o);
            a1 += __shfl_xor_sync(0xffffffffu, a1, o);
            a2 += __shfl_xor_sync(0xffffffffu, a2, o);
        }
        if (pend) fetch_row_entries();
        if (own) {
            if (RES) {
                a0 = e0 - a0;
                a1 = e1 - a1;
                a2 = e2 - a2;
                part[0] += a0 * a0 + a1 * a1 + a2 * a2;
            } else {
                part[0] += e0 * a0 + e1 * a1 + e2 * a2;
            }
            y[r3] = a0;
            y[r3 + 1] = a1;
            y[r3 + 2] = a2;
        }
    };
    // the next slice of the warp: its rows (one per rpw lanes), its steps
    auto next_slice = [&]() {
        if (sl >= sFirst) finish();
        ++sl;
        const bool isS = sl < nS;
        const int tpr = isS ? kTprS : kTprX;
        rpw = 32 / tpr;
        const int rl = (isS ? sl : sl - nS) * rpw + (lane % rpw);
        h = lane / rpw;
        own = rl < (isS ? A.S.nRows : A.X.nRows) && h == 0;
        r3 = own ? 3 * (long long)(isS ? A.S.row[rl] : A.X.row[rl]) : 0;
        pend = true;
        a0 = a1 = a2 = 0.0f;
        if (sl - sFirst < 32) {
            remS = tSteps[warp][sl - sFirst];
        } else {
            const SellDev<float> &P = isS ? A.S : A.X;
            const int ls = isS ? sl : sl - nS;
            remS = (int)((P.slicePtr[ls + 1] - P.slicePtr[ls]) >> 5);
        }
    };
    auto gather = [&](int st, int n, float (&xv)[C][3]) {
        const int *cs = reinterpret_cast<const int *>(ring + st * SB);
#pragma unroll
        for (int t = 0; t < C; ++t) {
            if (t < n) {
                const int c = cs[t * 32 + lane];
                xv[t][0] = __ldg(x + 3 * c);
                xv[t][1] = __ldg(x + 3 * c + 1);
                xv[t][2] = __ldg(x + 3 * c + 2);
            }
        }
    };
    LeanWalk cw = init;
    int curS = 1, curN = 0, nxtS = 1, nxtN = 0, cslot = 0, consumed = 0;
    long long curP = 0, nxtP = 0;
    uint32_t cpar = 0u;
    bool ok = true, have = cw.next(C, curS, curP, curN);
    float xa[C][3], xb[C][3];
    if (have) {
        ok = __all_sync(0xffffffffu, mbar_wait(bars, 0u, deadline));
        if (ok) gather(0, curN, xa);
    }
    // one stage: land and gather the next first, then the FMAs of this one
    // (switching rows where a slice ends), then refill this stage's slot
    auto stage = [&](float (&xc)[C][3], float (&xn)[C][3]) -> bool {
        if (!ok || !have) return false;
        const bool haveN = cw.next(C, nxtS, nxtP, nxtN);
        const int nslot = cslot + 1 == NS ? 0 : cslot + 1;
        const uint32_t npar = nslot == 0 ? cpar ^ 1u : cpar;
        if (haveN) {
            ok = __all_sync(0xffffffffu, mbar_wait(bars + nslot, npar, deadline));
            if (!ok) return false;
            gather(nslot, nxtN, xn);
        }
        const float *vs = reinterpret_cast<const float *>(ring + cslot * SB + C * 128);
#pragma unroll
        for (int t = 0; t < C; ++t) {
            if (t < curN) {
                if (remS == 0) next_slice();
                --remS;
                const float *v = vs + t * 288 + lane;
                a0 = fmaf(v[0], xc[t][0], a0);
                a0 = fmaf(v[32], xc[t][1], a0);
                a0 = fmaf(v[64], xc[t][2], a0);
                a1 = fmaf(v[96], xc[t][0], a1);
                a1 = fmaf(v[128], xc[t][1], a1);
                a1 = fmaf(v[160], xc[t][2], a1);
                a2 = fmaf(v[192], xc[t][0], a2);
                a2 = fmaf(v[224], xc[t][1], a2);
                a2 = fmaf(v[256], xc[t][2], a2);
            }
        }
        __syncwarp();
        if (pmore) issue();
        if (pend) fetch_row_entries();
        ++consumed;
        cslot = nslot;
        cpar = npar;
        curS = nxtS;
        curP = nxtP;
        curN = nxtN;
        have = haveN;
        return true;
    };
    while (stage(xa, xb) && stage(xb, xa)) {
    }
    if (ok) {
        if (sl >= sFirst) finish();
    } else {
        // a copy did not land in time: flag it, give the copies still in
        // flight a bounded chance to land, and leave the shared memory
        if (lane == 0) atomicExch(&sc->fault, 1);
        const unsigned long long drain = global_ns() + kDrainNs;
        for (int k = consumed; k < issued; ++k)
            mbar_wait(bars + k % NS, (uint32_t)(k / NS) & 1u, drain);
        __syncwarp();
    }
    if (fin == kFinDefer) {
        block_sum<float, 1>(part);
        if (threadIdx.x == 0)
            reinterpret_cast<float2 *>(partials)[blockIdx.x] = df_of((double)part[0]);
        return;
    }
    double tot[1];
    if (grid_sum<float, 1>(part, partials, &sc->ticket[0], tot) && threadIdx.x == 0) {
        if (sc->fault)
            sc->done = kFault;
        else
            finalize(sc, fin, slot, tot[0]);
    }
}

// the kernel of a shape: k_spmv_lean for the LEAN shapes, else k_spmv
template <typename T, bool RES, int SHAPE>
constexpr auto spmv_kernel() {
    if constexpr (SpmvCfg<T, SHAPE>::LEAN)
        return k_spmv_lean<RES, SHAPE>;
    else
        return k_spmv<T, RES, SHAPE>;
}

// Persistent grid of a shape: its resident blocks per SM times the SMs (at
// most one warp per slice); < 0 on a CUDA error.
template <typename T, int SHAPE>
int persistent_grid_of(int nSlicesTotal) {
    int dev = 0, sms = 0, nb = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return -1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
    const int smem = spmv_smem_bytes<T, SHAPE>();
    if (cudaFuncSetAttribute(spmv_kernel<T, false, SHAPE>(),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess ||
        cudaFuncSetAttribute(spmv_kernel<T, true, SHAPE>(),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, spmv_kernel<T, false, SHAPE>(),
                                                      kSpmvThreads, smem) != cudaSuccess ||
        nb < 1)
        return -1;
    const int need = (nSlicesTotal + kSpmvWarps - 1) / kSpmvWarps;
    return std::max(1, std::min(nb * sms, need));
}

template <typename T, bool RES, int SHAPE>
void launch_shape(const SpmvDev<T> &A, const T *x, T *y, const T *b, double *partials,
                  Scalars *sc, int fin, int slot, cudaStream_t st) {
    launch_pdl(spmv_kernel<T, RES, SHAPE>(), A.grid, kSpmvThreads, spmv_smem_bytes<T, SHAPE>(), st,
               A, x, y, b, partials, sc, fin, slot);
}

template <typename T>
int spmv_shape_count() { return SpmvShapes<T>::count; }
template int spmv_shape_count<float>();
template int spmv_shape_count<double>();

template <>
int spmv_persistent_grid<float>(int nSlicesTotal, int shape) {
    switch (shape) {
        case 0: return persistent_grid_of<float, 0>(nSlicesTotal);
        case 1: return persistent_grid_of<float, 1>(nSlicesTotal);
        case 2: return persistent_grid_of<float, 2>(nSlicesTotal);
        case 3: return persistent_grid_of<float, 3>(nSlicesTotal);
        case 4: return persistent_grid_of<float, 4>(nSlicesTotal);
        case 5: return persistent_grid_of<float, 5>(nSlicesTotal);
        case 6: return persistent_grid_of<float, 6>(nSlicesTotal);
        case 7: return persistent_grid_of<float, 7>(nSlicesTotal);
    }
    return -1;
}
template <>
int spmv_persistent_grid<double>(int nSlicesTotal, int shape) {
    switch (shape) {
        case 0: return persistent_grid_of<double, 0>(nSlicesTotal);
        case 1: return persistent_grid_of<double, 1>(nSlicesTotal);
        case 2: return persistent_grid_of<double, 2>(nSlicesTotal);
        case 3: return persistent_grid_of<double, 3>(nSlicesTotal);
    }
    return -1;
}

template <typename T, bool RES>
void launch_spmv_res(const SpmvDev<T> &A, const T *x, T *y, const T *b, double *partials,
                     Scalars *sc, int fin, int slot, cudaStream_t st) {
    switch (A.shape) {
        case 1: launch_shape<T, RES, 1>(A, x, y, b, partials, sc, fin, slot, st); return;
        case 2: launch_shape<T, RES, 2>(A, x, y, b, partials, sc, fin, slot, st); return;
        case 3: launch_shape<T, RES, 3>(A, x, y, b, partials, sc, fin, slot, st); return;
        case 4:
        case 5:
        case 6:
        case 7:
            if constexpr (SpmvShapes<T>::count > 7) {
                switch (A.shape) {
                    case 4: launch_shape<T, RES, 4>(A, x, y, b, partials, sc, fin, slot, st); return;
                    case 5: launch_shape<T, RES, 5>(A, x, y, b, partials, sc, fin, slot, st); return;
                    case 6: launch_shape<T, RES, 6>(A, x, y, b, partials, sc, fin, slot, st); return;
                    default: launch_shape<T, RES, 7>(A, x, y, b, partials, sc, fin, slot, st); return;
                }
            }
            break;
        default: break;
    }
    launch_shape<T, RES, 0>(A, x, y, b, partials, sc, fin, slot, st);
}

template <typename T>
void launch_spmv(const SpmvDev<T> &A, const T *x, T *y, const T *b, int residual_mode,
                 double *partials, Scalars *sc, int fin, int slot, cudaStream_t st) {
    if (residual_mode)
        launch_spmv_res<T, true>(A, x, y, b, partials, sc, fin, slot, st);
    else
        launch_spmv_res<T, false>(A, x, y, b, partials, sc, fin, slot, st);
}

template void launch_spmv<double>(const SpmvDev<double> &, const double *, double *,
                                  const double *, int, double *, Scalars *, int, int, cudaStream_t);
template void launch_spmv<float>(const SpmvDev<float> &, const float *, float *, const float *,
                                 int, double *, Scalars *, int, int, cudaStream_t);

// ---- dot products and mixed-precision conversions -------------------------

int device_sm_count() {
    constexpr int kMaxDev = 64;
    static int cache[kMaxDev] = {0};   // 0 = not queried yet; every writer stores the same value
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < kMaxDev && cache[dev] > 0) return cache[dev];
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return 1;
    if (dev < kMaxDev) cache[dev] = sms;
    return sms;
}


template <typename T>
__global__ void __launch_bounds__(kThreads)
k_dot(const T *__restrict__ a, const T *__restrict__ b, long long n, double *partials,
      Scalars *sc, int fin, int slot) {
    T part[1] = {T(0)};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        part[0] = fma(a[i], b[i], part[0]);
    double tot[1];
    if (grid_sum<T, 1>(part, partials, &sc->ticket[1], tot) && threadIdx.x == 0)
        finalize(sc, fin, slot, tot[0]);
}

template <typename T>
void launch_dot(const T *a, const T *b, long long n, double *partials, Scalars *sc, int fin,
                int slot, cudaStream_t st) {
    k_dot<T><<<2 * device_sm_count(), kThreads, 0, st>>>(a, b, n, partials, sc, fin, slot);
}
template void launch_dot<double>(const double *, const double *, long long, double *, Scalars *,
                                 int, int, cudaStream_t);
template void launch_dot<float>(const float *, const float *, long long, double *, Scalars *, int,
                                int, cudaStream_t);

static int grid_for(long long n) {
    const long long g = (n + kThreads - 1) / kThreads, cap = 4LL * device_sm_count();
    return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

__global__ void k_cast_f32(const double *__restrict__ a, float *__restrict__ b, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        b[i] = (float)a[i];
}

void launch_cast_f32(const double *a, float *b, long long n, cudaStream_t st) {
    if (n > 0) k_cast_f32<<<grid_for(n), kThreads, 0, st>>>(a, b, n);
}

}  // namespace xdcg
