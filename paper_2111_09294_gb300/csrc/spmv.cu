// Chunked node-blocked SpMV q = K p (Algorithm 1, the product K p_i) with
// the fused partial of p^T q, plus the plain vector kernels of the solve.
//
// K is stored as 3x3 blocks between "chunks" (3 consecutive dofs: the
// standard dofs of a node, its jump dofs, or one branch function's 3 dofs),
// so standard and enriched couplings of Eq. linear_system stream through the
// same code.  Values and column indices are read once per product with
// evict-first loads; the gathered x chunks stay in L1/L2.
#include "reduce.cuh"

namespace xdcg {

template <typename T>
__device__ __forceinline__ T ldcs(const T *p) { return __ldcs(p); }

// One slice of TPR-threads-per-row sliced ELL; returns this lane's share of
// the fused dot (x^T y, or y^T y in residual mode) in part.
template <typename T, bool RES, int TPR>
__device__ __forceinline__ void sell_slice(const SellDev<T> &P, int slice, int lane,
                                           const T *__restrict__ x, T *__restrict__ y,
                                           const T *__restrict__ b, T &part) {
    constexpr int RPW = 32 / TPR;
    const int rr = lane % RPW, h = lane / RPW;
    const int rl = slice * RPW + rr;
    const bool valid = rl < P.nRows;
    const int len = valid ? P.len[rl] : 0;
    long long base, cstep, vstep, ve;
    int steps;
    if (P.ilvSteps > 0) {             // interleaved: all slices step together
        base = 32LL * slice;
        steps = P.ilvSteps;
        cstep = 32LL * P.nSlices;
        ve = cstep;
        vstep = 9 * cstep;
    } else {                          // slice-blocked
        base = P.slicePtr[slice];
        steps = (int)((P.slicePtr[slice + 1] - base) >> 5);
        cstep = 32;
        ve = 32;
        vstep = 288;
    }
    const int *cp = P.col + base + lane;
    const T *vp = P.val + (P.ilvSteps > 0 ? base : 9 * base) + lane;
    T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll 4
    for (int st = 0; st < steps; ++st) {
        if (st * TPR + h < len) {
            const int c = __ldcs(cp + cstep * st);
            const T *v = vp + vstep * st;
            const T x0 = __ldg(x + 3 * c), x1 = __ldg(x + 3 * c + 1), x2 = __ldg(x + 3 * c + 2);
            a0 = fma(ldcs(v), x0, a0);
            a0 = fma(ldcs(v + ve), x1, a0);
            a0 = fma(ldcs(v + 2 * ve), x2, a0);
            a1 = fma(ldcs(v + 3 * ve), x0, a1);
            a1 = fma(ldcs(v + 4 * ve), x1, a1);
            a1 = fma(ldcs(v + 5 * ve), x2, a1);
            a2 = fma(ldcs(v + 6 * ve), x0, a2);
            a2 = fma(ldcs(v + 7 * ve), x1, a2);
            a2 = fma(ldcs(v + 8 * ve), x2, a2);
        }
    }
#pragma unroll
    for (int o = RPW; o < 32; o <<= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if (valid && h == 0) {
        const long long r3 = 3 * (long long)P.row[rl];
        if (RES) {
            a0 = b[r3] - a0;
            a1 = b[r3 + 1] - a1;
            a2 = b[r3 + 2] - a2;
            part = a0 * a0 + a1 * a1 + a2 * a2;
        } else {
            part = x[r3] * a0 + x[r3 + 1] * a1 + x[r3 + 2] * a2;
        }
        y[r3] = a0;
        y[r3 + 1] = a1;
        y[r3 + 2] = a2;
    }
}

template <typename T, bool RES>
__global__ void __launch_bounds__(kSpmvThreads)
k_spmv(SpmvDev<T> A, const T *__restrict__ x, T *__restrict__ y, const T *__restrict__ b,
       int nbS, double *partials, Scalars *sc, int fin, int slot) {
    if (sc->done != kRunning) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T part[1] = {T(0)};
    if ((int)blockIdx.x < nbS) {
        const int slice = blockIdx.x * kSpmvWarps + warp;
        if (slice < A.S.nSlices) sell_slice<T, RES, kTprS>(A.S, slice, lane, x, y, b, part[0]);
    } else {
        const int slice = (blockIdx.x - nbS) * kSpmvWarps + warp;
        if (slice < A.X.nSlices) sell_slice<T, RES, kTprX>(A.X, slice, lane, x, y, b, part[0]);
    }
    double tot[1];
    if (grid_sum<T, 1>(part, partials, &sc->ticket[0], tot) && threadIdx.x == 0)
        finalize(sc, fin, slot, tot[0]);
}

int spmv_grid(int nSlicesS, int nSlicesX) {
    return (nSlicesS + kSpmvWarps - 1) / kSpmvWarps + (nSlicesX + kSpmvWarps - 1) / kSpmvWarps;
}

template <typename T>
void launch_spmv(const SpmvDev<T> &A, const T *x, T *y, const T *b, int residual_mode,
                 double *partials, Scalars *sc, int fin, int slot, cudaStream_t st) {
    const int nbS = (A.S.nSlices + kSpmvWarps - 1) / kSpmvWarps;
    const int grid = spmv_grid(A.S.nSlices, A.X.nSlices);
    if (residual_mode)
        k_spmv<T, true><<<grid, kSpmvThreads, 0, st>>>(A, x, y, b, nbS, partials, sc, fin, slot);
    else
        k_spmv<T, false><<<grid, kSpmvThreads, 0, st>>>(A, x, y, b, nbS, partials, sc, fin, slot);
}

template void launch_spmv<double>(const SpmvDev<double> &, const double *, double *,
                                  const double *, int, double *, Scalars *, int, int, cudaStream_t);
template void launch_spmv<float>(const SpmvDev<float> &, const float *, float *, const float *,
                                 int, double *, Scalars *, int, int, cudaStream_t);

// ---- dot products and mixed-precision conversions -------------------------

constexpr int kDotBlocks = 304;   // 2 x 152 SMs

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
    k_dot<T><<<kDotBlocks, kThreads, 0, st>>>(a, b, n, partials, sc, fin, slot);
}
template void launch_dot<double>(const double *, const double *, long long, double *, Scalars *,
                                 int, int, cudaStream_t);
template void launch_dot<float>(const float *, const float *, long long, double *, Scalars *, int,
                                int, cudaStream_t);

__global__ void k_scale_to_f32(const double *__restrict__ r64, float *__restrict__ r32,
                               long long n, double s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        r32[i] = (float)(r64[i] * s);
}

__global__ void k_accumulate_f64(double *__restrict__ u64, const float *__restrict__ d32,
                                 long long n, double s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        u64[i] += s * (double)d32[i];
}

static int grid_for(long long n) {
    long long g = (n + kThreads - 1) / kThreads;
    return (int)(g < 4 * 152 ? (g > 0 ? g : 1) : 4 * 152);
}

void launch_scale_to_f32(const double *r64, float *r32, long long n, double s, cudaStream_t st) {
    k_scale_to_f32<<<grid_for(n), kThreads, 0, st>>>(r64, r32, n, s);
}

void launch_accumulate_f64(double *u64, const float *d32, long long n, double s, cudaStream_t st) {
    k_accumulate_f64<<<grid_for(n), kThreads, 0, st>>>(u64, d32, n, s);
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
