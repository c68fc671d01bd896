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

template <typename T, bool RES>
__global__ void __launch_bounds__(kThreads)
k_spmv(SpmvDev<T> A, const T *__restrict__ x, T *__restrict__ y, const T *__restrict__ b,
       int nbS, double *partials, Scalars *sc, int fin, int slot) {
    if (sc->done != kRunning) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T part[1] = {T(0)};
    if ((int)blockIdx.x < nbS) {
        const int slice = blockIdx.x * kWarps + warp;
        const int rl = slice * 32 + lane;
        if (slice < A.nSlices && rl < A.nS) {
            const int row = A.rowS[rl];
            const int len = A.lenS[rl];
            const long long base = A.slicePtr[slice];
            const int *cp = A.colS + base + lane;
            const T *vp = A.valS + 9 * base + lane;
            T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll 4
            for (int j = 0; j < len; ++j) {
                const int c = __ldcs(cp + 32 * j);
                const T *v = vp + 288 * j;
                const T x0 = __ldg(x + 3 * c), x1 = __ldg(x + 3 * c + 1), x2 = __ldg(x + 3 * c + 2);
                a0 = fma(ldcs(v), x0, a0);
                a0 = fma(ldcs(v + 32), x1, a0);
                a0 = fma(ldcs(v + 64), x2, a0);
                a1 = fma(ldcs(v + 96), x0, a1);
                a1 = fma(ldcs(v + 128), x1, a1);
                a1 = fma(ldcs(v + 160), x2, a1);
                a2 = fma(ldcs(v + 192), x0, a2);
                a2 = fma(ldcs(v + 224), x1, a2);
                a2 = fma(ldcs(v + 256), x2, a2);
            }
            T *yr = y + 3 * (long long)row;
            if (RES) {
                const T *br = b + 3 * (long long)row;
                a0 = br[0] - a0;
                a1 = br[1] - a1;
                a2 = br[2] - a2;
                part[0] = a0 * a0 + a1 * a1 + a2 * a2;
            } else {
                const T *xr = x + 3 * (long long)row;
                part[0] = xr[0] * a0 + xr[1] * a1 + xr[2] * a2;
            }
            yr[0] = a0;
            yr[1] = a1;
            yr[2] = a2;
        }
    } else {
        const int xi = (blockIdx.x - nbS) * kWarps + warp;
        if (xi < A.nX) {
            const int row = A.rowX[xi];
            const int len = A.lenX[xi];
            const long long base = A.ptrX[xi];
            T a0 = T(0), a1 = T(0), a2 = T(0);
            for (int t = lane; t < len; t += 32) {
                const int c = __ldcs(A.colX + base + t);
                const T *v = A.valX + 9 * base + 288 * (t >> 5) + (t & 31);
                const T x0 = __ldg(x + 3 * c), x1 = __ldg(x + 3 * c + 1), x2 = __ldg(x + 3 * c + 2);
                a0 = fma(ldcs(v), x0, a0);
                a0 = fma(ldcs(v + 32), x1, a0);
                a0 = fma(ldcs(v + 64), x2, a0);
                a1 = fma(ldcs(v + 96), x0, a1);
                a1 = fma(ldcs(v + 128), x1, a1);
                a1 = fma(ldcs(v + 160), x2, a1);
                a2 = fma(ldcs(v + 192), x0, a2);
                a2 = fma(ldcs(v + 224), x1, a2);
                a2 = fma(ldcs(v + 256), x2, a2);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a0 += __shfl_xor_sync(0xffffffffu, a0, o);
                a1 += __shfl_xor_sync(0xffffffffu, a1, o);
                a2 += __shfl_xor_sync(0xffffffffu, a2, o);
            }
            if (lane == 0) {
                T *yr = y + 3 * (long long)row;
                if (RES) {
                    const T *br = b + 3 * (long long)row;
                    a0 = br[0] - a0;
                    a1 = br[1] - a1;
                    a2 = br[2] - a2;
                    part[0] = a0 * a0 + a1 * a1 + a2 * a2;
                } else {
                    const T *xr = x + 3 * (long long)row;
                    part[0] = xr[0] * a0 + xr[1] * a1 + xr[2] * a2;
                }
                yr[0] = a0;
                yr[1] = a1;
                yr[2] = a2;
            }
        }
    }
    double tot[1];
    if (grid_sum<T, 1>(part, partials, &sc->ticket[0], tot) && threadIdx.x == 0)
        finalize(sc, fin, slot, tot[0]);
}

int spmv_grid(int nSlices, int nX) {
    return (nSlices + kWarps - 1) / kWarps + (nX + kWarps - 1) / kWarps;
}

template <typename T>
void launch_spmv(const SpmvDev<T> &A, const T *x, T *y, const T *b, int residual_mode,
                 double *partials, Scalars *sc, int fin, int slot, cudaStream_t st) {
    const int nbS = (A.nSlices + kWarps - 1) / kWarps;
    const int grid = spmv_grid(A.nSlices, A.nX);
    if (residual_mode)
        k_spmv<T, true><<<grid, kThreads, 0, st>>>(A, x, y, b, nbS, partials, sc, fin, slot);
    else
        k_spmv<T, false><<<grid, kThreads, 0, st>>>(A, x, y, b, nbS, partials, sc, fin, slot);
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
