// FP32 inner solve of the mixed-precision path, run on the block-scaled
// system  K~ = L^-1 K L^-T,  f~ = L^-1 r,  u = L^-T u~,  with L the FP64
// Cholesky factors of the node blocks (Eqs. block_jacobi, block_jacobi_enr).
//
// With M = L L^T the block-Jacobi preconditioner of Algorithm 3 becomes the
// identity, the deflation basis becomes Z~ = L^T Z, W~ = K~ Z~ = L^-1 W, and
// E = Z~^T K~ Z~ = Z^T K Z is unchanged; A-DEF2 on the scaled system produces
// the same iterates as on the original one in exact arithmetic.  In FP32 the
// scaling matters: the near-dependent enriched directions that give K its
// ~1e9 condition number are scaled out, so p^T K~ p stays positive where the
// unscaled FP32 recurrence breaks down.
#include "factor.cuh"
#include "reduce.cuh"

namespace xdcg {

// ---- set-up -----------------------------------------------------------------

__global__ void k_gather_f64(const int *__restrict__ src, long long n, const double *__restrict__ v,
                             double *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int s = src[i];
        out[i] = s >= 0 ? v[s] : 0.0;
    }
}

__global__ void k_gather_f32(const int *__restrict__ src, long long n, const double *__restrict__ v,
                             float *out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int s = src[i];
        out[i] = s >= 0 ? (float)v[s] : 0.0f;
    }
}

static int grid_of(long long n, int th) {
    const long long g = (n + th - 1) / th, cap = 8LL * device_sm_count();
    return (int)(g < cap ? (g > 0 ? g : 1) : cap);
}

void launch_gather(const int *src, long long n, const double *v, double *out64, float *out32,
                   cudaStream_t st) {
    if (n <= 0) return;
    if (out64) k_gather_f64<<<grid_of(n, 256), 256, 0, st>>>(src, n, v, out64);
    if (out32) k_gather_f32<<<grid_of(n, 256), 256, 0, st>>>(src, n, v, out32);
}

// K~_IJ = L_I^-1 K_IJ L_J^-T for every node-pair block, in place on a copy of K.
__global__ void k_scale_blocks(KinDev K, const int *__restrict__ blockRow, long long nnzb,
                               FacDev F, double *Kt) {
    const long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (p >= nnzb) return;
    const int I = blockRow[p], J = K.col[p];
    const int bI = K.dofStart[I + 1] - K.dofStart[I], bJ = K.dofStart[J + 1] - K.dofStart[J];
    double *B = Kt + K.valPtr[p];                       // bI x bJ, row-major
    const int lI = F.nodeList[I], tI = F.nodeIdx[I], lJ = F.nodeList[J], tJ = F.nodeIdx[J];
    for (int c = 0; c < bJ; ++c) fwd_solve(F, lI, tI, bI, B + c, bJ);   // columns: L_I^-1 B
    for (int r = 0; r < bI; ++r) fwd_solve(F, lJ, tJ, bJ, B + r * bJ, 1); // rows: (.) L_J^-T
}

void launch_scale_blocks(const KinDev &K, const int *blockRow, long long nnzb, const FacDev &F,
                         double *Kt, cudaStream_t st) {
    if (nnzb <= 0) return;
    k_scale_blocks<<<(int)((nnzb + 127) / 128), 128, 0, st>>>(K, blockRow, nnzb, F, Kt);
}

// deflation row j of a node (same rule as the unscaled path)
__device__ __forceinline__ void zrow(int j, int b, int menr, double X, double Y, double Z,
                                     double H, double (&o)[12]) {
#pragma unroll
    for (int c = 0; c < 12; ++c) o[c] = 0.0;
    const bool stdd = j < 3, jump = (b == 6 && j >= 3 && menr);
    if (!stdd && !jump) return;
    const int a = stdd ? j : j - 3;
    double r[6] = {0, 0, 0, 0, 0, 0};
    if (a == 0) { r[0] = 1.0; r[4] = Z; r[5] = -Y; }
    if (a == 1) { r[1] = 1.0; r[3] = -Z; r[5] = X; }
    if (a == 2) { r[2] = 1.0; r[3] = Y; r[4] = -X; }
    if (stdd) {
#pragma unroll
        for (int c = 0; c < 6; ++c) o[c] = r[c];
        if (menr) {
#pragma unroll
            for (int c = 0; c < 6; ++c) o[6 + c] = H * r[c];
        }
    } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) o[6 + c] = r[c];
    }
}

// Z~_I = L_I^T Z_I (b_I x M, row-major at zOff[t] for slot t holding node I), FP32.
__global__ void k_build_Zt(int nSlots, const int *slotNode, const int *dofStart, const int *sub,
                           const double *xrel, const signed char *hsign, const int *menr,
                           ZvalDev Zv, FacDev F, const long long *zOff, float *Zt) {
    const int ts = blockIdx.x * blockDim.x + threadIdx.x;
    if (ts >= nSlots) return;
    const int I = slotNode[ts];
    const int b = dofStart[I + 1] - dofStart[I];
    const int s = sub[I], me = menr[s], M = me ? 12 : 6;
    const double X = xrel[3 * I], Y = xrel[3 * I + 1], Z = xrel[3 * I + 2], H = hsign[I];
    const int l = F.nodeList[I], t = F.nodeIdx[I];
    double acc[15 * 12];
    for (int e = 0; e < b * M; ++e) acc[e] = 0.0;
    for (int j = 0; j < b; ++j) {
        double zr[12];
        if (Zv.v) {
            const double *r = Zv.v + Zv.off[I] + (long long)j * M;
            for (int c = 0; c < 12; ++c) zr[c] = c < M ? r[c] : 0.0;
        } else {
            zrow(j, b, me, X, Y, Z, H, zr);
        }
        bool any = false;
        for (int c = 0; c < M; ++c) any |= zr[c] != 0.0;
        if (!any) continue;
        for (int i = 0; i <= j; ++i) {
            const double lji = (i == j) ? 1.0 / Lent(F, l, t, j, j) : Lent(F, l, t, j, i);
            for (int c = 0; c < M; ++c) acc[i * M + c] += lji * zr[c];
        }
    }
    float *out = Zt + zOff[ts];
    for (int e = 0; e < b * M; ++e) out[e] = (float)acc[e];
}

void launch_build_Zt(int nSlots, const int *slotNode, const int *dofStart, const int *sub,
                     const double *xrel, const signed char *hsign, const int *menr,
                     const ZvalDev &Zv, const FacDev &F, const long long *zOff, float *Zt,
                     cudaStream_t st) {
    k_build_Zt<<<(nSlots + 127) / 128, 128, 0, st>>>(nSlots, slotNode, dofStart, sub, xrel, hsign,
                                                     menr, Zv, F, zOff, Zt);
}

// W~ = L^-1 W per W entry (b_I x M), FP32.
__global__ void k_scale_W(int nExt, const int *extBox, const int *extNode, const long long *wOff,
                          const int *menr, const int *dofStart, FacDev F, const double *W,
                          float *Wt) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nExt) return;
    const int I = extNode[e], M = menr[extBox[e]] ? 12 : 6;
    const int b = dofStart[I + 1] - dofStart[I];
    const int l = F.nodeList[I], t = F.nodeIdx[I];
    const double *Wb = W + wOff[e];
    for (int c = 0; c < M; ++c) {
        double x[15];
        for (int i = 0; i < b; ++i) x[i] = Wb[i * M + c];
        fwd_solve(F, l, t, b, x, 1);
        for (int i = 0; i < b; ++i) Wt[wOff[e] + i * M + c] = (float)x[i];
    }
}

void launch_scale_W(int nExt, const int *extBox, const int *extNode, const long long *wOff,
                    const int *menr, const int *dofStart, const FacDev &F, const double *W,
                    float *Wt, cudaStream_t st) {
    if (nExt == 0) return;
    k_scale_W<<<(nExt + 127) / 128, 128, 0, st>>>(nExt, extBox, extNode, wOff, menr, dofStart, F,
                                                  W, Wt);
}

// ---- outer-loop transforms (FP64) -----------------------------------------

// out = (float)(s L^-1 r) per node
// Node I has nat[I + 1] - nat[I] dofs (nat: the caller's numbering, where
// each node's dofs are consecutive and nodes follow one another); `in` and
// `ot` give where its dofs start in the input and the output vector.

// out = s L^-1 r per node
__global__ void k_fwd_scale(int nNodes, const int *nat, const int *in, const int *ot, FacDev F,
                            const double *r, double s, float *out) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nNodes) return;
    const int b = nat[I + 1] - nat[I], d0 = in[I], o0 = ot[I];
    const int t = F.nodeIdx[I];
    with_node_size(b, [&](auto Bc) {
        constexpr int B = decltype(Bc)::value;
        double x[B];
#pragma unroll
        for (int i = 0; i < B; ++i) x[i] = r[d0 + i];
        fwd_solve_fixed<B>(F, t, x);
#pragma unroll
        for (int i = 0; i < B; ++i) out[o0 + i] = (float)(s * x[i]);
    });
}

void launch_fwd_scale(int nNodes, const int *nat, const int *in, const int *ot, const FacDev &F,
                      const double *r, double s, float *out, cudaStream_t st) {
    k_fwd_scale<<<(nNodes + 127) / 128, 128, 0, st>>>(nNodes, nat, in, ot, F, r, s, out);
}

// u += scale L^-T ut per node
__global__ void k_bwd_accum(int nNodes, const int *nat, const int *in, const int *ot, FacDev F,
                            const float *ut, double scale, double *u) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nNodes) return;
    const int b = nat[I + 1] - nat[I], d0 = in[I], o0 = ot[I];
    const int t = F.nodeIdx[I];
    with_node_size(b, [&](auto Bc) {
        constexpr int B = decltype(Bc)::value;
        double x[B];
#pragma unroll
        for (int i = 0; i < B; ++i) x[i] = (double)ut[d0 + i];
        bwd_solve_fixed<B>(F, t, x);
#pragma unroll
        for (int i = 0; i < B; ++i) u[o0 + i] += scale * x[i];
    });
}

void launch_bwd_accum(int nNodes, const int *nat, const int *in, const int *ot, const FacDev &F,
                      const float *ut, double scale, double *u, cudaStream_t st) {
    k_bwd_accum<<<(nNodes + 127) / 128, 128, 0, st>>>(nNodes, nat, in, ot, F, ut, scale, u);
}

// out = x renumbered node by node (FP32 vectors)
__global__ void k_renumber(int nNodes, const int *nat, const int *in, const int *ot,
                           const float *x, float *out) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x;
    if (I >= nNodes) return;
    const int b = nat[I + 1] - nat[I], d0 = in[I], o0 = ot[I];
    for (int i = 0; i < b; ++i) out[o0 + i] = x[d0 + i];
}

void launch_renumber(int nNodes, const int *nat, const int *in, const int *ot, const float *x,
                     float *out, cudaStream_t st) {
    k_renumber<<<(nNodes + 127) / 128, 128, 0, st>>>(nNodes, nat, in, ot, x, out);
}

}  // namespace xdcg
