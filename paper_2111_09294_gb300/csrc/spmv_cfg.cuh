// Pipeline shapes of the bulk-copy SpMV kernels (single and batched).
#pragma once

#include "internal.h"

namespace xdcg {

// A shape: C steps per stage, NS stages per warp, MINB resident blocks per
// SM.  A step is one 32-lane column of the slice: 32 column indices and 9
// planes of 32 values (1280 bytes in FP32, 2432 in FP64).  GUARD skips the
// arithmetic of padding slots: worth a per-slice row length load in FP64,
// whose FMAs run at 1/64 of the FP32 rate on this GPU and bound the FP64
// product as much as its bytes do.  A context runs its precision's default
// shape (kSpmvDefaultShape*, internal.h) unless the set-up autotuner, which
// times every shape on the context's own matrix (xdcg_options.autotune),
// finds a faster one, or the caller pins one (xdcg_options.spmv_shape_*).
template <int C_, int NS_, int MINB_>
struct SpmvShapeOf {
    static constexpr int C = C_, NS = NS_, MINB = MINB_;
};
// LEAN shapes (FP32 only) run k_spmv_lean: stages of a fixed step count that
// run across slice boundaries, no per-stage metadata, the copy schedule
// walked by every lane (lane 0 issues the copies), the row switch tested per
// step; the same data layout, ring and arithmetic order per row.
template <typename T, int SHAPE> struct SpmvCfg;
template <bool G, bool L> struct SpmvFlags {
    static constexpr bool GUARD = G, LEAN = L;
};
template <> struct SpmvCfg<float, 0> : SpmvShapeOf<2, 3, 3>, SpmvFlags<false, false> {};
template <> struct SpmvCfg<float, 1> : SpmvShapeOf<1, 4, 4>, SpmvFlags<false, false> {};
template <> struct SpmvCfg<float, 2> : SpmvShapeOf<2, 4, 2>, SpmvFlags<false, false> {};
template <> struct SpmvCfg<float, 3> : SpmvShapeOf<1, 6, 3>, SpmvFlags<false, false> {};
template <> struct SpmvCfg<float, 4> : SpmvShapeOf<3, 3, 2>, SpmvFlags<false, false> {};
template <> struct SpmvCfg<float, 5> : SpmvShapeOf<2, 3, 3>, SpmvFlags<false, true> {};
template <> struct SpmvCfg<float, 6> : SpmvShapeOf<1, 6, 3>, SpmvFlags<false, true> {};
template <> struct SpmvCfg<float, 7> : SpmvShapeOf<2, 2, 4>, SpmvFlags<false, true> {};
template <> struct SpmvCfg<double, 0> : SpmvShapeOf<1, 3, 3>, SpmvFlags<true, false> {};
template <> struct SpmvCfg<double, 1> : SpmvShapeOf<1, 4, 2>, SpmvFlags<true, false> {};
template <> struct SpmvCfg<double, 2> : SpmvShapeOf<2, 2, 2>, SpmvFlags<true, false> {};
template <> struct SpmvCfg<double, 3> : SpmvShapeOf<1, 2, 4>, SpmvFlags<true, false> {};

template <typename T> struct SpmvShapes;
template <> struct SpmvShapes<float> { static constexpr int count = 8; };
template <> struct SpmvShapes<double> { static constexpr int count = 4; };

template <typename T, int SHAPE>
__host__ __device__ constexpr int stage_bytes() {
    return SpmvCfg<T, SHAPE>::C * (128 + 288 * (int)sizeof(T));
}

template <typename T, int SHAPE>
__host__ __device__ constexpr int spmv_smem_bytes() {
    return kSpmvWarps * SpmvCfg<T, SHAPE>::NS * (stage_bytes<T, SHAPE>() + 8 + 3 * 4);
}

}  // namespace xdcg
