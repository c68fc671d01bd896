// Pipeline shapes of the bulk-copy SpMV kernels (single and batched).
#pragma once

#include "internal.h"

namespace xdcg {

// A shape: C steps per stage, NS stages per warp, MINB resident blocks per
// SM.  A step is one 32-lane column of the slice: 32 column indices and 9
// planes of 32 values (1280 bytes in FP32, 2432 in FP64).  GUARD skips the
// arithmetic of padding slots: worth a per-slice row length load in FP64,
// whose FMAs run at 1/64 of the FP32 rate on this GPU and bound the FP64
// product as much as its bytes do.  Shape 0 of each precision is the
// default; the others are the candidates the set-up autotuner times on the
// context's own matrix (xdcg_options.autotune).
template <int C_, int NS_, int MINB_>
struct SpmvShapeOf {
    static constexpr int C = C_, NS = NS_, MINB = MINB_;
};
template <typename T, int SHAPE> struct SpmvCfg;
template <> struct SpmvCfg<float, 0> : SpmvShapeOf<2, 3, 3> { static constexpr bool GUARD = false; };
template <> struct SpmvCfg<float, 1> : SpmvShapeOf<1, 4, 4> { static constexpr bool GUARD = false; };
template <> struct SpmvCfg<float, 2> : SpmvShapeOf<2, 4, 2> { static constexpr bool GUARD = false; };
template <> struct SpmvCfg<float, 3> : SpmvShapeOf<1, 6, 3> { static constexpr bool GUARD = false; };
template <> struct SpmvCfg<float, 4> : SpmvShapeOf<3, 3, 2> { static constexpr bool GUARD = false; };
template <> struct SpmvCfg<double, 0> : SpmvShapeOf<1, 3, 3> { static constexpr bool GUARD = true; };
template <> struct SpmvCfg<double, 1> : SpmvShapeOf<1, 4, 2> { static constexpr bool GUARD = true; };
template <> struct SpmvCfg<double, 2> : SpmvShapeOf<2, 2, 2> { static constexpr bool GUARD = true; };
template <> struct SpmvCfg<double, 3> : SpmvShapeOf<1, 2, 4> { static constexpr bool GUARD = true; };

template <typename T> struct SpmvShapes;
template <> struct SpmvShapes<float> { static constexpr int count = 5; };
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
