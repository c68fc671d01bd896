// Pipeline shape of the bulk-copy SpMV kernels (single and batched).
#pragma once

#include "internal.h"

namespace xdcg {

// Per-precision pipeline shape: C steps per stage, NS stages per warp, MINB
// resident blocks per SM.  A step is one 32-lane column of the slice: 32
// column indices and 9 planes of 32 values (1280 bytes in FP32, 2432 in
// FP64).  GUARD skips the arithmetic of padding slots: worth a per-slice row
// length load in FP64, whose FMAs run at 1/64 of the FP32 rate on this GPU
// and bound the FP64 product as much as its bytes do.
template <typename T> struct SpmvCfg;
template <> struct SpmvCfg<float> {
    static constexpr int C = 2, NS = 3, MINB = 3;
    static constexpr bool GUARD = false;
};
template <> struct SpmvCfg<double> {
    static constexpr int C = 1, NS = 3, MINB = 3;
    static constexpr bool GUARD = true;
};

template <typename T>
__host__ __device__ constexpr int stage_bytes() { return SpmvCfg<T>::C * (128 + 288 * (int)sizeof(T)); }

template <typename T>
__host__ __device__ constexpr int spmv_smem_bytes() {
    return kSpmvWarps * SpmvCfg<T>::NS * (stage_bytes<T>() + 8 + 3 * 4);
}

}  // namespace xdcg
