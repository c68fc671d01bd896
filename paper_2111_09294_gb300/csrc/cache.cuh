// L2 residency hints.  Per iteration the FP32 path streams the matrix of
// K~ (about 170 MB at n = 373k, read once per product, evict-first loads)
// and re-reads a much smaller set: E^-1 (k^2 floats), the box blocks of
// Z~ and W~ and their row maps.  Loads of that set carry an evict-last L2
// cache policy (PTX createpolicy + ld.global.L2::cache_hint), so it tends to
// survive the matrix stream in the 129 MB L2 from one iteration to the next.
#pragma once

#include <cstdint>

namespace xdcg {

__device__ __forceinline__ uint64_t l2_keep_policy() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ float ld_keep(const float *a, uint64_t pol) {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ int ld_keep(const int *a, uint64_t pol) {
    int v;
    asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ float4 ld_keep(const float4 *a, uint64_t pol) {
    float4 v;
    asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(a), "l"(pol));
    return v;
}

}  // namespace xdcg
