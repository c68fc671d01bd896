// Programmatic dependent launch.  The kernels of the iteration loop are
// launched with programmatic stream serialisation: a kernel's blocks may be
// launched while its predecessor drains (each predecessor block counts as
// triggered when it exits; an explicit trigger, at kernel start or after a
// block's main work, measured slower), and
// they wait (griddepcontrol.wait) for the predecessor's completion and
// memory before touching anything it wrote.  Work that reads only set-up
// data (the SpMV's matrix stream) runs before the wait.  The wait is a no-op
// for a kernel launched without the attribute.
#pragma once

#include <cuda_runtime.h>

namespace xdcg {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), int grid, int block, size_t smem,
                       cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace xdcg
