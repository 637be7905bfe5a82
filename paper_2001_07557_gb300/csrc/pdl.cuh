// pdl.cuh -- programmatic dependent launch for the kernels of the solvers.
//
// A kernel launched with launch_pdl may be scheduled while the kernel before it
// in the stream is still draining: its blocks become resident as SMs free up
// and then wait in pdl_enter() until that kernel has completed and its writes
// are visible.  This removes most of the gap between consecutive kernels of a
// solver iteration (launch latency and the ramp of the next grid).
//
// Contract: every kernel launched with launch_pdl calls pdl_enter() before its
// first access to global memory.  A kernel whose predecessor is not a kernel
// (a copy, a memset, an event wait) is ordered as usual, and so is every
// dependency across streams.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace lq {

// Wait for the previous grid of the stream, then allow the next launch of the
// stream to be scheduled behind this one.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace lq
