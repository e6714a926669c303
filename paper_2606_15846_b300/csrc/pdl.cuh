// Programmatic dependent launch for chains of small kernels (the learner's
// update): a kernel launched with programmatic stream serialization may be
// scheduled while its predecessor on the stream still runs.  Every such
// kernel calls pdl_enter() first: it waits until the predecessor has
// completed and its writes are visible (so, transitively, everything before
// it), then lets its own successor be scheduled.  Launched without the
// attribute, both instructions return at once.
#pragma once
#include <cuda_runtime.h>

#include <utility>

namespace flashnav {

__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... K, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t stream, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<A>(args)...);
}

} // namespace flashnav
