// Programmatic dependent launch for the library's kernels.
//
// Every kernel is launched with programmatic stream serialisation and starts
// with pdl_enter(): griddepcontrol.wait returns once the kernel before it in
// the stream has completed and its writes are visible (a no-op without a
// prerequisite grid), then launch_dependents lets the next kernel's launch
// and setup proceed while this one runs.  Stream order and results are
// unchanged; the gap between the short kernels of a call (the dynamic
// re-partition is a chain of them) shrinks.
#ifndef SPMM_PDL_CUH
#define SPMM_PDL_CUH

#include <cuda_runtime.h>

#include <utility>

namespace spmm {

__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace spmm

#endif
