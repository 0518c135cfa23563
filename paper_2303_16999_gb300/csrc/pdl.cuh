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

#include <atomic>
#include <cstdint>
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

// Kernel attributes belong to a device: the dynamic shared-memory limit (and
// optionally all of L1 as shared memory) is set once per device; two threads
// racing here both set it, which is harmless.
template <typename... KArgs>
inline cudaError_t set_smem_attrs_once(std::atomic<uint64_t> &done, void (*kernel)(KArgs...),
                                       int smem_bytes, bool all_shared) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = 1ull << (dev & 63);
    if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (e == cudaSuccess && all_shared)
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
    return e;
}

}  // namespace spmm

#endif
