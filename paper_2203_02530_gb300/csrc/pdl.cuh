// Programmatic dependent launch for the kernels of the operation DAG.
//
// A kernel launched with launch_pdl may be scheduled as soon as every CTA of
// the kernel before it on the same stream has exited (or released it),
// before that kernel's completion has gone back through the front end.
// Every such kernel starts with pdl_begin(flags): by default it waits
// (griddepcontrol.wait) until the earlier kernel has completed and its
// writes are visible, and releases no successor early: CTAs launched early
// would wait on SMs that the kernels of the schedule's other streams could
// use.  The relaxed schedule mode passes two flags: kPdlNoWait (skip the
// wait: the kernel's operation has no DAG predecessor, it needs nothing from
// any other kernel of the product) and kPdlEarly (the next kernel of the
// stream is such a kernel, so release it as each CTA starts and let it fill
// this kernel's tail).
// Launched without the attribute (or with SPMV_NO_PDL=1 in the environment)
// the wait does nothing.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

namespace spmvk {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

enum { kPdlNoWait = 1, kPdlEarly = 2 };

// Start of a kernel of the operation DAG (see above).
__device__ __forceinline__ void pdl_begin(int flags) {
    if (!(flags & kPdlNoWait)) pdl_wait();
    if (flags & kPdlEarly) pdl_trigger();
}

inline bool pdl_enabled() {
    static const bool on = [] {
        const char* e = std::getenv("SPMV_NO_PDL");
        return !(e && std::strcmp(e, "0") != 0 && e[0] != '\0');
    }();
    return on;
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

}  // namespace spmvk
