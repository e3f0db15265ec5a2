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
// this kernel's tail).  The deferred mode passes kPdlDefer to a remote
// product whose stream predecessor writes none of its inputs but y: it reads
// A_R and the halo and forms its row sums before the wait, and waits only
// before its first access to y (and, at the latest, before it exits, so that
// its completion still implies the predecessor's); the predecessor, which
// waits for its own predecessor first, releases it as its CTAs start.
// Launched without the attribute (or with SPMV_NO_PDL=1 in the environment)
// the wait does nothing.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

namespace spmvk {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

enum { kPdlNoWait = 1, kPdlEarly = 2, kPdlDefer = 4 };

// Start of a kernel of the operation DAG (see above); kPdlDefer is ignored
// here (the kernel waits), so only kernels written for it can defer.
__device__ __forceinline__ void pdl_begin(int flags) {
    if (!(flags & kPdlNoWait)) pdl_wait();
    if (flags & kPdlEarly) pdl_trigger();
}

// Start of a kernel that honours kPdlDefer: it then skips the wait here and
// calls pdl_settle before touching y.
__device__ __forceinline__ void pdl_begin_deferrable(int flags) {
    if (!(flags & (kPdlNoWait | kPdlDefer))) pdl_wait();
    if (flags & kPdlEarly) pdl_trigger();
}

// A deferring kernel's wait, once per thread: before the thread's first
// access to y, and before it exits if it never made one.
__device__ __forceinline__ void pdl_settle(bool& pending) {
    if (pending) {
        pdl_wait();
        pending = false;
    }
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
