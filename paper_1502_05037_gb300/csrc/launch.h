// Launch bookkeeping: counts every kernel the library launches and, when a
// plan has timing enabled, brackets the launch with CUDA events on the
// plan's stream.
#pragma once
#include <cuda_runtime.h>

#include <utility>

struct purify_plan;

namespace purify {

struct Launch {
    purify_plan* p;
    const char* name;
    cudaEvent_t e0 = nullptr;
    Launch(purify_plan* plan, const char* kname);
    // Checks the launch status (throws on error) and records the end event.
    void done();
};

// Launch with programmatic stream serialisation: the kernel may be scheduled
// while its predecessor on the stream is still running (captured as a
// programmatic edge in graphs). Every kernel launched this way waits
// (pdl_wait) for the predecessor's completion and memory before it touches
// memory. Errors surface through cudaGetLastError (Launch::done).
template <typename... KArgs, typename... Args>
inline void launch_dependent(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
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
    (void)cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace purify
