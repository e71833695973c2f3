// Launch bookkeeping: counts every kernel the library launches and, when a
// plan has timing enabled, brackets the launch with CUDA events on the
// plan's stream.
#pragma once
#include <cuda_runtime.h>

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

}  // namespace purify
