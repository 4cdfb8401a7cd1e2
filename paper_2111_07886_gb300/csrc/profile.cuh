// Launch accounting shared by the launch wrappers (see profile.cu).
#pragma once

#include <nvtx3/nvToolsExt.h>

#include "pet_common.cuh"

namespace pet {

// NVTX range over a host-side phase (one subiteration, a whole reconstruction, a batch tick), for
// timeline tools; without a tool attached a push / pop is a no-op call.
class TraceRange {
public:
    explicit TraceRange(const char *name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange &) = delete;
    TraceRange &operator=(const TraceRange &) = delete;
};

// RAII scope around one kernel launch: counts it and, when profiling is on, brackets it with
// CUDA events on its stream.
class LaunchScope {
public:
    LaunchScope(int kind, cudaStream_t st);
    ~LaunchScope();
    LaunchScope(const LaunchScope &) = delete;
    LaunchScope &operator=(const LaunchScope &) = delete;

private:
    int kind_;
    cudaStream_t st_;
    bool active_;
    cudaEvent_t a_{}, b_{};
};

// Per-kernel timing is on (pet_profile_enable): work that normally runs on side streams beside
// other kernels (mu pass, objective) then runs on the caller's stream, so that each kernel's
// events bracket that kernel alone.
bool profile_active();

}  // namespace pet
