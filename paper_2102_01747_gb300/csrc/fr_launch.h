// fr_launch.h -- launchers the C ABI (fr_api.cu) calls; one per kernel family.
#pragma once

#include <cuda_runtime.h>

#include "fr_device.cuh"

namespace fr {

// requests per persistent launch: the table rides in the kernel parameters
// (64 x sizeof(DevReq) stays well inside the 32 KB parameter limit)
constexpr int kMaxReqPerLaunch = 64;

struct BatchArgs {
    unsigned long long *queue;  // queue head (zeroed before the launch)
    long long total_units;      // pixel slots over all requests
    int n_reqs;
    int refill_threshold;       // refill a warp once this many lanes are idle
    DevReq reqs[kMaxReqPerLaunch];
};

// one-ray-per-thread forward kernel for one request
cudaError_t launch_plain(const DevReq &R, int block, int unroll, bool count, cudaStream_t s);

// persistent forward kernel over A.n_reqs requests (memset of the queue head + launch)
cudaError_t launch_persist(const BatchArgs &A, int block, int ctas_per_sm, int unroll, bool count,
                           cudaStream_t s);

}  // namespace fr
