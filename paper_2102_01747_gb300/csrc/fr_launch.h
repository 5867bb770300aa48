// fr_launch.h -- launchers the C ABI (fr_api.cu) calls; one per kernel family.
#pragma once

#include <cuda_runtime.h>

#include "fr_device.cuh"

namespace fr {

// one-ray-per-thread forward kernel for one request
cudaError_t launch_plain(const DevReq &R, int block, int unroll, bool count, cudaStream_t s);

}  // namespace fr
