// fr_launch.h -- launchers the C ABI (fr_api.cu) calls; one per kernel family.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "fr_device.cuh"

namespace fr {

// An NVTX range over one C-ABI call, so that a profiler's timeline shows the
// calls beside their kernels (NVTX v3 is header-only; without a tool attached
// a push and a pop cost two indirect calls).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// requests per batch launch (either schedule): the table rides in the kernel parameters
// (64 x sizeof(DevReq) stays well inside the 32 KB parameter limit)
constexpr int kMaxReqPerLaunch = 64;

struct BatchArgs {
    unsigned long long *queue;  // queue head of the persistent schedule (zeroed before its launch)
    long long total_units;      // pixel slots (persistent) or CTAs (batch kernel) over all requests
    int n_reqs;
    int refill_threshold;       // refill a warp once this many lanes are idle
    DevReq reqs[kMaxReqPerLaunch];
};

// orbit iterations the adjoint keeps per DE (max_iter of a backward call)
constexpr int kMaxBwdIter = 64;

struct BwdArgs {
    DevReq R;                // the forward request (Julia)
    const float4 *saved;     // hit point + flags per pixel
    const float4 *d_rgba;    // cotangent of the float colour
    const float *d_depth;    // cotangent of the depth, may be NULL
    float *grad;             // 11 floats, accumulated
    double *acc;             // 11 double partial totals, zero on entry; NULL = the library's own
    unsigned int *done;      // finished-block count, zero on entry (with acc)
    float light_norm;        // |light dir| as given (before normalisation)
    float plane_norm;        // |plane n| as given
};

// adjoint of one Julia render (one thread per pixel, block reduction, atomics)
cudaError_t launch_backward(const BwdArgs &A, cudaStream_t s);

// one-ray-per-thread forward kernel for one request
cudaError_t launch_plain(const DevReq &R, int block, int unroll, bool count, cudaStream_t s);

// one-ray-per-thread kernel over A.n_reqs requests in one launch; reqs[r].unit_begin
// holds request r's first CTA, `ctas` the grid size; phong: some request uses
// Phong shading
cudaError_t launch_batch_plain(const BatchArgs &A, long long ctas, int block, int unroll, bool count,
                               bool phong, cudaStream_t s);

// the single-request kernel compiled with the Mandelbulb's analytic normal (unroll 1)
cudaError_t launch_plain_ban(const DevReq &R, int block, bool count, cudaStream_t s);

// the one-ray-per-thread kernels with a pixel's samples on R.spl adjacent lanes
// (unroll 1): one request, or a batch launch in which some request has spl > 1
cudaError_t launch_plain_lanes(const DevReq &R, int block, bool count, cudaStream_t s);
cudaError_t launch_batch_plain_lanes(const BatchArgs &A, long long ctas, int block, bool count, bool phong,
                                     cudaStream_t s);

// persistent warps over the tiles of A.n_reqs requests, each warp taking the
// next tile from the queue head A.queue (memset + launch); reqs[r].unit_begin
// holds request r's first tile, A.total_units the tiles of the launch
cudaError_t launch_batch_refill(const BatchArgs &A, int block, int unroll, bool count, bool phong, cudaStream_t s);
cudaError_t launch_batch_refill_lanes(const BatchArgs &A, int block, bool count, bool phong, cudaStream_t s);

// lane-state-machine forward kernel without the queue: one pixel per lane, all tiles launched
cudaError_t launch_lanes(const BatchArgs &A, int block, int unroll, bool count, bool phong, cudaStream_t s);

// persistent forward kernel over A.n_reqs requests (memset of the queue head + launch)
cudaError_t launch_persist(const BatchArgs &A, int block, int ctas_per_sm, int unroll, bool count, bool phong,
                           cudaStream_t s);

}  // namespace fr
