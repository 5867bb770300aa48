// fr_probe.cu -- the FP32 fused multiply-add throughput of the GPU the
// library runs on: the denominator of the renderer's FP32 roofline.
//
// Every thread runs kChains independent chains x <- x * a + b, each link one
// FFMA; kChains independent chains per thread and several warps per scheduler
// cover the FMA latency, so the count of links per second is the FMA pipes'
// issue rate.  a is just below 1 and b small, so the values stay finite; the
// chains' sum is stored once per thread so that none of them is dead code.
#include <cstdint>

#include "../../include/fr.h"

namespace fr {
fr_status set_error(fr_status st, const char *msg);
}

namespace {

constexpr int kChains = 8;     // independent chains per thread
constexpr int kUnroll = 16;    // links per chain per loop trip

__global__ void __launch_bounds__(256) ffma_probe_kernel(int iters, float a, float b, float *sink)
{
    const unsigned gid = blockIdx.x * blockDim.x + threadIdx.x;
    float x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = (float)(gid & 1023u) * 1e-6f + (float)k;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++) {
#pragma unroll
            for (int k = 0; k < kChains; k++) x[k] = fmaf(x[k], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    sink[gid] = s;
}

}  // namespace

extern "C" {

FR_API double fr_ffma_probe_flops(int32_t blocks, int32_t threads, int32_t iters)
{
    if (blocks < 1 || threads < 1 || iters < 1) return 0.0;
    return 2.0 * (double)blocks * (double)threads * (double)iters * kUnroll * kChains;
}

FR_API fr_status fr_ffma_probe(int32_t blocks, int32_t threads, int32_t iters, float *sink, void *stream)
{
    if (blocks < 1 || blocks > (1 << 20)) return fr::set_error(FR_EINVAL, "blocks outside 1..2^20");
    if (threads < 32 || threads > 256 || threads % 32) return fr::set_error(FR_EINVAL, "threads must be 32..256, x32");
    if (iters < 1) return fr::set_error(FR_EINVAL, "iters must be positive");
    if (!sink || ((uintptr_t)sink % 4)) return fr::set_error(FR_EINVAL, "sink is NULL or misaligned");
    ffma_probe_kernel<<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, 0.9999999f, 1e-7f, sink);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fr::set_error(FR_ECUDA, cudaGetErrorString(e));
    fr::set_error(FR_OK, "");
    return FR_OK;
}

}  // extern "C"
