// fr_static.cu -- fr_render_batch_static: the batched render without a
// caller-provided workspace, for callers that cannot allocate device memory.
//
// The persistent schedule (batch_kernel 0) needs one 256-byte queue head per
// launch of up to 64 requests.  fr_render_batch takes that scratch from the
// caller whichever schedule runs; this entry
// point takes it from a file-scope __device__ array instead, sized for the
// largest batch fr_render_batch accepts (4096 requests = 64 launches = 16 KB).
// Every GPU that loads the library holds the array until the process exits.
//
// Host code must not hand the array's name to a kernel: on the host it is only
// a stand-in symbol.  Its device address is looked up once per device with
// cudaGetSymbolAddress (on the first call made with that device current) and
// kept.  The batch itself then goes through the unchanged fr_render_batch,
// which zeroes each queue head with a memset on the stream before its launch,
// so what the previous call left in the array does not matter.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "../../include/fr.h"

namespace fr {
fr_status set_error(fr_status st, const char *msg);
}

namespace {

constexpr int kStaticLaunches = 64;  // 64 launches x 64 requests = 4096 requests
constexpr size_t kStaticBytes = 256 * kStaticLaunches;
constexpr int kStaticMaxRequests = 64 * kStaticLaunches;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

std::mutex g_static_mu;
void *g_static_addr[kMaxDevices];

}  // namespace

extern "C" {

FR_API fr_status fr_render_batch_static(const fr_request *reqs, int32_t n_reqs, void *stream)
{
    char msg[160];
    if (n_reqs < 1 || n_reqs > kStaticMaxRequests) {
        snprintf(msg, sizeof msg, "n_reqs %d outside 1..%d (the static workspace holds %d launches)",
                 n_reqs, kStaticMaxRequests, kStaticLaunches);
        return fr::set_error(FR_EINVAL, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        snprintf(msg, sizeof msg, "cudaGetDevice failed: %s", cudaGetErrorString(e));
        return fr::set_error(FR_ECUDA, msg);
    }
    if (dev < 0 || dev >= kMaxDevices) return fr::set_error(FR_EINVAL, "device ordinal beyond 63");
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        ws = g_static_addr[dev];
        if (!ws) {
            e = cudaGetSymbolAddress(&ws, g_static_ws);
            if (e != cudaSuccess || !ws) {
                snprintf(msg, sizeof msg, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return fr::set_error(FR_ECUDA, msg);
            }
            g_static_addr[dev] = ws;
        }
    }
    return fr_render_batch(reqs, n_reqs, ws, kStaticBytes, stream);
}

}  // extern "C"
