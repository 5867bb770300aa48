// fr_static.cu -- fr_render_batch_static: the batched render without a
// caller-provided workspace, for callers that cannot allocate device memory.
//
// The persistent schedules (batch_kernel 2, the default, and 0) need one
// 256-byte queue head per launch of up to 64 requests.  fr_render_batch takes
// that scratch from the caller whichever schedule runs; this entry
// point takes it from a file-scope __device__ array instead, sized for the
// largest batch fr_render_batch accepts (4096 requests = 64 launches = 16 KB).
// Every GPU that loads the library holds the array until the process exits.
//
// Host code must not hand the array's name to a kernel: on the host it is only
// a stand-in symbol.  Its device address comes from cudaGetSymbolAddress with
// the device current, on every call made outside a stream capture (so a
// context that was reset and re-created, which maps the array anew, is
// followed), and the last address seen on each device is kept for calls made
// while their stream is being captured, when no such lookup may run.  The
// batch itself then goes through the unchanged fr_render_batch, which zeroes
// each queue head with a memset on the stream before its launch, so what the
// previous call left in the array does not matter.
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/fr.h"
#include "fr_launch.h"

namespace fr {
fr_status set_error(fr_status st, const char *msg);
fr_status resolve_requests(const fr_request *reqs, int n_reqs, std::vector<DevReq> &all, bool &count);
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
    fr::NvtxRange range("fr_render_batch_static");
    char msg[160];
    if (!reqs) return fr::set_error(FR_EINVAL, "requests is NULL");
    if (n_reqs < 1 || n_reqs > kStaticMaxRequests) {
        snprintf(msg, sizeof msg, "n_reqs %d outside 1..%d (the static workspace holds %d launches)",
                 n_reqs, kStaticMaxRequests, kStaticLaunches);
        return fr::set_error(FR_EINVAL, msg);
    }
    {
        // every request is checked before the first CUDA call (which may create
        // the context); fr_render_batch checks them again, on the host only
        std::vector<fr::DevReq> all;
        bool count = false;
        const fr_status st = fr::resolve_requests(reqs, n_reqs, all, count);
        if (st != FR_OK) return st;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();  // leave no error behind for the next launch check
        snprintf(msg, sizeof msg, "cudaGetDevice failed: %s", cudaGetErrorString(e));
        return fr::set_error(FR_ECUDA, msg);
    }
    if (dev < 0 || dev >= kMaxDevices) return fr::set_error(FR_EINVAL, "device ordinal beyond 63");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing((cudaStream_t)stream, &cap);
    if (e != cudaSuccess) {
        cudaGetLastError();  // leave no error behind for the next launch check
        snprintf(msg, sizeof msg, "cudaStreamIsCapturing failed: %s", cudaGetErrorString(e));
        return fr::set_error(FR_ECUDA, msg);
    }
    void *ws = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_static_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            e = cudaGetSymbolAddress(&ws, g_static_ws);
            if (e != cudaSuccess || !ws) {
                cudaGetLastError();  // leave no error behind for the next launch check
                snprintf(msg, sizeof msg, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return fr::set_error(FR_ECUDA, msg);
            }
            g_static_addr[dev] = ws;
        } else {
            ws = g_static_addr[dev];
            if (!ws)
                return fr::set_error(FR_EINVAL, "the first fr_render_batch_static call on a device must come "
                                                "before any stream capture (it looks up the array's address)");
        }
    }
    return fr_render_batch(reqs, n_reqs, ws, kStaticBytes, stream);
}

}  // extern "C"
