// fr_plain.cu -- one ray per thread.  A warp owns a 4 x 8 tile of pixels (so
// its 32 rays start close together and diverge late); each thread runs its
// pixel's samples start to finish.  The request rides in the kernel's
// parameter space (__grid_constant__), read warp-uniformly from the constant
// bank.
#include "fr_launch.h"
#include "fr_trace.cuh"

namespace fr {

// Pixel of `lane` in tile number `tile` of request R.  Tiles are numbered in
// launch order (the hardware hands CTAs to SMs roughly in index order), laid
// over the image by R.tile_order: 0 rows of tiles top to bottom, 1 columns of
// tiles left to right, 2 rows bottom to top.  The grid is padded to whole
// CTAs; the padding tiles land past the image's right or bottom edge in every
// order, so their lanes fail the px < width, py < height test.
__device__ __forceinline__ void tile_pixel(const DevReq &R, long long tile, int lane, int &px, int &py)
{
    const long long tiles_y = (R.height + kTileH - 1) / kTileH;
    long long tx, ty;
    if (R.tile_order == 1) {
        tx = tile / tiles_y;
        ty = tile % tiles_y;
    } else {
        tx = tile % R.tiles_x;
        ty = tile / R.tiles_x;
        if (R.tile_order == 2 && ty < tiles_y) ty = tiles_y - 1 - ty;
    }
    px = (int)tx * kTileW + (lane & (kTileW - 1));
    py = (int)ty * kTileH + (lane / kTileW);
}

template <int KIND, int U, bool COUNT, bool PHONG>
__global__ void __launch_bounds__(256) plain_kernel(const __grid_constant__ DevReq R)
{
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tile = gtid >> 5;
    const int lane = threadIdx.x & 31;
    int px, py;
    tile_pixel(R, tile, lane, px, py);
    Counters cnt;
    if (COUNT)
        for (int k = 0; k < kNStats; k++) cnt.v[k] = 0;
    const bool valid = px < R.width && py < R.height;
    uint32_t c8 = 0;
    float depth = 0.0f;
    if (valid) render_pixel<KIND, U, COUNT, PHONG>(R, px, py, cnt, c8, depth);
    store_rgba8_depth(R, px, py, valid, c8, depth);
    if (COUNT) flush_counters(cnt, R.stats);
}

template <int KIND, int U, bool COUNT, bool PHONG = false>
static cudaError_t launch_plain_t(const DevReq &R, int block, cudaStream_t s)
{
    const long long tiles_y = (R.height + kTileH - 1) / kTileH;
    const long long threads = (long long)R.tiles_x * tiles_y * 32;
    const long long grid = (threads + block - 1) / block;
    plain_kernel<KIND, U, COUNT, PHONG><<<(unsigned)grid, block, 0, s>>>(R);
    return cudaGetLastError();
}

// Many requests in one launch of the same one-ray-per-thread code: the grid
// covers every tile of every request, each CTA inside one request (a request's
// tiles are padded to whole CTAs), so its kind and parameters are uniform and
// read from the kernel-parameter table.  The hardware block scheduler hands
// CTAs to SMs as they free up, so the requests' slow pixels overlap instead of
// each launch waiting for its own.  tile_begin of request r (in CTAs) is kept
// in reqs[r].unit_begin.
template <int U, bool COUNT, bool PHONG>
__global__ void __launch_bounds__(256) batch_plain_kernel(const __grid_constant__ BatchArgs A)
{
    const int warps = blockDim.x >> 5;
    const long long cta = blockIdx.x;
    int lo = 0, hi = A.n_reqs - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (A.reqs[mid].unit_begin <= cta)
            lo = mid;
        else
            hi = mid - 1;
    }
    const DevReq &R = A.reqs[lo];
    const long long tile = (cta - R.unit_begin) * warps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    int px, py;
    tile_pixel(R, tile, lane, px, py);
    Counters cnt;
    if (COUNT)
        for (int k = 0; k < kNStats; k++) cnt.v[k] = 0;
    const bool valid = px < R.width && py < R.height;
    uint32_t c8 = 0;
    float depth = 0.0f;
    if (valid) {
        if (R.kind == 0)
            render_pixel<0, U, COUNT, PHONG>(R, px, py, cnt, c8, depth);
        else
            render_pixel<1, U, COUNT, PHONG>(R, px, py, cnt, c8, depth);
    }
    store_rgba8_depth(R, px, py, valid, c8, depth);
    if (COUNT && R.stats) flush_counters(cnt, R.stats);
}

template <int U, bool COUNT, bool PHONG>
static cudaError_t launch_batch_plain_t(const BatchArgs &A, long long ctas, int block, cudaStream_t s)
{
    batch_plain_kernel<U, COUNT, PHONG><<<(unsigned)ctas, block, 0, s>>>(A);
    return cudaGetLastError();
}

// phong: some request of the launch uses Phong shading (the Phong-capable code
// then serves every request of the launch, at unroll 1)
cudaError_t launch_batch_plain(const BatchArgs &A, long long ctas, int block, int unroll, bool count,
                               bool phong, cudaStream_t s)
{
    if (phong) return count ? launch_batch_plain_t<1, true, true>(A, ctas, block, s)
                            : launch_batch_plain_t<1, false, true>(A, ctas, block, s);
    if (count) return launch_batch_plain_t<1, true, false>(A, ctas, block, s);
    if (unroll == 2) return launch_batch_plain_t<2, false, false>(A, ctas, block, s);
    return launch_batch_plain_t<1, false, false>(A, ctas, block, s);
}

// Phong requests run the Phong-capable instantiation at unroll 1
cudaError_t launch_plain(const DevReq &R, int block, int unroll, bool count, cudaStream_t s)
{
    if (R.shading) {
        if (R.kind == 0)
            return count ? launch_plain_t<0, 1, true, true>(R, block, s) : launch_plain_t<0, 1, false, true>(R, block, s);
        return count ? launch_plain_t<1, 1, true, true>(R, block, s) : launch_plain_t<1, 1, false, true>(R, block, s);
    }
    if (count) return R.kind == 0 ? launch_plain_t<0, 1, true>(R, block, s)
                                  : launch_plain_t<1, 1, true>(R, block, s);
    if (R.kind == 0) {
        if (unroll == 4) return launch_plain_t<0, 4, false>(R, block, s);
        if (unroll == 2) return launch_plain_t<0, 2, false>(R, block, s);
        return launch_plain_t<0, 1, false>(R, block, s);
    }
    if (unroll == 4) return launch_plain_t<1, 4, false>(R, block, s);
    if (unroll == 2) return launch_plain_t<1, 2, false>(R, block, s);
    return launch_plain_t<1, 1, false>(R, block, s);
}

}  // namespace fr
