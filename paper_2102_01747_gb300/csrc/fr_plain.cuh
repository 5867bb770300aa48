// fr_plain.cuh -- the one-ray-per-thread kernels (templates; instantiated in
// fr_plain.cu, and the single-request kernel with the Mandelbulb's analytic
// normal in fr_plain_an.cu).
// A warp owns a 4 x 8 tile of pixels (so its 32 rays start close together and
// diverge late); each thread runs its pixel's samples start to finish.  The
// request rides in the kernel's parameter space (__grid_constant__), read
// warp-uniformly from the constant bank.
#pragma once

#include "fr_launch.h"
#include "fr_trace.cuh"

namespace fr {

// Pixel and first sample of `lane` in tile number `tile` of request R.  A
// tile is 4 pixels wide and 8 / R.spl tall, pixel q of the tile (row-major)
// on lanes q * spl .. q * spl + spl - 1, sample k on the k-th of them.  Tiles
// are numbered in launch order (the hardware hands CTAs to SMs roughly in
// index order), laid over the image by R.tile_order: 0 rows of tiles top to
// bottom, 1 columns of tiles left to right, 2 rows bottom to top.  The grid is
// padded to whole CTAs; the padding tiles land past the image's right or
// bottom edge in every order, so their lanes fail the px < width, py < height
// test.
// spl is 1, 2, 4 or 8 (R.spl_log2 its log2) and width * height * spp < 2^31
// keeps a request below 2^26 tiles, so the arithmetic is 32-bit shifts and
// divisions.
template <bool LANES>
__device__ __forceinline__ void tile_pixel(const DevReq &R, long long tile, int lane, int &px, int &py,
                                           int &sample)
{
    const unsigned t = (unsigned)tile;
    const int spl_log2 = LANES ? R.spl_log2 : 0;
    const int th_log2 = 3 - spl_log2;  // tile height 8 / spl = 2^th_log2
    const unsigned tiles_y = ((unsigned)R.height + (1u << th_log2) - 1u) >> th_log2;
    unsigned tx, ty;
    if (R.tile_order == 1) {
        tx = t / tiles_y;
        ty = t - tx * tiles_y;
    } else {
        ty = t / (unsigned)R.tiles_x;
        tx = t - ty * (unsigned)R.tiles_x;
        if (R.tile_order == 2 && ty < tiles_y) ty = tiles_y - 1u - ty;
    }
    const int q = lane >> spl_log2;
    sample = lane & ((1 << spl_log2) - 1);
    px = (int)tx * kTileW + (q & (kTileW - 1));
    py = ((int)ty << th_log2) + (q / kTileW);
}


// One pixel of a lane (LANES false: each lane's pixel, all its samples in
// turn; LANES true: the samples of a pixel on R.spl adjacent lanes), called by
// all 32 lanes of the warp; the packed colour and depth of finished pixels go
// to the warp's quad store.
template <int KIND, int U, bool COUNT, bool PHONG, int BAN, bool LANES>
__device__ __forceinline__ void shade_tile(const DevReq &R, long long tile, Counters &cnt)
{
    const int lane = threadIdx.x & 31;
    int px, py, sample;
    tile_pixel<LANES>(R, tile, lane, px, py, sample);
    const bool valid = px < R.width && py < R.height;
    uint32_t c8 = 0;
    float depth = 0.0f;
    if constexpr (LANES) {
        render_pixel_lanes<KIND, U, COUNT, PHONG, BAN>(R, px, py, sample, valid, cnt, c8, depth);
        store_rgba8_depth(R, px, py, valid && sample == 0, c8, depth, R.spl);
    } else {
        if (valid) render_pixel<KIND, U, COUNT, PHONG, BAN>(R, px, py, cnt, c8, depth);
        store_rgba8_depth(R, px, py, valid, c8, depth);
    }
}

// BAN: compiled with the Mandelbulb's analytic normal (normal_at; 1 inline,
// 2 out of line)
template <int KIND, int U, bool COUNT, bool PHONG, int BAN, bool LANES = false>
__global__ void __launch_bounds__(256) plain_kernel(const __grid_constant__ DevReq R)
{
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    Counters cnt;
    if (COUNT)
        for (int k = 0; k < kNStats; k++) cnt.v[k] = 0;
    shade_tile<KIND, U, COUNT, PHONG, BAN, LANES>(R, gtid >> 5, cnt);
    if (COUNT) flush_counters(cnt, R.stats);
}

template <int KIND, int U, bool COUNT, bool PHONG = false, int BAN = 0, bool LANES = false>
static cudaError_t launch_plain_t(const DevReq &R, int block, cudaStream_t s)
{
    const long long threads = plain_tiles(R) * 32;
    const long long grid = (threads + block - 1) / block;
    plain_kernel<KIND, U, COUNT, PHONG, BAN, LANES><<<(unsigned)grid, block, 0, s>>>(R);
    return cudaGetLastError();
}

// Many requests in one launch of the same one-ray-per-thread code: the grid
// covers every tile of every request, each CTA inside one request (a request's
// tiles are padded to whole CTAs), so its kind and parameters are uniform and
// read from the kernel-parameter table.  The hardware block scheduler hands
// CTAs to SMs as they free up, so the requests' slow pixels overlap instead of
// each launch waiting for its own.  tile_begin of request r (in CTAs) is kept
// in reqs[r].unit_begin.
// Always compiled with the Mandelbulb's analytic normal (out of line), and held to 72
// registers (at most 256 threads per block, as fr_set_tuning enforces): left
// to itself the compiler takes 80, with which the 64-request mixed batch runs
// 36.0 ms against 33.3 (64 registers: 33.5).  fr_render_* can also launch it
// with one request (fr_tuning.single_kernel = 2, autotuned).
template <int U, bool COUNT, bool PHONG, bool LANES = false>
__global__ void __maxnreg__(72) batch_plain_kernel(const __grid_constant__ BatchArgs A)
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
    Counters cnt;
    if (COUNT)
        for (int k = 0; k < kNStats; k++) cnt.v[k] = 0;
    if (R.kind == 0)
        shade_tile<0, U, COUNT, PHONG, 2, LANES>(R, tile, cnt);
    else
        shade_tile<1, U, COUNT, PHONG, 2, LANES>(R, tile, cnt);
    if (COUNT && R.stats) flush_counters(cnt, R.stats);
}

template <int U, bool COUNT, bool PHONG, bool LANES = false>
static cudaError_t launch_batch_plain_t(const BatchArgs &A, long long ctas, int block, cudaStream_t s)
{
    batch_plain_kernel<U, COUNT, PHONG, LANES><<<(unsigned)ctas, block, 0, s>>>(A);
    return cudaGetLastError();
}

// Persistent warps over every tile of every request of a launch (the
// fr_render_batch schedule batch_kernel 2): the grid is as many CTAs as fit on
// the SMs at once, and each warp takes the next tile from one counter (the
// queue head in the caller's workspace, zeroed before the launch) as soon as
// its 32 lanes are done with the last, so no warp waits for the other warps
// of its CTA.  Tiles are numbered over the requests in launch order;
// reqs[r].unit_begin holds request r's first tile.  A warp's tiles come in
// increasing order, so its request cursor only moves forward.  The pixels
// are shade_tile's, so the images are the other schedules' bit for bit.
template <int U, bool COUNT, bool PHONG, bool LANES = false>
__global__ void __maxnreg__(72) batch_refill_kernel(const __grid_constant__ BatchArgs A)
{
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned long long total = (unsigned long long)A.total_units;
    int lo = 0;
    Counters cnt;
    if (COUNT)
        for (int k = 0; k < kNStats; k++) cnt.v[k] = 0;
    for (;;) {
        unsigned long long g = 0;
        if (lane == 0) g = atomicAdd(A.queue, 1ull);
        g = __shfl_sync(full, g, 0);
        if (g >= total) break;
        int r = lo;
        while (r + 1 < A.n_reqs && (unsigned long long)A.reqs[r + 1].unit_begin <= g) r++;
        if (COUNT && r != lo) {  // the counters belong to the request they were taken for
            if (A.reqs[lo].stats) flush_counters(cnt, A.reqs[lo].stats);
            for (int k = 0; k < kNStats; k++) cnt.v[k] = 0;
        }
        lo = r;
        const DevReq &R = A.reqs[lo];
        const long long tile = (long long)g - R.unit_begin;
        if (R.kind == 0)
            shade_tile<0, U, COUNT, PHONG, 2, LANES>(R, tile, cnt);
        else
            shade_tile<1, U, COUNT, PHONG, 2, LANES>(R, tile, cnt);
    }
    if (COUNT && A.reqs[lo].stats) flush_counters(cnt, A.reqs[lo].stats);
}

template <int U, bool COUNT, bool PHONG, bool LANES = false>
static cudaError_t launch_batch_refill_t(const BatchArgs &A, int block, cudaStream_t s)
{
    int dev = 0, sms = 0, fit = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, batch_refill_kernel<U, COUNT, PHONG, LANES>, block,
                                                           0)) != cudaSuccess)
        return e;
    if (fit < 1) return cudaErrorInvalidConfiguration;
    if ((e = cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    batch_refill_kernel<U, COUNT, PHONG, LANES><<<sms * fit, block, 0, s>>>(A);
    return cudaGetLastError();
}


}  // namespace fr
