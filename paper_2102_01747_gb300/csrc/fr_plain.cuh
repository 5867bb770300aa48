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
__device__ __forceinline__ void tile_pixel(const DevReq &R, long long tile, int lane, int &px, int &py,
                                           int &sample)
{
    const int th = kTileH / R.spl;
    const long long tiles_y = (R.height + th - 1) / th;
    long long tx, ty;
    if (R.tile_order == 1) {
        tx = tile / tiles_y;
        ty = tile % tiles_y;
    } else {
        tx = tile % R.tiles_x;
        ty = tile / R.tiles_x;
        if (R.tile_order == 2 && ty < tiles_y) ty = tiles_y - 1 - ty;
    }
    const int q = lane / R.spl;
    sample = lane - q * R.spl;
    px = (int)tx * kTileW + (q & (kTileW - 1));
    py = (int)ty * th + (q / kTileW);
}


// BAN: compiled with the Mandelbulb's analytic normal (normal_at)
template <int KIND, int U, bool COUNT, bool PHONG, bool BAN>
__global__ void __launch_bounds__(256) plain_kernel(const __grid_constant__ DevReq R)
{
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tile = gtid >> 5;
    const int lane = threadIdx.x & 31;
    int px, py, sample;
    tile_pixel(R, tile, lane, px, py, sample);
    Counters cnt;
    if (COUNT)
        for (int k = 0; k < kNStats; k++) cnt.v[k] = 0;
    const bool valid = px < R.width && py < R.height;
    uint32_t c8 = 0;
    float depth = 0.0f;
    render_pixel<KIND, U, COUNT, PHONG, BAN>(R, px, py, sample, valid, cnt, c8, depth);
    store_rgba8_depth(R, px, py, valid && sample == 0, c8, depth, R.spl);
    if (COUNT) flush_counters(cnt, R.stats);
}

template <int KIND, int U, bool COUNT, bool PHONG = false, bool BAN = false>
static cudaError_t launch_plain_t(const DevReq &R, int block, cudaStream_t s)
{
    const long long threads = plain_tiles(R) * 32;
    const long long grid = (threads + block - 1) / block;
    plain_kernel<KIND, U, COUNT, PHONG, BAN><<<(unsigned)grid, block, 0, s>>>(R);
    return cudaGetLastError();
}

// Many requests in one launch of the same one-ray-per-thread code: the grid
// covers every tile of every request, each CTA inside one request (a request's
// tiles are padded to whole CTAs), so its kind and parameters are uniform and
// read from the kernel-parameter table.  The hardware block scheduler hands
// CTAs to SMs as they free up, so the requests' slow pixels overlap instead of
// each launch waiting for its own.  tile_begin of request r (in CTAs) is kept
// in reqs[r].unit_begin.
// Always compiled with the Mandelbulb's analytic normal, and held to 72
// registers (at most 256 threads per block, as fr_set_tuning enforces): left
// to itself the compiler takes 80, with which the 64-request mixed batch runs
// 36.0 ms against 33.3 (64 registers: 33.5).  fr_render_* can also launch it
// with one request (fr_tuning.single_kernel = 2, autotuned).
template <int U, bool COUNT, bool PHONG>
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
    const int lane = threadIdx.x & 31;
    int px, py, sample;
    tile_pixel(R, tile, lane, px, py, sample);
    Counters cnt;
    if (COUNT)
        for (int k = 0; k < kNStats; k++) cnt.v[k] = 0;
    const bool valid = px < R.width && py < R.height;
    uint32_t c8 = 0;
    float depth = 0.0f;
    if (R.kind == 0)
        render_pixel<0, U, COUNT, PHONG, true>(R, px, py, sample, valid, cnt, c8, depth);
    else
        render_pixel<1, U, COUNT, PHONG, true>(R, px, py, sample, valid, cnt, c8, depth);
    store_rgba8_depth(R, px, py, valid && sample == 0, c8, depth, R.spl);
    if (COUNT && R.stats) flush_counters(cnt, R.stats);
}

template <int U, bool COUNT, bool PHONG>
static cudaError_t launch_batch_plain_t(const BatchArgs &A, long long ctas, int block, cudaStream_t s)
{
    batch_plain_kernel<U, COUNT, PHONG><<<(unsigned)ctas, block, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace fr
