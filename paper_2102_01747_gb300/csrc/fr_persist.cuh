// fr_persist.cuh -- persistent, divergence-compacting forward kernel (template;
// the queue-fed instantiations are in fr_persist.cu, the queue-less lane
// kernels in fr_lanes.cu, two translation units that compile in parallel).
//
// Why: in the one-ray-per-thread kernel a warp runs until its slowest lane is
// done, twice over: rays need 1..max_steps march steps, and every DE call
// needs 1..max_iter orbit steps (Mandelbulb 1080p: 2.7 on average, up to 12).
// Measured on that kernel at 1080p: 19 of 32 lanes active per issued
// instruction; on a batch of small images every launch is as long as its
// slowest pixel.
//
// Outcome, measured on 64 mixed requests: this kernel keeps no more lanes busy
// (18.5 of 32, like the one-ray-per-thread batch kernel) and its bookkeeping
// costs 179 thread instructions per orbit iteration against 139, so it is the
// alternative schedule (fr_tuning.batch_kernel = 0), not the default.
//
// How: CTAs stay resident (grid = SMs x resident CTAs).  Each lane holds one
// pixel's complete state (packed into few registers): its sample, the phase of
// the current ray (camera march, normal taps, shadow march), the march
// variables and one orbit in progress.  Every round of the warp loop advances
// each busy lane's orbit by a few steps (Julia: the unroll depth K, Mandelbulb:
// one); a lane whose orbit has escaped or reached max_iter turns it into a
// distance (Eq. 2), feeds it to its ray's state machine (march step, normal
// tap or shadow step, Listing "Julia Set ray cast") and starts its next orbit
// at once, so lanes never wait for each other's orbits or rays.  A finished
// pixel is stored and its lane refilled from one queue over every pixel of
// every request: once `refill_threshold` lanes are idle the warp takes exactly
// that many pixels with one atomicAdd on the queue head and hands them out by
// ballot rank.  (Reserving more than the idle lanes, to make the atomics rarer,
// measured slower: pixels parked in a busy warp starve the others at the end.)
//
// The orbit steps, the distance, the march update and the stencils are the
// same device functions, with every rounding step spelled out, that the
// one-ray-per-thread kernel uses, in the same order per ray, so the two
// kernels produce bit-identical images.
//
// The request table (<= 64 DevReq) travels in the kernel parameters
// (__grid_constant__) and is staged into shared memory by every CTA, since the
// lanes of one warp may read different requests.  The queue head lives in the
// caller's workspace and is zeroed by a memset before each launch.  No CTA
// waits on another: the only shared state is that counter.
#pragma once

#include "fr_launch.h"
#include "fr_trace.cuh"

namespace fr {

enum : uint32_t { PH_IDLE = 0, PH_PRIMARY = 1, PH_NORMAL = 2, PH_SHADOW = 3 };

// Lane state.  Small integers are packed:
//   pix  = px | py << 16
//   meta = req (bits 0-7) | phase (8-9) | tap (10-12) | fp (13) | sample (14-20)
//          | sample flags (21-23) | pixel flags (24-26) | mirror stage (27)
//   cnt  = orbit steps of the current DE (bits 0-10) | march steps (11-30)
// During the normal phase `ro` holds the current stencil tap point (the camera
// ray's origin is no longer needed there).
struct Lane {
    uint32_t pix, meta, cnt;
    float3 ro, rd;
    float t, t1, thit;
    float3 x;         // hit point of the current sample (of the mirror ray in the mirror stage)
    float3 g;         // stencil sum, then the unit normal
    float3 n0;        // Phong shading: the camera hit's normal while the mirror ray runs
    Orbit o;
    float4 acc;       // colour summed over samples
    float dmin;       // nearest hit over samples
};

__device__ __forceinline__ uint32_t L_req(const Lane &S) { return S.meta & 0xffu; }
__device__ __forceinline__ uint32_t L_phase(const Lane &S) { return (S.meta >> 8) & 3u; }
__device__ __forceinline__ void L_set_phase(Lane &S, uint32_t p) { S.meta = (S.meta & ~(3u << 8)) | (p << 8); }
__device__ __forceinline__ int L_tap(const Lane &S) { return (int)((S.meta >> 10) & 7u); }
__device__ __forceinline__ void L_set_tap(Lane &S, int k) { S.meta = (S.meta & ~(7u << 10)) | ((uint32_t)k << 10); }
__device__ __forceinline__ bool L_fp(const Lane &S) { return (S.meta >> 13) & 1u; }
__device__ __forceinline__ void L_set_fp(Lane &S, bool f) { S.meta = (S.meta & ~(1u << 13)) | ((uint32_t)f << 13); }
__device__ __forceinline__ int L_sample(const Lane &S) { return (int)((S.meta >> 14) & 127u); }
__device__ __forceinline__ void L_set_sample(Lane &S, int k) { S.meta = (S.meta & ~(127u << 14)) | ((uint32_t)k << 14); }
__device__ __forceinline__ uint32_t L_sflags(const Lane &S) { return (S.meta >> 21) & 7u; }
__device__ __forceinline__ void L_set_sflags(Lane &S, uint32_t f) { S.meta = (S.meta & ~(7u << 21)) | (f << 21); }
__device__ __forceinline__ uint32_t L_pflags(const Lane &S) { return (S.meta >> 24) & 7u; }
// mirror stage: the march / stencil in progress belongs to the Phong model's mirror ray
__device__ __forceinline__ bool L_rf(const Lane &S) { return (S.meta >> 27) & 1u; }
__device__ __forceinline__ void L_set_rf(Lane &S, bool f) { S.meta = (S.meta & ~(1u << 27)) | ((uint32_t)f << 27); }
__device__ __forceinline__ int L_px(const Lane &S) { return (int)(S.pix & 0xffffu); }
__device__ __forceinline__ int L_py(const Lane &S) { return (int)(S.pix >> 16); }
__device__ __forceinline__ int L_it(const Lane &S) { return (int)(S.cnt & 0x7ffu); }
__device__ __forceinline__ int L_steps(const Lane &S) { return (int)(S.cnt >> 11); }

// per-pixel counters of the counting variant, flushed when the pixel is stored
struct PixCount {
    unsigned long long v[kNStats];
};

// start a DE at p (the Mandelbulb's c is p; kept in `ro` for the normal taps,
// recomputed as ro + t rd during a march)
__device__ __forceinline__ void begin_de(Lane &S, const DevReq &R, float3 p)
{
    S.cnt &= ~0x7ffu;
    if (R.kind == 0)
        julia_init(S.o, p, R.slice_w);
    else
        bulb_init(S.o, p);
}

__device__ __forceinline__ long long pixel_index(const DevReq &R, const Lane &S)
{
    return (long long)L_py(S) * R.width + L_px(S);
}

template <bool COUNT>
__device__ __forceinline__ void store_and_idle(Lane &S, const DevReq &R, PixCount &pc)
{
    const long long idx = pixel_index(R, S);
    const float4 c = mean4(S.acc, R.spp);
    if (R.rgba8) R.rgba8[idx] = pack_rgba8(c);
    if (R.rgba) R.rgba[idx] = c;
    if (R.depth) R.depth[idx] = S.dmin;
    if (R.saved) {
        // the hit point of the nearest sample was written when it was found
        float *sv = reinterpret_cast<float *>(R.saved + idx);
        if (!(L_pflags(S) & kFlagHit)) {
            sv[0] = 0.0f;
            sv[1] = 0.0f;
            sv[2] = 0.0f;
        }
        sv[3] = __uint_as_float(L_pflags(S));
    }
    // the trap of the nearest hit was written when it was found
    if (R.trap && !(L_pflags(S) & kFlagHit)) R.trap[idx] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    L_set_phase(S, PH_IDLE);
    if (COUNT && R.stats) {
#pragma unroll
        for (int k = 0; k < kNStats; k++)
            if (pc.v[k]) atomicAdd(R.stats + k, pc.v[k]);
    }
}

// Start samples sample.. of the lane's pixel until one needs a DE; samples
// whose ray misses the search interval take the background.  When no sample
// is left the pixel is stored and the lane goes idle.
template <bool COUNT>
__device__ void begin_samples(Lane &S, const DevReq &R, PixCount &pc)
{
    int sample = L_sample(S);
    while (sample < R.spp) {
        float3 ro, rd;
        camera_ray(R, L_px(S), L_py(S), sample, ro, rd);
        if (COUNT) pc.v[kStatPrimaryRays] += 1;
        float t0, t1;
        bool fp;
        if (bounds(R, ro, rd, t0, t1, fp)) {
            L_set_sample(S, sample);
            L_set_phase(S, PH_PRIMARY);
            L_set_fp(S, fp);
            S.cnt = 0;
            S.ro = ro;
            S.rd = rd;
            S.t = t0;
            S.t1 = t1;
            begin_de(S, R, along(ro, rd, t0));
            return;
        }
        acc4(S.acc, R.bg);
        sample++;
    }
    L_set_sample(S, sample);
    store_and_idle<COUNT>(S, R, pc);
}

// the camera ray of the current sample hit at S.thit, S.x: keep the nearest
// hit over the samples (depth, saved hit point, orbit trap)
__device__ __forceinline__ void record_hit(Lane &S, const DevReq &R)
{
    if (S.thit < S.dmin) {
        S.dmin = S.thit;
        if (R.saved) {
            float *sv = reinterpret_cast<float *>(R.saved + pixel_index(R, S));
            sv[0] = S.x.x;
            sv[1] = S.x.y;
            sv[2] = S.x.z;
        }
        if (R.trap) R.trap[pixel_index(R, S)] = orbit_trap(R, S.x);
    }
}

template <bool COUNT>
__device__ __forceinline__ void finish_sample(Lane &S, const DevReq &R, float4 c, bool hit, PixCount &pc)
{
    acc4(S.acc, c);
    if (hit) S.meta |= L_sflags(S) << 24;
    L_set_sample(S, L_sample(S) + 1);
    begin_samples<COUNT>(S, R, pc);
}

// Phong shading of the sample once the colour along its mirror ray is known
template <bool COUNT>
__device__ __forceinline__ void finish_phong(Lane &S, const DevReq &R, float3 refl, PixCount &pc)
{
    float3 ro, rd;
    camera_ray(R, L_px(S), L_py(S), L_sample(S), ro, rd);
    const float vis = (L_sflags(S) & kFlagShadow) ? 0.0f : 1.0f;
    L_set_rf(S, false);
    finish_sample<COUNT>(S, R, shade_phong(R, S.n0, rd, vis, refl), true, pc);
}

// Phong shading: cast the mirror ray of the camera ray about the hit's normal
// S.g from x + 4 eps n (a miss, or an empty interval, sees the background)
template <bool COUNT>
__device__ __forceinline__ void start_mirror(Lane &S, const DevReq &R, PixCount &pc)
{
    float3 ro, rd;
    camera_ray(R, L_px(S), L_py(S), L_sample(S), ro, rd);
    S.n0 = S.g;
    if (COUNT) pc.v[kStatReflectRays] += 1;
    const float3 mo = offset_point(S.x, S.n0, R.shadow_off);
    const float3 md = mirror(rd, S.n0);
    float t0, t1;
    bool fp;
    if (!bounds(R, mo, md, t0, t1, fp)) {
        finish_phong<COUNT>(S, R, v3(R.bg), pc);
        return;
    }
    L_set_rf(S, true);
    L_set_phase(S, PH_PRIMARY);
    L_set_fp(S, fp);
    S.cnt = 0;
    S.ro = mo;
    S.rd = md;
    S.t = t0;
    S.t1 = t1;
    begin_de(S, R, along(mo, md, t0));
}

// the unit normal is in S.g: cast the shadow ray, then (Phong) the mirror ray,
// or shade the sample; in the mirror stage it is the mirror hit's normal
template <bool COUNT, bool PHONG>
__device__ __forceinline__ void after_normal(Lane &S, const DevReq &R, PixCount &pc)
{
    if constexpr (PHONG) {
        if (L_rf(S)) {  // the mirror ray's hit, lit by Phong without a shadow ray
            finish_phong<COUNT>(S, R, phong(R, S.g, S.rd, 1.0f), pc);
            return;
        }
    }
    if (R.shadows) {
        const float3 L = v3(R.light);
        const float3 so = offset_point(S.x, S.g, R.shadow_off);
        float s0, s1;
        bool sfp;
        if (COUNT) pc.v[kStatShadowRays] += 1;
        if (bounds(R, so, L, s0, s1, sfp)) {
            L_set_phase(S, PH_SHADOW);
            S.cnt = 0;
            S.ro = so;
            S.rd = L;
            S.t = s0;
            S.t1 = s1;
            begin_de(S, R, along(so, L, s0));
            return;
        }
    }
    if constexpr (PHONG) {
        if (R.shading) {
            start_mirror<COUNT>(S, R, pc);
            return;
        }
    }
    finish_sample<COUNT>(S, R, shade(R, S.g, 1.0f), true, pc);
}

// A DE call of the lane has finished with distance d: advance its ray.
// PHONG compiles the mirror stage in (requests still choose it with R.shading).
template <bool COUNT, bool PHONG>
__device__ void advance(Lane &S, const DevReq &R, float d, PixCount &pc)
{
    const uint32_t phase = L_phase(S);
    if (phase == PH_NORMAL) {
        int tap = L_tap(S);
        tap_accum(S.g, R.normal_mode, R.normal_h, tap, d);
        if (COUNT) pc.v[kStatNormalDE] += 1;
        tap++;
        const int taps = R.normal_mode == 0 ? 4 : 6;
        if (tap < taps) {
            L_set_tap(S, tap);
            S.ro = tap_point(S.x, R.normal_mode, R.normal_h, tap);
            begin_de(S, R, S.ro);
            return;
        }
        S.g = finish_normal(S.g, S.rd);
        after_normal<COUNT, PHONG>(S, R, pc);
        return;
    }
    // one step of a camera or shadow march
    const int steps = L_steps(S) + 1;
    S.cnt = (uint32_t)steps << 11;
    const bool rf = PHONG && L_rf(S);
    if (COUNT) pc.v[phase == PH_SHADOW ? kStatShadowDE : (rf ? kStatReflectDE : kStatPrimaryDE)] += 1;
    bool hit = d < R.eps;
    bool miss = false;
    if (!hit) {
        S.t = march_step(S.t, d, R.max_step);
        if (S.t > S.t1)
            miss = true;
        else if (steps >= R.max_steps)
            hit = true;  // out of steps inside the interval: the listing reports a hit
    }
    if (!hit && !miss) {
        begin_de(S, R, along(S.ro, S.rd, S.t));
        return;
    }
    if (phase == PH_SHADOW) {
        if (hit) L_set_sflags(S, L_sflags(S) | kFlagShadow);
        if constexpr (PHONG) {
            if (R.shading) {
                start_mirror<COUNT>(S, R, pc);
                return;
            }
        }
        finish_sample<COUNT>(S, R, shade(R, S.g, hit ? 0.0f : 1.0f), true, pc);
        return;
    }
    if (miss) {
        if constexpr (PHONG) {
            if (rf) {
                finish_phong<COUNT>(S, R, v3(R.bg), pc);  // the mirror ray sees the background
                return;
            }
        }
        finish_sample<COUNT>(S, R, R.bg, false, pc);
        return;
    }
    S.x = along(S.ro, S.rd, S.t);
    if (!rf) {
        S.thit = S.t;
        L_set_sflags(S, kFlagHit);
        record_hit(S, R);
    }
    if (L_fp(S) && steps == 1) {  // first sample on the cut plane is inside: the cut face
        S.g = v3(R.plane_hat);
        if (!rf) L_set_sflags(S, kFlagHit | kFlagFace);
        after_normal<COUNT, PHONG>(S, R, pc);
        return;
    }
    if (R.normal_mode == 2) {  // analytic normal: one orbit with tangents, no stencil
        int trips;
        S.g = R.kind == 0 ? julia_analytic_normal(R, S.x, S.rd, trips)
                          : bulb_analytic_normal(R, R.power, S.x, S.rd, trips);
        if (COUNT) {
            pc.v[kStatNormalDE] += 1;
            pc.v[kStatOrbit] += trips;
        }
        after_normal<COUNT, PHONG>(S, R, pc);
        return;
    }
    L_set_phase(S, PH_NORMAL);
    L_set_tap(S, 0);
    S.g = v3(0.0f, 0.0f, 0.0f);
    S.ro = tap_point(S.x, R.normal_mode, R.normal_h, 0);
    begin_de(S, R, S.ro);
}

// Queue unit u -> (request, pixel).  Units of a request are its 4 x 8 tiles
// times 32 lanes; slots past the image edge of a ragged tile are empty.
template <bool COUNT>
__device__ __forceinline__ void start_pixel(Lane &S, long long u, const DevReq *sreq,
                                            const long long *sbegin, int nq, PixCount &pc)
{
    int lo = 0, hi = nq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sbegin[mid] <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    const DevReq &R = sreq[lo];
    // 64-bit: with the ragged tiles' padding a request can hold more than 2^31
    // slots even though width * height * spp < 2^31
    const long long local = u - sbegin[lo];
    const long long tile = local >> 5;
    const int w = (int)(local & 31);
    const long long ty = tile / R.tiles_x;
    const int px = (int)(tile - ty * R.tiles_x) * kTileW + (w & (kTileW - 1));
    const int py = (int)ty * kTileH + (w / kTileW);
    if (px >= R.width || py >= R.height) return;  // empty slot: the lane stays idle
    S.pix = (uint32_t)px | ((uint32_t)py << 16);
    S.meta = (uint32_t)lo;  // phase idle, sample 0, flags 0
    S.acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    S.dmin = __int_as_float(0x7f800000);
    if (COUNT)
#pragma unroll
        for (int k = 0; k < kNStats; k++) pc.v[k] = 0;
    begin_samples<COUNT>(S, R, pc);
}

// resident 256-thread CTAs the register budget is fitted to
#ifndef FR_PERSIST_MIN_BLOCKS
#define FR_PERSIST_MIN_BLOCKS 2
#endif

// REFILL = false is the same lane state machine without the queue: every warp
// takes the 32 pixel slots of one tile at launch (grid = all tiles) and ends
// when its lanes are done.  Lanes of different phases still share one DE code
// path and never wait for each other's orbits, but nothing is refilled.
template <int KJ, bool COUNT, bool REFILL, bool PHONG>
__global__ void __launch_bounds__(256, FR_PERSIST_MIN_BLOCKS) persist_kernel(const __grid_constant__ BatchArgs A)
{
    extern __shared__ float4 smem[];
    DevReq *sreq = reinterpret_cast<DevReq *>(smem);
    __shared__ long long sbegin[kMaxReqPerLaunch];
    const int nq = A.n_reqs;
    {
        // stage the request table: parameter space -> shared memory
        const float4 *src = reinterpret_cast<const float4 *>(A.reqs);
        const int words = nq * (int)(sizeof(DevReq) / sizeof(float4));
        for (int i = threadIdx.x; i < words; i += blockDim.x) smem[i] = src[i];
        for (int i = threadIdx.x; i < nq; i += blockDim.x) sbegin[i] = A.reqs[i].unit_begin;
    }
    __syncthreads();

    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const unsigned long long total = (unsigned long long)A.total_units;
    Lane S;
    S.meta = 0;  // idle
    PixCount pc;
#pragma unroll
    for (int k = 0; k < kNStats; k++) pc.v[k] = 0;
    bool exhausted = false;
    if (!REFILL) {
        const long long u = ((long long)blockIdx.x * blockDim.x + threadIdx.x);
        if ((unsigned long long)u < total) start_pixel<COUNT>(S, u, sreq, sbegin, nq, pc);
        exhausted = true;
    }

    for (;;) {
        // ---- refill idle lanes (warp-uniform control flow): one atomicAdd takes
        // exactly as many queue units as the warp has idle lanes
        unsigned idle = __ballot_sync(FULL, L_phase(S) == PH_IDLE);
        while (idle != 0u && !exhausted && (__popc(idle) >= A.refill_threshold || idle == FULL)) {
            const int n = __popc(idle);
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(A.queue, (unsigned long long)n);
            base = __shfl_sync(FULL, base, 0);
            if (base + (unsigned long long)n >= total) exhausted = true;
            if (L_phase(S) == PH_IDLE) {
                const unsigned long long u = base + (unsigned long long)__popc(idle & below);
                if (u < total) start_pixel<COUNT>(S, (long long)u, sreq, sbegin, nq, pc);
            }
            idle = __ballot_sync(FULL, L_phase(S) == PH_IDLE);
        }
        if (idle == FULL && exhausted) break;
        // ---- a few orbit steps for every busy lane, then the ray's next move
        if (L_phase(S) != PH_IDLE) {
            const DevReq &R = sreq[L_req(S)];
            if (R.kind == 0) {
                const float4 c = R.c;
                bool done = false;
                if (R.power == 2) {
#pragma unroll
                    for (int j = 0; j < KJ; j++)
                        if (!done) {
                            julia2_step(S.o, c);
                            S.cnt++;
                            done = (S.o.m > R.esc2) || (L_it(S) >= R.max_iter);
                        }
                } else {
#pragma unroll
                    for (int j = 0; j < KJ; j++)
                        if (!done) {
                            julia3_step(S.o, c);
                            S.cnt++;
                            done = (S.o.m > R.esc2) || (L_it(S) >= R.max_iter);
                        }
                }
                if (done) {
                    if (COUNT) pc.v[kStatOrbit] += L_it(S);
                    advance<COUNT, PHONG>(S, R, julia_dist(S.o), pc);
                }
            } else {
                const float3 cpt = (L_phase(S) == PH_NORMAL) ? S.ro : along(S.ro, S.rd, S.t);
                if (R.bulb_alg)
                    bulb_step_alg(S.o, cpt, R.power);
                else
                    bulb_step(S.o, cpt, R.power);
                S.cnt++;
                if ((S.o.m > R.esc2) || (L_it(S) >= R.max_iter)) {
                    if (COUNT) pc.v[kStatOrbit] += L_it(S);
                    advance<COUNT, PHONG>(S, R, bulb_dist(S.o), pc);
                }
            }
        }
    }
}

template <int KJ, bool COUNT, bool REFILL, bool PHONG = false>
static cudaError_t launch_persist_t(const BatchArgs &A, int block, int ctas_per_sm, cudaStream_t s)
{
    const size_t smem = (size_t)A.n_reqs * sizeof(DevReq);
    if constexpr (!REFILL) {  // (if constexpr: each unit instantiates only its own kernels)
        const long long grid = (A.total_units + block - 1) / block;
        persist_kernel<KJ, COUNT, false, PHONG><<<(unsigned)grid, block, smem, s>>>(A);
        return cudaGetLastError();
    } else {
        int dev = 0, sms = 0, fit = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, persist_kernel<KJ, COUNT, true, PHONG>, block,
                                                               smem)) !=
            cudaSuccess)
            return e;
        if (fit < 1) return cudaErrorInvalidConfiguration;
        const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < fit) ? ctas_per_sm : fit;
        if ((e = cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
        persist_kernel<KJ, COUNT, true, PHONG><<<sms * per_sm, block, smem, s>>>(A);
        return cudaGetLastError();
    }
}

static_assert(sizeof(BatchArgs) <= 32764, "the request table must fit the kernel parameter space");

}  // namespace fr

