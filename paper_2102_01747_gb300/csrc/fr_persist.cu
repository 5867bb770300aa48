// fr_persist.cu -- persistent, divergence-compacting forward kernel.
//
// Why: in the one-ray-per-thread kernel a warp runs until its slowest lane is
// done, twice over: rays need 1..max_steps march steps, and every DE call
// needs 1..max_iter orbit steps (Mandelbulb 1080p: 2.7 on average, up to 12).
// Measured on that kernel: 10 of 32 lanes active per issued instruction and a
// long tail of nearly empty SMs.
//
// How: CTAs stay resident (grid = SMs x resident CTAs).  Each lane holds one
// pixel's complete state: its sample, the phase of the current ray (camera
// march, normal taps, shadow march), the march variables and one orbit in
// progress.  Every round of the warp loop advances each lane's orbit by a few
// steps (Julia: the unroll depth K, Mandelbulb: one); a lane whose orbit has
// escaped or reached max_iter turns it into a distance (Eq. 2), feeds it to
// its ray's state machine (march step, normal tap or shadow step, Listing
// "Julia Set ray cast") and starts its next orbit right away, so lanes never
// wait for each other's orbits or rays.  A finished pixel is stored and its
// lane refilled from one queue over every pixel of every request: once
// `refill_threshold` lanes are idle the warp takes that many pixels with a
// single atomicAdd and hands them out by ballot rank.  A warp is short of work
// only at the very end of the queue.
//
// The orbit steps, the distance, the march update and the stencils are the
// same device functions the one-ray-per-thread kernel uses, in the same order
// per ray, so both kernels produce the same image.
//
// The request table (<= 64 DevReq) travels in the kernel parameters
// (__grid_constant__) and is staged into shared memory by every CTA, since the
// lanes of one warp may read different requests.  The queue head lives in the
// caller's workspace and is zeroed by a memset before each launch.  No CTA
// waits on another: the only shared state is that counter.
#include "fr_launch.h"
#include "fr_trace.cuh"

namespace fr {

enum : int { PH_IDLE = 0, PH_PRIMARY = 1, PH_NORMAL = 2, PH_SHADOW = 3 };

struct Lane {
    int req;          // request index (shared-memory table)
    int px, py, sample;
    int phase;
    int steps;        // DE calls of the current march
    int tap;          // current stencil tap
    int it;           // orbit steps of the current DE
    bool fp;          // march interval starts on the cut plane
    float3 ro, rd;
    float t, t1;
    float thit;       // depth of the current sample's camera-ray hit
    float3 x;         // hit point of the current sample
    float3 g;         // stencil sum, then the unit normal
    float3 cpt;       // point of the current DE (the Mandelbulb's c)
    Orbit o;
    uint32_t sflags;  // flags of the current sample
    float4 acc;       // colour summed over samples
    float dmin;       // nearest hit over samples
    float3 xbest;
    uint32_t pflags;  // flags ORed over samples
};

// per-pixel counters of the counting variant, flushed when the pixel is stored
struct PixCount {
    unsigned long long v[kNStats];
};

__device__ __forceinline__ void begin_de(Lane &S, const DevReq &R, float3 p)
{
    S.cpt = p;
    S.it = 0;
    if (R.kind == 0)
        julia_init(S.o, p, R.slice_w);
    else
        bulb_init(S.o, p);
}

template <bool COUNT>
__device__ __forceinline__ void store_and_idle(Lane &S, const DevReq &R, PixCount &pc)
{
    const float fs = (float)R.spp;
    const float4 acc = make_float4(S.acc.x / fs, S.acc.y / fs, S.acc.z / fs, S.acc.w / fs);
    store_pixel(R, S.px, S.py, acc, S.dmin, S.xbest, S.pflags);
    S.phase = PH_IDLE;
    if (COUNT && R.stats) {
#pragma unroll
        for (int k = 0; k < kNStats; k++)
            if (pc.v[k]) atomicAdd(R.stats + k, pc.v[k]);
    }
}

// Start samples S.sample.. of the lane's pixel until one needs a DE; samples
// whose ray misses the search interval take the background.  When no sample
// is left the pixel is stored and the lane goes idle.
template <bool COUNT>
__device__ void begin_samples(Lane &S, const DevReq &R, PixCount &pc)
{
    while (S.sample < R.spp) {
        float3 ro, rd;
        camera_ray(R, S.px, S.py, S.sample, ro, rd);
        if (COUNT) pc.v[kStatPrimaryRays] += 1;
        float t0, t1;
        bool fp;
        if (bounds(R, ro, rd, t0, t1, fp)) {
            S.phase = PH_PRIMARY;
            S.ro = ro;
            S.rd = rd;
            S.t = t0;
            S.t1 = t1;
            S.fp = fp;
            S.steps = 0;
            begin_de(S, R, along(ro, rd, t0));
            return;
        }
        S.acc.x += R.bg.x;
        S.acc.y += R.bg.y;
        S.acc.z += R.bg.z;
        S.acc.w += R.bg.w;
        S.sample++;
    }
    store_and_idle<COUNT>(S, R, pc);
}

template <bool COUNT>
__device__ __forceinline__ void finish_sample(Lane &S, const DevReq &R, float4 c, bool hit, PixCount &pc)
{
    S.acc.x += c.x;
    S.acc.y += c.y;
    S.acc.z += c.z;
    S.acc.w += c.w;
    if (hit) {
        if (S.thit < S.dmin) {
            S.dmin = S.thit;
            S.xbest = S.x;
        }
        S.pflags |= S.sflags;
    }
    S.sample++;
    begin_samples<COUNT>(S, R, pc);
}

// the unit normal is in S.g: cast the shadow ray, or shade the sample
template <bool COUNT>
__device__ __forceinline__ void after_normal(Lane &S, const DevReq &R, PixCount &pc)
{
    if (R.shadows) {
        const float3 L = v3(R.light);
        const float3 so = S.x + S.g * R.shadow_off;
        float s0, s1;
        bool sfp;
        if (COUNT) pc.v[kStatShadowRays] += 1;
        if (bounds(R, so, L, s0, s1, sfp)) {
            S.phase = PH_SHADOW;
            S.ro = so;
            S.rd = L;
            S.t = s0;
            S.t1 = s1;
            S.steps = 0;
            begin_de(S, R, along(so, L, s0));
            return;
        }
    }
    finish_sample<COUNT>(S, R, shade(R, S.g, 1.0f), true, pc);
}

// A DE call of the lane has finished with distance d: advance its ray.
template <bool COUNT>
__device__ void advance(Lane &S, const DevReq &R, float d, PixCount &pc)
{
    if (S.phase == PH_NORMAL) {
        tap_accum(S.g, R.normal_mode, R.normal_h, S.tap, d);
        if (COUNT) pc.v[kStatNormalDE] += 1;
        S.tap++;
        const int taps = R.normal_mode == 0 ? 4 : 6;
        if (S.tap < taps) {
            begin_de(S, R, tap_point(S.x, R.normal_mode, R.normal_h, S.tap));
            return;
        }
        S.g = finish_normal(S.g, S.rd);
        after_normal<COUNT>(S, R, pc);
        return;
    }
    // one step of a camera or shadow march
    S.steps++;
    if (COUNT) pc.v[S.phase == PH_PRIMARY ? kStatPrimaryDE : kStatShadowDE] += 1;
    bool hit = d < R.eps;
    bool miss = false;
    if (!hit) {
        S.t += (d < R.max_step) ? d : R.max_step;
        if (S.t > S.t1)
            miss = true;
        else if (S.steps >= R.max_steps)
            hit = true;  // out of steps inside the interval: the listing reports a hit
    }
    if (!hit && !miss) {
        begin_de(S, R, along(S.ro, S.rd, S.t));
        return;
    }
    if (S.phase == PH_SHADOW) {
        if (hit) S.sflags |= kFlagShadow;
        finish_sample<COUNT>(S, R, shade(R, S.g, hit ? 0.0f : 1.0f), true, pc);
        return;
    }
    if (miss) {
        finish_sample<COUNT>(S, R, R.bg, false, pc);
        return;
    }
    S.thit = S.t;
    S.x = along(S.ro, S.rd, S.t);
    S.sflags = kFlagHit;
    if (S.fp && S.steps == 1) {  // first sample on the cut plane is inside: the cut face
        S.g = v3(R.plane_hat);
        S.sflags |= kFlagFace;
        after_normal<COUNT>(S, R, pc);
        return;
    }
    S.phase = PH_NORMAL;
    S.tap = 0;
    S.g = v3(0.0f, 0.0f, 0.0f);
    begin_de(S, R, tap_point(S.x, R.normal_mode, R.normal_h, 0));
}

// Queue unit u -> (request, pixel).  Units of a request are its 8 x 4 tiles
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
    const long long local = u - sbegin[lo];
    const long long tile = local >> 5;
    const int w = (int)(local & 31);
    const int px = (int)(tile % R.tiles_x) * kTileW + (w & (kTileW - 1));
    const int py = (int)(tile / R.tiles_x) * kTileH + (w / kTileW);
    if (px >= R.width || py >= R.height) return;  // empty slot: the lane stays idle
    S.req = lo;
    S.px = px;
    S.py = py;
    S.sample = 0;
    S.acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    S.dmin = __int_as_float(0x7f800000);
    S.xbest = v3(0.0f, 0.0f, 0.0f);
    S.pflags = 0;
    if (COUNT)
#pragma unroll
        for (int k = 0; k < kNStats; k++) pc.v[k] = 0;
    begin_samples<COUNT>(S, R, pc);
}

// resident 256-thread CTAs the register budget is fitted to (3 -> <= 85 registers, 24 warps per SM)
#ifndef FR_PERSIST_MIN_BLOCKS
#define FR_PERSIST_MIN_BLOCKS 2
#endif

template <int KJ, bool COUNT>
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
    S.phase = PH_IDLE;
    S.req = 0;
    PixCount pc;
#pragma unroll
    for (int k = 0; k < kNStats; k++) pc.v[k] = 0;
    bool exhausted = false;

    for (;;) {
        // ---- refill idle lanes (warp-uniform control flow)
        unsigned idle = __ballot_sync(FULL, S.phase == PH_IDLE);
        while (idle != 0u && !exhausted && (__popc(idle) >= A.refill_threshold || idle == FULL)) {
            const int n = __popc(idle);
            const int leader = __ffs(idle) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(A.queue, (unsigned long long)n);
            base = __shfl_sync(FULL, base, leader);
            if (base + (unsigned long long)n >= total) exhausted = true;
            if (S.phase == PH_IDLE) {
                const unsigned long long u = base + (unsigned long long)__popc(idle & below);
                if (u < total) start_pixel<COUNT>(S, (long long)u, sreq, sbegin, nq, pc);
            }
            idle = __ballot_sync(FULL, S.phase == PH_IDLE);
        }
        if (idle == FULL) {
            if (exhausted) break;
            continue;
        }
        // ---- a few orbit steps for every busy lane, then the ray's next move
        if (S.phase != PH_IDLE) {
            const DevReq &R = sreq[S.req];
            bool done = false;
            if (R.kind == 0) {
                const float4 c = R.c;
                if (R.power == 2) {
#pragma unroll
                    for (int j = 0; j < KJ; j++)
                        if (!done) {
                            julia2_step(S.o, c);
                            S.it++;
                            done = (S.o.m > R.esc2) || (S.it >= R.max_iter);
                        }
                } else {
#pragma unroll
                    for (int j = 0; j < KJ; j++)
                        if (!done) {
                            julia3_step(S.o, c);
                            S.it++;
                            done = (S.o.m > R.esc2) || (S.it >= R.max_iter);
                        }
                }
                if (done) {
                    if (COUNT) pc.v[kStatOrbit] += S.it;
                    advance<COUNT>(S, R, julia_dist(S.o), pc);
                }
            } else {
                bulb_step(S.o, S.cpt, R.power);
                S.it++;
                if ((S.o.m > R.esc2) || (S.it >= R.max_iter)) {
                    if (COUNT) pc.v[kStatOrbit] += S.it;
                    advance<COUNT>(S, R, bulb_dist(S.o), pc);
                }
            }
        }
    }
}

template <int KJ, bool COUNT>
static cudaError_t launch_persist_t(const BatchArgs &A, int block, int ctas_per_sm, cudaStream_t s)
{
    const size_t smem = (size_t)A.n_reqs * sizeof(DevReq);
    int dev = 0, sms = 0, fit = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, persist_kernel<KJ, COUNT>, block, smem)) !=
        cudaSuccess)
        return e;
    if (fit < 1) return cudaErrorInvalidConfiguration;
    const int per_sm = (ctas_per_sm > 0 && ctas_per_sm < fit) ? ctas_per_sm : fit;
    if ((e = cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), s)) != cudaSuccess) return e;
    persist_kernel<KJ, COUNT><<<sms * per_sm, block, smem, s>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_persist(const BatchArgs &A, int block, int ctas_per_sm, int unroll, bool count,
                           cudaStream_t s)
{
    if (count) return launch_persist_t<2, true>(A, block, ctas_per_sm, s);
    if (unroll == 4) return launch_persist_t<4, false>(A, block, ctas_per_sm, s);
    if (unroll == 2) return launch_persist_t<2, false>(A, block, ctas_per_sm, s);
    return launch_persist_t<1, false>(A, block, ctas_per_sm, s);
}

}  // namespace fr
