// fr_trace.cuh -- the one-ray-per-thread path built on fr_device.cuh: the
// march loop, the normal stencils, one traced sample (interval -> march ->
// normal -> shadow -> shade) and one pixel (samples -> mean colour, nearest
// depth -> store).
#pragma once

#include "fr_device.cuh"

namespace fr {

// Sphere tracing (Listing "Julia Set ray cast"): from t0, d = DE(ro + t rd);
// d < eps -> hit; t += min(d, max_step); t > t1 -> miss; running out of steps
// inside the interval is reported as a hit at the current t.
template <int KIND, int U, bool COUNT>
__device__ __forceinline__ bool march(const DevReq &R, float3 ro, float3 rd, float t0, float t1,
                                      float &t_out, int &steps_out, Counters &cnt, int slot)
{
    float t = t0;
    int steps = 0;
    bool hit = true;
    for (int i = 0; i < R.max_steps; i++) {
        int trips;
        float d = de<KIND, U>(R, along(ro, rd, t), trips);
        steps++;
        if (COUNT) cnt.v[kStatOrbit] += trips;
        if (d < R.eps) break;
        t = march_step(t, d, R.max_step);
        if (t > t1) {
            hit = false;
            break;
        }
    }
    if (COUNT) cnt.v[slot] += steps;
    t_out = t;
    steps_out = steps;
    return hit;
}

// Normal = normalised gradient of the DE at x from the stencil taps of
// tap_point / tap_accum (tetrahedral Eq. 5 or central differences), or the
// analytic normal (one orbit carrying its Jacobian); a zero or non-finite
// gradient gives -rd.  The Mandelbulb's analytic normal is compiled only into
// the BAN instantiations (requests that ask for it are launched there): its
// orbit is a third inlined copy of the trig step, and carried in every kernel
// it slowed the Phong frame by 7 % (instruction fetch).  BAN 1 inlines it (the
// single-request kernels for such requests), BAN 2 calls it out of line (the
// batch kernels, which carry it for every launch).
template <int KIND, int U, bool COUNT, int BAN>
__device__ __forceinline__ float3 normal_at(const DevReq &R, float3 x, float3 rd, Counters &cnt)
{
    if ((KIND == 0 || BAN) && R.normal_mode == 2) {
        int trips;
        const float3 n = KIND == 0 ? julia_analytic_normal(R, x, rd, trips)
                                   : BAN == 2 ? bulb_analytic_normal_ool(R, KIND == 2 ? 8 : R.power, x, rd, trips)
                                                 : bulb_analytic_normal(R, KIND == 2 ? 8 : R.power, x, rd, trips);
        if (COUNT) {
            cnt.v[kStatNormalDE] += 1;
            cnt.v[kStatOrbit] += trips;
        }
        return n;
    }
    const int taps = R.normal_mode == 0 ? 4 : 6;
    float3 g = v3(0.0f, 0.0f, 0.0f);
    for (int k = 0; k < taps; k++) {
        int trips;
        const float d = de<KIND, U>(R, tap_point(x, R.normal_mode, R.normal_h, k), trips);
        tap_accum(g, R.normal_mode, R.normal_h, k, d);
        if (COUNT) cnt.v[kStatOrbit] += trips;
    }
    if (COUNT) cnt.v[kStatNormalDE] += taps;
    return finish_normal(g, rd);
}

// One camera sample: interval, march, normal (the plane's for a cut-face hit:
// interval starts on the plane and the first DE sample is already inside),
// optional shadow ray from x + 4 eps n toward the light, Lambert shading.
//
// The camera ray and the shadow ray go through one march loop (two passes of
// one loop body) and the stencil has its own loop, so the DE is inlined twice.
// Inlined three times (a march loop per ray), the Mandelbulb's math-library
// code left the warps stalling on instruction fetch (5.0 stalls per issued
// instruction against 0.9; 1.31 against 1.03 ms for the 1080p frame).  A
// single call site for all DE evaluations (one loop whose trips pick the point
// by phase) measured slower again (1.10 ms; Julia 256^2 0.149 against
// 0.117 ms): its phase bookkeeping costs more than the smaller code saves.
template <int KIND, int U, bool COUNT, int BAN>
__device__ __forceinline__ float4 trace_sample(const DevReq &R, float3 ro, float3 rd, float &t_hit,
                                               uint32_t &flags, float3 &xhit, Counters &cnt)
{
    flags = 0;
    t_hit = __int_as_float(0x7f800000);
    float t0, t1, t;
    bool fp;
    int steps;
    if (!bounds(R, ro, rd, t0, t1, fp)) return R.bg;
    float3 mro = ro, mrd = rd;  // the ray being marched
    float3 x = v3(0.0f, 0.0f, 0.0f), n = x;
    uint32_t fl = 0;
    float vis = 1.0f;
#pragma unroll 1
    for (int pass = 0; pass < 2; pass++) {
        const bool hit = march<KIND, U, COUNT>(R, mro, mrd, t0, t1, t, steps, cnt,
                                               pass == 0 ? kStatPrimaryDE : kStatShadowDE);
        if (pass == 1) {
            if (hit) {
                vis = 0.0f;
                fl |= kFlagShadow;
            }
            break;
        }
        if (!hit) return R.bg;
        x = along(ro, rd, t);
        t_hit = t;
        fl = kFlagHit;
        if (fp && steps == 1) {
            n = v3(R.plane_hat);
            fl |= kFlagFace;
        } else {
            n = normal_at<KIND, U, COUNT, BAN>(R, x, rd, cnt);
        }
        if (!R.shadows) break;
        if (COUNT) cnt.v[kStatShadowRays] += 1;
        mro = offset_point(x, n, R.shadow_off);
        mrd = v3(R.light);
        bool sfp;
        if (!bounds(R, mro, mrd, t0, t1, sfp)) break;
    }
    flags = fl;
    xhit = x;
    return shade(R, n, vis);
}

// The same sample with the closest-hit model of Sec. 3.1 available (requests
// with R.shading set): after the optional shadow ray a third pass marches the
// mirror ray from x + 4 eps n; its hit is lit by Phong without a shadow ray or
// a further bounce (a miss sees the background), and the result is weighted
// by Fresnel-Schlick in shade_phong.  The two hits' normals share one stencil
// call, so the DE is still inlined twice.  Kept apart from the Lambert-only
// loop above, which holds fewer live values.
template <int KIND, int U, bool COUNT, int BAN>
__device__ __forceinline__ float4 trace_sample_phong(const DevReq &R, float3 ro, float3 rd, float &t_hit,
                                                     uint32_t &flags, float3 &xhit, Counters &cnt)
{
    flags = 0;
    t_hit = __int_as_float(0x7f800000);
    float t0, t1, t;
    bool fp;
    int steps;
    if (!bounds(R, ro, rd, t0, t1, fp)) return R.bg;
    enum { kCamera = 0, kShadow = 1, kReflect = 2 };
    float3 mro = ro, mrd = rd;  // the ray being marched
    float3 x = v3(0.0f, 0.0f, 0.0f), n = x;
    float3 refl = v3(R.bg);     // colour along the mirror ray (Phong shading)
    uint32_t fl = 0;
    float vis = 1.0f;
    int pass = kCamera;
#pragma unroll 1
    for (;;) {
        const bool hit = march<KIND, U, COUNT>(R, mro, mrd, t0, t1, t, steps, cnt,
                                               pass == kCamera   ? kStatPrimaryDE
                                               : pass == kShadow ? kStatShadowDE
                                                                 : kStatReflectDE);
        if (pass == kShadow) {
            if (hit) {
                vis = 0.0f;
                fl |= kFlagShadow;
            }
        } else {
            if (!hit) {
                if (pass == kCamera) return R.bg;
                break;  // the mirror ray sees the background
            }
            const float3 xh = along(mro, mrd, t);
            const bool face = fp && steps == 1;
            const float3 nh = face ? v3(R.plane_hat) : normal_at<KIND, U, COUNT, BAN>(R, xh, mrd, cnt);
            if (pass == kReflect) {
                refl = phong(R, nh, mrd, 1.0f);  // no shadow ray, no further bounce
                break;
            }
            x = xh;
            n = nh;
            t_hit = t;
            fl = kFlagHit | (face ? kFlagFace : 0u);
        }
        // the next ray from the hit: the shadow ray, then the mirror ray
        if (pass == kCamera && R.shadows) {
            if (COUNT) cnt.v[kStatShadowRays] += 1;
            mro = offset_point(x, n, R.shadow_off);
            mrd = v3(R.light);
            if (bounds(R, mro, mrd, t0, t1, fp)) {
                pass = kShadow;
                continue;
            }
        }
        if (!R.shading) break;
        if (COUNT) cnt.v[kStatReflectRays] += 1;
        mro = offset_point(x, n, R.shadow_off);
        mrd = mirror(rd, n);
        if (!bounds(R, mro, mrd, t0, t1, fp)) break;
        pass = kReflect;
    }
    flags = fl;
    xhit = x;
    return R.shading ? shade_phong(R, n, rd, vis, refl) : shade(R, n, vis);
}

// One pixel: spp samples, mean colour, nearest hit depth, hit point of the
// nearest hit, OR of the flags; the per-pixel extras (float RGBA, saved state,
// trap) are stored here, the packed colour and the depth are returned for the
// warp's quad store (store_rgba8_depth).  PHONG compiles the Phong +
// mirror-ray path in (requests still choose it with R.shading); without it the
// Lambert-only code keeps fewer registers.
template <int KIND, int U, bool COUNT, bool PHONG, int BAN = 0>
__device__ __forceinline__ void render_pixel(const DevReq &R, int px, int py, Counters &cnt, uint32_t &c8,
                                             float &depth)
{
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float dmin = __int_as_float(0x7f800000);
    float3 xh = v3(0.0f, 0.0f, 0.0f);
    uint32_t fl = 0;
    for (int s = 0; s < R.spp; s++) {
        float3 ro, rd, x;
        float t;
        uint32_t f;
        camera_ray(R, px, py, s, ro, rd);
        if (COUNT) cnt.v[kStatPrimaryRays] += 1;
        float4 c;
        if constexpr (PHONG)
            c = trace_sample_phong<KIND, U, COUNT, BAN>(R, ro, rd, t, f, x, cnt);
        else
            c = trace_sample<KIND, U, COUNT, BAN>(R, ro, rd, t, f, x, cnt);
        acc4(acc, c);
        if ((f & kFlagHit) && t < dmin) {
            dmin = t;
            xh = x;
        }
        fl |= f;
    }
    const float4 mean = mean4(acc, R.spp);
    store_pixel_extras(R, (long long)py * R.width + px, mean, xh, fl);
    c8 = pack_rgba8(mean);
    depth = dmin;
}

// The same pixel, called by all 32 lanes of the warp together, with its spp
// samples on R.spl adjacent lanes: sample k on the k-th when R.spl = spp (2, 4
// or 8), all samples in turn on one lane when R.spl = 1 (requests of a batch
// launch that some other request's spl > 1 put on this code).  With spl = spp
// the warp's 32 rays come from 32 / spp neighbouring pixels (a tile
// 4 x 8 / spp pixels) whose samples are a fraction of a pixel apart, so they
// take nearly the same march and orbit lengths and keep more lanes busy.  The
// pixel's first lane folds in the other lanes' results in sample order -- the
// same additions in the same order as render_pixel's loop -- so both layouts
// give the same bits; its results are the pixel's.  `valid`: the pixel lies
// inside the image.  (Kernels of their own: carried in the one-lane kernels,
// this code cost the 1080p frame 2.5 %.)
template <int KIND, int U, bool COUNT, bool PHONG, int BAN = 0>
__device__ __forceinline__ void render_pixel_lanes(const DevReq &R, int px, int py, int sample, bool valid,
                                                   Counters &cnt, uint32_t &c8, float &depth)
{
    float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float dmin = __int_as_float(0x7f800000);
    float3 xh = v3(0.0f, 0.0f, 0.0f);
    uint32_t fl = 0;
    if (valid) {
        for (int s = sample; s < R.spp; s += R.spl) {
            float3 ro, rd, x;
            float t;
            uint32_t f;
            camera_ray(R, px, py, s, ro, rd);
            if (COUNT) cnt.v[kStatPrimaryRays] += 1;
            float4 c;
            if constexpr (PHONG)
                c = trace_sample_phong<KIND, U, COUNT, BAN>(R, ro, rd, t, f, x, cnt);
            else
                c = trace_sample<KIND, U, COUNT, BAN>(R, ro, rd, t, f, x, cnt);
            acc4(acc, c);
            if ((f & kFlagHit) && t < dmin) {
                dmin = t;
                xh = x;
            }
            fl |= f;
        }
    }
    if (R.spl > 1) {
        // the pixel's samples from its lanes, in sample order: every lane folds,
        // so the shuffles read each lane's own sample (c0 .. f0)
        const unsigned full = 0xffffffffu;
        const int first = (threadIdx.x & 31) & ~(R.spl - 1);
        const float4 c0 = acc;
        const float t0 = dmin;
        const float3 x0 = xh;
        const uint32_t f0 = fl;
        acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        dmin = __int_as_float(0x7f800000);
        fl = 0;
        for (int j = 0; j < R.spl; j++) {
            const float4 cj = make_float4(__shfl_sync(full, c0.x, first + j), __shfl_sync(full, c0.y, first + j),
                                          __shfl_sync(full, c0.z, first + j), __shfl_sync(full, c0.w, first + j));
            const float tj = __shfl_sync(full, t0, first + j);
            const float3 xj = v3(__shfl_sync(full, x0.x, first + j), __shfl_sync(full, x0.y, first + j),
                                 __shfl_sync(full, x0.z, first + j));
            const uint32_t fj = __shfl_sync(full, f0, first + j);
            acc4(acc, cj);
            if ((fj & kFlagHit) && tj < dmin) {
                dmin = tj;
                xh = xj;
            }
            fl |= fj;
        }
    }
    const float4 mean = mean4(acc, R.spp);
    if (valid && sample == 0) store_pixel_extras(R, (long long)py * R.width + px, mean, xh, fl);
    c8 = pack_rgba8(mean);
    depth = dmin;
}

}  // namespace fr
