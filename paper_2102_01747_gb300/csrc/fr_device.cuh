// fr_device.cuh -- device-side building blocks of the sphere tracer (sm_103a).
//
// One request is a DevReq: the public parameter structs of include/fr.h resolved
// on the host into what the kernels read (camera basis, normalised light,
// squared radii, output pointers).  Every routine here computes in FP32 with
// the accurate CUDA math library (no --use_fast_math, no __xxxf intrinsics);
// the compiler may contract a*b+c into FFMA.
//
// Paper passages (da Silva, Novello, Lopes, Velho, "Real-time rendering of
// complex fractals"):
//   julia_de   Listing "Julia Set distance", Eqs. 2-4 (degree p, slice w)
//   bulb_de    Listing "Mandelbulb distance", Eq. 1 (White-Nylander power)
//   bounds     Sec. 3.1: search interval [eps, 7000] clipped by a bounding
//              sphere and the cutting plane (Fig. 1)
//   march      Listing "Julia Set ray cast" (step min(d, max_step), hit d < eps,
//              miss t > t1, step cap counts as a hit)
//   normal     Eq. 5 / Listing "Normal calculation" (tetrahedral), or central
//              differences
//   shade      Lambert closest-hit with an optional shadow ray
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fr {

constexpr int kTileW = 8;   // a warp covers an 8 x 4 tile of pixels
constexpr int kTileH = 4;

// statistics slots (same order as FR_STAT_* in include/fr.h)
constexpr int kStatPrimaryRays = 0, kStatShadowRays = 1, kStatPrimaryDE = 2,
              kStatNormalDE = 3, kStatShadowDE = 4, kStatOrbit = 5, kNStats = 6;

constexpr uint32_t kFlagHit = 1u, kFlagFace = 2u, kFlagShadow = 4u;

struct __align__(16) DevReq {
    float4 c;             // Julia constant (real, i, j, k)
    int kind;             // 0 Julia, 1 Mandelbulb
    int power;            // Julia p or Mandelbulb n
    int max_iter;
    int max_steps;
    float slice_w;
    float esc2;           // Julia escape_r2, Mandelbulb bailout^2
    float eps;
    float max_step;
    float bound_r2;
    float normal_h;       // resolved stencil size
    float shadow_off;     // 4 * eps
    int normal_mode;      // 0 tetra, 1 central
    int plane_on;
    int shadows;
    int spp;
    int pad0;
    float4 plane;         // n.xyz, offset
    float4 plane_hat;     // n / |n|
    float4 eye;
    float4 fwd;
    float4 right;
    float4 up;
    float th;             // tan(fov_y / 2)
    float th_aspect;      // th * width / height
    float inv_w, inv_h;
    int width, height;
    int tiles_x;
    uint32_t seed;
    float4 light;         // normalised direction toward the light
    float4 albedo;
    float ka, kd;
    float pad1, pad2;
    float4 bg;
    uint32_t *rgba8;
    float4 *rgba;
    float *depth;
    float4 *saved;
    unsigned long long *stats;
    long long unit_begin; // first queue unit of this request inside a batch
    long long n_units;    // tiles * 32
};

// ------------------------------------------------------------------ vectors
__device__ __forceinline__ float3 v3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 v3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return v3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 normalize3(float3 a)
{
    float l = sqrtf(dot3(a, a));
    return v3(a.x / l, a.y / l, a.z / l);
}
// ro + t * rd, one FFMA per component
__device__ __forceinline__ float3 along(float3 ro, float3 rd, float t)
{
    return v3(fmaf(rd.x, t, ro.x), fmaf(rd.y, t, ro.y), fmaf(rd.z, t, ro.z));
}

// ------------------------------------------------------------------ jitter
// splitmix64 (Steele, Lea, Flood 2014): golden-ratio increment, then the
// xor-shift-multiply finaliser.  Counter = (seed << 40) + pixel*spp + sample;
// top 24 bits -> sx, next 24 bits -> sy (exact multiples of 2^-24).
__device__ __forceinline__ uint64_t splitmix64(uint64_t s)
{
    uint64_t z = s + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

__device__ __forceinline__ void camera_ray(const DevReq &R, int px, int py, int sample, float3 &ro,
                                           float3 &rd)
{
    float sx = 0.5f, sy = 0.5f;
    if (R.spp > 1) {
        uint64_t ctr = ((uint64_t)R.seed << 40) +
                       ((uint64_t)py * (uint64_t)R.width + (uint64_t)px) * (uint64_t)R.spp +
                       (uint64_t)sample;
        uint64_t h = splitmix64(ctr);
        sx = (float)(uint32_t)(h >> 40) * (1.0f / 16777216.0f);
        sy = (float)(uint32_t)((h >> 16) & 0xffffffULL) * (1.0f / 16777216.0f);
    }
    float uu = ((float)px + sx) * R.inv_w;
    float vv = ((float)py + sy) * R.inv_h;
    float ax = (2.0f * uu - 1.0f) * R.th_aspect;
    float ay = (1.0f - 2.0f * vv) * R.th;
    rd = normalize3(v3(R.fwd) + v3(R.right) * ax + v3(R.up) * ay);
    ro = v3(R.eye);
}

// ------------------------------------------------------------------ interval
// Bounding sphere |x|^2 <= R^2 gives [t0, t1]; t0 >= eps (tmin = kPrecis),
// t1 <= 7000 (tmax); the plane keeps dot(n, x) <= offset.  from_plane is set
// when the interval starts where the ray enters the kept half-space.
__device__ __forceinline__ bool bounds(const DevReq &R, float3 ro, float3 rd, float &t0, float &t1,
                                       bool &from_plane)
{
    float b = dot3(ro, rd);
    float cc = dot3(ro, ro) - R.bound_r2;
    float disc = b * b - cc;
    if (!(disc >= 0.0f)) return false;
    float s = sqrtf(disc);
    t0 = fmaxf(-b - s, R.eps);
    t1 = fminf(-b + s, 7000.0f);
    from_plane = false;
    if (R.plane_on) {
        float3 n = v3(R.plane);
        float a = dot3(n, ro) - R.plane.w;
        float bb = dot3(n, rd);
        if (bb == 0.0f) {
            if (a > 0.0f) return false;
        } else {
            float ts = -a / bb;
            if (bb > 0.0f) {
                t1 = fminf(t1, ts);
            } else if (ts > t0) {
                t0 = ts;
                from_plane = true;
            }
        }
    }
    return t0 <= t1;
}

// ------------------------------------------------------------------ distance estimators
// Quaternion Julia DE, degree 2: |z'|^2 *= 4 |z|^2 before each z <- z^2 + c,
// z^2 = (x^2 - |v|^2, 2 x v) for z = (x, v); stop once |z|^2 > esc2;
// d = 0.25 log|z|^2 sqrt(|z|^2 / |z'|^2).
template <int U>
__device__ __forceinline__ float julia_de2(const float4 c, float slice_w, int max_iter, float esc2,
                                           float3 p, int &trips)
{
    float x = p.x, y = p.y, z = p.z, w = slice_w;
    float m2 = x * x + y * y + z * z + w * w;
    float dz2 = 1.0f;
    int i = 0;
#pragma unroll U
    for (int k = 0; k < max_iter; k++) {
        dz2 *= 4.0f * m2;
        float tx = x + x;
        float nx = x * x - (y * y + z * z + w * w) + c.x;
        y = tx * y + c.y;
        z = tx * z + c.z;
        w = tx * w + c.w;
        x = nx;
        m2 = x * x + y * y + z * z + w * w;
        i++;
        if (m2 > esc2) break;
    }
    trips = i;
    return 0.25f * logf(m2) * sqrtf(m2 / dz2);
}

// degree 3 (the listing's cube): |z'|^2 *= 9 |z|^4, z^3 = (x^3 - 3x|v|^2, (3x^2 - |v|^2) v)
template <int U>
__device__ __forceinline__ float julia_de3(const float4 c, float slice_w, int max_iter, float esc2,
                                           float3 p, int &trips)
{
    float x = p.x, y = p.y, z = p.z, w = slice_w;
    float m2 = x * x + y * y + z * z + w * w;
    float dz2 = 1.0f;
    int i = 0;
#pragma unroll U
    for (int k = 0; k < max_iter; k++) {
        dz2 *= 9.0f * (m2 * m2);
        float x2 = x * x;
        float v2 = y * y + z * z + w * w;
        float f = 3.0f * x2 - v2;
        float nx = x * (x2 - 3.0f * v2) + c.x;
        y = f * y + c.y;
        z = f * z + c.z;
        w = f * w + c.w;
        x = nx;
        m2 = x * x + y * y + z * z + w * w;
        i++;
        if (m2 > esc2) break;
    }
    trips = i;
    return 0.25f * logf(m2) * sqrtf(m2 / dz2);
}

// Mandelbulb DE: w0 = c, m = |w|^2, dz = 1; per trip dz <- n r^(n-1) dz + 1 and
// w <- r^n (sin b sin a, cos b, sin b cos a) + c with b = n acos(w.y / r) (y/r
// clamped to [-1, 1]), a = n atan2(w.x, w.z); stop once m > bailout^2;
// d = 0.25 log(m) sqrt(m) / dz.  r = 0 gives the zero power.
template <int U>
__device__ __forceinline__ float bulb_de(int n, int max_iter, float esc2, float3 c, int &trips)
{
    float wx = c.x, wy = c.y, wz = c.z;
    float m = wx * wx + wy * wy + wz * wz;
    float dz = 1.0f;
    const float nf = (float)n;
    int i = 0;
#pragma unroll U
    for (int k = 0; k < max_iter; k++) {
        float r = sqrtf(m);
        dz = nf * powf(r, nf - 1.0f) * dz + 1.0f;
        float px = 0.0f, py = 0.0f, pz = 0.0f;
        if (r > 0.0f) {
            float ct = fminf(fmaxf(wy / r, -1.0f), 1.0f);
            float b = nf * acosf(ct);
            float a = nf * atan2f(wx, wz);
            float sb, cb, sa, ca;
            sincosf(b, &sb, &cb);
            sincosf(a, &sa, &ca);
            float rn = powf(r, nf);
            px = rn * (sb * sa);
            py = rn * cb;
            pz = rn * (sb * ca);
        }
        wx = px + c.x;
        wy = py + c.y;
        wz = pz + c.z;
        m = wx * wx + wy * wy + wz * wz;
        i++;
        if (m > esc2) break;
    }
    trips = i;
    return 0.25f * logf(m) * sqrtf(m) / dz;
}

template <int KIND, int U>
__device__ __forceinline__ float de(const DevReq &R, float3 p, int &trips)
{
    if (KIND == 0) {
        if (R.power == 2) return julia_de2<U>(R.c, R.slice_w, R.max_iter, R.esc2, p, trips);
        return julia_de3<U>(R.c, R.slice_w, R.max_iter, R.esc2, p, trips);
    }
    return bulb_de<U>(R.power, R.max_iter, R.esc2, p, trips);
}

// ------------------------------------------------------------------ shading
__device__ __forceinline__ float4 shade(const DevReq &R, float3 n, float vis)
{
    float ndl = dot3(n, v3(R.light));
    float diff = ndl > 0.0f ? ndl : 0.0f;
    float k = R.ka + R.kd * diff * vis;
    return make_float4(R.albedo.x * k, R.albedo.y * k, R.albedo.z * k, 1.0f);
}

// round-half-up of clamp(x, 0, 1) * 255 (NaN -> 0)
__device__ __forceinline__ uint32_t quantize(float x)
{
    float y = fminf(fmaxf(x, 0.0f), 1.0f);
    return (uint32_t)floorf(__fadd_rn(__fmul_rn(y, 255.0f), 0.5f));
}

__device__ __forceinline__ uint32_t pack_rgba8(float4 c)
{
    return quantize(c.x) | (quantize(c.y) << 8) | (quantize(c.z) << 16) | (quantize(c.w) << 24);
}

// per-thread event counters (only kept in the counting kernels)
struct Counters {
    unsigned long long v[kNStats];
};

__device__ __forceinline__ void flush_counters(const Counters &c, unsigned long long *stats)
{
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int k = 0; k < kNStats; k++) {
        unsigned long long s = c.v[k];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(full, s, o);
        if ((threadIdx.x & 31) == 0 && s) atomicAdd(stats + k, s);
    }
}

// write one finished pixel
__device__ __forceinline__ void store_pixel(const DevReq &R, int px, int py, float4 acc, float dmin,
                                            float3 xhit, uint32_t flags)
{
    const long long idx = (long long)py * R.width + px;
    if (R.rgba8) R.rgba8[idx] = pack_rgba8(acc);
    if (R.rgba) R.rgba[idx] = acc;
    if (R.depth) R.depth[idx] = dmin;
    if (R.saved) R.saved[idx] = make_float4(xhit.x, xhit.y, xhit.z, __uint_as_float(flags));
}

}  // namespace fr
