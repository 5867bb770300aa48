// fr_device.cuh -- device-side building blocks of the sphere tracer (sm_103a).
//
// One request is a DevReq: the public parameter structs of include/fr.h resolved
// on the host into what the kernels read (camera basis, normalised light,
// squared radii, output pointers).  Every routine here computes in FP32 with
// the accurate CUDA math library or, for the Mandelbulb power's angles, the
// routines of fr_math.cuh (same error bounds, measured; no --use_fast_math,
// no approximate __xxxf intrinsics) and spells out every rounding step
// (mul/add/sub/dvd, fmaf), so that all kernels compute the same bits for the
// same ray.
//
// Paper passages (da Silva, Novello, Lopes, Velho, "Real-time rendering of
// complex fractals"):
//   julia_de   Listing "Julia Set distance", Eqs. 2-4 (degree p, slice w)
//   bulb_de    Listing "Mandelbulb distance", Eq. 1 (White-Nylander power)
//   bounds     Sec. 3.1: search interval [eps, 7000] clipped by a bounding
//              sphere and the cutting plane (Fig. 1)
//   march      Listing "Julia Set ray cast" (step min(d, max_step), hit d < eps,
//              miss t > t1, step cap counts as a hit)
//   normal     Eq. 5 / Listing "Normal calculation" (tetrahedral), central
//              differences, or grad G / |grad G| from the orbit's Jacobian
//              (Sec. 2; julia_analytic_normal, bulb_analytic_normal)
//   shade      Lambert closest-hit with an optional shadow ray, or Phong with
//              a Fresnel-weighted mirror ray (Listing "Closest-hit shader")
//   orbit_trap the listings' colour parameters
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "fr_math.cuh"

namespace fr {

// A warp covers a 4 x 8 tile of pixels (4 wide, 8 tall).  Measured against
// 8 x 4 and 16 x 2 tiles: 4 x 8 is the fastest (1-4 %), 16 x 2 the slowest.
constexpr int kTileW = 4;
constexpr int kTileH = 8;

// statistics slots (same order as FR_STAT_* in include/fr.h)
constexpr int kStatPrimaryRays = 0, kStatShadowRays = 1, kStatPrimaryDE = 2,
              kStatNormalDE = 3, kStatShadowDE = 4, kStatOrbit = 5, kStatReflectRays = 6,
              kStatReflectDE = 7, kNStats = 8;

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
    int bulb_alg;         // Mandelbulb power without transcendental calls
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
    float k_spec, shininess;  // Phong highlight weight and exponent
    float refl_coef;          // weight of the reflected colour
    int shading;              // 0 Lambert, 1 Phong + reflection bounce
    int quad_store;           // rgba8 / depth rows may be written 4 pixels per 16-byte store
    int tile_order;           // order of the tiles over the grid (fr_tuning.tile_order)
    int spl;                  // one-ray-per-thread kernels: lanes per pixel (1, or spp when the
                              // pixel's samples run on adjacent lanes; fr_tuning.sample_lanes)
    int spl_log2;             // log2(spl)
    float4 bg;
    uint32_t *rgba8;
    float4 *rgba;
    float *depth;
    float4 *saved;
    unsigned long long *stats;
    float4 *trap;
    long long unit_begin; // first queue unit of this request inside a batch
    long long n_units;    // tiles * 32
};

// warps (tiles of 4 x 8 / spl pixels) one request takes in the one-ray-per-thread kernels
__host__ __device__ __forceinline__ long long plain_tiles(const DevReq &R)
{
    const int th = kTileH / R.spl;
    return (long long)R.tiles_x * ((R.height + th - 1) / th);
}

// ------------------------------------------------------------------ arithmetic
// Every rounding step below is spelled out (fmaf = one fused multiply-add,
// __fmul_rn / __fadd_rn / __fsub_rn / __fdiv_rn = one rounded operation that
// the compiler may not fuse).  Left to itself the compiler fuses a*b + c
// depending on the surrounding code, so the same function inlined into two
// kernels could round differently; written out, every kernel that calls these
// routines computes bit-identical values for the same ray.
__device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float dvd(float a, float b) { return __fdiv_rn(a, b); }

// ------------------------------------------------------------------ vectors
__device__ __forceinline__ float3 v3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 v3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b)
{
    return fmaf(a.z, b.z, fmaf(a.y, b.y, mul(a.x, b.x)));
}
__device__ __forceinline__ float3 normalize3(float3 a)
{
    const float l = sqrtf(dot3(a, a));
    return v3(dvd(a.x, l), dvd(a.y, l), dvd(a.z, l));
}
// ro + t * rd
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
    const float uu = mul(add((float)px, sx), R.inv_w);
    const float vv = mul(add((float)py, sy), R.inv_h);
    const float ax = mul(fmaf(2.0f, uu, -1.0f), R.th_aspect);
    const float ay = mul(fmaf(-2.0f, vv, 1.0f), R.th);
    rd = normalize3(v3(fmaf(R.up.x, ay, fmaf(R.right.x, ax, R.fwd.x)),
                       fmaf(R.up.y, ay, fmaf(R.right.y, ax, R.fwd.y)),
                       fmaf(R.up.z, ay, fmaf(R.right.z, ax, R.fwd.z))));
    ro = v3(R.eye);
}

// ------------------------------------------------------------------ interval
// Bounding sphere |x|^2 <= R^2 gives [t0, t1]; t0 >= eps (tmin = kPrecis),
// t1 <= 7000 (tmax); the plane keeps dot(n, x) <= offset.  from_plane is set
// when the interval starts where the ray enters the kept half-space.
__device__ __forceinline__ bool bounds(const DevReq &R, float3 ro, float3 rd, float &t0, float &t1,
                                       bool &from_plane)
{
    const float b = dot3(ro, rd);
    const float cc = sub(dot3(ro, ro), R.bound_r2);
    const float disc = fmaf(b, b, -cc);
    if (!(disc >= 0.0f)) return false;
    const float s = sqrtf(disc);
    t0 = fmaxf(sub(-b, s), R.eps);
    t1 = fminf(sub(s, b), 7000.0f);
    from_plane = false;
    if (R.plane_on) {
        const float3 n = v3(R.plane);
        const float a = sub(dot3(n, ro), R.plane.w);
        const float bb = dot3(n, rd);
        if (bb == 0.0f) {
            if (a > 0.0f) return false;
        } else {
            const float ts = dvd(-a, bb);
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
// Each DE is written as init / one orbit step / distance so that the one-ray-
// per-thread kernel (whole orbit in a loop) and the persistent kernel (orbit
// steps interleaved with other lanes' work) run exactly the same arithmetic.
//
// Quaternion Julia (Listing "Julia Set distance", Eqs. 2-4): z0 = (p, slice_w),
// |z'|^2 = 1; each step multiplies |z'|^2 by p^2 |z|^(2(p-1)) and then sets
// z <- z^p + c; the orbit stops once |z|^2 > esc2 or after max_iter steps;
// d = 0.25 log|z|^2 sqrt(|z|^2 / |z'|^2) (= 0.5 |z| log|z| / |z'|).
struct Orbit {
    float a, b, c, d;  // Julia: z = (a, b, c, d)      Mandelbulb: w = (a, b, c)
    float dz;          // Julia: |z'|^2                Mandelbulb: |w'|
    float m;           // |z|^2 (|w|^2) of the current iterate
};

__device__ __forceinline__ float norm2_4(float a, float b, float c, float d)
{
    return fmaf(d, d, fmaf(c, c, fmaf(b, b, mul(a, a))));
}

__device__ __forceinline__ void julia_init(Orbit &o, float3 p, float slice_w)
{
    o.a = p.x; o.b = p.y; o.c = p.z; o.d = slice_w;
    o.m = norm2_4(o.a, o.b, o.c, o.d);
    o.dz = 1.0f;
}

// degree 2: z^2 = (x^2 - |v|^2, 2 x v) for z = (x, v); |z'|^2 *= 4 |z|^2
__device__ __forceinline__ void julia2_step(Orbit &o, const float4 c)
{
    o.dz = mul(o.dz, mul(4.0f, o.m));
    const float tx = add(o.a, o.a);
    const float v2 = fmaf(o.d, o.d, fmaf(o.c, o.c, mul(o.b, o.b)));
    const float nx = add(fmaf(o.a, o.a, -v2), c.x);
    o.b = fmaf(tx, o.b, c.y);
    o.c = fmaf(tx, o.c, c.z);
    o.d = fmaf(tx, o.d, c.w);
    o.a = nx;
    o.m = norm2_4(o.a, o.b, o.c, o.d);
}

// degree 3 (the listing's cube): z^3 = (x^3 - 3x|v|^2, (3x^2 - |v|^2) v); |z'|^2 *= 9 |z|^4
__device__ __forceinline__ void julia3_step(Orbit &o, const float4 c)
{
    o.dz = mul(o.dz, mul(9.0f, mul(o.m, o.m)));
    const float x2 = mul(o.a, o.a);
    const float v2 = fmaf(o.d, o.d, fmaf(o.c, o.c, mul(o.b, o.b)));
    const float f = fmaf(3.0f, x2, -v2);
    const float nx = fmaf(o.a, fmaf(-3.0f, v2, x2), c.x);
    o.b = fmaf(f, o.b, c.y);
    o.c = fmaf(f, o.c, c.z);
    o.d = fmaf(f, o.d, c.w);
    o.a = nx;
    o.m = norm2_4(o.a, o.b, o.c, o.d);
}

__device__ __forceinline__ float julia_dist(const Orbit &o)
{
    // (|z'|^2 can underflow to 0 only after |z| has, and m / 0 = inf is held
    // finite for sqrt_own: the distance is then as large as float allows)
    return mul(mul(0.25f, log_own(o.m)), sqrt_own(fminf(dvd(o.m, o.dz), 3.40282347e38f)));
}

// Mandelbulb (Listing "Mandelbulb distance", Eq. 1): w0 = c, dz = 1; each step
// dz <- n r^(n-1) dz + 1 and w <- r^n (sin b sin a, cos b, sin b cos a) + c with
// r = |w|, b = n acos(w.y / r) (y/r clamped to [-1, 1]), a = n atan2(w.x, w.z);
// r = 0 gives the zero power.  d = 0.25 log(m) sqrt(m) / dz.  The integer
// powers r^(n-1) and r^n are products (ipow) rather than two calls of the
// general powf: the same quantities in a few multiplications.
__device__ __forceinline__ void bulb_init(Orbit &o, float3 p)
{
    o.a = p.x; o.b = p.y; o.c = p.z; o.d = 0.0f;
    o.m = dot3(p, p);
    o.dz = 1.0f;
}

// The listing's angles of w for the power n, in half-turns (x 1/pi):
// b = n acos(u) with u = w.y / r clamped to [-1, 1], a = n atan2(w.x, w.z).
// In half-turns sin and cos need no range reduction by pi (sincospi_own);
// acospi and atan2pi return the angles in half-turns directly (all three in
// fr_math.cuh).  u is w.y times 1 / r (ir, from the seed that gave r, so the
// angle does not wait for r).  Returns u.
__device__ __forceinline__ float bulb_angles(float3 w, float ir, float nf, float &b, float &a)
{
    const float u = fminf(fmaxf(mul(w.y, ir), -1.0f), 1.0f);
    b = mul(nf, acospi(u));
    a = mul(nf, atan2pi(w.x, w.z));
    return u;
}

// r^k for an integer 0 <= k < 16 by binary exponentiation (each product
// rounded once, so r^7 carries at most 4 roundings).  Unrolled over the four
// bits of k with the products selected, not branched on: the same products in
// the same order as the loop over k's bits (res starts at 1, and 1 * b is b
// exactly), without its data-dependent branches.
__device__ __forceinline__ float ipow(float r, int k)
{
    float res = 1.0f, b = r;
#pragma unroll
    for (int bit = 0; bit < 4; bit++) {
        const float p = mul(res, b);
        res = ((k >> bit) & 1) ? p : res;
        b = mul(b, b);
    }
    return res;
}

// r^(n-1): straight-line for the paper's n = 8, binary exponentiation otherwise
__device__ __forceinline__ float rpow_nm1(float r, int n)
{
    if (n == 8) {
        const float r2 = mul(r, r), r4 = mul(r2, r2);
        return mul(mul(r4, r2), r);
    }
    return ipow(r, n - 1);
}

__device__ __forceinline__ void bulb_step(Orbit &o, float3 cpt, int n)
{
    const float nf = (float)n;
    float ir;
    const float r = sqrt_rsqrt_own(o.m, ir);
    const float rn1 = rpow_nm1(r, n);  // r^(n-1) (the listing's pow(sqrt(m), n-1))
    o.dz = fmaf(mul(nf, rn1), o.dz, 1.0f);
    float px = 0.0f, py = 0.0f, pz = 0.0f;
    if (r > 0.0f) {
        float b, a;
        bulb_angles(v3(o.a, o.b, o.c), ir, nf, b, a);
        float sb, cb, sa, ca;
        sincospi_own(b, &sb, &cb);
        sincospi_own(a, &sa, &ca);
        const float rn = mul(rn1, r);  // r^n (the listing's pow(r, n))
        px = mul(rn, mul(sb, sa));
        py = mul(rn, cb);
        pz = mul(rn, mul(sb, ca));
    }
    o.a = add(px, cpt.x);
    o.b = add(py, cpt.y);
    o.c = add(pz, cpt.z);
    o.m = dot3(v3(o.a, o.b, o.c), v3(o.a, o.b, o.c));
}

// (c + i s)^k for an integer 1 <= k <= 16 by binary exponentiation of complex
// numbers; the bits of k select multiplications instead of branching on them
__device__ __forceinline__ void cpow_int(float c, float s, int k, float &rc, float &rs)
{
    float ac = 1.0f, as = 0.0f, bc = c, bs = s;
#pragma unroll
    for (int bit = 0; bit < 5; bit++) {
        const float tc = fmaf(ac, bc, -mul(as, bs));
        const float ts = fmaf(ac, bs, mul(as, bc));
        const bool take = (k >> bit) & 1;
        ac = take ? tc : ac;
        as = take ? ts : as;
        const float sc = fmaf(bc, bc, -mul(bs, bs));
        bs = mul(2.0f, mul(bc, bs));
        bc = sc;
    }
    rc = ac;
    rs = as;
}

// (c + i s)^8: three squarings
__device__ __forceinline__ void cpow8(float c, float s, float &rc, float &rs)
{
#pragma unroll
    for (int i = 0; i < 3; i++) {
        const float sc = fmaf(c, c, -mul(s, s));
        s = mul(2.0f, mul(c, s));
        c = sc;
    }
    rc = c;
    rs = s;
}

// The same step with Eq. 1 evaluated without transcendental calls: with
// r = |w| and rho = |(w.x, w.z)|, the angles of the listing have
// cos b0 = w.y / r, sin b0 = rho / r (b0 in [0, pi]) and cos a0 = w.z / rho,
// sin a0 = w.x / rho, so (cos n b0, sin n b0) and (cos n a0, sin n a0) are the
// n-th powers of the unit complex numbers cos + i sin (de Moivre).  On the
// polar axis (rho = 0) a0 is taken as 0.  n = 8 (the paper's power) takes
// three squarings; other n go through cpow_int.
__device__ __forceinline__ void bulb_step_alg(Orbit &o, float3 cpt, int n)
{
    const float nf = (float)n;
    float ir;
    const float r = sqrt_rsqrt_own(o.m, ir);  // r and 1 / r
    const float rn1 = rpow_nm1(r, n);
    o.dz = fmaf(mul(nf, rn1), o.dz, 1.0f);
    float px = 0.0f, py = 0.0f, pz = 0.0f;
    if (r > 0.0f) {
        const float rho2 = fmaf(o.c, o.c, mul(o.a, o.a));
        const float cb0 = fminf(fmaxf(mul(o.b, ir), -1.0f), 1.0f);
        float irho;
        const float rho = sqrt_rsqrt_own(rho2, irho);  // rho and 1 / rho
        const float sb0 = mul(rho, ir);
        float ca0 = 1.0f, sa0 = 0.0f;
        if (rho > 0.0f) {
            ca0 = mul(o.c, irho);
            sa0 = mul(o.a, irho);
        }
        float cb, sb, ca, sa;
        if (n == 8) {
            cpow8(cb0, sb0, cb, sb);
            cpow8(ca0, sa0, ca, sa);
        } else {
            cpow_int(cb0, sb0, n, cb, sb);
            cpow_int(ca0, sa0, n, ca, sa);
        }
        const float rn = mul(rn1, r);
        px = mul(rn, mul(sb, sa));
        py = mul(rn, cb);
        pz = mul(rn, mul(sb, ca));
    }
    o.a = add(px, cpt.x);
    o.b = add(py, cpt.y);
    o.c = add(pz, cpt.z);
    o.m = dot3(v3(o.a, o.b, o.c), v3(o.a, o.b, o.c));
}

__device__ __forceinline__ float bulb_dist(const Orbit &o)
{
    // dz >= 1; above 2^126 (it overflows to inf after ~12 steps at r ~ 2) the
    // distance is below 1e-37 either way: dz is held at 2^126 for quot
    return quot(mul(mul(0.25f, log_own(o.m)), sqrt_own(o.m)), fminf(o.dz, 8.507059e37f));
}

// whole-orbit DEs (one-ray-per-thread kernel); trips = orbit loop trips
template <int U>
__device__ __forceinline__ float julia_de2(const float4 c, float slice_w, int max_iter, float esc2,
                                           float3 p, int &trips)
{
    Orbit o;
    julia_init(o, p, slice_w);
    int i = 0;
#pragma unroll U
    for (int k = 0; k < max_iter; k++) {
        julia2_step(o, c);
        i++;
        if (o.m > esc2) break;
    }
    trips = i;
    return julia_dist(o);
}

template <int U>
__device__ __forceinline__ float julia_de3(const float4 c, float slice_w, int max_iter, float esc2,
                                           float3 p, int &trips)
{
    Orbit o;
    julia_init(o, p, slice_w);
    int i = 0;
#pragma unroll U
    for (int k = 0; k < max_iter; k++) {
        julia3_step(o, c);
        i++;
        if (o.m > esc2) break;
    }
    trips = i;
    return julia_dist(o);
}

template <int U>
__device__ __forceinline__ float bulb_orbit(int n, int max_iter, float esc2, float3 c, int alg, int &trips)
{
    Orbit o;
    bulb_init(o, c);
    int i = 0;
#pragma unroll U
    for (int k = 0; k < max_iter; k++) {
        if (alg)
            bulb_step_alg(o, c, n);
        else
            bulb_step(o, c, n);
        i++;
        if (o.m > esc2) break;
    }
    trips = i;
    return bulb_dist(o);
}

// The orbit loop is copied for each form of the step (transcendental or de
// Moivre) and, in each, for the paper's power n = 8 compiled with n a
// constant (the straight-line r^7), so that the loop tests neither; the other
// powers share the copy with n at run time.  Every copy makes the same
// products in the same order.
template <int U>
__device__ __forceinline__ float bulb_de(int n, int max_iter, float esc2, float3 c, int alg, int &trips)
{
    if (alg) {
        if (n == 8) return bulb_orbit<U>(8, max_iter, esc2, c, 1, trips);
        return bulb_orbit<U>(n, max_iter, esc2, c, 1, trips);
    }
    if (n == 8) return bulb_orbit<U>(8, max_iter, esc2, c, 0, trips);
    return bulb_orbit<U>(n, max_iter, esc2, c, 0, trips);
}

// KIND: 0 the Julia set, 1 the Mandelbulb, 2 the Mandelbulb of a request
// whose power is 8 (the kernel then holds no code for other powers)
template <int KIND, int U>
__device__ __forceinline__ float de(const DevReq &R, float3 p, int &trips)
{
    if (KIND == 0) {
        if (R.power == 2) return julia_de2<U>(R.c, R.slice_w, R.max_iter, R.esc2, p, trips);
        return julia_de3<U>(R.c, R.slice_w, R.max_iter, R.esc2, p, trips);
    }
    return bulb_de<U>(KIND == 2 ? 8 : R.power, R.max_iter, R.esc2, p, R.bulb_alg, trips);
}

// ------------------------------------------------------------------ orbit traps
// Colour parameters of the DE at a point, as the listings hand them to the
// closest-hit stage.  Mandelbulb (Listing "Mandelbulb distance"): the running
// minimum of (|w.x|, |w.y|, |w.z|, m), started at w0 = c and updated after
// each step with the new w and the m of the step before, returned as
// (final m, min |w.y|, min |w.z|, min m).  Julia (Listing "Julia Set
// distance"): the count of steps that did not escape, with the final |z|^2.
__device__ __forceinline__ float4 orbit_trap(const DevReq &R, float3 p)
{
    Orbit o;
    if (R.kind == 0) {
        julia_init(o, p, R.slice_w);
        int n = 0;
        for (int k = 0; k < R.max_iter; k++) {
            if (R.power == 2)
                julia2_step(o, R.c);
            else
                julia3_step(o, R.c);
            if (o.m > R.esc2) break;
            n++;
        }
        return make_float4((float)n, o.m, 0.0f, 0.0f);
    }
    bulb_init(o, p);
    float4 t = make_float4(fabsf(o.a), fabsf(o.b), fabsf(o.c), o.m);
    for (int k = 0; k < R.max_iter; k++) {
        const float m_prev = o.m;
        if (R.bulb_alg)
            bulb_step_alg(o, p, R.power);
        else
            bulb_step(o, p, R.power);
        t = make_float4(fminf(t.x, fabsf(o.a)), fminf(t.y, fabsf(o.b)), fminf(t.z, fabsf(o.c)),
                        fminf(t.w, m_prev));
        if (o.m > R.esc2) break;
    }
    return make_float4(o.m, t.y, t.z, t.w);
}

// ------------------------------------------------------------------ analytic normal
// Sec. 2: on the set grad d = grad G / |grad G|, and grad G at x is parallel to
// J^T z_N, J = dz_N / dz_0 (G = lim log|z_N| / p^N).  The three slice
// directions of J are carried through the orbit as tangent quaternions
// (forward mode): t <- D(z^p)[t], with
//   p = 2: D[t] = z t + t z = (2(a ta - v.tv), 2(a tv + ta v))        z = (a, v)
//   p = 3: D[t] = ((3a^2 - 3|v|^2) ta - 6a v.tv, (6a ta - 2 v.tv) v + (3a^2 - |v|^2) tv)
// and the gradient is (z_N . t_x, z_N . t_y, z_N . t_z).  The orbit runs with
// the same step function and stop rule as the DE.
__device__ __forceinline__ void tangent_step(float4 &t, const Orbit &o, int p)
{
    const float vdt = fmaf(o.d, t.w, fmaf(o.c, t.z, mul(o.b, t.y)));
    if (p == 2) {
        const float na = mul(2.0f, fmaf(o.a, t.x, -vdt));
        t.y = mul(2.0f, fmaf(o.a, t.y, mul(t.x, o.b)));
        t.z = mul(2.0f, fmaf(o.a, t.z, mul(t.x, o.c)));
        t.w = mul(2.0f, fmaf(o.a, t.w, mul(t.x, o.d)));
        t.x = na;
        return;
    }
    const float v2 = fmaf(o.d, o.d, fmaf(o.c, o.c, mul(o.b, o.b)));
    const float a2 = mul(o.a, o.a);
    const float f = fmaf(3.0f, a2, -v2);
    const float s = fmaf(6.0f * o.a, t.x, mul(-2.0f, vdt));  // coefficient of v
    const float na = fmaf(mul(3.0f, sub(a2, v2)), t.x, mul(-6.0f * o.a, vdt));
    t.y = fmaf(s, o.b, mul(f, t.y));
    t.z = fmaf(s, o.c, mul(f, t.z));
    t.w = fmaf(s, o.d, mul(f, t.w));
    t.x = na;
}

// g = (z_N . t_x, z_N . t_y, z_N . t_z), not normalised (the adjoint needs |g|)
__device__ __forceinline__ float3 julia_analytic_grad(const DevReq &R, float3 x, int &trips)
{
    Orbit o;
    julia_init(o, x, R.slice_w);
    float4 tx = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
    float4 ty = make_float4(0.0f, 1.0f, 0.0f, 0.0f);
    float4 tz = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
    int i = 0;
    for (int k = 0; k < R.max_iter; k++) {
        tangent_step(tx, o, R.power);
        tangent_step(ty, o, R.power);
        tangent_step(tz, o, R.power);
        if (R.power == 2)
            julia2_step(o, R.c);
        else
            julia3_step(o, R.c);
        i++;
        if (o.m > R.esc2) break;
    }
    trips = i;
    return v3(fmaf(o.d, tx.w, fmaf(o.c, tx.z, fmaf(o.b, tx.y, mul(o.a, tx.x)))),
              fmaf(o.d, ty.w, fmaf(o.c, ty.z, fmaf(o.b, ty.y, mul(o.a, ty.x)))),
              fmaf(o.d, tz.w, fmaf(o.c, tz.z, fmaf(o.b, tz.y, mul(o.a, tz.x)))));
}

__device__ __forceinline__ float3 julia_analytic_normal(const DevReq &R, float3 x, float3 rd, int &trips)
{
    const float3 g = julia_analytic_grad(R, x, trips);
    const float l = sqrtf(dot3(g, g));
    if (!(l > 0.0f) || !isfinite(l)) return v3(-rd.x, -rd.y, -rd.z);
    return v3(dvd(g.x, l), dvd(g.y, l), dvd(g.z, l));
}

// ------------------------------------------------------------------ normal stencils
// Tap k of the stencil around x and its contribution to the gradient sum g.
// Tetrahedral (Eq. 5, Listing "Normal calculation"): taps x + h nu_k with
// nu = (1,-1,-1), (-1,-1,1), (-1,1,-1), (1,1,1), g += (h nu_k) d_k.
// Central: taps x +- h e_j in the order +x, -x, +y, -y, +z, -z,
// g_j = d(x + h e_j) - d(x - h e_j).
__device__ __forceinline__ float3 tap_point(float3 x, int mode, float h, int k)
{
    if (mode == 0) {
        const float sx = (k == 0 || k == 3) ? h : -h;
        const float sy = (k >= 2) ? h : -h;
        const float sz = (k == 1 || k == 3) ? h : -h;
        return v3(add(x.x, sx), add(x.y, sy), add(x.z, sz));
    }
    const float s = (k & 1) ? -h : h;
    return v3(k < 2 ? add(x.x, s) : x.x, (k >> 1) == 1 ? add(x.y, s) : x.y, k >= 4 ? add(x.z, s) : x.z);
}

__device__ __forceinline__ void tap_accum(float3 &g, int mode, float h, int k, float d)
{
    if (mode == 0) {
        const float sx = (k == 0 || k == 3) ? h : -h;
        const float sy = (k >= 2) ? h : -h;
        const float sz = (k == 1 || k == 3) ? h : -h;
        g.x = fmaf(sx, d, g.x);
        g.y = fmaf(sy, d, g.y);
        g.z = fmaf(sz, d, g.z);
        return;
    }
    const int j = k >> 1;
    if (j == 0)
        g.x = (k & 1) ? sub(g.x, d) : d;
    else if (j == 1)
        g.y = (k & 1) ? sub(g.y, d) : d;
    else
        g.z = (k & 1) ? sub(g.z, d) : d;
}

// unit gradient, -rd when it is zero or not finite
__device__ __forceinline__ float3 finish_normal(float3 g, float3 rd)
{
    const float l = sqrtf(dot3(g, g));
    if (!(l > 0.0f) || !isfinite(l)) return v3(-rd.x, -rd.y, -rd.z);
    return v3(dvd(g.x, l), dvd(g.y, l), dvd(g.z, l));
}

// Analytic normal of the Mandelbulb: the construction of julia_analytic_normal
// with G = lim log|w_N| / n^N and J = dw_N / dc.  c enters every step of Eq. 1,
// so a column d of J follows d <- DP(w) d + e from d_0 = e (e the column's unit
// vector), where DP is the Jacobian of the power
// P(w) = r^n (sin b sin a, cos b, sin b cos a) in the listing's angles
// (u = w.y / r, b = n acos u, a = n atan2(w.x, w.z)):
//   dr = (w . d) / r,  du = (d.y r - w.y dr) / r^2,  db = -n du / sqrt(1 - u^2),
//   da = n (w.z d.x - w.x d.z) / (w.x^2 + w.z^2),  d(r^n) = n r^(n-1) dr,
// with db (da) taken as 0 on the polar axis where sqrt(1 - u^2) (w.x^2 + w.z^2)
// vanishes.  Gradient component k = w_N . (column k); the orbit stops where the
// DE's does.  The orbit runs once per column, each pass carrying one column:
// all three columns in one pass held 16 more registers across the whole
// one-ray-per-thread kernel (48 -> 64 for the Mandelbulb), a cost every pixel
// pays, while three passes cost hit pixels three orbits, one fewer than the
// tetrahedral stencil.  Each pass repeats the same operations on w, so the
// orbit, its length and the stop are the same in all three.  n is the
// request's power, the literal 8 in kernels compiled for that power.
__device__ __forceinline__ float3 bulb_analytic_normal(const DevReq &R, int n, float3 x, float3 rd, int &trips)
{
    const float nf = (float)n;
    float3 g = v3(0.0f, 0.0f, 0.0f);
    int i = 0;
#pragma unroll 1
    for (int col = 0; col < 3; col++) {
        float3 w = x;
        float3 d = v3(col == 0 ? 1.0f : 0.0f, col == 1 ? 1.0f : 0.0f, col == 2 ? 1.0f : 0.0f);
        i = 0;
        for (int k = 0; k < R.max_iter; k++) {
            i++;
            float ir;
            const float r = sqrt_rsqrt_own(dot3(w, w), ir);
            float3 P = v3(0.0f, 0.0f, 0.0f), dP = P;
            if (r > 0.0f) {
                float b, a;
                const float u = bulb_angles(w, ir, nf, b, a);  // as bulb_step
                float sb, cb, sa, ca;
                sincospi_own(b, &sb, &cb);
                sincospi_own(a, &sa, &ca);
                const float rn1 = rpow_nm1(r, n);
                const float rn = mul(rn1, r);
                P = v3(mul(rn, mul(sb, sa)), mul(rn, cb), mul(rn, mul(sb, ca)));
                const float rho2 = fmaf(w.z, w.z, mul(w.x, w.x));
                // the divisions by r, r^2, sqrt(1 - u^2) and rho^2 as products with the
                // reciprocals (ir from the step's seed; 1/sqrt(1 - u^2) and 1/rho from
                // one seed each; zero below the normal range, on the polar axis)
                float isu, irho;
                const float su = sqrt_rsqrt_own(fmaxf(fmaf(-u, u, 1.0f), 0.0f), isu);
                const float rho = sqrt_rsqrt_own(rho2, irho);
                const float dr = mul(dot3(w, d), ir);
                const float du = mul(mul(fmaf(-w.y, dr, mul(d.y, r)), ir), ir);
                const float db = su > 0.0f ? mul(mul(-nf, du), isu) : 0.0f;
                const float da = rho > 0.0f ? mul(mul(mul(nf, fmaf(w.z, d.x, -mul(w.x, d.z))), irho), irho) : 0.0f;
                const float drn = mul(mul(nf, rn1), dr);
                const float cbdb = mul(cb, db), sbda = mul(sb, da);
                dP = v3(fmaf(drn, mul(sb, sa), mul(rn, fmaf(cbdb, sa, mul(ca, sbda)))),
                        fmaf(drn, cb, -mul(rn, mul(sb, db))),
                        fmaf(drn, mul(sb, ca), mul(rn, fmaf(cbdb, ca, -mul(sa, sbda)))));
            }
            d = v3(col == 0 ? add(dP.x, 1.0f) : dP.x, col == 1 ? add(dP.y, 1.0f) : dP.y,
                   col == 2 ? add(dP.z, 1.0f) : dP.z);
            w = v3(add(P.x, x.x), add(P.y, x.y), add(P.z, x.z));
            if (dot3(w, w) > R.esc2) break;
        }
        const float gk = dot3(w, d);
        if (col == 0) g.x = gk;
        else if (col == 1) g.y = gk;
        else g.z = gk;
    }
    trips = i;
    return finish_normal(g, rd);
}

// The same normal out of line, for the batch kernels: they carry it for the
// few requests that ask for it, and inlined it is a third copy of the trig
// orbit in every one of them (the 64-request mixed batch, which has no such
// request, runs 1.7 % faster with it out of line).
static __device__ __noinline__ float3 bulb_analytic_normal_ool(const DevReq &R, int n, float3 x, float3 rd,
                                                               int &trips)
{
    return bulb_analytic_normal(R, n, x, rd, trips);
}

// shadow-ray origin x + off n
__device__ __forceinline__ float3 offset_point(float3 x, float3 n, float off)
{
    return v3(fmaf(n.x, off, x.x), fmaf(n.y, off, x.y), fmaf(n.z, off, x.z));
}

// ------------------------------------------------------------------ shading
__device__ __forceinline__ float4 shade(const DevReq &R, float3 n, float vis)
{
    const float ndl = dot3(n, v3(R.light));
    const float diff = ndl > 0.0f ? ndl : 0.0f;
    const float k = fmaf(mul(R.kd, diff), vis, R.ka);
    return make_float4(mul(R.albedo.x, k), mul(R.albedo.y, k), mul(R.albedo.z, k), 1.0f);
}

// Phong (the closest-hit shader of Sec. 3.1; its helpers are not listed):
// albedo (ka + kd max(0, n.L) vis) + k_spec vis max(0, r.(-d))^shininess with
// r = 2 (n.L) n - L the light mirrored about n, no highlight where n.L <= 0.
__device__ __forceinline__ float3 phong(const DevReq &R, float3 n, float3 d, float vis)
{
    const float3 L = v3(R.light);
    const float ndl = dot3(n, L);
    const float diff = ndl > 0.0f ? ndl : 0.0f;
    const float k = fmaf(mul(R.kd, diff), vis, R.ka);
    float spec = 0.0f;
    if (ndl > 0.0f) {
        const float two_ndl = mul(2.0f, ndl);
        const float3 r = v3(fmaf(n.x, two_ndl, -L.x), fmaf(n.y, two_ndl, -L.y), fmaf(n.z, two_ndl, -L.z));
        const float rv = -dot3(r, d);
        spec = powf(rv > 0.0f ? rv : 0.0f, R.shininess);
    }
    const float hl = mul(mul(R.k_spec, spec), vis);
    return v3(fmaf(R.albedo.x, k, hl), fmaf(R.albedo.y, k, hl), fmaf(R.albedo.z, k, hl));
}

// mirror direction of d about the unit normal n: d - 2 (n.d) n
__device__ __forceinline__ float3 mirror(float3 d, float3 n)
{
    const float m = mul(-2.0f, dot3(n, d));
    return v3(fmaf(n.x, m, d.x), fmaf(n.y, m, d.y), fmaf(n.z, m, d.z));
}

// Phong at the hit plus refl_coef * Fresnel-Schlick * (colour along the mirror
// ray), F = albedo + (1 - albedo) (1 - cos)^5, cos = max(0, -n.rd), per channel.
__device__ __forceinline__ float4 shade_phong(const DevReq &R, float3 n, float3 rd, float vis, float3 refl)
{
    const float3 base = phong(R, n, rd, vis);
    float c = -dot3(n, rd);
    c = c > 0.0f ? c : 0.0f;
    const float u = sub(1.0f, c);
    const float u2 = mul(u, u);
    const float w = mul(mul(u2, u2), u);
    const float fr = fmaf(sub(1.0f, R.albedo.x), w, R.albedo.x);
    const float fg = fmaf(sub(1.0f, R.albedo.y), w, R.albedo.y);
    const float fb = fmaf(sub(1.0f, R.albedo.z), w, R.albedo.z);
    return make_float4(fmaf(mul(R.refl_coef, fr), refl.x, base.x), fmaf(mul(R.refl_coef, fg), refl.y, base.y),
                       fmaf(mul(R.refl_coef, fb), refl.z, base.z), 1.0f);
}

// round-half-up of clamp(x, 0, 1) * 255 (NaN -> 0)
__device__ __forceinline__ uint32_t quantize(float x)
{
    const float y = fminf(fmaxf(x, 0.0f), 1.0f);
    return (uint32_t)floorf(add(mul(y, 255.0f), 0.5f));
}

__device__ __forceinline__ uint32_t pack_rgba8(float4 c)
{
    return quantize(c.x) | (quantize(c.y) << 8) | (quantize(c.z) << 16) | (quantize(c.w) << 24);
}

// running sum over samples and the mean
__device__ __forceinline__ void acc4(float4 &acc, float4 c)
{
    acc.x = add(acc.x, c.x);
    acc.y = add(acc.y, c.y);
    acc.z = add(acc.z, c.z);
    acc.w = add(acc.w, c.w);
}
__device__ __forceinline__ float4 mean4(float4 acc, int spp)
{
    const float fs = (float)spp;
    return make_float4(dvd(acc.x, fs), dvd(acc.y, fs), dvd(acc.z, fs), dvd(acc.w, fs));
}

// march update t += min(d, max_step)
__device__ __forceinline__ float march_step(float t, float d, float max_step)
{
    return add(t, (d < max_step) ? d : max_step);
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

// Per-pixel stores of everything but the packed colour and the depth: float
// RGBA, saved state, orbit trap (16 bytes per pixel each).
__device__ __forceinline__ void store_pixel_extras(const DevReq &R, long long idx, float4 acc, float3 xhit,
                                                   uint32_t flags)
{
    if (R.rgba) R.rgba[idx] = acc;
    if (R.saved) R.saved[idx] = make_float4(xhit.x, xhit.y, xhit.z, __uint_as_float(flags));
    if (R.trap) R.trap[idx] = (flags & kFlagHit) ? orbit_trap(R, xhit) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
}

// Packed colour and depth of a warp's tile, called by all 32 lanes together
// (valid: the lane holds a finished pixel inside the image).  Pixel q of the
// tile sits on lane q * spl (spl lanes per pixel), and the tile is 4 pixels
// wide, so the 4 adjacent pixels of a tile row are on lanes spl apart: where
// the row is complete and the image width and both buffers allow 16-byte
// alignment (quad_store), the row's first pixel lane gathers them by shuffles
// and writes one 16-byte store per buffer; otherwise every valid lane writes
// its own 4 bytes.
__device__ __forceinline__ void store_rgba8_depth(const DevReq &R, int px, int py, bool valid, uint32_t c8,
                                                  float d, int spl = 1)
{
    static_assert(kTileW == 4, "a tile row is one 16-byte quad");
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint32_t c1 = __shfl_down_sync(full, c8, spl), c2 = __shfl_down_sync(full, c8, 2 * spl),
                   c3 = __shfl_down_sync(full, c8, 3 * spl);
    const float d1 = __shfl_down_sync(full, d, spl), d2 = __shfl_down_sync(full, d, 2 * spl),
                d3 = __shfl_down_sync(full, d, 3 * spl);
    const int first = lane & ~(4 * spl - 1);  // the row's first pixel lane
    const unsigned ok = __ballot_sync(full, valid);
    const unsigned want = (1u << first) | (1u << (first + spl)) | (1u << (first + 2 * spl)) |
                          (1u << (first + 3 * spl));
    const bool row = (ok & want) == want;
    const long long idx = (long long)py * R.width + px;
    if (R.quad_store && row) {
        if (lane == first) {
            if (R.rgba8) *reinterpret_cast<uint4 *>(R.rgba8 + idx) = make_uint4(c8, c1, c2, c3);
            if (R.depth) *reinterpret_cast<float4 *>(R.depth + idx) = make_float4(d, d1, d2, d3);
        }
    } else if (valid) {
        if (R.rgba8) R.rgba8[idx] = c8;
        if (R.depth) R.depth[idx] = d;
    }
}

}  // namespace fr
