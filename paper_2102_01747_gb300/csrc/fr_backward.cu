// fr_backward.cu -- adjoint of the Julia render by implicit differentiation.
//
// Forward state: the hit point x of every pixel and its flags (hit, cut face,
// shadowed), saved by the forward kernels.  Nothing of the march is kept: the
// march is not differentiated.  At a surface hit the march has converged onto
// the level set of the distance estimate d(x; c) through x, so the hit depth
// t along the unit ray rd moves with a parameter theta as
//     dt/dtheta = -(dd/dtheta) / (grad_x d . rd)          (implicit function)
// The normal is the normalised stencil sum g = sum_k w_k d(x + o_k) of the
// forward pass; it moves through each tap's own dependence on c and through x.
// The analytic normal's g = J^T z_N (Sec. 2) moves through c and x inside its
// own orbit (julia_normal_vjp).
// Lambert shading moves through n and through L = dir/|dir|.  A cut-face hit
// sits on the plane: t = (o - n.ro)/(n.rd), normal n/|n|.
//
// d and its partial derivatives with respect to the point and to c come from
// reverse mode through the orbit of Eqs. 3-4: the orbit is recomputed from the
// point with the forward pass's own step function (so d, and with it the
// normal, are bit-identical to the forward pass), its iterates are kept in a
// per-thread array, and the adjoint runs back through
//     z_{k+1} = z_k^p + c,   |z'|^2 = prod_k p^2 |z_k|^(2(p-1)),
//     d = 0.25 log|z_N|^2 sqrt(|z_N|^2 / |z'|^2).
// Escape counts, hit status and shadow visibility are held fixed.
//
// One thread per pixel; the 11 partial sums (dc[4], dn[3], doffset, ddir[3])
// are reduced per warp with shuffles, per block in shared memory, and across
// blocks in a double accumulator that the last block adds to the caller's
// gradient (reproducible bits; see backward_kernel).
#include "fr_launch.h"
#include "fr_trace.cuh"

namespace fr {

// transpose of the Jacobian of q -> q^2 at z, applied to yb
__device__ __forceinline__ float4 jt_square(float4 z, float4 yb)
{
    const float vdy = z.y * yb.y + z.z * yb.z + z.w * yb.w;
    return make_float4(2.0f * (z.x * yb.x + vdy), 2.0f * (z.x * yb.y - z.y * yb.x),
                       2.0f * (z.x * yb.z - z.z * yb.x), 2.0f * (z.x * yb.w - z.w * yb.x));
}

// transpose of the Jacobian of q -> q^3 = (a^3 - 3a|v|^2, (3a^2 - |v|^2) v) at z
__device__ __forceinline__ float4 jt_cube(float4 z, float4 yb)
{
    const float a = z.x;
    const float v2 = z.y * z.y + z.z * z.z + z.w * z.w;
    const float f = 3.0f * a * a - v2;
    const float vdy = z.y * yb.y + z.z * yb.z + z.w * yb.w;
    const float s = -6.0f * a * yb.x - 2.0f * vdy;  // coefficient of v in vbar
    return make_float4((3.0f * a * a - 3.0f * v2) * yb.x + 6.0f * a * vdy, s * z.y + f * yb.y,
                       s * z.z + f * yb.z, s * z.w + f * yb.w);
}

// d(p) with d d / d p (gx) and d d / d c (gc) by reverse mode; d as in julia_de2/3
template <int P>
__device__ float julia_de_grad(const DevReq &R, float3 p, float3 &gx, float4 &gc)
{
    float4 zs[kMaxBwdIter];
    Orbit o;
    julia_init(o, p, R.slice_w);
    int n = 0;
    for (int k = 0; k < R.max_iter; k++) {
        zs[k] = make_float4(o.a, o.b, o.c, o.d);
        if (P == 2)
            julia2_step(o, R.c);
        else
            julia3_step(o, R.c);
        n++;
        if (o.m > R.esc2) break;
    }
    const float d = julia_dist(o);
    const float m = o.m;
    // d = 0.25 log(m) sqrt(m / D):  dd/dm = 0.25 sqrt(m/D) (1 + 0.5 log m) / m
    const float dd_dm = 0.25f * sqrtf(m / o.dz) * (1.0f + 0.5f * logf(m)) / m;
    float4 zb = make_float4(2.0f * dd_dm * o.a, 2.0f * dd_dm * o.b, 2.0f * dd_dm * o.c, 2.0f * dd_dm * o.d);
    float4 cb = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int k = n - 1; k >= 0; k--) {
        cb.x += zb.x;
        cb.y += zb.y;
        cb.z += zb.z;
        cb.w += zb.w;
        const float4 z = zs[k];
        float4 nb = (P == 2) ? jt_square(z, zb) : jt_cube(z, zb);
        // |z'|^2 carries p^2 |z_k|^(2(p-1)):  dd/dz_k += -d (p-1) z_k / |z_k|^2
        const float mk = z.x * z.x + z.y * z.y + z.z * z.z + z.w * z.w;
        const float coef = -d * (float)(P - 1) / mk;
        nb.x += coef * z.x;
        nb.y += coef * z.y;
        nb.z += coef * z.z;
        nb.w += coef * z.w;
        zb = nb;
    }
    gx = v3(zb.x, zb.y, zb.z);
    gc = cb;
    return d;
}

// transpose of z -> D(z^3)[t] (the tangent map of the cube, differentiated in
// z with t fixed), applied to b.  With z = (a, v), t = (ta, tv):
//   D(z^3)[t] = (3(a^2 - |v|^2) ta - 6a v.tv,  s v + f tv),
//   s = 6a ta - 2 v.tv,  f = 3a^2 - |v|^2.
__device__ __forceinline__ float4 jt_dcube(float4 z, float4 t, float4 b)
{
    const float a = z.x, ta = t.x;
    const float vdt = z.y * t.y + z.z * t.z + z.w * t.w;
    const float vdb = z.y * b.y + z.z * b.z + z.w * b.w;
    const float tdb = t.y * b.y + t.z * b.z + t.w * b.w;
    const float s = 6.0f * a * ta - 2.0f * vdt;
    const float ab = b.x * (6.0f * a * ta - 6.0f * vdt) + 6.0f * ta * vdb + 6.0f * a * tdb;
    const float cv = -6.0f * ta * b.x - 2.0f * tdb;  // coefficient of v
    const float ct = -6.0f * a * b.x - 2.0f * vdb;   // coefficient of tv
    return make_float4(ab, cv * z.y + ct * t.y + s * b.y, cv * z.z + ct * t.z + s * b.z,
                       cv * z.w + ct * t.w + s * b.w);
}

// phi = z_N . tau_N, tau the orbit's tangent along u (tau_0 = (u, 0)): the
// analytic normal's g (Sec. 2, julia_analytic_grad) contracted with u.
// Returns d phi / d x (the slice's three directions) and d phi / d c by
// reverse mode through the pair recursion (z, tau) -> (z^p + c, D(z^p)[tau]),
// the orbit recomputed with the forward pass's step functions.
template <int P>
__device__ void julia_normal_vjp(const DevReq &R, float3 x, float3 u, float3 &gx, float4 &gc)
{
    float4 zs[kMaxBwdIter], ts[kMaxBwdIter];
    Orbit o;
    julia_init(o, x, R.slice_w);
    float4 tau = make_float4(u.x, u.y, u.z, 0.0f);
    int n = 0;
    for (int k = 0; k < R.max_iter; k++) {
        zs[k] = make_float4(o.a, o.b, o.c, o.d);
        ts[k] = tau;
        tangent_step(tau, o, P);
        if (P == 2)
            julia2_step(o, R.c);
        else
            julia3_step(o, R.c);
        n++;
        if (o.m > R.esc2) break;
    }
    float4 zb = tau;                                   // d phi / d z_N
    float4 tb = make_float4(o.a, o.b, o.c, o.d);       // d phi / d tau_N
    float4 cb = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int k = n - 1; k >= 0; k--) {
        cb.x += zb.x;
        cb.y += zb.y;
        cb.z += zb.z;
        cb.w += zb.w;
        const float4 z = zs[k], t = ts[k];
        float4 nzb = (P == 2) ? jt_square(z, zb) : jt_cube(z, zb);
        // D(z^2)[t] = z t + t z is symmetric in (z, t), so its z-derivative is the square's at t
        const float4 dz = (P == 2) ? jt_square(t, tb) : jt_dcube(z, t, tb);
        nzb.x += dz.x;
        nzb.y += dz.y;
        nzb.z += dz.z;
        nzb.w += dz.w;
        tb = (P == 2) ? jt_square(z, tb) : jt_cube(z, tb);
        zb = nzb;
    }
    gx = v3(zb.x, zb.y, zb.z);
    gc = cb;
}

// weight vector of stencil tap k in g = sum_k w_k d_k (see tap_accum)
__device__ __forceinline__ float3 tap_weight(int mode, float h, int k)
{
    if (mode == 0) {
        return v3((k == 0 || k == 3) ? h : -h, (k >= 2) ? h : -h, (k == 1 || k == 3) ? h : -h);
    }
    const float s = (k & 1) ? -1.0f : 1.0f;
    const int j = k >> 1;
    return v3(j == 0 ? s : 0.0f, j == 1 ? s : 0.0f, j == 2 ? s : 0.0f);
}

// Cut-face hit: t = (o - n.ro) / (n.rd), normal n/|n|; Lambert through n and L
__device__ __forceinline__ void face_grad(const BwdArgs &A, float3 x, float3 rd, float3 L, float W, float vis,
                                          float gd, float gsum[11])
{
    const DevReq &R = A.R;
    const float3 nh = v3(R.plane_hat);
    const float3 nraw = v3(R.plane);
    const float ndl = dot3(nh, L);
    const float act = ndl > 0.0f ? W * R.kd * vis : 0.0f;
    const float nrd = dot3(nraw, rd);
    gsum[4] += act * (L.x - nh.x * ndl) / A.plane_norm - gd * x.x / nrd;
    gsum[5] += act * (L.y - nh.y * ndl) / A.plane_norm - gd * x.y / nrd;
    gsum[6] += act * (L.z - nh.z * ndl) / A.plane_norm - gd * x.z / nrd;
    gsum[7] += gd / nrd;
    gsum[8] += act * (nh.x - L.x * ndl) / A.light_norm;
    gsum[9] += act * (nh.y - L.y * ndl) / A.light_norm;
    gsum[10] += act * (nh.z - L.z * ndl) / A.light_norm;
}

// The Mandelbulb has no parameter c and its surface hits move with neither
// the plane nor the light: only Lambert's n.L moves, through the light
// direction, with n the forward pass's normal at the saved hit.
__device__ void pixel_grad_bulb(const BwdArgs &A, int px, int py, float gsum[11])
{
    const DevReq &R = A.R;
    const long long idx = (long long)py * R.width + px;
    const float4 sv = A.saved[idx];
    const uint32_t flags = __float_as_uint(sv.w);
    if (!(flags & kFlagHit)) return;
    const float4 dr = A.d_rgba[idx];
    const float W = dr.x * R.albedo.x + dr.y * R.albedo.y + dr.z * R.albedo.z;
    const float gd = A.d_depth ? A.d_depth[idx] : 0.0f;
    const float vis = (flags & kFlagShadow) ? 0.0f : 1.0f;
    float3 ro, rd;
    camera_ray(R, px, py, 0, ro, rd);
    const float3 x = v3(sv.x, sv.y, sv.z);
    const float3 L = v3(R.light);
    if (flags & kFlagFace) {
        face_grad(A, x, rd, L, W, vis, gd, gsum);
        return;
    }
    Counters cnt;
    const float3 n = normal_at<1, 1, false, true>(R, x, rd, cnt);
    const float ndl = dot3(n, L);
    const float act = ndl > 0.0f ? W * R.kd * vis : 0.0f;
    gsum[8] += act * (n.x - L.x * ndl) / A.light_norm;
    gsum[9] += act * (n.y - L.y * ndl) / A.light_norm;
    gsum[10] += act * (n.z - L.z * ndl) / A.light_norm;
}

template <int P>
__device__ void pixel_grad(const BwdArgs &A, int px, int py, float gsum[11])
{
    const DevReq &R = A.R;
    const long long idx = (long long)py * R.width + px;
    const float4 sv = A.saved[idx];
    const uint32_t flags = __float_as_uint(sv.w);
    if (!(flags & kFlagHit)) return;
    const float4 dr = A.d_rgba[idx];
    const float W = dr.x * R.albedo.x + dr.y * R.albedo.y + dr.z * R.albedo.z;
    const float gd = A.d_depth ? A.d_depth[idx] : 0.0f;
    const float vis = (flags & kFlagShadow) ? 0.0f : 1.0f;
    float3 ro, rd;
    camera_ray(R, px, py, 0, ro, rd);
    const float3 x = v3(sv.x, sv.y, sv.z);
    const float3 L = v3(R.light);

    if (flags & kFlagFace) {
        face_grad(A, x, rd, L, W, vis, gd, gsum);
        return;
    }

    float3 gx0;
    float4 gc0;
    const float d0 = julia_de_grad<P>(R, x, gx0, gc0);
    (void)d0;
    const float srd = dot3(gx0, rd);
    const float4 dtdc = make_float4(-gc0.x / srd, -gc0.y / srd, -gc0.z / srd, -gc0.w / srd);

    const bool analytic = R.normal_mode == 2;
    const int taps = analytic ? 0 : (R.normal_mode == 0 ? 4 : 6);
    float grd[6];
    float4 gck[6];
    float3 g = v3(0.0f, 0.0f, 0.0f);
    if (analytic) {
        int trips;
        g = julia_analytic_grad(R, x, trips);
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
        if (k < taps) {
            float3 gxk;
            const float dk = julia_de_grad<P>(R, tap_point(x, R.normal_mode, R.normal_h, k), gxk, gck[k]);
            grd[k] = dot3(gxk, rd);
            tap_accum(g, R.normal_mode, R.normal_h, k, dk);
        }
    }
    const float gl = sqrtf(dot3(g, g));
    if (!(gl > 0.0f) || !isfinite(gl)) return;  // the forward used -rd: no gradient
    const float3 n = v3(g.x / gl, g.y / gl, g.z / gl);
    const float ndl = dot3(n, L);
    const float act = ndl > 0.0f ? W * R.kd * vis : 0.0f;
    // u = act (I - n n^T) L / |g|; dLoss/dc = sum_k (u . w_k) (gc_k + (gx_k . rd) dt/dc) + gd dt/dc
    const float3 u = v3(act * (L.x - n.x * ndl) / gl, act * (L.y - n.y * ndl) / gl,
                        act * (L.z - n.z * ndl) / gl);
    float s = gd;  // coefficient of dt/dc
    float4 gcsum = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (analytic) {
        // g = J^T z_N moves through c and through x:  u . dg = d(g . u)
        float3 gxu;
        julia_normal_vjp<P>(R, x, u, gxu, gcsum);
        s += dot3(gxu, rd);
    }
#pragma unroll
    for (int k = 0; k < 6; k++) {
        if (k < taps) {
            const float uw = dot3(u, tap_weight(R.normal_mode, R.normal_h, k));
            gcsum.x += uw * gck[k].x;
            gcsum.y += uw * gck[k].y;
            gcsum.z += uw * gck[k].z;
            gcsum.w += uw * gck[k].w;
            s += uw * grd[k];
        }
    }
    gsum[0] += gcsum.x + s * dtdc.x;
    gsum[1] += gcsum.y + s * dtdc.y;
    gsum[2] += gcsum.z + s * dtdc.z;
    gsum[3] += gcsum.w + s * dtdc.w;
    gsum[8] += act * (n.x - L.x * ndl) / A.light_norm;
    gsum[9] += act * (n.y - L.y * ndl) / A.light_norm;
    gsum[10] += act * (n.z - L.z * ndl) / A.light_norm;
}

// The library's gradient accumulator (11 doubles) and count of finished
// blocks, used by calls that bring no workspace; both return to zero at the
// end of every call.  A call with a workspace uses the 11 doubles and the
// count there instead.
__device__ double g_bwd_acc[11];
__device__ unsigned int g_bwd_done;

template <int P>
__global__ void __launch_bounds__(256) backward_kernel(const __grid_constant__ BwdArgs A)
{
    const DevReq &R = A.R;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long tile = gtid >> 5;
    const int lane = threadIdx.x & 31;
    const int px = (int)(tile % R.tiles_x) * kTileW + (lane & (kTileW - 1));
    const int py = (int)(tile / R.tiles_x) * kTileH + (lane / kTileW);
    float gsum[11];
#pragma unroll
    for (int k = 0; k < 11; k++) gsum[k] = 0.0f;
    if (px < R.width && py < R.height) {
        if constexpr (P == 0)
            pixel_grad_bulb(A, px, py, gsum);
        else
            pixel_grad<P>(A, px, py, gsum);
    }

    __shared__ float part[8][11];
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 11; k++) {
        float v = gsum[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) part[warp][k] = v;
    }
    __syncthreads();
    // Block sums go into a double accumulator, so their order (which block
    // finishes first) moves the total by about 1e-16 relative, far below the
    // float rounding it gets at the end: the same inputs give the same
    // gradient bits (unless a total falls that close to a float rounding
    // boundary).  The last block to finish converts the totals to float once,
    // adds them to the caller's gradient and clears the accumulator for the
    // next call.  No block waits for another: the last one is the one whose
    // ticket completes the count (fence, then count).
    double *acc = A.acc ? A.acc : g_bwd_acc;
    unsigned int *done = A.acc ? A.done : &g_bwd_done;
    if (threadIdx.x < 11) {
        float v = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += part[w][threadIdx.x];
        if (v != 0.0f) atomicAdd(acc + threadIdx.x, (double)v);
    }
    __threadfence();
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        if (threadIdx.x < 11) {
            // read and clear in one step
            const unsigned long long bits =
                atomicExch(reinterpret_cast<unsigned long long *>(acc + threadIdx.x), 0ull);
            A.grad[threadIdx.x] += (float)__longlong_as_double((long long)bits);
        }
        if (threadIdx.x == 0) *done = 0u;
    }
}

cudaError_t launch_backward(const BwdArgs &A, cudaStream_t s)
{
    const int block = 256;
    const long long tiles_y = (A.R.height + kTileH - 1) / kTileH;
    const long long threads = (long long)A.R.tiles_x * tiles_y * 32;
    const long long grid = (threads + block - 1) / block;
    if (A.R.kind == 1)  // Mandelbulb (P = 0)
        backward_kernel<0><<<(unsigned)grid, block, 0, s>>>(A);
    else if (A.R.power == 2)
        backward_kernel<2><<<(unsigned)grid, block, 0, s>>>(A);
    else
        backward_kernel<3><<<(unsigned)grid, block, 0, s>>>(A);
    return cudaGetLastError();
}

}  // namespace fr
