// fr_api.cu -- the C ABI of include/fr.h: argument checks on the host, the
// resolution of the public structs into DevReq, launch-shape selection and
// error reporting.  No device memory is allocated here.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/fr.h"
#include "fr_launch.h"

namespace {

thread_local std::string g_err;

fr_status fail(fr_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

std::mutex g_tuning_mu;
fr_tuning g_tuning = {128, 1, 64, 0, 16, 4, 0, 2, 0, 1};

fr_tuning tuning()
{
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    return g_tuning;
}

bool finite_n(const float *v, int n)
{
    for (int i = 0; i < n; i++)
        if (!std::isfinite(v[i])) return false;
    return true;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

struct F3 {
    float x, y, z;
};
F3 f3(const float *v) { return {v[0], v[1], v[2]}; }
F3 sub(F3 a, F3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
F3 cross(F3 a, F3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
float dot(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
float4 f4(F3 a, float w = 0.0f) { return make_float4(a.x, a.y, a.z, w); }

// normalise in float; false if the length is zero or not finite
bool normalize(F3 &a)
{
    float l = std::sqrt(dot(a, a));
    if (!(l > 0.0f) || !std::isfinite(l)) return false;
    a = {a.x / l, a.y / l, a.z / l};
    return true;
}

fr_status resolve_march(fr::DevReq &R, int max_iter, float bound_radius, int max_steps, float eps,
                        float max_step, int normal_mode, float normal_h)
{
    if (max_iter < 1 || max_iter > 1024) return fail(FR_EINVAL, "max_iter %d outside 1..1024", max_iter);
    if (!(bound_radius > 0.0f) || !std::isfinite(bound_radius))
        return fail(FR_EINVAL, "bound_radius must be positive and finite");
    if (max_steps < 1 || max_steps > 100000)
        return fail(FR_EINVAL, "max_steps %d outside 1..100000", max_steps);
    if (!(eps > 0.0f) || !std::isfinite(eps)) return fail(FR_EINVAL, "eps must be positive and finite");
    if (!(max_step > 0.0f) || !std::isfinite(max_step))
        return fail(FR_EINVAL, "max_step must be positive and finite");
    if (normal_mode != FR_NORMAL_TETRA && normal_mode != FR_NORMAL_CENTRAL && normal_mode != FR_NORMAL_ANALYTIC)
        return fail(FR_EINVAL, "normal_mode %d unknown", normal_mode);
    if (!(normal_h >= 0.0f) || !std::isfinite(normal_h))
        return fail(FR_EINVAL, "normal_h must be >= 0 and finite");
    R.max_iter = max_iter;
    R.bound_r2 = bound_radius * bound_radius;
    R.max_steps = max_steps;
    R.eps = eps;
    R.max_step = max_step;
    R.normal_mode = normal_mode;
    // default stencil: the listing's 0.5773 * kPrecis (|h nu| = eps) or 1e-4
    R.normal_h = normal_h > 0.0f ? normal_h : (normal_mode == FR_NORMAL_TETRA ? 0.5773f * eps : 1e-4f);
    R.shadow_off = 4.0f * eps;
    return FR_OK;
}

fr_status resolve_julia(fr::DevReq &R, const fr_julia_params *P)
{
    if (!P) return fail(FR_EINVAL, "julia params is NULL");
    if (P->p != 2 && P->p != 3) return fail(FR_EINVAL, "julia degree p=%d (2 or 3 supported)", P->p);
    if (!finite_n(P->c, 4) || !std::isfinite(P->slice_w)) return fail(FR_EINVAL, "julia c / slice_w not finite");
    if (!(P->escape_r2 > 0.0f) || !std::isfinite(P->escape_r2))
        return fail(FR_EINVAL, "escape_r2 must be positive and finite");
    R.kind = FR_KIND_JULIA;
    R.c = make_float4(P->c[0], P->c[1], P->c[2], P->c[3]);
    R.power = P->p;
    R.slice_w = P->slice_w;
    R.esc2 = P->escape_r2;
    return resolve_march(R, P->max_iter, P->bound_radius, P->max_steps, P->eps, P->max_step,
                         P->normal_mode, P->normal_h);
}

fr_status resolve_bulb(fr::DevReq &R, const fr_bulb_params *P)
{
    if (!P) return fail(FR_EINVAL, "mandelbulb params is NULL");
    if (P->n < 2 || P->n > 16) return fail(FR_EINVAL, "mandelbulb power n=%d outside 2..16", P->n);
    if (!(P->bailout > 0.0f) || !std::isfinite(P->bailout))
        return fail(FR_EINVAL, "bailout must be positive and finite");
    R.kind = FR_KIND_BULB;
    R.c = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    R.power = P->n;
    R.slice_w = 0.0f;
    R.esc2 = P->bailout * P->bailout;
    if (P->algebraic != 0 && P->algebraic != 1) return fail(FR_EINVAL, "algebraic must be 0 or 1");
    R.bulb_alg = P->algebraic;
    return resolve_march(R, P->max_iter, P->bound_radius, P->max_steps, P->eps, P->max_step,
                         P->normal_mode, P->normal_h);
}

// camera, light, plane and (when out != NULL) the output buffers
fr_status resolve_common(fr::DevReq &R, const fr_plane *pl, const fr_camera *cam, const fr_light *li,
                         const fr_image *out, bool need_out = true)
{
    if (!cam) return fail(FR_EINVAL, "camera is NULL");
    if (!li) return fail(FR_EINVAL, "light is NULL");
    if (need_out && !out) return fail(FR_EINVAL, "image is NULL");
    if (cam->width < 1 || cam->height < 1) return fail(FR_EINVAL, "image %dx%d is empty", cam->width, cam->height);
    if (cam->width > 65535 || cam->height > 65535)
        return fail(FR_EINVAL, "image sides are limited to 65535 (got %dx%d)", cam->width, cam->height);
    if (cam->spp < 1 || cam->spp > 64) return fail(FR_EINVAL, "spp %d outside 1..64", cam->spp);
    if ((long long)cam->width * cam->height * cam->spp >= (1LL << 31))
        return fail(FR_EINVAL, "width*height*spp must stay below 2^31");
    if (!finite_n(cam->eye, 3) || !finite_n(cam->target, 3) || !finite_n(cam->up, 3))
        return fail(FR_EINVAL, "camera vectors not finite");
    if (!(cam->fov_y_deg > 0.0f && cam->fov_y_deg < 180.0f))
        return fail(FR_EINVAL, "fov_y_deg %g outside (0, 180)", (double)cam->fov_y_deg);
    F3 fwd = sub(f3(cam->target), f3(cam->eye));
    if (!normalize(fwd)) return fail(FR_EINVAL, "camera eye equals target");
    F3 right = cross(fwd, f3(cam->up));
    if (!normalize(right)) return fail(FR_EINVAL, "camera up is parallel to the view direction");
    F3 up = cross(right, fwd);
    const float th = std::tan(0.5f * cam->fov_y_deg * 0.017453292519943295f);
    R.eye = f4(f3(cam->eye));
    R.fwd = f4(fwd);
    R.right = f4(right);
    R.up = f4(up);
    R.th = th;
    R.th_aspect = th * ((float)cam->width / (float)cam->height);
    R.inv_w = 1.0f / (float)cam->width;
    R.inv_h = 1.0f / (float)cam->height;
    R.width = cam->width;
    R.height = cam->height;
    R.tiles_x = (cam->width + fr::kTileW - 1) / fr::kTileW;
    R.spp = cam->spp;
    R.seed = cam->seed;
    const long long tiles_y = (cam->height + fr::kTileH - 1) / fr::kTileH;
    R.n_units = (long long)R.tiles_x * tiles_y * 32;
    R.unit_begin = 0;
    R.spl = 1;
    R.spl_log2 = 0;

    if (!finite_n(li->dir, 3) || !finite_n(li->albedo, 3) || !finite_n(li->background, 4) ||
        !std::isfinite(li->k_ambient) || !std::isfinite(li->k_diffuse))
        return fail(FR_EINVAL, "light values not finite");
    F3 L = f3(li->dir);
    if (!normalize(L)) return fail(FR_EINVAL, "light direction is zero");
    R.light = f4(L);
    R.albedo = make_float4(li->albedo[0], li->albedo[1], li->albedo[2], 0.0f);
    R.ka = li->k_ambient;
    R.kd = li->k_diffuse;
    R.shadows = li->shadows ? 1 : 0;
    R.bg = make_float4(li->background[0], li->background[1], li->background[2], li->background[3]);
    if (li->shading != FR_SHADE_LAMBERT && li->shading != FR_SHADE_PHONG)
        return fail(FR_EINVAL, "shading %d unknown", li->shading);
    R.shading = li->shading;
    if (R.shading == FR_SHADE_PHONG) {
        if (!(li->k_specular >= 0.0f) || !std::isfinite(li->k_specular))
            return fail(FR_EINVAL, "k_specular must be finite and >= 0");
        if (!(li->shininess >= 1.0f && li->shininess <= 4096.0f))
            return fail(FR_EINVAL, "shininess outside 1..4096");
        if (!(li->reflect_coef >= 0.0f && li->reflect_coef <= 1.0f))
            return fail(FR_EINVAL, "reflect_coef outside 0..1");
        R.k_spec = li->k_specular;
        R.shininess = li->shininess;
        R.refl_coef = li->reflect_coef;
    }

    R.plane_on = (pl && pl->enabled) ? 1 : 0;
    R.plane = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    R.plane_hat = R.plane;
    if (R.plane_on) {
        if (!finite_n(pl->n, 3) || !std::isfinite(pl->offset)) return fail(FR_EINVAL, "plane not finite");
        F3 n = f3(pl->n);
        if (!normalize(n)) return fail(FR_EINVAL, "plane normal is zero");
        R.plane = make_float4(pl->n[0], pl->n[1], pl->n[2], pl->offset);
        R.plane_hat = f4(n);
    }

    if (!need_out) return FR_OK;
    if (!out->rgba8 && !out->rgba && !out->depth && !out->saved && !out->stats && !out->trap)
        return fail(FR_EINVAL, "image has no output buffer");
    if (!aligned(out->rgba8, 4) || !aligned(out->depth, 4) || !aligned(out->rgba, 16) ||
        !aligned(out->saved, 16) || !aligned(out->stats, 8) || !aligned(out->trap, 16))
        return fail(FR_EINVAL, "output buffer misaligned (rgba/saved/trap 16 B, rgba8/depth 4 B, stats 8 B)");
    R.rgba8 = out->rgba8;
    R.rgba = reinterpret_cast<float4 *>(out->rgba);
    R.depth = out->depth;
    // rows of 4 adjacent pixels start on 16-byte boundaries of both buffers
    R.quad_store = (cam->width % 4 == 0 && aligned(out->rgba8, 16) && aligned(out->depth, 16)) ? 1 : 0;
    R.saved = reinterpret_cast<float4 *>(out->saved);
    R.stats = out->stats;
    R.trap = reinterpret_cast<float4 *>(out->trap);
    return FR_OK;
}

// lanes per pixel of the one-ray-per-thread kernels: the pixel's samples on
// adjacent lanes when the tuning asks for it and spp is 2, 4 or 8
int lanes_per_pixel(const fr_tuning &tu, const fr::DevReq &R)
{
    return (tu.sample_lanes && (R.spp == 2 || R.spp == 4 || R.spp == 8)) ? R.spp : 1;
}

void set_lanes(fr::DevReq &R, int spl)
{
    R.spl = spl;
    R.spl_log2 = spl == 8 ? 3 : spl == 4 ? 2 : spl == 2 ? 1 : 0;
}

fr_status launched(cudaError_t e)
{
    if (e != cudaSuccess) return fail(FR_ECUDA, "CUDA launch failed: %s", cudaGetErrorString(e));
    g_err.clear();
    return FR_OK;
}

}  // namespace

namespace fr {
// error reporting for entry points defined in other translation units
fr_status set_error(fr_status st, const char *msg) { return fail(st, "%s", msg); }

// Checks every request of a batch and resolves it into all[i] (no CUDA call);
// count is set when some request asks for the statistics counters.  The
// message of the first bad request names its index.
fr_status resolve_requests(const fr_request *reqs, int n_reqs, std::vector<DevReq> &all, bool &count)
{
    if (!reqs) return fail(FR_EINVAL, "requests is NULL");
    if (n_reqs < 1 || n_reqs > 4096) return fail(FR_EINVAL, "n_reqs %d outside 1..4096", n_reqs);
    all.assign((size_t)n_reqs, DevReq{});
    count = false;
    for (int i = 0; i < n_reqs; i++) {
        DevReq &R = all[(size_t)i];
        std::memset(&R, 0, sizeof R);
        const fr_request &q = reqs[i];
        fr_status st;
        if (q.kind == FR_KIND_JULIA)
            st = resolve_julia(R, &q.julia);
        else if (q.kind == FR_KIND_BULB)
            st = resolve_bulb(R, &q.bulb);
        else
            st = fail(FR_EINVAL, "kind %d unknown", q.kind);
        if (st == FR_OK) st = resolve_common(R, &q.plane, &q.camera, &q.light, &q.out);
        if (st != FR_OK) {
            g_err = "request " + std::to_string(i) + ": " + g_err;
            return st;
        }
        count = count || q.out.stats != nullptr;
    }
    return FR_OK;
}
}  // namespace fr

extern "C" {

FR_API int32_t fr_abi_version(void) { return 3; }

FR_API const char *fr_last_error(void) { return g_err.c_str(); }

FR_API fr_status fr_get_tuning(fr_tuning *out)
{
    if (!out) return fail(FR_EINVAL, "tuning is NULL");
    *out = tuning();
    return FR_OK;
}

FR_API fr_status fr_set_tuning(const fr_tuning *t)
{
    if (!t) return fail(FR_EINVAL, "tuning is NULL");
    auto block_ok = [](int b) { return b >= 32 && b <= 256 && b % 32 == 0; };
    auto unroll_ok = [](int u) { return u == 1 || u == 2 || u == 4; };
    if (!block_ok(t->plain_block) || !block_ok(t->persist_block))
        return fail(FR_EINVAL, "block sizes must be multiples of 32 in 32..256");
    if (!unroll_ok(t->plain_unroll) || !(unroll_ok(t->persist_unroll) || t->persist_unroll == 8))
        return fail(FR_EINVAL, "unroll depth must be 1, 2 or 4 (persistent: also 8)");
    if (t->persist_ctas_per_sm < 0 || t->persist_ctas_per_sm > 32)
        return fail(FR_EINVAL, "persist_ctas_per_sm outside 0..32");
    if (t->refill_threshold < 1 || t->refill_threshold > 32)
        return fail(FR_EINVAL, "refill_threshold outside 1..32");
    if (t->single_kernel < 0 || t->single_kernel > 2) return fail(FR_EINVAL, "single_kernel must be 0, 1 or 2");
    if (t->batch_kernel < 0 || t->batch_kernel > 2) return fail(FR_EINVAL, "batch_kernel must be 0, 1 or 2");
    if (t->tile_order < 0 || t->tile_order > 2) return fail(FR_EINVAL, "tile_order must be 0, 1 or 2");
    if (t->sample_lanes != 0 && t->sample_lanes != 1) return fail(FR_EINVAL, "sample_lanes must be 0 or 1");
    std::lock_guard<std::mutex> lk(g_tuning_mu);
    g_tuning = *t;
    return FR_OK;
}

// one request through the configured single-request kernel
static fr_status launch_single(const fr::DevReq &R, bool count, void *stream)
{
    const fr_tuning tu = tuning();
    if (tu.single_kernel == 1) {
        static thread_local fr::BatchArgs A;
        A.reqs[0] = R;
        A.reqs[0].unit_begin = 0;
        A.n_reqs = 1;
        A.total_units = R.n_units;
        A.refill_threshold = 1;
        A.queue = nullptr;
        return launched(fr::launch_lanes(A, tu.plain_block, tu.persist_unroll, count, R.shading != 0,
                                         (cudaStream_t)stream));
    }
    if (tu.single_kernel == 2) {
        // width * height * spp < 2^31 keeps a request below 2^26 tiles in either
        // layout (32 lanes per tile): the grid stays below the 2^31 - 1 CTA limit
        static thread_local fr::BatchArgs A;
        const long long warps_per_cta = tu.plain_block / 32;
        A.reqs[0] = R;
        A.reqs[0].unit_begin = 0;
        A.reqs[0].tile_order = tu.tile_order;
        set_lanes(A.reqs[0], lanes_per_pixel(tu, R));
        const long long ctas = (fr::plain_tiles(A.reqs[0]) + warps_per_cta - 1) / warps_per_cta;
        A.n_reqs = 1;
        A.total_units = ctas;
        A.refill_threshold = 1;
        A.queue = nullptr;
        return launched(fr::launch_batch_plain(A, ctas, tu.plain_block, tu.plain_unroll, count, R.shading != 0,
                                               (cudaStream_t)stream));
    }
    fr::DevReq Q = R;
    Q.tile_order = tu.tile_order;
    set_lanes(Q, lanes_per_pixel(tu, R));
    return launched(fr::launch_plain(Q, tu.plain_block, tu.plain_unroll, count, (cudaStream_t)stream));
}

FR_API fr_status fr_render_julia(const fr_julia_params *params, const fr_plane *plane,
                                 const fr_camera *camera, const fr_light *light, const fr_image *out,
                                 void *stream)
{
    fr::NvtxRange range("fr_render_julia");
    fr::DevReq R;
    std::memset(&R, 0, sizeof R);
    fr_status st = resolve_julia(R, params);
    if (st != FR_OK) return st;
    if ((st = resolve_common(R, plane, camera, light, out)) != FR_OK) return st;
    return launch_single(R, out->stats != nullptr, stream);
}

FR_API fr_status fr_render_mandelbulb(const fr_bulb_params *params, const fr_plane *plane,
                                      const fr_camera *camera, const fr_light *light,
                                      const fr_image *out, void *stream)
{
    fr::NvtxRange range("fr_render_mandelbulb");
    fr::DevReq R;
    std::memset(&R, 0, sizeof R);
    fr_status st = resolve_bulb(R, params);
    if (st != FR_OK) return st;
    if ((st = resolve_common(R, plane, camera, light, out)) != FR_OK) return st;
    return launch_single(R, out->stats != nullptr, stream);
}

// one 256-byte slot (queue head) per launch of up to kMaxReqPerLaunch requests
FR_API size_t fr_batch_workspace_bytes(int32_t n_reqs)
{
    if (n_reqs < 1) return 0;
    return (size_t)256 * (size_t)((n_reqs + fr::kMaxReqPerLaunch - 1) / fr::kMaxReqPerLaunch);
}

FR_API fr_status fr_render_batch(const fr_request *reqs, int32_t n_reqs, void *workspace,
                                 size_t ws_bytes, void *stream)
{
    fr::NvtxRange range("fr_render_batch");
    if (!reqs) return fail(FR_EINVAL, "requests is NULL");
    if (n_reqs < 1 || n_reqs > 4096) return fail(FR_EINVAL, "n_reqs %d outside 1..4096", n_reqs);
    if (!workspace) return fail(FR_EINVAL, "workspace is NULL");
    if (!aligned(workspace, 256)) return fail(FR_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < fr_batch_workspace_bytes(n_reqs))
        return fail(FR_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, fr_batch_workspace_bytes(n_reqs));
    // check every request before launching anything
    static thread_local fr::BatchArgs A;
    std::vector<fr::DevReq> all;
    bool count = false;
    {
        const fr_status st = fr::resolve_requests(reqs, n_reqs, all, count);
        if (st != FR_OK) return st;
    }
    const fr_tuning tu = tuning();
    for (fr::DevReq &R : all) set_lanes(R, tu.batch_kernel != 0 ? lanes_per_pixel(tu, R) : 1);

    // costliest requests first: the cheap ones then fill in behind the costly
    // ones' slow pixels at the end of the launch (outputs travel with their
    // request).  Estimated cost: pixels x samples x orbit-iteration cap, x 6
    // for the Mandelbulb (its step is about six Julia steps of instructions),
    // x 1.4 with shadow rays.  Measured on 64 mixed requests: 32.6 ms against
    // 33.1 ms ordered by pixels alone.
    std::vector<int> order((size_t)n_reqs);
    for (int i = 0; i < n_reqs; i++) order[(size_t)i] = i;
    auto cost = [&](int i) {
        const fr::DevReq &R = all[(size_t)i];
        return (double)R.n_units * R.spp * R.max_iter * (R.kind == FR_KIND_BULB ? 6.0 : 1.0) *
               (R.shadows ? 1.4 : 1.0);
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
    const long long warps_per_cta = tu.plain_block / 32;
    auto ctas_of = [&](const fr::DevReq &R) { return (fr::plain_tiles(R) + warps_per_cta - 1) / warps_per_cta; };
    if (tu.batch_kernel == 1)  // the grid of each launch must fit the 2^31 - 1 CTA limit
        for (int first = 0; first < n_reqs; first += fr::kMaxReqPerLaunch) {
            long long ctas = 0;
            for (int i = first; i < std::min(n_reqs, first + fr::kMaxReqPerLaunch); i++)
                ctas += ctas_of(all[(size_t)order[(size_t)i]]);
            if (ctas > 2147483647LL)
                return fail(FR_EINVAL, "one launch of this batch would need %lld CTAs (at most 2^31 - 1)", ctas);
        }
    for (int first = 0, chunk = 0; first < n_reqs; first += fr::kMaxReqPerLaunch, chunk++) {
        const int n = std::min(fr::kMaxReqPerLaunch, n_reqs - first);
        A.n_reqs = n;
        A.refill_threshold = tu.refill_threshold;
        A.queue = reinterpret_cast<unsigned long long *>(static_cast<char *>(workspace) + 256 * (size_t)chunk);
        fr_status st;
        if (tu.batch_kernel == 2) {
            long long tiles = 0;
            for (int i = 0; i < n; i++) {
                A.reqs[i] = all[(size_t)order[(size_t)(first + i)]];
                A.reqs[i].unit_begin = tiles;
                A.reqs[i].tile_order = tu.tile_order;
                tiles += fr::plain_tiles(A.reqs[i]);
            }
            A.total_units = tiles;
            bool phong = false;
            for (int i = 0; i < n; i++) phong = phong || A.reqs[i].shading != 0;
            st = launched(fr::launch_batch_refill(A, tu.plain_block, tu.plain_unroll, count, phong,
                                                  (cudaStream_t)stream));
        } else if (tu.batch_kernel == 1) {
            long long ctas = 0;
            for (int i = 0; i < n; i++) {
                A.reqs[i] = all[(size_t)order[(size_t)(first + i)]];
                A.reqs[i].unit_begin = ctas;
                A.reqs[i].tile_order = tu.tile_order;
                ctas += ctas_of(A.reqs[i]);
            }
            A.total_units = ctas;
            bool phong = false;
            for (int i = 0; i < n; i++) phong = phong || A.reqs[i].shading != 0;
            st = launched(fr::launch_batch_plain(A, ctas, tu.plain_block, tu.plain_unroll, count, phong,
                                                 (cudaStream_t)stream));
        } else {
            long long units = 0;
            for (int i = 0; i < n; i++) {
                A.reqs[i] = all[(size_t)order[(size_t)(first + i)]];
                A.reqs[i].unit_begin = units;
                units += A.reqs[i].n_units;
            }
            A.total_units = units;
            bool phong = false;
            for (int i = 0; i < n; i++) phong = phong || A.reqs[i].shading != 0;
            st = launched(fr::launch_persist(A, tu.persist_block, tu.persist_ctas_per_sm, tu.persist_unroll,
                                             count, phong, (cudaStream_t)stream));
        }
        if (st != FR_OK) return st;
    }
    return FR_OK;
}

static fr_status resolve_backward_common(fr::BwdArgs &A, const fr_plane *plane, const fr_camera *camera,
                                         const fr_light *light, const float *saved, const float *d_rgba,
                                         const float *d_depth, float *grad);

// checks and resolves the arguments of a backward call into A (acc/done left NULL)
static fr_status resolve_backward(fr::BwdArgs &A, const fr_julia_params *params, const fr_plane *plane,
                                  const fr_camera *camera, const fr_light *light, const float *saved,
                                  const float *d_rgba, const float *d_depth, float *grad)
{
    std::memset(&A, 0, sizeof A);
    fr_status st = resolve_julia(A.R, params);
    if (st != FR_OK) return st;
    if (params->max_iter > fr::kMaxBwdIter)
        return fail(FR_EINVAL, "backward keeps at most %d orbit iterations (max_iter %d)", fr::kMaxBwdIter,
                    params->max_iter);
    return resolve_backward_common(A, plane, camera, light, saved, d_rgba, d_depth, grad);
}

static fr_status resolve_backward_common(fr::BwdArgs &A, const fr_plane *plane, const fr_camera *camera,
                                         const fr_light *light, const float *saved, const float *d_rgba,
                                         const float *d_depth, float *grad)
{
    fr_status st;
    if (light && light->shading != FR_SHADE_LAMBERT)
        return fail(FR_EINVAL, "backward supports Lambert shading");
    if (!camera) return fail(FR_EINVAL, "camera is NULL");
    if (camera->spp != 1) return fail(FR_EINVAL, "backward needs spp == 1 (got %d)", camera->spp);
    if (!saved || !d_rgba || !grad) return fail(FR_EINVAL, "saved, d_rgba and grad must be given");
    if (!aligned(saved, 16) || !aligned(d_rgba, 16) || !aligned(d_depth, 4) || !aligned(grad, 4))
        return fail(FR_EINVAL, "buffer misaligned (saved/d_rgba 16 B, d_depth/grad 4 B)");
    if ((st = resolve_common(A.R, plane, camera, light, nullptr, false)) != FR_OK) return st;
    A.saved = reinterpret_cast<const float4 *>(saved);
    A.d_rgba = reinterpret_cast<const float4 *>(d_rgba);
    A.d_depth = d_depth;
    A.grad = grad;
    A.light_norm = std::sqrt(light->dir[0] * light->dir[0] + light->dir[1] * light->dir[1] +
                             light->dir[2] * light->dir[2]);
    A.plane_norm = A.R.plane_on ? std::sqrt(plane->n[0] * plane->n[0] + plane->n[1] * plane->n[1] +
                                            plane->n[2] * plane->n[2])
                                : 1.0f;
    return FR_OK;
}

FR_API fr_status fr_render_backward(const fr_julia_params *params, const fr_plane *plane,
                                    const fr_camera *camera, const fr_light *light, const float *saved,
                                    const float *d_rgba, const float *d_depth, float *grad, void *stream)
{
    fr::NvtxRange range("fr_render_backward");
    fr::BwdArgs A;
    const fr_status st = resolve_backward(A, params, plane, camera, light, saved, d_rgba, d_depth, grad);
    if (st != FR_OK) return st;
    return launched(fr::launch_backward(A, (cudaStream_t)stream));
}

FR_API fr_status fr_render_backward_mandelbulb(const fr_bulb_params *params, const fr_plane *plane,
                                               const fr_camera *camera, const fr_light *light,
                                               const float *saved, const float *d_rgba, const float *d_depth,
                                               float *grad, void *workspace, size_t ws_bytes, void *stream)
{
    fr::NvtxRange range("fr_render_backward_mandelbulb");
    if (workspace && !aligned(workspace, 16)) return fail(FR_EINVAL, "workspace must be 16-byte aligned");
    if (workspace && ws_bytes < fr_backward_workspace_bytes())
        return fail(FR_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, fr_backward_workspace_bytes());
    fr::BwdArgs A;
    std::memset(&A, 0, sizeof A);
    fr_status st = resolve_bulb(A.R, params);
    if (st != FR_OK) return st;
    if ((st = resolve_backward_common(A, plane, camera, light, saved, d_rgba, d_depth, grad)) != FR_OK)
        return st;
    if (workspace) {
        A.acc = static_cast<double *>(workspace);
        A.done = reinterpret_cast<unsigned int *>(static_cast<char *>(workspace) + 11 * sizeof(double));
        const cudaError_t e =
            cudaMemsetAsync(workspace, 0, fr_backward_workspace_bytes(), (cudaStream_t)stream);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return launched(e);
        }
    }
    return launched(fr::launch_backward(A, (cudaStream_t)stream));
}

// 11 doubles, then the finished-block count, padded to 128 bytes
FR_API size_t fr_backward_workspace_bytes(void) { return 128; }

FR_API fr_status fr_render_backward_ws(const fr_julia_params *params, const fr_plane *plane,
                                       const fr_camera *camera, const fr_light *light, const float *saved,
                                       const float *d_rgba, const float *d_depth, float *grad,
                                       void *workspace, size_t ws_bytes, void *stream)
{
    fr::NvtxRange range("fr_render_backward_ws");
    if (!workspace) return fail(FR_EINVAL, "workspace is NULL");
    if (!aligned(workspace, 16)) return fail(FR_EINVAL, "workspace must be 16-byte aligned");
    if (ws_bytes < fr_backward_workspace_bytes())
        return fail(FR_ENOMEM, "workspace %zu bytes < %zu needed", ws_bytes, fr_backward_workspace_bytes());
    fr::BwdArgs A;
    const fr_status st = resolve_backward(A, params, plane, camera, light, saved, d_rgba, d_depth, grad);
    if (st != FR_OK) return st;
    A.acc = static_cast<double *>(workspace);
    A.done = reinterpret_cast<unsigned int *>(static_cast<char *>(workspace) + 11 * sizeof(double));
    // the kernel leaves the workspace zeroed, but a workspace fresh from the
    // allocator (or left by a failed launch) is cleared here, in stream order
    const cudaError_t e = cudaMemsetAsync(workspace, 0, fr_backward_workspace_bytes(), (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();  // clear the error state so later calls start clean
        return launched(e);
    }
    return launched(fr::launch_backward(A, (cudaStream_t)stream));
}

}  // extern "C"
