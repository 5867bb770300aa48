/*
 * fr.h -- C ABI of libfr, a GB300 (sm_103a) CUDA renderer for distance-estimated
 * sphere tracing of the quaternion Julia set and the degree-n Mandelbulb.
 *
 * Method (da Silva, Novello, Lopes, Velho, "Real-time rendering of complex
 * fractals"):
 *   - quaternion Julia set of f(q) = q^p + c, seen through the 3D slice
 *     q = (x, y, z, slice_w), optionally cut by a plane            Sec. 1.1, Fig. 1
 *   - Mandelbulb of f(v) = v^n + c with the White-Nylander power    Sec. 1.2, Eq. 1
 *   - distance estimate d = 0.5 |f^k| log|f^k| / |(f^k)'| from the orbit and its
 *     running derivative                                           Eq. 2, Eqs. 3-4,
 *                                      Listings "Julia Set distance", "Mandelbulb distance"
 *   - sphere tracing from t = eps in steps of min(d, max_step) inside the
 *     interval left by a bounding sphere and the cutting plane     Listing "Julia Set ray cast", Sec. 3.1
 *   - normal = normalised gradient of d, tetrahedral (Eq. 5, Listing "Normal
 *     calculation") or central differences, or grad G / |grad G| from the
 *     orbit's Jacobian (Sec. 2)
 *   - closest-hit shading: Lambert with one directional light and an optional
 *     shadow ray, or the Phong + Fresnel-weighted mirror ray of Listing
 *     "Closest-hit shader"; the listings' orbit-trap colour parameters as an
 *     optional output
 *   - the adjoint of the Julia render by implicit differentiation at the hit
 *     (Sec. 2's level-set relations)
 *
 * Conventions shared by every entry point:
 *   - Device memory belongs to the caller.  Every pointer in fr_image, the
 *     gradient and the batch workspace is a device pointer (cudaMalloc or a
 *     torch CUDA tensor); the parameter structs and the request array are host
 *     memory, read before the call returns.
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy default
 *     stream).  The library allocates no device memory.
 *   - Parameters are checked on the host first.  A bad argument returns
 *     FR_EINVAL, launches nothing and leaves a message for fr_last_error().
 *     A failed launch returns FR_ECUDA.  Results are defined once the stream
 *     reaches the work.
 *   - Images are row-major, row 0 at the top, pixel (x, y) at index y*width + x.
 *     rgba8 packs r | g<<8 | b<<16 | a<<24, each channel round-half-up of
 *     clamp(value, 0, 1) * 255.  Depth is the ray parameter t of the nearest hit
 *     along the unit view ray (world units), +inf where no sample hit.
 *   - With spp > 1 the colour is the mean over the pixel's samples (sub-pixel
 *     offsets from splitmix64 of (seed << 40) + pixel*spp + sample) and the depth
 *     the smallest hit t.
 */
#ifndef FR_H
#define FR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FR_API __attribute__((visibility("default")))
#else
#define FR_API
#endif

typedef enum {
    FR_OK = 0,
    FR_EINVAL = 1,     /* bad argument; nothing launched                          */
    FR_ECUDA = 2,      /* a CUDA call failed (message in fr_last_error)           */
    FR_ETIMEOUT = 3,   /* reserved: no kernel of this library waits on another    */
    FR_ENOMEM = 4,     /* caller-provided workspace too small                     */
    FR_ENOTIMPL = 5    /* combination not supported                               */
} fr_status;

enum { FR_KIND_JULIA = 0, FR_KIND_BULB = 1 };
enum { FR_NORMAL_TETRA = 0, FR_NORMAL_CENTRAL = 1, FR_NORMAL_ANALYTIC = 2 };
enum { FR_SHADE_LAMBERT = 0, FR_SHADE_PHONG = 1 };

/* indices into fr_image.stats */
enum {
    FR_STAT_PRIMARY_RAYS = 0,  /* camera rays traced (width*height*spp)              */
    FR_STAT_SHADOW_RAYS = 1,   /* shadow rays cast (one per shaded hit when enabled)  */
    FR_STAT_PRIMARY_DE = 2,    /* distance-estimator calls of camera-ray marches      */
    FR_STAT_NORMAL_DE = 3,     /* distance-estimator calls of the normal stencils     */
    FR_STAT_SHADOW_DE = 4,     /* distance-estimator calls of shadow-ray marches      */
    FR_STAT_ORBIT_ITERS = 5,   /* orbit loop trips summed over all DE calls           */
    FR_STAT_REFLECT_RAYS = 6,  /* reflection rays cast (one per hit, Phong shading)   */
    FR_STAT_REFLECT_DE = 7,    /* distance-estimator calls of reflection-ray marches  */
    FR_NSTATS = 8
};

/* Pinhole camera.  Forward = target - eye, right = forward x up, vertical field
 * of view fov_y_deg in (0, 180).  One sample per pixel sits at the pixel centre. */
typedef struct {
    float eye[3], target[3], up[3];
    float fov_y_deg;
    int32_t width, height;   /* 1..65535, width*height*spp < 2^31      */
    int32_t spp;             /* samples per pixel, 1..64               */
    uint32_t seed;           /* jitter seed (used when spp > 1)        */
} fr_camera;

/* Directional light and the closest-hit model.
 * FR_SHADE_LAMBERT:
 *   hit:  rgb = albedo * (k_ambient + k_diffuse * max(0, n . L) * visible), a = 1
 * FR_SHADE_PHONG (the closest-hit shader of Sec. 3.1: Phong lighting plus a
 * reflection ray weighted by the Fresnel-Schlick reflectance; its helpers are
 * not listed, so the model is stated here):
 *   phong(n, d, vis) = albedo * (k_ambient + k_diffuse * max(0, n . L) * vis)
 *                      + k_specular * vis * max(0, r . (-d))^shininess,
 *                      r = 2 (n . L) n - L, no highlight where n . L <= 0
 *   hit:  rgb = phong(n, rd, visible) + reflect_coef * F * refl, a = 1, where
 *         F = albedo + (1 - albedo) (1 - max(0, -n . rd))^5 per channel, and
 *         refl = phong(n2, rr, 1) at the first hit of the mirror ray
 *         rr = rd - 2 (n . rd) n from x + 4 eps n (normal n2 by the request's
 *         normal scheme, no shadow ray, no further bounce), background rgb on
 *         a miss
 *   miss: rgba = background
 * Every forward kernel runs both models; the adjoint (fr_render_backward)
 * refuses the Phong model with FR_EINVAL. */
typedef struct {
    float dir[3];            /* toward the light; normalised here, must be non-zero */
    float albedo[3];
    float k_ambient, k_diffuse;
    int32_t shadows;         /* 1: one shadow ray per hit, start x + 4 eps n      */
    float background[4];
    int32_t shading;         /* FR_SHADE_LAMBERT or FR_SHADE_PHONG                 */
    float k_specular;        /* >= 0 (Phong)                                       */
    float shininess;         /* 1..4096 (Phong)                                    */
    float reflect_coef;      /* 0..1; the listing uses 0.1 (Phong)                 */
} fr_light;

/* Cutting plane (Sec. 3.1, Fig. 1): points with dot(n, x) > offset are removed.
 * A ray whose search interval starts on the plane and whose first DE sample is
 * already below eps hits the cut face; its normal is n / |n|. */
typedef struct {
    int32_t enabled;
    float n[3];              /* non-zero when enabled                  */
    float offset;
} fr_plane;

/* Quaternion Julia set, f(q) = q^p + c (Listing "Julia Set distance" with
 * degree p; the listing itself uses p = 3, the text of Sec. 1.1 p = 2). */
typedef struct {
    float c[4];              /* (real, i, j, k)                                   */
    int32_t p;               /* 2 or 3                                            */
    float slice_w;           /* k-component of the 3D slice (0 in the listing)    */
    int32_t max_iter;        /* orbit iteration cap, 1..1024                      */
    float escape_r2;         /* escape once |q|^2 > escape_r2 (listing: 256)      */
    float bound_radius;      /* bounding sphere at the origin, > 0                */
    int32_t max_steps;       /* march step cap, 1..100000 (listing: 1024)         */
    float eps;               /* hit threshold kPrecis, > 0                        */
    float max_step;          /* step clamp (listing: 0.2), > 0                    */
    int32_t normal_mode;     /* FR_NORMAL_TETRA, FR_NORMAL_CENTRAL, or FR_NORMAL_ANALYTIC:
                                grad d = grad G / |grad G| on the set (Sec. 2), from the
                                orbit's derivative carried alongside it (no stencil) */
    float normal_h;          /* stencil size; 0 = 0.5773*eps (tetra), 1e-4 (central) */
} fr_julia_params;

/* Mandelbulb, f(v) = v^n + c with the orbit started at w0 = c (Listing
 * "Mandelbulb distance"; the listing uses n = 8, 4 iterations, |w|^2 > 256). */
typedef struct {
    int32_t n;               /* power, 2..16                                      */
    int32_t max_iter;        /* orbit iteration cap, 1..1024                      */
    float bailout;           /* escape once |w| > bailout, > 0                    */
    float bound_radius;
    int32_t max_steps;
    float eps;
    float max_step;
    int32_t normal_mode;     /* as for the Julia set; FR_NORMAL_ANALYTIC carries
                                J = dw/dc through Eq. 1 (J <- DP(w) J + I) and
                                takes grad G along J^T w_N                       */
    float normal_h;
    int32_t algebraic;       /* 0: the listing's acos/atan2/sin/cos power; 1: the same
                                Eq. 1 by de Moivre powers of cos + i sin, no
                                transcendental calls in the orbit loop           */
} fr_bulb_params;

/* Output buffers (device).  Any may be NULL except that at least one of rgba8,
 * rgba, depth, saved, stats, trap must be given.  Alignment: rgba, saved and
 * trap 16 bytes, the others 4 (stats 8). */
typedef struct {
    uint32_t *rgba8;             /* width*height packed colour                        */
    float *rgba;                 /* width*height*4 mean colour before quantisation     */
    float *depth;                /* width*height nearest hit t, +inf on a miss         */
    float *saved;                /* width*height*4: hit point x, y, z and flag bits    */
                                 /* (1 hit, 2 cut face, 4 shadowed) as a float's bits; */
                                 /* the state fr_render_backward reads                 */
    unsigned long long *stats;   /* FR_NSTATS counters, ADDED to (zero them first)     */
    float *trap;                 /* width*height*4 orbit-trap values of the DE at the  */
                                 /* nearest hit point, (0,0,0,0) on a miss.  Mandelbulb: */
                                 /* the listing's resColor = (final |w|^2, min |w.y|,   */
                                 /* min |w.z|, min |w|^2); Julia: (iterations before    */
                                 /* escape -- the listing's second output --, final    */
                                 /* |z|^2, 0, 0).  One extra DE per hit pixel.          */
} fr_image;

/* One request of a batch.  `kind` selects which parameter block is read. */
typedef struct {
    int32_t kind;            /* FR_KIND_JULIA or FR_KIND_BULB */
    fr_julia_params julia;
    fr_bulb_params bulb;
    fr_plane plane;
    fr_camera camera;
    fr_light light;
    fr_image out;
} fr_request;

/* Launch shapes; the autotuner writes them, every later call reads them. */
typedef struct {
    int32_t plain_block;         /* threads per block of the one-ray-per-thread kernel (32..256, x32) */
    int32_t plain_unroll;        /* orbit-loop unroll depth: 1, 2 or 4                  */
    int32_t persist_block;       /* threads per block of the persistent kernel          */
    int32_t persist_ctas_per_sm; /* resident CTAs per SM; 0 = as many as fit            */
    int32_t refill_threshold;    /* refill a warp once this many lanes are idle (1..32) */
    int32_t persist_unroll;      /* Julia orbit steps per scheduling round: 1, 2, 4, 8  */
    int32_t single_kernel;       /* fr_render_julia/mandelbulb: 0 nested loops per thread,
                                    1 lane state machine (one DE call site), no queue,
                                    2 the batch kernel (batch_kernel 1's code, which
                                    the compiler allocates differently) with the one
                                    request.  Same images bit for bit.               */
    int32_t batch_kernel;        /* fr_render_batch: 0 persistent kernel with the pixel
                                    queue and the lane state machine, 1 one-ray-per-thread
                                    kernel over every tile of every request in one launch
                                    (plain_block threads), 2 (default) the same per-pixel
                                    code in persistent warps, each taking the next tile of
                                    the launch from the queue head as soon as its lanes
                                    are done                                           */
    int32_t tile_order;          /* how the one-ray-per-thread kernels lay their 4 x 8
                                    tiles, in launch order, over each image: 0 (default)
                                    rows top to bottom, 1 columns left to right, 2 rows
                                    bottom to top.  The hardware starts CTAs roughly in
                                    index order, so this decides which part of the frame
                                    runs first; images are the same bit for bit.      */
    int32_t sample_lanes;        /* one-ray-per-thread kernels with spp 2, 4 or 8: 1 (default)
                                    the pixel's samples on spp adjacent lanes (a warp
                                    covers 4 x 8 / spp pixels, whose jittered rays take
                                    nearly the same marches), 0 each lane runs its
                                    pixel's samples in turn (4 x 8 pixels per warp).
                                    Same images bit for bit.                           */
} fr_tuning;

/* Render one quaternion Julia image with the one-ray-per-thread kernel
 * (camera ray -> interval -> march -> normal -> shadow -> shade -> store).
 * plane may be NULL (no cut).  Errors: FR_EINVAL, FR_ECUDA. */
FR_API fr_status fr_render_julia(const fr_julia_params *params, const fr_plane *plane,
                                 const fr_camera *camera, const fr_light *light,
                                 const fr_image *out, void *stream);

/* Same for the Mandelbulb. */
FR_API fr_status fr_render_mandelbulb(const fr_bulb_params *params, const fr_plane *plane,
                                      const fr_camera *camera, const fr_light *light,
                                      const fr_image *out, void *stream);

/* Device workspace a batch of n_reqs requests needs (bytes, 256-aligned start). */
FR_API size_t fr_batch_workspace_bytes(int32_t n_reqs);

/* Render n_reqs requests (mixed kinds and sizes) with one kernel launch per 64
 * requests (costliest first: pixels x samples x iteration cap, weighted by
 * fractal and shadows).  Three schedules, picked by fr_tuning.batch_kernel:
 *   2 (default)  one-ray-per-thread code in persistent CTAs over every tile of
 *                every request: each warp takes the next 32-pixel tile of the
 *                launch from the queue head as soon as its lanes are done, so
 *                the slow pixels of different requests overlap and no warp
 *                waits for the other warps of its CTA;
 *   1            the same per-pixel code as a grid over every tile of every
 *                request: each CTA belongs to one request and the hardware
 *                block scheduler hands CTAs to SMs as they free up;
 *   0            persistent CTAs, each warp pulling pixels from one queue over
 *                all requests and refilling idle lanes as rays finish.
 * Images are the same bit for bit either way (and equal fr_render_julia /
 * fr_render_mandelbulb of each request).  The request table travels in the
 * kernel's parameters, so the call is at most a memset of the queue heads plus
 * one launch per 64 requests, with no host synchronisation and no copy: it can
 * be captured into a CUDA graph and replayed.  `workspace` (device,
 * >= fr_batch_workspace_bytes(n_reqs) bytes, 256-byte aligned) holds the
 * queue heads of schedules 0 and 2 and is overwritten; two batches in flight at once need two
 * workspaces.  reqs is host memory.  1 <= n_reqs <= 4096.  Errors: FR_EINVAL
 * (also when one launch's 64 requests would need more than 2^31 - 1 CTAs),
 * FR_ENOMEM (workspace too small), FR_ECUDA. */
FR_API fr_status fr_render_batch(const fr_request *reqs, int32_t n_reqs, void *workspace,
                                 size_t ws_bytes, void *stream);

/* fr_render_batch without a caller-provided workspace.  The paper has no
 * counterpart: this is for callers that cannot allocate device memory -- a
 * plugin whose host application owns every device allocation, or a frame loop
 * that may not call cudaMalloc once running (it can synchronise the device and
 * break frame pacing).  The queue heads live in a 16 KB file-scope __device__
 * array of the library, enough for the largest batch fr_render_batch accepts
 * (4096 requests); every GPU that loads the library keeps it until exit.  The
 * requests are checked before any CUDA call.  A call made while `stream` is not
 * being captured looks the array's address up (cudaGetSymbolAddress, with the
 * current device), so a device reset in between is followed; a call made
 * during a stream capture reuses the address last looked up on that device,
 * so the first call on a device must come before any capture (otherwise
 * FR_EINVAL).  Nothing is allocated: no cudaMalloc, cudaFree or allocating
 * library call.  The array is shared by every call (each launch zeroes its own
 * queue head first), so calls that overlap on the GPU -- on different streams,
 * or from different threads -- race on it; serialise them.  Errors: as
 * fr_render_batch, plus FR_EINVAL for n_reqs outside 1..4096. */
FR_API fr_status fr_render_batch_static(const fr_request *reqs, int32_t n_reqs, void *stream);

/* Vector-Jacobian product of a Julia render (spp = 1) by implicit
 * differentiation at the hit point: for surface hits
 *     dt/dtheta = -(dd/dtheta) / (grad_x d . rd),
 * the normal's dependence through the stencil taps (or, for the analytic
 * normal, through J^T z_N by reverse mode over the orbit and its tangent),
 * Lambert's through n and L;
 * cut-face hits through t = (offset - n.ro)/(n.rd) and the normal n/|n|.
 * The orbit is recomputed from the hit point saved by the forward call (same
 * parameters, out.saved given).  Escape counts, hit status and shadow
 * visibility are held fixed.
 *   saved    width*height*4 floats from the forward call (device)
 *   d_rgba   width*height*4 cotangent of fr_image.rgba (device; alpha ignored)
 *   d_depth  width*height cotangent of the depth (device, may be NULL; miss
 *            pixels ignored)
 *   grad     11 floats (device), ADDED to: dc[4], dplane_n[3], dplane_offset,
 *            dlight_dir[3]
 * The pixels' contributions are summed in double on the device (a per-device
 * accumulator of the library that every call clears when it ends), so the
 * result does not depend on the order the GPU runs the pixels in: the same
 * inputs give the same gradient bits.  Calls that overlap on the GPU (on
 * different streams, or from different threads) share that accumulator and
 * race on it; serialise them, or give each its own workspace through
 * fr_render_backward_ws.
 * Errors: FR_EINVAL (spp != 1, Phong shading, NULL buffers, bad parameters),
 * FR_ECUDA. */
FR_API fr_status fr_render_backward(const fr_julia_params *params, const fr_plane *plane,
                                    const fr_camera *camera, const fr_light *light,
                                    const float *saved, const float *d_rgba, const float *d_depth,
                                    float *grad, void *stream);

/* fr_render_backward with the double accumulator in caller-owned device
 * memory instead of the library's, so that calls with different workspaces
 * may overlap on the GPU (different streams or threads; one workspace per call
 * in flight).  The call clears the workspace on `stream` before its kernel and
 * the kernel leaves it cleared; its contents between calls carry nothing.
 *   workspace  device memory, 16-byte aligned, fr_backward_workspace_bytes()
 *              bytes (11 doubles and a block counter)
 * Same result bits as fr_render_backward for the same inputs.
 * Errors: FR_EINVAL (workspace NULL or misaligned, and as fr_render_backward),
 * FR_ENOMEM (ws_bytes too small), FR_ECUDA.  The workspace is checked before
 * anything else. */
FR_API size_t fr_backward_workspace_bytes(void);

/* Vector-Jacobian product of a Mandelbulb render (spp = 1, Lambert), same
 * cotangents and 11-float layout as fr_render_backward.  The fractal has no
 * parameter c (grad[0..3] gets nothing); a surface hit moves with neither the
 * cut plane nor the light, so it adds only Lambert's d(n.L)/d(light dir) with
 * n the forward pass's normal at the saved hit, and a cut-face hit adds the
 * plane's and the light's terms as in fr_render_backward.
 *   workspace  NULL (the library's accumulator: calls must not overlap) or
 *              fr_backward_workspace_bytes() bytes of device memory, 16-byte
 *              aligned, as for fr_render_backward_ws
 * Errors: FR_EINVAL (spp != 1, Phong shading, NULL buffers, bad parameters,
 * misaligned workspace), FR_ENOMEM (ws_bytes too small), FR_ECUDA. */
FR_API fr_status fr_render_backward_mandelbulb(const fr_bulb_params *params, const fr_plane *plane,
                                               const fr_camera *camera, const fr_light *light,
                                               const float *saved, const float *d_rgba, const float *d_depth,
                                               float *grad, void *workspace, size_t ws_bytes, void *stream);
FR_API fr_status fr_render_backward_ws(const fr_julia_params *params, const fr_plane *plane,
                                       const fr_camera *camera, const fr_light *light,
                                       const float *saved, const float *d_rgba, const float *d_depth,
                                       float *grad, void *workspace, size_t ws_bytes, void *stream);

/* Diagnostic, with no counterpart in the paper: the FP32 fused multiply-add
 * rate of this GPU, the denominator of the renderer's FP32 roofline.  Launches
 * `blocks` x `threads` threads (threads 32..256, a multiple of 32), each running
 * 8 independent chains of iters * 16 fused multiply-adds, and writes one float
 * per thread to `sink` (device, blocks * threads floats, 4-byte aligned) so
 * that no chain is dead code.  Time it with events on `stream`;
 * fr_ffma_probe_flops gives the FP32 operations of one launch (2 per FFMA; 0
 * for non-positive arguments).  Errors: FR_EINVAL, FR_ECUDA. */
FR_API fr_status fr_ffma_probe(int32_t blocks, int32_t threads, int32_t iters, float *sink, void *stream);
FR_API double fr_ffma_probe_flops(int32_t blocks, int32_t threads, int32_t iters);

/* Read / replace the process-wide launch shapes (checked; FR_EINVAL if out of range). */
FR_API fr_status fr_get_tuning(fr_tuning *out);
FR_API fr_status fr_set_tuning(const fr_tuning *t);

/* Message of the calling thread's last failure ("" if none). */
FR_API const char *fr_last_error(void);

/* ABI version of this header (increments on any layout change). */
FR_API int32_t fr_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif
