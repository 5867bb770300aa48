/*
 * fr_oracle.h -- plain, slow CPU oracle for distance-estimated sphere tracing
 * of the quaternion Julia set and the degree-n Mandelbulb.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package's smoke() check
 * and the benchmark's CPU-baseline leg may load this library.  The product
 * path (the CUDA library) shares no code, header or constant with it.
 *
 * Everything is written once in a precision-generic body (fr_oracle_body.inc)
 * and compiled twice: the *_d entry points compute in double, the *_f entry
 * points in float.  Parameters always arrive as doubles; the float build
 * rounds each one to float on entry.  Compile with -ffp-contract=off so that
 * no multiply-add is fused behind the reader's back.
 *
 * Passages of the paper ("Real-time rendering of complex fractals",
 * da Silva, Novello, Lopes, Velho) followed by each part:
 *   quaternion Julia set, f(z)=z^p+c over the quaternions   Sec. 1.1
 *   Mandelbulb and the White-Nylander power (Eq. 1)         Sec. 1.2
 *   distance estimate d = |f^n| log|f^n| / |(f^n)'|         Eq. 2, Eqs. 3-4
 *   Julia distance listing (dz2 recursion, 0.25 log m2 ...) Listing "Julia Set distance"
 *   Mandelbulb distance listing                             Listing "Mandelbulb distance"
 *   sphere-tracing loop (tmin = eps, step clamp 0.2)        Listing "Julia Set ray cast"
 *   interval clip by bounding sphere and cutting plane      Sec. 3.1 (text before that listing)
 *   tetrahedral gradient                                    Eq. 5 and Listing "Normal calculation"
 *   hit -> normal -> shade                                  Listings "JuliaDistance", "Closest-hit shader"
 *   Phong + Fresnel-Schlick reflection bounce               closest-hit listing of Sec. 3.1
 *   analytic normal grad G / |grad G| (Julia, Mandelbulb)   Sec. 2
 *   gradient of the Julia render (dual numbers)             Sec. 2, implicit differentiation
 *
 * Every part is pinned by tests/test_oracle_*.py against something other than
 * itself (closed forms, complex-arithmetic orbits, brute force, finite
 * differences, symmetries).  Parity unpinned: the DE's upper bracket in 3D
 * (only the lower bound has a theorem), the colour at a mirror ray's hit (its
 * structure is pinned, not its value), orbit-trap values of orbits that stay
 * bounded, and whole images beyond their component pins (the paper prints no
 * values).
 */
#ifndef FR_ORACLE_H
#define FR_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_JULIA = 0, ORC_BULB = 1 };
enum { ORC_NORMAL_TETRA = 0, ORC_NORMAL_CENTRAL = 1, ORC_NORMAL_ANALYTIC = 2 };
enum { ORC_SHADE_LAMBERT = 0, ORC_SHADE_PHONG = 1 };

/* One render request.  All reals are doubles; the float build rounds them. */
typedef struct {
    int kind;                 /* ORC_JULIA or ORC_BULB */
    /* quaternion Julia: f(q) = q^p + c, 3D slice q = (x, y, z, slice_w) */
    double c[4];
    int p;                    /* 2 or 3 */
    double slice_w;
    double escape_r2;         /* escape when |q|^2 > escape_r2 */
    /* Mandelbulb: f(v) = v^n + c, orbit starts at w0 = c */
    int n;
    double bailout;           /* escape when |w| > bailout */
    /* shared */
    int max_iter;             /* orbit iteration cap */
    double bound_radius;      /* bounding sphere at the origin */
    int max_steps;            /* march step cap */
    double eps;               /* hit threshold (kPrecis) */
    double max_step;          /* step clamp (0.2 in the listing) */
    int normal_mode;          /* ORC_NORMAL_* */
    double normal_h;          /* <= 0: mode default */
    /* cutting plane: keep points with dot(plane_n, x) <= plane_o */
    int plane_enabled;
    double plane_n[3];
    double plane_o;
    /* pinhole camera */
    double eye[3], target[3], up[3];
    double fov_y_deg;
    int width, height, spp;
    uint32_t seed;
    /* directional light and Lambert shading */
    double light_dir[3];      /* toward the light; normalised by the oracle */
    double albedo[3];
    double k_ambient, k_diffuse;
    int shadows;
    double background[4];
    /* closest-hit model: ORC_SHADE_LAMBERT, or ORC_SHADE_PHONG = Phong lighting
     * plus one reflection bounce weighted by Fresnel-Schlick (the paper's
     * closest-hit listing for the Julia set) */
    int shading;
    double k_specular;        /* white specular weight */
    double shininess;         /* Phong exponent */
    double reflect_coef;      /* weight of the reflected colour (0.1 in the listing) */
} orc_scene;

/* Per-pixel outputs.  Any pointer may be NULL. */
typedef struct {
    float *rgba;              /* n x 4, unquantised mean colour          */
    uint32_t *rgba8;          /* n, r | g<<8 | b<<16 | a<<24              */
    float *depth;             /* n, min hit t over samples, +inf on miss  */
    int32_t *flags;           /* n, OR over samples: 1 hit, 2 cut face, 4 shadowed */
    int64_t *stats;           /* n x 7: primary DE calls, normal DE calls, shadow DE calls,
                                 orbit iterations, shadow rays, reflection DE calls,
                                 reflection rays                           */
    double *rgba64;           /* n x 4, same as rgba at the render precision (double build) */
    double *depth64;          /* n */
    float *trap;              /* n x 4, orbit-trap colour parameters at the nearest hit
                                 (Mandelbulb listing: (m, min|w.y|, min|w.z|, min m);
                                 Julia listing: (iterations before escape, |z|^2, 0, 0)) */
} orc_outputs;

/* Render pixels[i] (linear index y*width + x) for i < n_pixels; pixels == NULL
 * renders the whole image in row-major order.  Threads split the list in an
 * interleaved way; results do not depend on the thread count.
 * Returns 0 on success, -1 on a parameter it cannot take. */
int orc_render_d(const orc_scene *s, const int64_t *pixels, int64_t n_pixels,
                 const orc_outputs *out, int n_threads);
int orc_render_f(const orc_scene *s, const int64_t *pixels, int64_t n_pixels,
                 const orc_outputs *out, int n_threads);

/* Building blocks exposed for the pins. */
void orc_qmul_d(const double a[4], const double b[4], double out[4]);
void orc_qmul_f(const float a[4], const float b[4], float out[4]);
void orc_qpow_d(const double q[4], int p, double out[4]);
void orc_bulb_pow_d(const double v[3], int n, double out[3]);
void orc_bulb_pow_f(const float v[3], int n, float out[3]);
/* distance estimate at a 3D point; *n_out = non-escaping iterations,
 * *trips_out = orbit loop trips, *m2_out = final squared modulus */
double orc_de_d(const orc_scene *s, const double p[3], int *n_out, int *trips_out, double *m2_out);
float orc_de_f(const orc_scene *s, const float p[3], int *n_out, int *trips_out, float *m2_out);
/* 2D escape-time Julia set (Sec. 1.1): trips until |z|^2 > escape_r2, or max_iter */
int orc_julia2d_escape_d(double zr, double zi, double cr, double ci, int max_iter, double escape_r2);
/* search interval after the bounding sphere and the cut; returns 1 if non-empty */
int orc_bounds_d(const orc_scene *s, const double ro[3], const double rd[3],
                 double *t0, double *t1, int *from_plane);
/* camera ray of sample `sample` of pixel (px, py) */
void orc_camera_ray_d(const orc_scene *s, int px, int py, int sample, double ro[3], double rd[3]);
void orc_camera_ray_f(const orc_scene *s, int px, int py, int sample, float ro[3], float rd[3]);
uint64_t orc_splitmix64(uint64_t state);
void orc_jitter(uint32_t seed, int64_t pixel, int spp, int sample, double *sx, double *sy);

/* Test fields for the marcher and the gradient schemes (kind: 0 sphere
 * |p - q| - r with prm = (qx, qy, qz, r); 1 affine a.p + b with prm = (ax, ay, az, b);
 * 2 quadratic p^T A p + g.p with prm = (A row-major 9, g 3)). */
int orc_march_field_d(int kind, const double *prm, const double ro[3], const double rd[3],
                      double t0, double t1, int max_steps, double eps, double max_step,
                      double *t_out, int *steps_out);
void orc_normal_field_d(int kind, const double *prm, const double p[3], int mode, double h,
                        const double rd[3], double n_out[3]);
/* Lambert closed-hit shading of one sample and the 8-bit quantiser */
void orc_shade_d(const orc_scene *s, const double n[3], double vis, double rgba_out[4]);
/* Phong closest-hit colour of one sample seen along rd, with visibility vis,
 * plus reflect_coef * Fresnel-Schlick(albedo) * refl_rgb (the reflected colour) */
void orc_shade_phong_d(const orc_scene *s, const double n[3], const double rd[3], double vis,
                       const double refl_rgb[3], double rgba_out[4]);
/* unit normal at a point by the scene's normal mode (tetrahedral, central, or
 * analytic: grad G / |grad G| of the Julia set or the Mandelbulb); rd is the
 * fallback direction's ray */
void orc_normal_scene_d(const orc_scene *s, const double p[3], const double rd[3], double n[3]);
void orc_normal_scene_f(const orc_scene *s, const float p[3], const float rd[3], float n[3]);
/* orbit-trap colour parameters of the DE at a point (see orc_outputs.trap) */
void orc_trap_d(const orc_scene *s, const double p[3], double out[4]);
void orc_trap_f(const orc_scene *s, const float p[3], float out[4]);
uint32_t orc_quantize_d(double x);
uint32_t orc_quantize_f(float x);

/* Reference gradient of the loss
 *     L = sum_pixels mask * ( sum_ch d_rgba[ch] * rgba[ch] + d_depth * depth )
 * i.e. the vector-Jacobian product of the Julia render with cotangents d_rgba
 * (width*height*4) and d_depth (width*height, may be NULL), by implicit
 * differentiation at the hit point, with forward-mode dual numbers in double.
 * grad[0..3] = dL/dc, grad[4..6] = dL/dplane_n, grad[7] = dL/dplane_o,
 * grad[8..10] = dL/dlight_dir.  spp must be 1.  mask may be NULL. */
int orc_julia_grad_d(const orc_scene *s, const double *d_rgba, const double *d_depth,
                     const uint8_t *mask, double grad[11], int n_threads);

/* The same for a Mandelbulb render: the fractal has no parameter c
 * (grad[0..3] = 0), so surface hits move only through Lambert's n.L (light
 * direction) and cut-face hits through the plane and the light. */
int orc_bulb_grad_d(const orc_scene *s, const double *d_rgba, const double *d_depth,
                    const uint8_t *mask, double grad[11], int n_threads);

#ifdef __cplusplus
}
#endif
#endif
