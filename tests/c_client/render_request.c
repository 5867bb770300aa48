/*
 * render_request.c -- a client of libfr.so written in plain C99: no Python,
 * no PyTorch.  It reads one request's parameter structs from a file, renders
 * it with fr_render_julia or fr_render_mandelbulb into device buffers it
 * allocates itself, and writes the packed colours and depths back out.
 *
 *   render_request <params.bin> <out.bin> [grad.bin]
 *
 * params.bin: int32 kind (FR_KIND_JULIA or FR_KIND_BULB), then the
 * fr_julia_params or fr_bulb_params, fr_plane, fr_camera and fr_light structs,
 * byte for byte as laid out by include/fr.h.
 * out.bin: width*height uint32 packed colours, then width*height float depths.
 * grad.bin (Julia requests only): the 11 floats fr_render_backward_ws returns
 * for the loss 0.5 |rgba|^2 of the float colour (cotangent = the colour
 * itself), with the hit state saved by a second forward call.
 * Exit status: 0 on success, 1 on bad usage or I/O, 2 when a call fails.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "fr.h"

static int read_exact(FILE *f, void *p, size_t n)
{
    return fread(p, 1, n, f) == n;
}

/* forward with the float colour and the saved hit state, then the adjoint of
 * 0.5 |rgba|^2 into a zeroed 11-float gradient; writes the gradient to path */
static int backward(const fr_julia_params *jp, const fr_plane *plane, const fr_camera *cam,
                    const fr_light *light, size_t n, cudaStream_t stream, const char *path)
{
    float *d_rgba = NULL, *d_saved = NULL, *d_grad = NULL;
    void *ws = NULL;
    const size_t ws_bytes = fr_backward_workspace_bytes();
    if (cudaMalloc((void **)&d_rgba, n * 4 * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&d_saved, n * 4 * sizeof(float)) != cudaSuccess ||
        cudaMalloc((void **)&d_grad, 11 * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&ws, ws_bytes) != cudaSuccess ||
        cudaMemsetAsync(d_grad, 0, 11 * sizeof(float), stream) != cudaSuccess)
        return 1;
    fr_image img;
    memset(&img, 0, sizeof img);
    img.rgba = d_rgba;
    img.saved = d_saved;
    fr_status st = fr_render_julia(jp, plane, cam, light, &img, stream);
    if (st == FR_OK)
        st = fr_render_backward_ws(jp, plane, cam, light, d_saved, d_rgba, NULL, d_grad, ws, ws_bytes, stream);
    if (st != FR_OK) {
        fprintf(stderr, "backward failed (%d): %s\n", (int)st, fr_last_error());
        return 1;
    }
    float grad[11];
    if (cudaMemcpyAsync(grad, d_grad, sizeof grad, cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return 1;
    FILE *f = fopen(path, "wb");
    const int ok = f && fwrite(grad, sizeof(float), 11, f) == 11;
    if (f) fclose(f);
    cudaFree(d_rgba);
    cudaFree(d_saved);
    cudaFree(d_grad);
    cudaFree(ws);
    return ok ? 0 : 1;
}

int main(int argc, char **argv)
{
    int32_t kind;
    fr_julia_params jp;
    fr_bulb_params bp;
    fr_plane plane;
    fr_camera cam;
    fr_light light;
    if (argc != 3 && argc != 4) {
        fprintf(stderr, "usage: %s params.bin out.bin [grad.bin]\n", argv[0]);
        return 1;
    }
    FILE *in = fopen(argv[1], "rb");
    if (!in) return 1;
    int ok = read_exact(in, &kind, sizeof kind);
    if (ok && kind == FR_KIND_JULIA)
        ok = read_exact(in, &jp, sizeof jp);
    else if (ok && kind == FR_KIND_BULB)
        ok = read_exact(in, &bp, sizeof bp);
    else
        ok = 0;
    ok = ok && read_exact(in, &plane, sizeof plane) && read_exact(in, &cam, sizeof cam) &&
         read_exact(in, &light, sizeof light);
    fclose(in);
    if (!ok || cam.width < 1 || cam.height < 1 || (argc == 4 && kind != FR_KIND_JULIA)) {
        fprintf(stderr, "bad parameter file\n");
        return 1;
    }

    const size_t n = (size_t)cam.width * (size_t)cam.height;
    uint32_t *d_rgba8 = NULL;
    float *d_depth = NULL;
    cudaStream_t stream;
    if (cudaMalloc((void **)&d_rgba8, n * sizeof(uint32_t)) != cudaSuccess ||
        cudaMalloc((void **)&d_depth, n * sizeof(float)) != cudaSuccess ||
        cudaStreamCreate(&stream) != cudaSuccess) {
        fprintf(stderr, "CUDA setup failed\n");
        return 2;
    }
    fr_image img;
    memset(&img, 0, sizeof img);
    img.rgba8 = d_rgba8;
    img.depth = d_depth;
    fr_status st = kind == FR_KIND_JULIA ? fr_render_julia(&jp, &plane, &cam, &light, &img, stream)
                                         : fr_render_mandelbulb(&bp, &plane, &cam, &light, &img, stream);
    if (st != FR_OK) {
        fprintf(stderr, "render failed (%d): %s\n", (int)st, fr_last_error());
        return 2;
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess) {
        fprintf(stderr, "render did not complete\n");
        return 2;
    }

    uint32_t *rgba8 = (uint32_t *)malloc(n * sizeof(uint32_t));
    float *depth = (float *)malloc(n * sizeof(float));
    if (!rgba8 || !depth ||
        cudaMemcpy(rgba8, d_rgba8, n * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(depth, d_depth, n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
        fprintf(stderr, "copy back failed\n");
        return 2;
    }
    FILE *out = fopen(argv[2], "wb");
    ok = out && fwrite(rgba8, sizeof(uint32_t), n, out) == n && fwrite(depth, sizeof(float), n, out) == n;
    if (out) fclose(out);
    free(rgba8);
    free(depth);
    if (ok && argc == 4 && backward(&jp, &plane, &cam, &light, n, stream, argv[3]) != 0) return 2;
    cudaFree(d_rgba8);
    cudaFree(d_depth);
    cudaStreamDestroy(stream);
    if (!ok) return 1;
    printf("rendered %dx%d with ABI version %d\n", (int)cam.width, (int)cam.height, (int)fr_abi_version());
    return 0;
}
