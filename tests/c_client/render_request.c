/*
 * render_request.c -- a client of libfr.so written in plain C99: no Python,
 * no PyTorch.  It reads one request's parameter structs from a file, renders
 * it with fr_render_julia or fr_render_mandelbulb into device buffers it
 * allocates itself, and writes the packed colours and depths back out.
 *
 *   render_request <params.bin> <out.bin>
 *
 * params.bin: int32 kind (FR_KIND_JULIA or FR_KIND_BULB), then the
 * fr_julia_params or fr_bulb_params, fr_plane, fr_camera and fr_light structs,
 * byte for byte as laid out by include/fr.h.
 * out.bin: width*height uint32 packed colours, then width*height float depths.
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

int main(int argc, char **argv)
{
    int32_t kind;
    fr_julia_params jp;
    fr_bulb_params bp;
    fr_plane plane;
    fr_camera cam;
    fr_light light;
    if (argc != 3) {
        fprintf(stderr, "usage: %s params.bin out.bin\n", argv[0]);
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
    if (!ok || cam.width < 1 || cam.height < 1) {
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
    cudaFree(d_rgba8);
    cudaFree(d_depth);
    cudaStreamDestroy(stream);
    if (!ok) return 1;
    printf("rendered %dx%d with ABI version %d\n", (int)cam.width, (int)cam.height, (int)fr_abi_version());
    return 0;
}
