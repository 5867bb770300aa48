// Accuracy of the orbit step's own transcendental routines (fr_math.cuh)
// against double precision on the device, beside the CUDA library routines
// they replace.  Prints one line of key=value pairs; tests/test_math_gpu.py
// compiles, runs and checks it.
#include <cmath>
#include <cstdint>
#include <cstdio>

#include "fr_math.cuh"

using namespace fr;

// error of got in units of the float ulp at ref (ulp of the smallest normal for ref = 0)
__device__ double ulps(float got, double ref)
{
    const float a = fabsf((float)ref);
    const float up = a == 0.0f ? 1.17549435e-38f : nextafterf(a, INFINITY) - a;
    return fabs((double)got - ref) / (double)up;
}

// maxima kept as fixed-point integers (atomicMax on unsigned long long)
__device__ void keep_max(unsigned long long *slot, double v)
{
    atomicMax(slot, (unsigned long long)fmin(v * 1e9, 1.8e19));
}

__device__ float lcg_unit(uint64_t &s)
{
    s = s * 6364136223846793005ULL + 1442695040888963407ULL;
    return (float)((s >> 40) & 0xffffff) * (1.0f / 16777216.0f);
}

enum { kAtanOwn, kAtanLib, kAtanAbs, kAcosOwn, kAcosLib, kAcosAbs, kSinAbsOwn, kCosAbsOwn,
       kSinAbsLib, kCosAbsLib, kQuot, kSqrtOwn, kLogOwn, kLogLib, kRsqrtOwn, kSlots };

__global__ void atan2_kernel(unsigned long long *m, long long n)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t s = 0x9e3779b97f4a7c15ULL ^ (uint64_t)i;
        float y = (lcg_unit(s) * 2.0f - 1.0f) * 2.0f, x = (lcg_unit(s) * 2.0f - 1.0f) * 2.0f;
        const int scale = (int)(lcg_unit(s) * 4.0f);
        if (scale == 1) y *= 1e-3f;
        if (scale == 2) x *= 1e-3f;
        const double ref = atan2((double)y, (double)x) / M_PI;
        const float own = atan2pi(y, x);
        keep_max(&m[kAtanOwn], ulps(own, ref));
        keep_max(&m[kAtanLib], ulps(__fmul_rn(atan2f(y, x), 0.318309886183790671538f), ref));
        keep_max(&m[kAtanAbs], fabs((double)own - ref) * 1e6);
        // y / x for |y| <= |x|: within one ulp (faithful)
        const float ax = fmaxf(fabsf(x), 1e-30f);
        const float q = quot(copysignf(fminf(fabsf(y), ax), y), ax);
        keep_max(&m[kQuot], ulps(q, (double)copysignf(fminf(fabsf(y), ax), y) / (double)ax));
    }
}

__global__ void acos_kernel(unsigned long long *m, long long n)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = (float)(-1.0 + 2.0 * (double)i / (double)(n - 1));
        const double ref = acos((double)x) / M_PI;
        const float own = acospi(x);
        keep_max(&m[kAcosOwn], ulps(own, ref));
        keep_max(&m[kAcosLib], ulps(__fmul_rn(acosf(x), 0.318309886183790671538f), ref));
        keep_max(&m[kAcosAbs], fabs((double)own - ref) * 1e6);
    }
}

__global__ void sincos_kernel(unsigned long long *m, long long n)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = (float)(-16.0 + 32.0 * (double)i / (double)(n - 1));
        const double rs = sin(M_PI * (double)x), rc = cos(M_PI * (double)x);
        float s1, c1, s2, c2;
        sincospi_own(x, &s1, &c1);
        sincospif(x, &s2, &c2);
        keep_max(&m[kSinAbsOwn], fabs(s1 - rs) * 1e6);
        keep_max(&m[kCosAbsOwn], fabs(c1 - rc) * 1e6);
        keep_max(&m[kSinAbsLib], fabs(s2 - rs) * 1e6);
        keep_max(&m[kCosAbsLib], fabs(c2 - rc) * 1e6);
    }
}

__global__ void sqrt_log_kernel(unsigned long long *m, long long n)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        uint64_t s = 0x2545f4914f6cdd1dULL ^ (uint64_t)i;
        // log-uniform over [2^-126, 2^20] and uniform over [1/2, 2] in turn
        const float x = (i & 1) ? 0.5f + 1.5f * lcg_unit(s)
                                : exp2f(-126.0f + 146.0f * lcg_unit(s));
        keep_max(&m[kSqrtOwn], ulps(sqrt_own(x), sqrt((double)x)));
        float inv;
        const float r2 = sqrt_rsqrt_own(x, inv);
        keep_max(&m[kRsqrtOwn], ulps(inv, 1.0 / sqrt((double)x)));
        if (r2 != sqrt_own(x)) keep_max(&m[kRsqrtOwn], 1e9);  // the same bits as sqrt_own
        const double rl = log((double)x);
        keep_max(&m[kLogOwn], ulps(log_own(x), rl));
        keep_max(&m[kLogLib], ulps(logf(x), rl));
    }
}

// special points, one thread
__global__ void special_kernel(float *o)
{
    const float z = 0.0f;
    o[0] = atan2pi(z, z);
    o[1] = atan2pi(-z, z);
    o[2] = atan2pi(z, -z);
    o[3] = atan2pi(-z, -z);
    o[4] = atan2pi(1.0f, 0.0f);
    o[5] = atan2pi(0.0f, -1.0f);
    o[6] = atan2pi(1.0f, 1.0f);
    o[7] = acospi(1.0f);
    o[8] = acospi(-1.0f);
    o[9] = acospi(0.0f);
    float s, c;
    sincospi_own(8.0f, &s, &c);
    o[10] = s;
    o[11] = c;
    sincospi_own(-1.5f, &s, &c);
    o[12] = s;
    o[13] = c;
    o[14] = sqrt_own(0.0f);
    o[15] = sqrt_own(4.0f);
    o[16] = sqrt_own(1e-40f);
    o[17] = log_own(1.0f);
    o[18] = log_own(0.0f);
    o[19] = log_own(2.0f);
}

int main()
{
    unsigned long long *m = nullptr;
    float *sp = nullptr;
    if (cudaMalloc(&m, kSlots * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc(&sp, 20 * sizeof(float)) != cudaSuccess) {
        fprintf(stderr, "cudaMalloc failed\n");
        return 1;
    }
    cudaMemset(m, 0, kSlots * sizeof(unsigned long long));
    atan2_kernel<<<152 * 8, 256>>>(m, 1LL << 27);
    acos_kernel<<<152 * 8, 256>>>(m, 1LL << 26);
    sincos_kernel<<<152 * 8, 256>>>(m, 1LL << 26);
    sqrt_log_kernel<<<152 * 8, 256>>>(m, 1LL << 26);
    special_kernel<<<1, 1>>>(sp);
    unsigned long long h[kSlots];
    float hs[20];
    cudaMemcpy(h, m, sizeof h, cudaMemcpyDeviceToHost);
    cudaMemcpy(hs, sp, sizeof hs, cudaMemcpyDeviceToHost);
    const cudaError_t err = cudaDeviceSynchronize();
    if (err != cudaSuccess) {
        fprintf(stderr, "CUDA error %s\n", cudaGetErrorString(err));
        return 1;
    }
    const char *names[kSlots] = {"atan2pi_ulp", "atan2f_ulp", "atan2pi_abs_e6", "acospi_ulp", "acosf_ulp",
                                 "acospi_abs_e6", "sinpi_abs_e6", "cospi_abs_e6", "sincospif_sin_abs_e6",
                                 "sincospif_cos_abs_e6", "quot_ulp", "sqrt_own_ulp", "log_own_ulp",
                                 "logf_ulp", "rsqrt_own_ulp"};
    for (int k = 0; k < kSlots; k++) printf("%s=%.6g ", names[k], (double)h[k] / 1e9);
    printf("special=");
    for (int k = 0; k < 20; k++) printf("%s%.9g", k ? "," : "", hs[k]);
    printf("\n");
    return 0;
}
