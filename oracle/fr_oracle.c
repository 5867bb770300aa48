/*
 * fr_oracle.c -- CPU oracle, compiled twice from one body (double and float).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.
 */
#include <math.h>
#include <tgmath.h>
#include <stdint.h>
#include <pthread.h>
#include "fr_oracle.h"

/* splitmix64 (Steele, Lea and Flood, 2014; the public-domain reference
 * generator by Vigna): add the golden-ratio increment, then the
 * xor-shift-multiply finaliser. */
uint64_t orc_splitmix64(uint64_t state)
{
    uint64_t z = state + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Sub-pixel offset of one sample: the counter (seed << 40) + pixel*spp + sample
 * is hashed once; the top 24 bits give sx and the next 24 bits give sy, each
 * a multiple of 2^-24 in [0, 1), exact in float. */
void orc_jitter(uint32_t seed, int64_t pixel, int spp, int sample, double *sx, double *sy)
{
    uint64_t ctr = ((uint64_t)seed << 40) + (uint64_t)pixel * (uint64_t)spp + (uint64_t)sample;
    uint64_t h = orc_splitmix64(ctr);
    *sx = (double)(h >> 40) * (1.0 / 16777216.0);
    *sy = (double)((h >> 16) & 0xffffffULL) * (1.0 / 16777216.0);
}

/* 2D escape-time Julia set (Sec. 1.1): iterate z <- z^2 + c over the complex
 * numbers; return the number of trips until |z|^2 > escape_r2 (max_iter when
 * the orbit never leaves). */
int orc_julia2d_escape_d(double zr, double zi, double cr, double ci, int max_iter, double escape_r2)
{
    for (int i = 0; i < max_iter; i++) {
        double nr = zr * zr - zi * zi + cr;
        double ni = 2.0 * zr * zi + ci;
        zr = nr;
        zi = ni;
        if (zr * zr + zi * zi > escape_r2) return i + 1;
    }
    return max_iter;
}

#define CAT_(a, b) a##b
#define CAT(a, b) CAT_(a, b)

#define R double
#define F(name) CAT(name, _d)
#define K(x) ((double)(x))
#include "fr_oracle_body.inc"
#undef R
#undef F
#undef K

#include "fr_oracle_grad.inc"

#define R float
#define F(name) CAT(name, _f)
#define K(x) ((float)(x))
#include "fr_oracle_body.inc"
#undef R
#undef F
#undef K
