// fr_plain_lanes.cu -- the one-ray-per-thread kernels of fr_plain.cuh with a
// pixel's 2, 4 or 8 samples on adjacent lanes (LANES, render_pixel_lanes), for
// requests with R.spl > 1 (a translation unit of its own so that it compiles
// in parallel with the rest).  Unroll depth 1; Phong requests take the
// Phong-capable instantiation, the Mandelbulb's analytic normal the BAN one,
// and Lambert Mandelbulb requests of the power 8 one compiled for that power.
#include "fr_plain.cuh"

namespace fr {

cudaError_t launch_plain_lanes(const DevReq &R, int block, bool count, cudaStream_t s)
{
    if (R.kind == 0) {
        if (R.shading)
            return count ? launch_plain_t<0, 1, true, true, false, true>(R, block, s)
                         : launch_plain_t<0, 1, false, true, false, true>(R, block, s);
        return count ? launch_plain_t<0, 1, true, false, false, true>(R, block, s)
                     : launch_plain_t<0, 1, false, false, false, true>(R, block, s);
    }
    if (R.normal_mode == 2) {
        if (R.shading)
            return count ? launch_plain_t<1, 1, true, true, true, true>(R, block, s)
                         : launch_plain_t<1, 1, false, true, true, true>(R, block, s);
        return count ? launch_plain_t<1, 1, true, false, true, true>(R, block, s)
                     : launch_plain_t<1, 1, false, false, true, true>(R, block, s);
    }
    if (R.shading)
        return count ? launch_plain_t<1, 1, true, true, false, true>(R, block, s)
                     : launch_plain_t<1, 1, false, true, false, true>(R, block, s);
    if (count) return launch_plain_t<1, 1, true, false, false, true>(R, block, s);
    return R.power == 8 ? launch_plain_t<2, 1, false, false, false, true>(R, block, s)
                        : launch_plain_t<1, 1, false, false, false, true>(R, block, s);
}

cudaError_t launch_batch_plain_lanes(const BatchArgs &A, long long ctas, int block, bool count, bool phong,
                                     cudaStream_t s)
{
    if (phong) return count ? launch_batch_plain_t<1, true, true, true>(A, ctas, block, s)
                            : launch_batch_plain_t<1, false, true, true>(A, ctas, block, s);
    return count ? launch_batch_plain_t<1, true, false, true>(A, ctas, block, s)
                 : launch_batch_plain_t<1, false, false, true>(A, ctas, block, s);
}

cudaError_t launch_batch_refill_lanes(const BatchArgs &A, int block, bool count, bool phong, cudaStream_t s)
{
    if (phong) return count ? launch_batch_refill_t<1, true, true, true>(A, block, s)
                            : launch_batch_refill_t<1, false, true, true>(A, block, s);
    return count ? launch_batch_refill_t<1, true, false, true>(A, block, s)
                 : launch_batch_refill_t<1, false, false, true>(A, block, s);
}

}  // namespace fr
