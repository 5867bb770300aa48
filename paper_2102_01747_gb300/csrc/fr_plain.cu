// fr_plain.cu -- launches of the one-ray-per-thread kernels of fr_plain.cuh
// (single requests that ask for the Mandelbulb's analytic normal go to
// fr_plain_an.cu).
#include "fr_plain.cuh"

namespace fr {

// phong: some request of the launch uses Phong shading (the Phong-capable code
// then serves every request of the launch, at unroll 1)
cudaError_t launch_batch_plain(const BatchArgs &A, long long ctas, int block, int unroll, bool count,
                               bool phong, cudaStream_t s)
{
    for (int i = 0; i < A.n_reqs; i++)
        if (A.reqs[i].spl > 1) return launch_batch_plain_lanes(A, ctas, block, count, phong, s);
    if (phong) return count ? launch_batch_plain_t<1, true, true>(A, ctas, block, s)
                            : launch_batch_plain_t<1, false, true>(A, ctas, block, s);
    if (count) return launch_batch_plain_t<1, true, false>(A, ctas, block, s);
    if (unroll == 2) return launch_batch_plain_t<2, false, false>(A, ctas, block, s);
    return launch_batch_plain_t<1, false, false>(A, ctas, block, s);
}

cudaError_t launch_batch_refill(const BatchArgs &A, int block, int unroll, bool count, bool phong, cudaStream_t s)
{
    for (int i = 0; i < A.n_reqs; i++)
        if (A.reqs[i].spl > 1) return launch_batch_refill_lanes(A, block, count, phong, s);
    if (phong) return count ? launch_batch_refill_t<1, true, true>(A, block, s)
                            : launch_batch_refill_t<1, false, true>(A, block, s);
    if (count) return launch_batch_refill_t<1, true, false>(A, block, s);
    if (unroll == 2) return launch_batch_refill_t<2, false, false>(A, block, s);
    return launch_batch_refill_t<1, false, false>(A, block, s);
}

// Phong requests run the Phong-capable instantiation at unroll 1; Mandelbulb
// requests of the paper's power 8 (not counting) an instantiation for that
// power
cudaError_t launch_plain(const DevReq &R, int block, int unroll, bool count, cudaStream_t s)
{
    if (R.spl > 1) return launch_plain_lanes(R, block, count, s);
    if (R.kind == 1 && R.normal_mode == 2) return launch_plain_ban(R, block, count, s);
    if (R.shading) {
        if (R.kind == 0)
            return count ? launch_plain_t<0, 1, true, true>(R, block, s) : launch_plain_t<0, 1, false, true>(R, block, s);
        if (count) return launch_plain_t<1, 1, true, true>(R, block, s);
        return R.power == 8 ? launch_plain_t<2, 1, false, true>(R, block, s) : launch_plain_t<1, 1, false, true>(R, block, s);
    }
    if (count) return R.kind == 0 ? launch_plain_t<0, 1, true>(R, block, s)
                                  : launch_plain_t<1, 1, true>(R, block, s);
    if (R.kind == 0) {
        if (unroll == 4) return launch_plain_t<0, 4, false>(R, block, s);
        if (unroll == 2) return launch_plain_t<0, 2, false>(R, block, s);
        return launch_plain_t<0, 1, false>(R, block, s);
    }
    if (R.power == 8) {
        if (unroll == 4) return launch_plain_t<2, 4, false>(R, block, s);
        if (unroll == 2) return launch_plain_t<2, 2, false>(R, block, s);
        return launch_plain_t<2, 1, false>(R, block, s);
    }
    if (unroll == 4) return launch_plain_t<1, 4, false>(R, block, s);
    if (unroll == 2) return launch_plain_t<1, 2, false>(R, block, s);
    return launch_plain_t<1, 1, false>(R, block, s);
}

}  // namespace fr
