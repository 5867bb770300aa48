// fr_plain_an.cu -- the single-request kernel of fr_plain.cuh compiled with the
// Mandelbulb's analytic normal, for requests that ask for it (a translation
// unit of its own so that it compiles in parallel with the rest); requests of
// the power 8 take the instantiation compiled for that power.
#include "fr_plain.cuh"

namespace fr {

cudaError_t launch_plain_ban(const DevReq &R, int block, bool count, cudaStream_t s)
{
    if (R.shading) {
        if (count) return launch_plain_t<1, 1, true, true, true>(R, block, s);
        return R.power == 8 ? launch_plain_t<2, 1, false, true, true>(R, block, s)
                            : launch_plain_t<1, 1, false, true, true>(R, block, s);
    }
    if (count) return launch_plain_t<1, 1, true, false, true>(R, block, s);
    return R.power == 8 ? launch_plain_t<2, 1, false, false, true>(R, block, s)
                        : launch_plain_t<1, 1, false, false, true>(R, block, s);
}

}  // namespace fr
