// fr_lanes.cu -- launches of the lane state machine of fr_persist.cuh without
// the queue: one pixel per lane, every tile launched (fr_tuning.single_kernel = 1).
#include "fr_persist.cuh"

namespace fr {

cudaError_t launch_lanes(const BatchArgs &A, int block, int unroll, bool count, bool phong, cudaStream_t s)
{
    if (phong) return count ? launch_persist_t<4, true, false, true>(A, block, 0, s)
                            : launch_persist_t<4, false, false, true>(A, block, 0, s);
    if (count) return launch_persist_t<4, true, false>(A, block, 0, s);
    if (unroll == 8) return launch_persist_t<8, false, false>(A, block, 0, s);
    if (unroll == 2) return launch_persist_t<2, false, false>(A, block, 0, s);
    return launch_persist_t<4, false, false>(A, block, 0, s);
}

}  // namespace fr
