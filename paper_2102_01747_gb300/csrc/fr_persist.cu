// fr_persist.cu -- launches of the queue-fed persistent kernel of fr_persist.cuh
// (fr_tuning.batch_kernel = 0).
#include "fr_persist.cuh"

namespace fr {

// phong: some request of the launch uses Phong shading (the Phong-capable
// instantiation then serves every request of the launch, at unroll 4)
cudaError_t launch_persist(const BatchArgs &A, int block, int ctas_per_sm, int unroll, bool count, bool phong,
                           cudaStream_t s)
{
    if (phong) return count ? launch_persist_t<4, true, true, true>(A, block, ctas_per_sm, s)
                            : launch_persist_t<4, false, true, true>(A, block, ctas_per_sm, s);
    if (count) return launch_persist_t<4, true, true>(A, block, ctas_per_sm, s);
    if (unroll == 8) return launch_persist_t<8, false, true>(A, block, ctas_per_sm, s);
    if (unroll == 4) return launch_persist_t<4, false, true>(A, block, ctas_per_sm, s);
    if (unroll == 2) return launch_persist_t<2, false, true>(A, block, ctas_per_sm, s);
    return launch_persist_t<1, false, true>(A, block, ctas_per_sm, s);
}

}  // namespace fr
