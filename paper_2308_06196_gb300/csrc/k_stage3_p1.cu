// k_stage3_p1.cu -- hexahedral stage kernels of degree p = 1 (all octant variants).
#include "k_stage3.cuh"

namespace bgk {
cudaError_t prepare_stage3_p1() { return prepare3<2>(); }
cudaError_t launch_stage3_p1(const StageArgs &A, int mode, int oct, cudaStream_t s)
{
    return launch3_any<2>(A, mode, oct, s);
}
}  // namespace bgk
