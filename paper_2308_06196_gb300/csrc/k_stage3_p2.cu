// k_stage3_p2.cu -- hexahedral stage kernels of degree p = 2 (all octant variants).
#include "k_stage3.cuh"

namespace bgk {
cudaError_t prepare_stage3_p2() { return prepare3<3>(); }
cudaError_t launch_stage3_p2(const StageArgs &A, int mode, int oct, cudaStream_t s)
{
    return launch3_any<3>(A, mode, oct, s);
}
}  // namespace bgk
