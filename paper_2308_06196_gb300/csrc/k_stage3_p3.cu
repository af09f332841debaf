// k_stage3_p3.cu -- hexahedral stage kernels of degree p = 3 (all octant variants).
#include "k_stage3.cuh"

namespace bgk {
cudaError_t prepare_stage3_p3() { return prepare3<4>(); }
cudaError_t launch_stage3_p3(const StageArgs &A, int mode, int oct, cudaStream_t s)
{
    return launch3_any<4>(A, mode, oct, s);
}
}  // namespace bgk
