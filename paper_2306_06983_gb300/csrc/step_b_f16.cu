// Instantiations of the fused step kernel: Model B, binary16 population deviations, N = 2..8.
#include "step_kernel.cuh"

namespace nlbm {

cudaError_t launch_step_b_f16(int ns, const StepParams &p, int tx, int ty, cudaStream_t st)
{
    return launch_step_model<1, 2>(ns, p, tx, ty, st);
}

}  // namespace nlbm
