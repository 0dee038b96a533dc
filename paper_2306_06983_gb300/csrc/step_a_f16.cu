// Instantiations of the fused step kernel: Model A, binary16 population deviations, N = 2..8.
#include "step_kernel.cuh"

namespace nlbm {

cudaError_t launch_step_a_f16(int ns, const StepParams &p, int tx, int ty, cudaStream_t st)
{
    return launch_step_model<0, 2>(ns, p, tx, ty, st);
}

}  // namespace nlbm
