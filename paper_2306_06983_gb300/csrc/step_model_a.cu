// Instantiations of the fused step kernel for Model A (N = 2..8).
#include "step_kernel.cuh"

namespace nlbm {

cudaError_t launch_step_model_a(int ns, const StepParams &p, int tx, int ty, cudaStream_t st)
{
    return launch_step_model<0>(ns, p, tx, ty, st);
}

}  // namespace nlbm
