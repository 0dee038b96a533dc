// Instantiations of the fused step kernel for Model B (N = 2..8).
#include "step_kernel.cuh"

namespace nlbm {

cudaError_t launch_step_model_b(int ns, const StepParams &p, int tx, int ty, cudaStream_t st)
{
    return launch_step_model<1>(ns, p, tx, ty, st);
}

}  // namespace nlbm
