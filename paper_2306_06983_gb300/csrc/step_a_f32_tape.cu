// Instantiations of the fused step kernel that also writes the adjoint's
// tape: Model A, FP32 populations, 128-thread blocks, N = 2..8.
#include "step_kernel.cuh"

namespace nlbm {

cudaError_t launch_step_tape_a_f32(int ns, const StepParams &p, cudaStream_t st)
{
    if (!p.tape) return cudaErrorInvalidValue;
    switch (ns) {
#define NLBM_CASE(K) \
    case K: return launch_step_nst<K, 0, 128, 0, true>(p, 0, st);
        NLBM_CASE(1) NLBM_CASE(2) NLBM_CASE(3) NLBM_CASE(4) NLBM_CASE(5) NLBM_CASE(6) NLBM_CASE(7)
#undef NLBM_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace nlbm
