// Ensemble of independent simulations in one persistent launch per step.
//
// Every simulation keeps its own state and parameter block (StepParams, in
// device memory); the host builds a table of tiles -- (simulation, strip,
// row chunk) -- over all of them, largest simulations first.  A grid of
// exactly the resident blocks of the device takes tiles in table order from
// a global counter and runs the same fused step (step_tile) on each, with the
// tile's parameter block copied into shared memory.  Model A and Model B
// simulations share the launch (the model is read per tile), and so do
// simulations whose pulls are staged as row windows and those that are not.
// Simulations never exchange data, so no block waits on another; the only
// cross-block traffic is the tile counter.
#include <atomic>

#include "step_kernel.cuh"

namespace nlbm {

template <int NS, int T>
__global__ void __launch_bounds__(T) batch_step_kernel(const StepParams *__restrict__ params,
                                                        const BatchTile *__restrict__ tiles, int ntiles,
                                                        int *counters, int parity)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ StepParams s_P;
    __shared__ int s_k;
    // the other counter is the next launch's; this launch's was cleared by
    // the previous one (or at creation)
    pdl_wait();
    if (blockIdx.x == 0 && threadIdx.x == 0) counters[parity ^ 1] = 0;
    for (;;) {
        if (threadIdx.x == 0) s_k = atomicAdd(&counters[parity], 1);
        __syncthreads();
        const int k = s_k;
        if (k >= ntiles) break;
        const BatchTile tl = tiles[k];
        const int *src = reinterpret_cast<const int *>(params + tl.sim);
        int *dst = reinterpret_cast<int *>(&s_P);
        for (int i = threadIdx.x; i < (int)(sizeof(StepParams) / sizeof(int)); i += T) dst[i] = src[i];
        __syncthreads();
        if (s_P.row_window) {
            if (s_P.model == 0)
                step_tile<NS, 0, T, 0, true>(s_P, tl.x0, tl.y0, tl.ty, smem);
            else
                step_tile<NS, 1, T, 0, true>(s_P, tl.x0, tl.y0, tl.ty, smem);
        } else {
            if (s_P.model == 0)
                step_tile<NS, 0, T, 0, false>(s_P, tl.x0, tl.y0, tl.ty, smem);
            else
                step_tile<NS, 1, T, 0, false>(s_P, tl.x0, tl.y0, tl.ty, smem);
        }
        __syncthreads();   // s_k, s_P and the rings are reused by the next tile
    }
}

namespace {

template <int NS, int T>
cudaError_t configure(int *blocks)
{
    static_assert(sizeof(StepParams) % sizeof(int) == 0, "parameter block copied as ints");
    const size_t smem = step_smem_bytes<NS, T, 0, true>();
    // resident blocks per device, 0 until configured (threads that race here
    // compute and store the same value)
    static std::atomic<int> resident[64];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    int r = resident[dev].load(std::memory_order_acquire);
    if (!r) {
        e = cudaFuncSetAttribute(batch_step_kernel<NS, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_step_kernel<NS, T>, T, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        r = per_sm * sms > 0 ? per_sm * sms : 1;
        resident[dev].store(r, std::memory_order_release);
    }
    *blocks = r;
    return cudaSuccess;
}

template <int NS, int T>
cudaError_t launch_nt(const StepParams *d_params, const BatchTile *d_tiles, int ntiles, int *d_counters,
                      int parity, cudaStream_t st)
{
    int blocks = 0;
    cudaError_t e = configure<NS, T>(&blocks);
    if (e != cudaSuccess) return e;
    const int grid = ntiles < blocks ? (ntiles > 0 ? ntiles : 1) : blocks;
    return launch_pdl(batch_step_kernel<NS, T>, dim3(grid), dim3(T), step_smem_bytes<NS, T, 0, true>(), st, d_params,
                      d_tiles, ntiles, d_counters, parity);
}

template <int NS>
cudaError_t launch_n(int tx, const StepParams *d_params, const BatchTile *d_tiles, int ntiles, int *d_counters,
                     int parity, cudaStream_t st)
{
    switch (tx) {
    case 64: return launch_nt<NS, 64>(d_params, d_tiles, ntiles, d_counters, parity, st);
    case 128: return launch_nt<NS, 128>(d_params, d_tiles, ntiles, d_counters, parity, st);
    case 256: return launch_nt<NS, 256>(d_params, d_tiles, ntiles, d_counters, parity, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace

cudaError_t launch_batch_step(int ns, int tx, const StepParams *d_params, const BatchTile *d_tiles,
                              int ntiles, int *d_counters, int parity, cudaStream_t st)
{
    switch (ns) {
#define NLBM_CASE(K) \
    case K: return launch_n<K>(tx, d_params, d_tiles, ntiles, d_counters, parity, st);
        NLBM_CASE(1) NLBM_CASE(2) NLBM_CASE(3) NLBM_CASE(4) NLBM_CASE(5) NLBM_CASE(6) NLBM_CASE(7)
#undef NLBM_CASE
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace nlbm
