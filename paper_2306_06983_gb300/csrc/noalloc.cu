// Per-phase volume reduction whose scratch lives in a fixed, library-owned
// device array instead of caller memory, for callers that cannot hand the
// library any extra device allocation (see nlbm_phase_mass_noalloc in
// include/nlbm.h).
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "../../include/nlbm.h"
#include "nlbm_internal.cuh"

namespace {

// FP64 partial sums of the two-kernel reduction: kMassBlocks blocks times
// (N + 1) values (N volumes and a divergence flag), for N up to kMaxPhases.
// Every GPU that loads the library keeps this array (36.9 KB) until the
// process exits.  The reduction overwrites every entry it later reads, so
// nothing needs to be cleared between calls.
constexpr int kScratchDoubles = nlbm::kMassBlocks * (nlbm::kMaxPhases + 1);
static __device__ __align__(256) double g_mass_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {nullptr};
void *g_scratch_ctx[kMaxDevices] = {nullptr};   // context the address was looked up in

// The current context of the calling thread (the driver's cuCtxGetCurrent,
// reached through the runtime so that the library needs no link against
// libcuda); nullptr if it cannot be obtained.
void *current_context()
{
    typedef int (*get_ctx_fn)(void **);
    static get_ctx_fn fn = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<get_ctx_fn>(p);
        looked_up = true;
    }
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0) ctx = nullptr;
    return ctx;
}

// Rejections are reported by status code and one line on stderr (this entry
// point has no handle to carry an error text).
void set_err(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    fputs("nlbm_phase_mass_noalloc: ", stderr);
    vfprintf(stderr, fmt, ap);
    fputc('\n', stderr);
    va_end(ap);
}

// Device address of the scratch array on the current device.  The host-side
// name g_mass_scratch is only a stand-in; the address a kernel may use comes
// from cudaGetSymbolAddress, looked up once per device with that device
// current, and again whenever the calling thread's current context differs
// from the one the address was taken in (a caller's own driver context, or
// the primary context re-created after cudaDeviceReset).
nlbm_status scratch_for_current_device(double **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_err("cudaGetDevice: %s", cudaGetErrorString(e));
        return NLBM_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_err("device ordinal %d outside 0..%d", dev, kMaxDevices - 1);
        return NLBM_EINVAL;
    }
    // (cudaGetDevice has made the device's primary context current if the
    // thread had none, so the context read here is the one the kernels use)
    void *ctx = current_context();
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_mass_scratch);
        if (e != cudaSuccess || !p) {
            set_err("cudaGetSymbolAddress of the reduction scratch: %s", cudaGetErrorString(e));
            return NLBM_ECUDA;
        }
        g_scratch_ptr[dev] = static_cast<double *>(p);
        g_scratch_ctx[dev] = ctx;
    }
    *out = g_scratch_ptr[dev];
    return NLBM_OK;
}

}  // namespace

extern "C" nlbm_status nlbm_phase_mass_noalloc(const float *dev_phi, int32_t n_phases,
                                               int64_t n_nodes, double *dev_mass,
                                               int32_t *dev_flag, void *cuda_stream)
{
    if (!dev_phi || !dev_mass || !dev_flag) {
        set_err("dev_phi, dev_mass and dev_flag must be device pointers, not NULL");
        return NLBM_EINVAL;
    }
    if (n_phases < 2 || n_phases > nlbm::kMaxPhases) {
        set_err("n_phases=%d outside 2..%d (the static scratch holds %d doubles)", n_phases,
                nlbm::kMaxPhases, kScratchDoubles);
        return NLBM_EINVAL;
    }
    if (n_nodes < 1 || n_nodes > ((int64_t)1 << 28)) {
        set_err("n_nodes=%lld outside 1..%lld", (long long)n_nodes, (long long)1 << 28);
        return NLBM_EINVAL;
    }
    double *scratch = nullptr;
    nlbm_status st = scratch_for_current_device(&scratch);
    if (st != NLBM_OK) return st;
    cudaError_t e = nlbm::launch_phase_mass(n_phases - 1, dev_phi, (unsigned)n_nodes, scratch,
                                            dev_mass, reinterpret_cast<int *>(dev_flag),
                                            static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) {
        set_err("phase-mass kernels: %s", cudaGetErrorString(e));
        return NLBM_ECUDA;
    }
    return NLBM_OK;
}
