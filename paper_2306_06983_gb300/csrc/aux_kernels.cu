// Initial state, moment export and the FP64 per-phase volume reduction.
#include "nlbm_internal.cuh"

namespace nlbm {

namespace {

__constant__ int kCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int kCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

// Initial state of a fluid at rest (u = 0, P = 0): the populations that the
// first pull must see are the equilibria f_i = w_i phi_p (Eq. (19)) and
// g_i = lambda_i(P = 0) = 0 (Eq. (22)).  With pull streaming the stored
// post-collision value f*_i(x) is read by node z = x + c_i, or by x itself
// when that link crosses a bounce-back wall, so f*_i(x) = w_i phi(z).  The
// rest population is phi - 5 phi/9 formed with error-free subtractions, so
// the nine values a node receives sum to its phi up to one rounding.
__device__ __forceinline__ float init_two_sum(float a, float b, float &e)
{
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

template <int NS>
__global__ void init_kernel(const StepParams P, float *u_other)
{
    const unsigned pl = P.plane;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < pl; k += gridDim.x * blockDim.x) {
        const int x = k % P.nx, y = k / P.nx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int tx = x + kCx[i], ty = y + kCy[i];
            const bool out_x = tx < 0 || tx >= P.nx, out_y = ty < 0 || ty >= P.ny;
            unsigned src;
            if ((out_x && P.wall_x) || (out_y && P.wall_y)) {
                src = k;
            } else {
                if (tx < 0) tx += P.nx;
                if (tx >= P.nx) tx -= P.nx;
                if (ty < 0) ty += P.ny;
                if (ty >= P.ny) ty -= P.ny;
                src = (unsigned)ty * P.nx + tx;
            }
#pragma unroll
            for (int p = 0; p < NS; ++p) {
                const float phi = P.phi[(size_t)p * pl + src];
                const float p9 = phi * (1.f / 9.f);
                float v;
                if (i == 0) {
                    float e1, e2;
                    const float a1 = init_two_sum(phi, -4.f * p9, e1);
                    const float a2 = init_two_sum(a1, -p9, e2);
                    v = a2 + (e1 + e2);
                } else {
                    v = i < 5 ? p9 : 0.25f * p9;
                }
                P.fout[((size_t)p * 9 + i) * pl + k] = v;
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) P.gout[(size_t)i * pl + k] = 0.f;
        P.uout[k] = 0.f;
        P.uout[pl + k] = 0.f;
        u_other[k] = 0.f;
        u_other[pl + k] = 0.f;
        P.mphi[k] = 0.f;
        P.mphi[pl + k] = 0.f;
        P.pout[k] = 0.f;
    }
}

// Initial state with 16-bit storage.  The first pull must see the
// equilibria f_i = w_i phi (Eq. (19)) and g_i = 0: the stored moving
// deviations are 0 (the puller adds w_i phi of itself, and 3 w_i P with
// P = 0), and the FP32 rest population of node z is phi(z) minus the eight
// values z reconstructs, summed with the compensation the step kernel uses.
__device__ __forceinline__ float init_w(int i) { return i == 0 ? 4.f / 9.f : (i < 5 ? 1.f / 9.f : 1.f / 36.f); }

template <int NS>
__global__ void init16_kernel(const StepParams P, float *u_other, float *p_other)
{
    const unsigned pl = P.plane;
    unsigned short *f16 = (unsigned short *)P.fout;
    unsigned short *g16 = (unsigned short *)P.gout;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < pl; k += gridDim.x * blockDim.x) {
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            const float phi = P.phi[(size_t)p * pl + k];
            float r[9];
#pragma unroll
            for (int i = 1; i < 9; ++i) r[i] = __fmaf_rn(init_w(i), phi, 0.f);
            float e13, e24, e57, e68, ea, eb, es, e0;
            const float s13 = init_two_sum(r[1], r[3], e13), s24 = init_two_sum(r[2], r[4], e24);
            const float s57 = init_two_sum(r[5], r[7], e57), s68 = init_two_sum(r[6], r[8], e68);
            const float sa = init_two_sum(s13, s24, ea), sb = init_two_sum(s57, s68, eb);
            const float S = init_two_sum(sa, sb, es);
            const float E = ((e13 + e24) + (e57 + e68)) + ((ea + eb) + es);
            const float a0 = init_two_sum(phi, -S, e0);
            P.f0out[(size_t)p * pl + k] = a0 + (e0 - E);
#pragma unroll
            for (int i = 0; i < 8; ++i) f16[((size_t)p * 8 + i) * pl + k] = 0;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) g16[(size_t)i * pl + k] = 0;
        P.uout[k] = 0.f;
        P.uout[pl + k] = 0.f;
        u_other[k] = 0.f;
        u_other[pl + k] = 0.f;
        P.mphi[k] = 0.f;
        P.mphi[pl + k] = 0.f;
        P.pout[k] = 0.f;
        p_other[k] = 0.f;
    }
}

template <int NS>
__global__ void export_kernel(const float *__restrict__ phi_aux, const float *__restrict__ u,
                              const float *__restrict__ Pf, unsigned pl, float *phi_out,
                              float *u_out, float *p_out)
{
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < pl; k += gridDim.x * blockDim.x) {
        if (phi_out) {
            float s = 0.f;
#pragma unroll
            for (int p = 0; p < NS; ++p) {
                const float v = phi_aux[(size_t)p * pl + k];
                phi_out[(size_t)p * pl + k] = v;
                s += v;
            }
            phi_out[(size_t)NS * pl + k] = 1.f - s;   // Sec. 4: phi_N = 1 - sum
        }
        if (u_out) {
            u_out[k] = u[k];
            u_out[pl + k] = u[pl + k];
        }
        if (p_out) p_out[k] = Pf[k];
    }
}

constexpr int kMassThreads = 256;

// Per-block FP64 partial volumes of all N phases plus a divergence flag
// (non-finite or outside [-0.5, 1.5]); fixed grid and block size, so the
// summation order -- and the result -- are reproducible bit for bit.
template <int NS>
__global__ void __launch_bounds__(kMassThreads) mass_partial_kernel(const float *__restrict__ phi,
                                                                    unsigned pl, double *partials)
{
    constexpr int N = NS + 1;
    double acc[N];
#pragma unroll
    for (int p = 0; p < N; ++p) acc[p] = 0.0;
    double bad = 0.0;
    for (unsigned k = blockIdx.x * kMassThreads + threadIdx.x; k < pl; k += gridDim.x * kMassThreads) {
        double s = 0.0;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            const float v = phi[(size_t)p * pl + k];
            acc[p] += (double)v;
            s += (double)v;
            if (!(v >= -0.5f && v <= 1.5f)) bad = 1.0;   // also catches NaN
        }
        const double vN = 1.0 - s;
        acc[NS] += vN;
        if (!(vN >= -0.5 && vN <= 1.5)) bad = 1.0;
    }
    __shared__ double red[kMassThreads / 32][N + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int p = 0; p <= N; ++p) {
        double v = p < N ? acc[p] : bad;
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_down_sync(0xffffffffu, v, o);
            v = p < N ? v + w : fmax(v, w);
        }
        if (lane == 0) red[warp][p] = v;
    }
    __syncthreads();
    if (threadIdx.x <= N) {
        const int p = threadIdx.x;
        double v = red[0][p];
        for (int w = 1; w < kMassThreads / 32; ++w) v = p < N ? v + red[w][p] : fmax(v, red[w][p]);
        partials[(size_t)blockIdx.x * (N + 1) + p] = v;
    }
}

// Sums the per-block partials in a fixed order: mass[p] for p < N,
// flag = 1 if any block saw a diverged value.
__global__ void mass_final_kernel(const double *__restrict__ partials, int nblocks, int N,
                                  double *mass, int *flag)
{
    __shared__ double red[kMassThreads];
    for (int p = 0; p <= N; ++p) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nblocks; b += kMassThreads) {
            const double w = partials[(size_t)b * (N + 1) + p];
            v = p < N ? v + w : fmax(v, w);
        }
        red[threadIdx.x] = v;
        __syncthreads();
        for (int s = kMassThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s)
                red[threadIdx.x] = p < N ? red[threadIdx.x] + red[threadIdx.x + s]
                                         : fmax(red[threadIdx.x], red[threadIdx.x + s]);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            if (p < N) mass[p] = red[0];
            else *flag = red[0] > 0.0 ? 1 : 0;
        }
        __syncthreads();
    }
}

int grid_for(unsigned pl, int threads)
{
    unsigned b = (pl + threads - 1) / threads;
    if (b > 65535u * 16u) b = 65535u * 16u;
    return (int)(b ? b : 1);
}

}  // namespace

cudaError_t launch_init(int ns, const StepParams &p, cudaStream_t st)
{
    // p.uin is the second velocity buffer (both are zeroed).
    const int threads = 256, blocks = grid_for(p.plane, threads);
    float *u_other = const_cast<float *>(p.uin);
    if (p.f0out) {   // 16-bit storage; p.pin is the second pressure buffer
        float *p_other = const_cast<float *>(p.pin);
        switch (ns) {
#define NLBM_CASE(K) \
    case K: init16_kernel<K><<<blocks, threads, 0, st>>>(p, u_other, p_other); break;
            NLBM_CASE(1) NLBM_CASE(2) NLBM_CASE(3) NLBM_CASE(4) NLBM_CASE(5) NLBM_CASE(6) NLBM_CASE(7)
#undef NLBM_CASE
        default: return cudaErrorInvalidValue;
        }
        return cudaGetLastError();
    }
    switch (ns) {
#define NLBM_CASE(K) \
    case K: init_kernel<K><<<blocks, threads, 0, st>>>(p, u_other); break;
        NLBM_CASE(1) NLBM_CASE(2) NLBM_CASE(3) NLBM_CASE(4) NLBM_CASE(5) NLBM_CASE(6) NLBM_CASE(7)
#undef NLBM_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_export(int ns, const float *phi_aux, const float *u, const float *Pf,
                          unsigned plane, float *phi_out, float *u_out, float *p_out,
                          cudaStream_t st)
{
    const int threads = 256, blocks = grid_for(plane, threads);
    switch (ns) {
#define NLBM_CASE(K)                                                                          \
    case K:                                                                                   \
        export_kernel<K><<<blocks, threads, 0, st>>>(phi_aux, u, Pf, plane, phi_out, u_out,   \
                                                     p_out);                                  \
        break;
        NLBM_CASE(1) NLBM_CASE(2) NLBM_CASE(3) NLBM_CASE(4) NLBM_CASE(5) NLBM_CASE(6) NLBM_CASE(7)
#undef NLBM_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_phase_mass(int ns, const float *phi_aux, unsigned plane, double *partials,
                              double *mass_out, int *flag_out, cudaStream_t st)
{
    switch (ns) {
#define NLBM_CASE(K)                                                                         \
    case K:                                                                                  \
        mass_partial_kernel<K><<<kMassBlocks, kMassThreads, 0, st>>>(phi_aux, plane, partials); \
        break;
        NLBM_CASE(1) NLBM_CASE(2) NLBM_CASE(3) NLBM_CASE(4) NLBM_CASE(5) NLBM_CASE(6) NLBM_CASE(7)
#undef NLBM_CASE
    default: return cudaErrorInvalidValue;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    mass_final_kernel<<<1, kMassThreads, 0, st>>>(partials, kMassBlocks, ns + 1, mass_out, flag_out);
    return cudaGetLastError();
}

}  // namespace nlbm
