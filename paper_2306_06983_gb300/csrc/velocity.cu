// A state that starts in motion (nlbm_set_velocity): the populations of a
// fluid moving with a given velocity field u0 over the phase fields set by
// nlbm_set_phi, FP32 storage.
//
// Pass 1, per node z: grad phi_p (Eq. (27)), the source R_p (Eqs. (2)-(4))
// and m_phi (Eq. (13)) of the initial fields -- stored as the previous m_phi
// of the first step -- and the pressure P' = -c_s^2 u0 . grad rho /
// (2 (1 - w_0)) for which Eq. (25c) recovers P = 0 from the populations; u0
// becomes the previous velocity of the first step.
// Pass 2, per node x: the stored post-collision value f*_i(x) is what node
// z = x + c_i pulls (x itself across a bounce-back wall, as the opposite
// direction), so it is that node's equilibrium f^eq_i(phi(z), u0(z)) of
// Eq. (19) and g^eq_i(z) of Eq. (22) with P', rho(z) and m = rho u0 + m_phi;
// the rest population is phi minus the eight values the node pulls, summed
// with error-free transformations, so the nine sum to phi up to one rounding.
#include "nlbm_internal.cuh"
#include "step_kernel.cuh"

namespace nlbm {

namespace {

__constant__ int vCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int vCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
__constant__ int vOpp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

// Node of (x, y) on the lattice: periodic wrap, or the mirror image across
// a half-way bounce-back wall (phi mirrored, zero normal gradient).
__device__ __forceinline__ unsigned image_node(const StepParams &P, int x, int y)
{
    bool f;
    return (unsigned)map_axis(y, P.ny, P.wall_y, f) * P.nx + map_axis(x, P.nx, P.wall_x, f);
}

__device__ __forceinline__ float vel_two_sum(float a, float b, float &e)
{
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

template <int NS, int MODEL>
__global__ void velocity_prep_kernel(const StepParams P, const float *__restrict__ u0, float *u_prev,
                                     float *p_init)
{
    constexpr int N = NS + 1;
    const unsigned pl = P.plane;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < pl; k += gridDim.x * blockDim.x) {
        const int x = k % P.nx, y = k / P.nx;
        float ph[N], gx[N], gy[N];
        float sph = 0.f, sgx = 0.f, sgy = 0.f;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            const float *f = P.phi + (size_t)p * pl;
            float ax = 0.f, ay = 0.f;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const float v = f[image_node(P, x + vCx[i], y + vCy[i])];
                const float w = w_of(i);
                ax += 3.f * w * vCx[i] * v;
                ay += 3.f * w * vCy[i] * v;
            }
            ph[p] = f[k];
            gx[p] = ax;
            gy[p] = ay;
            sph += ph[p];
            sgx += ax;
            sgy += ay;
        }
        ph[NS] = 1.f - sph;
        gx[NS] = -sgx;
        gy[NS] = -sgy;
        float Rx[NS], Ry[NS], mx, my;
        source_terms<NS, MODEL>(P, ph, gx, gy, Rx, Ry);
        mass_flux<NS>(P, gx, gy, Rx, Ry, mx, my);
        P.mphi[k] = mx;
        P.mphi[pl + k] = my;
        float grx = 0.f, gry = 0.f;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            grx += P.drho[p] * gx[p];
            gry += P.drho[p] * gy[p];
        }
        const float ux = u0[k], uy = u0[pl + k];
        u_prev[k] = ux;
        u_prev[pl + k] = uy;
        // P' = -c_s^2 u.grad rho / (2 (1 - w_0)), c_s^2 = 1/3, w_0 = 4/9
        p_init[k] = -0.3f * (ux * grx + uy * gry);
    }
}

template <int NS>
__global__ void velocity_pop_kernel(const StepParams P, const float *__restrict__ u0,
                                    const float *__restrict__ p_init)
{
    const unsigned pl = P.plane;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < pl; k += gridDim.x * blockDim.x) {
        const int x = k % P.nx, y = k / P.nx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            // the node that pulls f*_i(x), and as which direction
            int tx = x + vCx[i], ty = y + vCy[i], di = i;
            const bool out_x = tx < 0 || tx >= P.nx, out_y = ty < 0 || ty >= P.ny;
            unsigned z;
            if ((out_x && P.wall_x) || (out_y && P.wall_y)) {
                z = k;
                di = vOpp[i];
            } else {
                tx = tx < 0 ? tx + P.nx : (tx >= P.nx ? tx - P.nx : tx);
                ty = ty < 0 ? ty + P.ny : (ty >= P.ny ? ty - P.ny : ty);
                z = (unsigned)ty * P.nx + tx;
            }
            const float ux = u0[z], uy = u0[pl + z];
            const float cu = 3.f * (vCx[di] * ux + vCy[di] * uy);   // c_i . u / c_s^2
            float rho = P.rhoN;
#pragma unroll
            for (int p = 0; p < NS; ++p) {
                const float phi = P.phi[(size_t)p * pl + z];
                rho += P.drho[p] * phi;
                float v;
                if (i == 0) {
                    // f*_0 = phi - sum of the eight equilibria node x pulls
                    float r[9];
#pragma unroll
                    for (int j = 1; j < 9; ++j)
                        r[j] = w_of(j) * phi * (1.f + 3.f * (vCx[j] * ux + vCy[j] * uy));
                    float e13, e24, e57, e68, ea, eb, es, e0;
                    const float s13 = vel_two_sum(r[1], r[3], e13), s24 = vel_two_sum(r[2], r[4], e24);
                    const float s57 = vel_two_sum(r[5], r[7], e57), s68 = vel_two_sum(r[6], r[8], e68);
                    const float sa = vel_two_sum(s13, s24, ea), sb = vel_two_sum(s57, s68, eb);
                    const float S = vel_two_sum(sa, sb, es);
                    const float E = ((e13 + e24) + (e57 + e68)) + ((ea + eb) + es);
                    const float a0 = vel_two_sum(phi, -S, e0);
                    v = a0 + (e0 - E);
                } else {
                    v = w_of(di) * phi * (1.f + cu);
                }
                P.fout[((size_t)p * 9 + i) * pl + k] = v;
            }
            if (i > 0) {
                // g^eq_i = lambda_i + w_i [c_i.(rho u)/c_s^2 + (m u):(c_i c_i - c_s^2 I)/(2 c_s^4)],
                // lambda_i = w_i P / c_s^2, m = rho u + m_phi
                const float mx = rho * ux + P.mphi[z], my = rho * uy + P.mphi[pl + z];
                const float cm = vCx[di] * mx + vCy[di] * my, cuu = vCx[di] * ux + vCy[di] * uy;
                const float mu_ = mx * ux + my * uy;
                const float w = w_of(di);
                P.gout[(size_t)(i - 1) * pl + k] =
                    w * (3.f * p_init[z] + rho * cu + 4.5f * (cm * cuu - (1.f / 3.f) * mu_));
            }
        }
    }
}

}  // namespace

cudaError_t launch_velocity_state(int ns, int model, const StepParams &p, const float *u0, float *u_prev,
                                  float *p_scratch, cudaStream_t st)
{
    const int threads = 256;
    unsigned b = (p.plane + threads - 1) / threads;
    if (b > 65535u * 16u) b = 65535u * 16u;
    const int blocks = (int)(b ? b : 1);
    switch (ns) {
#define NLBM_CASE(K)                                                                                      \
    case K:                                                                                               \
        if (model == 0)                                                                                   \
            velocity_prep_kernel<K, 0><<<blocks, threads, 0, st>>>(p, u0, u_prev, p_scratch);             \
        else                                                                                              \
            velocity_prep_kernel<K, 1><<<blocks, threads, 0, st>>>(p, u0, u_prev, p_scratch);             \
        velocity_pop_kernel<K><<<blocks, threads, 0, st>>>(p, u0, p_scratch);                             \
        break;
        NLBM_CASE(1) NLBM_CASE(2) NLBM_CASE(3) NLBM_CASE(4) NLBM_CASE(5) NLBM_CASE(6) NLBM_CASE(7)
#undef NLBM_CASE
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace nlbm
