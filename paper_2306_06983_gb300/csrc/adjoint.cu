// Reverse (adjoint) of the fused step, Models A and B, periodic axes or
// half-way bounce-back walls (without wetting), gravity, FP32.
//
// For a loss L(phi(T)) the adjoint runs the steps backwards.  For each step t
// it first rebuilds the step's intermediate fields from the step's input
// state (the "tape": phi, j, the pulled g, grad phi, lap phi, R, m_phi, w and
// F, three per-node passes), then takes the adjoint through the step in four
// per-node passes, each the transpose of a forward stage:
//   rev1  pointwise at x: both collisions (Eqs. (18)-(24)), the macroscopic
//         relations (Eqs. (25b), (25c), (13)), the mixture rules (Eqs. (11),
//         (12)) and F_s with the chemical potentials (Eqs. (16), (17));
//   rev2  transpose of F_c's stencil (gather of the F adjoint), then w,
//         m_phi (Eq. (13)) and the source (Model A, Eq. (2); Model B,
//         Eqs. (3), (4)) pointwise;
//   rev3  transposes of the isotropic gradient and Laplacian (Eq. (27));
//   rev4  transpose of the pull (streaming) and of the moments
//         phi = sum f_i, j = sum c_i f_i (Eq. (25a)).
// The adjoint of the step's inputs is the seed of the previous step.  The
// derivatives are those of the exact-arithmetic step; the exact-sum devices
// of the forward kernel (compensated sums, paired populations) change only
// rounding.  Per-node contributions to dL/d sigma_pq and dL/dM are summed
// in FP64 in a fixed order each step.
#include "nlbm_internal.cuh"
#include "adjoint.cuh"

namespace nlbm {

namespace {

__constant__ int aCx[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
__constant__ int aCy[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

__device__ __forceinline__ float wgt(int i) { return i == 0 ? 4.f / 9.f : (i < 5 ? 1.f / 9.f : 1.f / 36.f); }

__constant__ int aOpp[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

__device__ __forceinline__ unsigned wrap_node(int x, int y, int nx, int ny)
{
    x = x < 0 ? x + nx : (x >= nx ? x - nx : x);
    y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    return (unsigned)y * nx + x;
}

// Boundaries (half-way bounce-back walls on x and/or y, periodic otherwise),
// for positions at most one node outside the lattice.
// Whether (x, y) lies beyond a wall.
__device__ __forceinline__ bool beyond_wall(const StepParams &P, int x, int y)
{
    return (P.wall_x && (x < 0 || x >= P.nx)) || (P.wall_y && (y < 0 || y >= P.ny));
}
// The node a position stands for: periodic wrap, or the mirror image
// across a wall (a ghost node, whose phi is that of its image); fx, fy
// report mirroring across an x or a y wall.
__device__ __forceinline__ unsigned image_node(const StepParams &P, int x, int y, bool &fx, bool &fy)
{
    fx = P.wall_x && (x < 0 || x >= P.nx);
    fy = P.wall_y && (y < 0 || y >= P.ny);
    x = x < 0 ? (fx ? -1 - x : x + P.nx) : (x >= P.nx ? (fx ? 2 * P.nx - 1 - x : x - P.nx) : x);
    y = y < 0 ? (fy ? -1 - y : y + P.ny) : (y >= P.ny ? (fy ? 2 * P.ny - 1 - y : y - P.ny) : y);
    return (unsigned)y * P.nx + x;
}
// The positions that stand for node (x, y): itself and the ghost nodes
// beyond the walls it touches (up to 4 on a lattice one node wide with
// walls on both axes); returns their number, the first being the node.
__device__ __forceinline__ int standins(const StepParams &P, int x, int y, int (&px)[9], int (&py)[9])
{
    int xs[3] = {x, 0, 0}, ys[3] = {y, 0, 0}, nxs = 1, nys = 1;
    if (P.wall_x) {
        if (x == 0) xs[nxs++] = -1;
        if (x == P.nx - 1) xs[nxs++] = P.nx;
    }
    if (P.wall_y) {
        if (y == 0) ys[nys++] = -1;
        if (y == P.ny - 1) ys[nys++] = P.ny;
    }
    int n = 0;
    for (int b = 0; b < nys; ++b)
        for (int a = 0; a < nxs; ++a) {
            px[n] = xs[a];
            py[n] = ys[b];
            ++n;
        }
    return n;
}
// w = m_phi,x u_y - u_x m_phi,y at a ghost of a node, from the node's m_phi
// and previous velocity: the ghost's m_phi is the mirror image (normal
// component negated) and its velocity the no-slip ghost -u per mirroring,
// so w = s1 m_x u_y + s2 u_x m_y with s1 = -1 across a y wall, s2 = +1
// across an x wall (s1 = 1, s2 = -1 at the node itself).
__device__ __forceinline__ float w_sign1(bool fx, bool fy) { (void)fx; return fy ? -1.f : 1.f; }
__device__ __forceinline__ float w_sign2(bool fx, bool fy) { (void)fy; return fx ? 1.f : -1.f; }

// Model A's weight w(phi) = max(phi, 0)^n (Eq. (2)) and dw/dphi
// (n max(phi, 0)^(n-1); 0 where phi <= 0).  Integer n in 1..8 by
// multiplication, as in the forward kernel.
__device__ __forceinline__ float wa(const StepParams &P, float ph)
{
    const float pc = fmaxf(ph, 0.f);
    if (P.model_n_int > 0) {
        float w = pc;
        for (int k = 1; k < P.model_n_int; ++k) w *= pc;
        return w;
    }
    return pc > 0.f ? powf(pc, P.model_n) : 0.f;
}
__device__ __forceinline__ float dwa(const StepParams &P, float ph)
{
    if (!(ph > 0.f)) return 0.f;
    if (P.model_n_int > 0) {
        float w = 1.f;
        for (int k = 1; k < P.model_n_int; ++k) w *= ph;
        return (float)P.model_n_int * w;
    }
    return P.model_n * powf(ph, P.model_n - 1.f);
}

// 1 / |v| of a unit vector n = v / |v|: smooth reading 1 / sqrt(|v|^2 +
// delta^2), else 1 / |v| with n = 0 (returned 0) below the threshold.
__device__ __forceinline__ float unit_r(const StepParams &P, float n2)
{
    return P.unit_delta2 > 0.f ? rsqrtf(n2 + P.unit_delta2) : (n2 > 1e-24f ? rsqrtf(n2) : 0.f);
}

// g'(s) = 2 s (1 - s) (1 - 2 s) and its derivative (Eq. (17)).
__device__ __forceinline__ float gp1(float s) { return 2.f * s * (1.f - s) * (1.f - 2.f * s); }
__device__ __forceinline__ float gp2(float s) { return 2.f - 12.f * s + 12.f * s * s; }

// ------------------------------------------------------------------ tape

// Pull and moments: phi_p, j_p (Eq. (25a)) and the pulled flow populations.
template <int NS>
__global__ void tape_pull_kernel(const StepParams P, AdjTape T)
{
    const unsigned pl = P.plane;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < pl; k += gridDim.x * blockDim.x) {
        const int x = k % P.nx, y = k / P.nx;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            float ph = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                // pulled from x - c_i, or bounced back at a wall (f*_opp(i) of the node)
                const bool bb = beyond_wall(P, x - aCx[i], y - aCy[i]);
                const float f = bb ? P.fin[((size_t)p * 9 + aOpp[i]) * pl + k]
                                   : P.fin[((size_t)p * 9 + i) * pl + wrap_node(x - aCx[i], y - aCy[i], P.nx, P.ny)];
                ph += f;
                jx += aCx[i] * f;
                jy += aCy[i] * f;
            }
            T.phi[(size_t)p * pl + k] = ph;
            T.j[(size_t)(2 * p) * pl + k] = jx;
            T.j[(size_t)(2 * p + 1) * pl + k] = jy;
        }
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const bool bb = beyond_wall(P, x - aCx[i], y - aCy[i]);
            T.g[(size_t)(i - 1) * pl + k] = bb ? P.gin[(size_t)(aOpp[i] - 1) * pl + k]
                                               : P.gin[(size_t)(i - 1) * pl + wrap_node(x - aCx[i], y - aCy[i], P.nx, P.ny)];
        }
    }
}

// grad phi and lap phi (Eq. (27)) of phases 1..N-1, the source (Model A,
// Eq. (2); Model B, Eqs. (3), (4)), m_phi (Eq. (13)) and w = m_phi,x u_y -
// u_x m_phi,y with the previous velocity.
template <int NS, int MODEL>
__global__ void tape_stencil_kernel(const StepParams P, AdjTape T)
{
    constexpr int N = NS + 1;
    const unsigned pl = P.plane;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < pl; k += gridDim.x * blockDim.x) {
        const int x = k % P.nx, y = k / P.nx;
        float ph[N], gx[N], gy[N];
        float sph = 0.f, sgx = 0.f, sgy = 0.f;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            const float *f = T.phi + (size_t)p * pl;
            const float c = f[k];
            float ax = 0.f, ay = 0.f, lap = 0.f;
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                bool fx, fy;
                const float v = f[image_node(P, x + aCx[i], y + aCy[i], fx, fy)];
                ax += 3.f * wgt(i) * aCx[i] * v;
                ay += 3.f * wgt(i) * aCy[i] * v;
                lap += 6.f * wgt(i) * (v - c);
            }
            ph[p] = c;
            gx[p] = ax;
            gy[p] = ay;
            T.grad[(size_t)(2 * p) * pl + k] = ax;
            T.grad[(size_t)(2 * p + 1) * pl + k] = ay;
            T.lap[(size_t)p * pl + k] = lap;
            sph += c;
            sgx += ax;
            sgy += ay;
        }
        ph[NS] = 1.f - sph;
        gx[NS] = -sgx;
        gy[NS] = -sgy;
        float Rx[NS], Ry[NS];
#pragma unroll
        for (int p = 0; p < NS; ++p) Rx[p] = Ry[p] = 0.f;
        if constexpr (MODEL == 0) {
            // R_p = a_p n_p - w_p / (sum_q w_q) sum_q a_q n_q, a_q = 4 phi_q (1 - phi_q) / eps
            float ax[N], ay[N], S = 0.f, Vx = 0.f, Vy = 0.f;
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const float ar = P.four_over_eps * ph[q] * (1.f - ph[q]) * unit_r(P, gx[q] * gx[q] + gy[q] * gy[q]);
                ax[q] = ar * gx[q];
                ay[q] = ar * gy[q];
                S += wa(P, ph[q]);
                Vx += ax[q];
                Vy += ay[q];
            }
#pragma unroll
            for (int p = 0; p < NS; ++p) {
                const float b = wa(P, ph[p]) / S;
                Rx[p] = ax[p] - b * Vx;
                Ry[p] = ay[p] - b * Vy;
            }
        } else {
#pragma unroll
            for (int p = 0; p < N; ++p)
#pragma unroll
                for (int q = p + 1; q < N; ++q) {
                    const float vx = ph[q] * gx[p] - ph[p] * gx[q], vy = ph[q] * gy[p] - ph[p] * gy[q];
                    const float r = unit_r(P, vx * vx + vy * vy);
                    const float c = P.four_over_eps * ph[p] * ph[q] * r;
                    if (p < NS) { Rx[p] += c * vx; Ry[p] += c * vy; }
                    if (q < NS) { Rx[q] -= c * vx; Ry[q] -= c * vy; }
                }
        }
        float mx = 0.f, my = 0.f;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            T.R[(size_t)(2 * p) * pl + k] = Rx[p];
            T.R[(size_t)(2 * p + 1) * pl + k] = Ry[p];
            mx += P.drho[p] * (gx[p] - Rx[p]);
            my += P.drho[p] * (gy[p] - Ry[p]);
        }
        mx *= -P.mob;
        my *= -P.mob;
        T.mphi[k] = mx;
        T.mphi[pl + k] = my;
        T.w[k] = mx * P.uin[pl + k] - P.uin[k] * my;
    }
}

// Chemical potentials of all N phases at one node (Eq. (17)).
template <int NS>
__device__ __forceinline__ void chem_pot(const StepParams &P, const float (&ph)[NS + 1], const float (&lap)[NS + 1],
                                         float (&mu)[NS + 1])
{
    constexpr int N = NS + 1;
    float g[N];
#pragma unroll
    for (int p = 0; p < N; ++p) {
        g[p] = gp1(ph[p]);
        mu[p] = 0.f;
    }
#pragma unroll
    for (int p = 0; p < N; ++p)
#pragma unroll
        for (int q = p + 1; q < N; ++q) {
            const float G = gp1(ph[p] + ph[q]);
            mu[p] += P.beta2[p][q] * (g[p] - G) + P.kap[p][q] * lap[q];
            mu[q] += P.beta2[p][q] * (g[q] - G) + P.kap[p][q] * lap[p];
        }
}

// F = F_s + F_c + F_g (Eq. (16), the lagged-velocity F_c and gravity rho g).
template <int NS>
__global__ void tape_force_kernel(const StepParams P, AdjTape T)
{
    constexpr int N = NS + 1;
    const unsigned pl = P.plane;
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < pl; k += gridDim.x * blockDim.x) {
        const int x = k % P.nx, y = k / P.nx;
        float ph[N], lap[N], mu[N];
        float sph = 0.f, sl = 0.f;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            ph[p] = T.phi[(size_t)p * pl + k];
            lap[p] = T.lap[(size_t)p * pl + k];
            sph += ph[p];
            sl += lap[p];
        }
        ph[NS] = 1.f - sph;
        lap[NS] = -sl;
        chem_pot<NS>(P, ph, lap, mu);
        float rho = P.rhoN;
#pragma unroll
        for (int p = 0; p < NS; ++p) rho += P.drho[p] * ph[p];
        float Fx = 0.f, Fy = 0.f;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            const float d = mu[p] - mu[NS];
            Fx += d * T.grad[(size_t)(2 * p) * pl + k];
            Fy += d * T.grad[(size_t)(2 * p + 1) * pl + k];
        }
        float dxw = 0.f, dyw = 0.f;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            bool fx, fy;
            const unsigned n = image_node(P, x + aCx[i], y + aCy[i], fx, fy);
            float v = T.w[n];
            if (fx || fy) {
                const float mx = T.mphi[n], my = T.mphi[pl + n], ux = P.uin[n], uy = P.uin[pl + n];
                v = w_sign1(fx, fy) * mx * uy + w_sign2(fx, fy) * ux * my;
            }
            dxw += 3.f * wgt(i) * aCx[i] * v;
            dyw += 3.f * wgt(i) * aCy[i] * v;
        }
        T.F[k] = Fx + 0.5f * dyw + rho * P.gx;
        T.F[pl + k] = Fy - 0.5f * dxw + rho * P.gy;
    }
}

// ---------------------------------------------------------------- reverse

// rev1: pointwise adjoint of the collisions and everything between the
// tape fields and them.  Seeds at x: A.lf_out (f*), A.lg_out (g*), A.lphi_out
// (phi(t): the next step's phi_prev and the loss), A.lu_out, A.lm_out.
template <int NS>
__device__ __forceinline__ void rev_collide_node(const StepParams &P, const AdjTape &T, const AdjFields &A, unsigned k)
{
    constexpr int N = NS + 1;
    constexpr int NP = N * (N - 1) / 2;
    const unsigned pl = P.plane;
    {
        // ---------------- forward values at x
        float ph[N], lap[N], gx[NS], gy[NS], jx[NS], jy[NS], Rx[NS], Ry[NS], php[NS];
        float sph = 0.f, sl = 0.f, rho = P.rhoN, mu = P.muN, grx = 0.f, gry = 0.f, rho_prev = P.rhoN;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            ph[p] = __ldg(T.phi + (size_t)p * pl + k);
            lap[p] = __ldg(T.lap + (size_t)p * pl + k);
            gx[p] = __ldg(T.grad + (size_t)(2 * p) * pl + k);
            gy[p] = __ldg(T.grad + (size_t)(2 * p + 1) * pl + k);
            jx[p] = __ldg(T.j + (size_t)(2 * p) * pl + k);
            jy[p] = __ldg(T.j + (size_t)(2 * p + 1) * pl + k);
            Rx[p] = __ldg(T.R + (size_t)(2 * p) * pl + k);
            Ry[p] = __ldg(T.R + (size_t)(2 * p + 1) * pl + k);
            php[p] = __ldg(P.phi_prev + (size_t)p * pl + k);
            sph += ph[p];
            sl += lap[p];
            rho += P.drho[p] * ph[p];
            mu += P.dmu[p] * ph[p];
            grx += P.drho[p] * gx[p];
            gry += P.drho[p] * gy[p];
            rho_prev += P.drho[p] * php[p];
        }
        ph[NS] = 1.f - sph;
        lap[NS] = -sl;
        double gacc[NP + 1];   // updated at the end; loaded before the first store
#pragma unroll
        for (int q = 0; q <= NP; ++q) gacc[q] = A.gacc[(size_t)q * pl + k];
        float g[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) g[i] = __ldg(T.g + (size_t)(i - 1) * pl + k);
        const float Fx = __ldg(T.F + k), Fy = __ldg(T.F + pl + k);
        const float mphx = __ldg(T.mphi + k), mphy = __ldg(T.mphi + pl + k);
        const float upx = __ldg(P.uin + k), upy = __ldg(P.uin + pl + k);
        const float mpx = __ldg(P.mphi + k), mpy = __ldg(P.mphi + pl + k);   // m_phi of step t-1
        const float sg = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
        const float jgx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
        const float jgy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
        const float d58 = (g[5] + g[6]) + (g[7] + g[8]);
        const float Pxx = (g[1] + g[3]) + d58, Pyy = (g[2] + g[4]) + d58, Pxy = (g[5] - g[6]) + (g[7] - g[8]);
        const float ux = (jgx + 0.5f * Fx) / rho, uy = (jgy + 0.5f * Fy) / rho;
        const float mx = rho * ux + mphx, my = rho * uy + mphy;
        const float ugr = ux * grx + uy * gry;
        const float mu_t = mx * ux + my * uy;
        const float mu_prev = (rho_prev * upx + mpx) * upx + (rho_prev * upy + mpy) * upy;
        const float Pr = 0.6f * (sg + 0.5f * ugr - (1.f / 3.f) * mu_t - (1.f / 3.f) * mu_prev);
        const float den = 6.f * mu + rho;
        const float s2 = 2.f * rho / den, c2 = 1.f - s2, h2 = 1.f - 0.5f * s2;
        const float Qxx = mx * ux, Qyy = my * uy, Qxy = 0.5f * (mx * uy + my * ux);
        const float dQxx = mphx * ux - mpx * upx, dQyy = mphy * uy - mpy * upy;
        const float dQxy = 0.5f * ((mphx * uy + mphy * ux) - (mpx * upy + mpy * upx));
        const float Mxx = 2.f * ux * Fx + dQxx + (2.f / 3.f) * ux * grx + (1.f / 3.f) * ugr;
        const float Myy = 2.f * uy * Fy + dQyy + (2.f / 3.f) * uy * gry + (1.f / 3.f) * ugr;
        const float Mxy = ux * Fy + Fx * uy + dQxy + (1.f / 3.f) * (ux * gry + grx * uy);

        // ---------------- adjoint accumulators
        float a_ph[N], a_lap[N], a_gx[NS], a_gy[NS], a_Rx[NS], a_Ry[NS], a_php[NS];
#pragma unroll
        for (int p = 0; p < N; ++p) { a_ph[p] = 0.f; a_lap[p] = 0.f; }
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            a_ph[p] = __ldg(A.lphi_out + (size_t)p * pl + k);
            a_gx[p] = a_gy[p] = a_Rx[p] = a_Ry[p] = a_php[p] = 0.f;
        }
        float a_ux = __ldg(A.lu_out + k), a_uy = __ldg(A.lu_out + pl + k);
        float a_mphx = __ldg(A.lm_out + k), a_mphy = __ldg(A.lm_out + pl + k);
        float a_upx = 0.f, a_upy = 0.f, a_mpx = 0.f, a_mpy = 0.f;
        float a_Fx = 0.f, a_Fy = 0.f, a_rho = 0.f, a_mu = 0.f, a_grx = 0.f, a_gry = 0.f, a_s1 = 0.f;

        // ---------------- flow collision (Eqs. (21)-(24)) reversed
        float lg[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) lg[i] = __ldg(A.lg_out + (size_t)(i - 1) * pl + k);
        const float a_m1 = 0.5f * (lg[1] - lg[3]);
        const float a_m2 = 0.5f * (lg[2] - lg[4]);
        const float a_m3 = 0.5f * (lg[1] + lg[3]);
        const float a_m4 = 0.5f * (lg[2] + lg[4]);
        const float a_m5 = 0.25f * ((lg[5] - lg[6]) + (lg[7] - lg[8]));
        const float a_m6 = -0.5f * (lg[2] - lg[4]) + 0.25f * ((lg[5] + lg[6]) - (lg[7] + lg[8]));
        const float a_m7 = -0.5f * (lg[1] - lg[3]) + 0.25f * ((lg[5] - lg[6]) - (lg[7] - lg[8]));
        const float a_m8 = -0.5f * ((lg[1] + lg[2]) + (lg[3] + lg[4])) + 0.25f * ((lg[5] + lg[6]) + (lg[7] + lg[8]));
        // m8 = (P + Qxx + Qyy)/3 + (Mxx + Myy)/6 - ugr/18
        float a_P = a_m8 / 3.f, a_Qxx = a_m8 / 3.f, a_Qyy = a_m8 / 3.f;
        float a_Mxx = a_m8 / 6.f, a_Myy = a_m8 / 6.f, a_ugr = -a_m8 / 18.f;
        // m7 = rho ux/3 + Fx/6, m6 = rho uy/3 + Fy/6
        a_rho += (a_m7 * ux + a_m6 * uy) / 3.f;
        a_ux += a_m7 * rho / 3.f;
        a_uy += a_m6 * rho / 3.f;
        a_Fx += a_m7 / 6.f;
        a_Fy += a_m6 / 6.f;
        // m5 = c2 Pxy + s2 Qxy + h2 Mxy; m4, m3 likewise
        float a_Pxy = c2 * a_m5, a_Qxy = s2 * a_m5, a_Mxy = h2 * a_m5;
        float a_s2 = (-Pxy + Qxy - 0.5f * Mxy) * a_m5;
        float a_Pyy = c2 * a_m4;
        a_P += s2 * a_m4;
        a_Qyy += s2 * a_m4;
        a_Myy += h2 * a_m4;
        a_s2 += (-Pyy + Pr + Qyy - 0.5f * Myy) * a_m4;
        float a_Pxx = c2 * a_m3;
        a_P += s2 * a_m3;
        a_Qxx += s2 * a_m3;
        a_Mxx += h2 * a_m3;
        a_s2 += (-Pxx + Pr + Qxx - 0.5f * Mxx) * a_m3;
        // m1 = jgx + Fx, m2 = jgy + Fy
        float a_jgx = a_m1, a_jgy = a_m2;
        a_Fx += a_m1;
        a_Fy += a_m2;
        // Mxy, Myy, Mxx
        a_ux += a_Mxy * (Fy + gry / 3.f);
        a_uy += a_Mxy * (Fx + grx / 3.f);
        a_Fx += a_Mxy * uy;
        a_Fy += a_Mxy * ux;
        a_grx += a_Mxy * uy / 3.f;
        a_gry += a_Mxy * ux / 3.f;
        float a_dQxy = a_Mxy;
        a_uy += a_Myy * (2.f * Fy + (2.f / 3.f) * gry);
        a_Fy += 2.f * uy * a_Myy;
        a_gry += (2.f / 3.f) * uy * a_Myy;
        a_ugr += a_Myy / 3.f;
        float a_dQyy = a_Myy;
        a_ux += a_Mxx * (2.f * Fx + (2.f / 3.f) * grx);
        a_Fx += 2.f * ux * a_Mxx;
        a_grx += (2.f / 3.f) * ux * a_Mxx;
        a_ugr += a_Mxx / 3.f;
        float a_dQxx = a_Mxx;
        // dQ terms
        a_mphx += 0.5f * uy * a_dQxy + ux * a_dQxx;
        a_mphy += 0.5f * ux * a_dQxy + uy * a_dQyy;
        a_ux += 0.5f * mphy * a_dQxy + mphx * a_dQxx;
        a_uy += 0.5f * mphx * a_dQxy + mphy * a_dQyy;
        a_mpx -= 0.5f * upy * a_dQxy + upx * a_dQxx;
        a_mpy -= 0.5f * upx * a_dQxy + upy * a_dQyy;
        a_upx -= 0.5f * mpy * a_dQxy + mpx * a_dQxx;
        a_upy -= 0.5f * mpx * a_dQxy + mpy * a_dQyy;
        // Q terms: Qxx = mx ux, Qyy = my uy, Qxy = (mx uy + my ux)/2
        float a_mx = ux * a_Qxx + 0.5f * uy * a_Qxy;
        float a_my = uy * a_Qyy + 0.5f * ux * a_Qxy;
        a_ux += mx * a_Qxx + 0.5f * my * a_Qxy;
        a_uy += my * a_Qyy + 0.5f * mx * a_Qxy;
        // s2 = 2 rho / (6 mu + rho)
        a_rho += a_s2 * 12.f * mu / (den * den);
        a_mu += -a_s2 * 12.f * rho / (den * den);
        // ---------------- phase collisions (Eqs. (18)-(20)) reversed
        const float s1 = P.s1, h1 = (1.f - 0.5f * s1) / 3.f;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            float lf[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) lf[i] = __ldg(A.lf_out + ((size_t)p * 9 + i) * pl + k);
            const float phi = ph[p];
            const float Gx = 3.f * (phi * ux - php[p] * upx) + Rx[p];
            const float Gy = 3.f * (phi * uy - php[p] * upy) + Ry[p];
            float a_phi = (4.f / 9.f) * lf[0] + ((lf[1] + lf[2]) + (lf[3] + lf[4])) / 9.f +
                          ((lf[5] + lf[6]) + (lf[7] + lf[8])) / 36.f;
            const float a_A = 0.5f * (lf[1] - lf[3]), a_B = 0.5f * (lf[2] - lf[4]);
            const float a_C = -0.5f * (lf[2] - lf[4]) + 0.25f * ((lf[5] - lf[7]) + (lf[6] - lf[8]));
            const float a_D = -0.5f * (lf[1] - lf[3]) + 0.25f * ((lf[5] - lf[7]) - (lf[6] - lf[8]));
            // C = phi uy/3 + Gy/18, D = phi ux/3 + Gx/18
            a_phi += (a_C * uy + a_D * ux) / 3.f;
            a_uy += a_C * phi / 3.f;
            a_ux += a_D * phi / 3.f;
            float a_Gy = a_C / 18.f, a_Gx = a_D / 18.f;
            // A = (1 - s1) jx + s1 phi ux + h1 Gx, B likewise
            A.lj[(size_t)(2 * p) * pl + k] = (1.f - s1) * a_A;
            A.lj[(size_t)(2 * p + 1) * pl + k] = (1.f - s1) * a_B;
            a_phi += s1 * (ux * a_A + uy * a_B);
            a_ux += s1 * phi * a_A;
            a_uy += s1 * phi * a_B;
            a_Gx += h1 * a_A;
            a_Gy += h1 * a_B;
            a_s1 += (-jx[p] + phi * ux - Gx / 6.f) * a_A + (-jy[p] + phi * uy - Gy / 6.f) * a_B;
            // G = 3 (phi u - phi_prev u_prev) + R
            a_phi += 3.f * (ux * a_Gx + uy * a_Gy);
            a_ux += 3.f * phi * a_Gx;
            a_uy += 3.f * phi * a_Gy;
            a_php[p] -= 3.f * (upx * a_Gx + upy * a_Gy);
            a_upx -= 3.f * php[p] * a_Gx;
            a_upy -= 3.f * php[p] * a_Gy;
            a_Rx[p] += a_Gx;
            a_Ry[p] += a_Gy;
            a_ph[p] += a_phi;
        }

        // ---------------- pressure (Eq. (25c)) and m (Eq. (13)) reversed
        a_ugr += 0.3f * a_P;
        const float a_mut = -0.2f * a_P, a_mup = -0.2f * a_P;
        // mu_prev = (rho_prev up + mp) . up
        const float a_rhop = a_mup * (upx * upx + upy * upy);
        a_upx += a_mup * (2.f * rho_prev * upx + mpx);
        a_upy += a_mup * (2.f * rho_prev * upy + mpy);
        a_mpx += a_mup * upx;
        a_mpy += a_mup * upy;
#pragma unroll
        for (int p = 0; p < NS; ++p) a_php[p] += P.drho[p] * a_rhop;
        // mu_t = m . u
        a_mx += a_mut * ux;
        a_my += a_mut * uy;
        a_ux += a_mut * mx;
        a_uy += a_mut * my;
        // ugr = u . grad rho
        a_ux += a_ugr * grx;
        a_uy += a_ugr * gry;
        a_grx += a_ugr * ux;
        a_gry += a_ugr * uy;
        // m = rho u + m_phi
        a_rho += a_mx * ux + a_my * uy;
        a_ux += rho * a_mx;
        a_uy += rho * a_my;
        a_mphx += a_mx;
        a_mphy += a_my;
        // u = (jg + F/2) / rho (Eq. (25b))
        a_jgx += a_ux / rho;
        a_jgy += a_uy / rho;
        a_Fx += 0.5f * a_ux / rho;
        a_Fy += 0.5f * a_uy / rho;
        a_rho -= (a_ux * ux + a_uy * uy) / rho;
        // sg, jg and Pi of the pulled flow populations (P = 0.6 (sg + ...))
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const float cx = (float)aCx[i], cy = (float)aCy[i];
            A.lg_pull[(size_t)(i - 1) * pl + k] = 0.6f * a_P + (cx * a_jgx + cy * a_jgy) + cx * cx * a_Pxx +
                                                  cy * cy * a_Pyy + cx * cy * a_Pxy;
        }

        // ---------------- gravity F_g = rho g in the total force
        a_rho += a_Fx * P.gx + a_Fy * P.gy;
        // ---------------- mixture rules (Eqs. (11), (12)) and F_s (Eqs. (16), (17))
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            a_ph[p] += P.drho[p] * a_rho + P.dmu[p] * a_mu;
            a_gx[p] += P.drho[p] * a_grx;
            a_gy[p] += P.drho[p] * a_gry;
        }
        float mu_c[N];
        chem_pot<NS>(P, ph, lap, mu_c);
        float a_muc[N];
        a_muc[NS] = 0.f;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            a_muc[p] = a_Fx * gx[p] + a_Fy * gy[p];
            a_muc[NS] -= a_muc[p];
            const float d = mu_c[p] - mu_c[NS];
            a_gx[p] += d * a_Fx;
            a_gy[p] += d * a_Fy;
        }
        float dsig[NP > 0 ? NP : 1];
        int pair = 0;
#pragma unroll
        for (int p = 0; p < N; ++p)
#pragma unroll
            for (int q = p + 1; q < N; ++q) {
                const float s = ph[p] + ph[q];
                const float b = P.beta2[p][q], kq = P.kap[p][q];
                const float G2 = gp2(s);
                a_ph[p] += a_muc[p] * b * (gp2(ph[p]) - G2) - a_muc[q] * b * G2;
                a_ph[q] += a_muc[q] * b * (gp2(ph[q]) - G2) - a_muc[p] * b * G2;
                a_lap[q] += kq * a_muc[p];
                a_lap[p] += kq * a_muc[q];
                // beta2 = 6 sigma / eps, kap = 3 eps sigma / 4
                const float G1 = gp1(s);
                dsig[pair++] = a_muc[p] * (P.six_over_eps * (gp1(ph[p]) - G1) + P.three_eps_over_4 * lap[q]) +
                               a_muc[q] * (P.six_over_eps * (gp1(ph[q]) - G1) + P.three_eps_over_4 * lap[p]);
            }
        // phase N = 1 - sum: fold its adjoints onto phases 1..N-1
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            a_ph[p] -= a_ph[NS];
            a_lap[p] -= a_lap[NS];
        }

        // ---------------- outputs
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            A.lphi_pw[(size_t)p * pl + k] = a_ph[p];
            A.llap[(size_t)p * pl + k] = a_lap[p];
            A.lgrad[(size_t)(2 * p) * pl + k] = a_gx[p];
            A.lgrad[(size_t)(2 * p + 1) * pl + k] = a_gy[p];
            A.lR[(size_t)(2 * p) * pl + k] = a_Rx[p];
            A.lR[(size_t)(2 * p + 1) * pl + k] = a_Ry[p];
            A.lphi_in[(size_t)p * pl + k] = a_php[p];
        }
        A.lF[k] = a_Fx;
        A.lF[pl + k] = a_Fy;
        A.lmphi[k] = a_mphx;
        A.lmphi[pl + k] = a_mphy;
        A.lu_in[k] = a_upx;
        A.lu_in[pl + k] = a_upy;
        A.lm_in[k] = a_mpx;
        A.lm_in[pl + k] = a_mpy;
#pragma unroll
        for (int q = 0; q < NP; ++q) A.gacc[(size_t)q * pl + k] = gacc[q] + (double)dsig[q];
        // s1 = 1 / (1/2 + 3 M): d s1 / dM = -3 s1^2
        A.gacc[(size_t)NP * pl + k] = gacc[NP] + (double)(-3.f * s1 * s1 * a_s1);
    }
}


// rev2: F_c's stencil transposed (gather of the F adjoint at the
// neighbours), then w, m_phi and the source (Model A or B) at the node.
template <int NS, int MODEL, bool WALLS>
__device__ __forceinline__ void rev_source_node(const StepParams &P, const AdjTape &T, const AdjFields &A, unsigned k)
{
    constexpr int N = NS + 1;
    constexpr int NP = N * (N - 1) / 2;
    const unsigned pl = P.plane;
    {
        const int x = k % P.nx, y = k / P.nx;
        // F_c(x) = (1/2 d_y w, -1/2 d_x w): w at position z enters F_c(z -
        // c_i) with weight 3 w_i c_i; the positions holding this node's w
        // are the node and, next to a wall, its ghosts (w there formed from
        // this node's m_phi and u with the signs s1, s2 of w_sign1/2).
        float a_w = 0.f, a_ws1 = 0.f, a_ws2 = 0.f;
        if constexpr (!WALLS) {
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                const unsigned n = wrap_node(x - aCx[i], y - aCy[i], P.nx, P.ny);
                a_w += 3.f * wgt(i) * (0.5f * aCy[i] * __ldg(A.lF + n) - 0.5f * aCx[i] * __ldg(A.lF + pl + n));
            }
            a_ws1 = a_w;
            a_ws2 = -a_w;
        } else {
            int px[9], py[9];
            const int ns = standins(P, x, y, px, py);
            for (int s = 0; s < ns; ++s) {
                const bool fx = px[s] < 0 || px[s] >= P.nx, fy = py[s] < 0 || py[s] >= P.ny;
                float aw = 0.f;
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const int zx = px[s] - aCx[i], zy = py[s] - aCy[i];
                    if (beyond_wall(P, zx, zy)) continue;
                    const unsigned n = wrap_node(zx, zy, P.nx, P.ny);
                    aw += 3.f * wgt(i) * (0.5f * aCy[i] * __ldg(A.lF + n) - 0.5f * aCx[i] * __ldg(A.lF + pl + n));
                }
                a_ws1 += w_sign1(fx, fy) * aw;
                a_ws2 += w_sign2(fx, fy) * aw;
            }
        }
        const float upx = __ldg(P.uin + k), upy = __ldg(P.uin + pl + k);
        const float mphx = __ldg(T.mphi + k), mphy = __ldg(T.mphi + pl + k);
        // w = s1 mx uy + s2 ux my (previous velocity)
        const float a_mx = __ldg(A.lmphi + k) + a_ws1 * upy;
        const float a_my = __ldg(A.lmphi + pl + k) + a_ws2 * upx;
        // the values this pass updates, loaded before its first store (the
        // compiler may not move a load across a store to another field)
        const float lux = A.lu_in[k], luy = A.lu_in[pl + k];
        const double gM = A.gacc[(size_t)NP * pl + k];
        float pw[NS];
#pragma unroll
        for (int p = 0; p < NS; ++p) pw[p] = A.lphi_pw[(size_t)p * pl + k];
        // m_phi = -M sum_p drho_p (grad phi_p - R_p)
        float ph[N], gx[N], gy[N], a_ph[N], a_gx[N], a_gy[N], a_Rx[NS], a_Ry[NS];
        float sph = 0.f, sgx = 0.f, sgy = 0.f, dM = 0.f;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            ph[p] = __ldg(T.phi + (size_t)p * pl + k);
            gx[p] = __ldg(T.grad + (size_t)(2 * p) * pl + k);
            gy[p] = __ldg(T.grad + (size_t)(2 * p + 1) * pl + k);
            sph += ph[p];
            sgx += gx[p];
            sgy += gy[p];
            a_ph[p] = 0.f;
            a_gx[p] = A.lgrad[(size_t)(2 * p) * pl + k] - P.mob * P.drho[p] * a_mx;
            a_gy[p] = A.lgrad[(size_t)(2 * p + 1) * pl + k] - P.mob * P.drho[p] * a_my;
            a_Rx[p] = __ldg(A.lR + (size_t)(2 * p) * pl + k) + P.mob * P.drho[p] * a_mx;
            a_Ry[p] = __ldg(A.lR + (size_t)(2 * p + 1) * pl + k) + P.mob * P.drho[p] * a_my;
            const float Rx = __ldg(T.R + (size_t)(2 * p) * pl + k), Ry = __ldg(T.R + (size_t)(2 * p + 1) * pl + k);
            dM -= P.drho[p] * ((gx[p] - Rx) * a_mx + (gy[p] - Ry) * a_my);
        }
        ph[NS] = 1.f - sph;
        gx[NS] = -sgx;
        gy[NS] = -sgy;
        a_ph[NS] = a_gx[NS] = a_gy[NS] = 0.f;
        if constexpr (MODEL == 0) {
            // Model A source: R_p = A_p - beta_p V with A_q = a_q n_q, a_q =
            // 4 phi_q (1 - phi_q) / eps, n_q = grad phi_q / s_q, V = sum_q A_q
            // (all N phases), beta_p = w_p / S, w_q = max(phi_q, 0)^n, S =
            // sum_q w_q.  Adjoints: the A-adjoint of phase q is its R-adjoint
            // (0 for phase N) minus sum_p beta_p (R-adjoint of p); the
            // w-adjoint is (b_q - sum_p b_p beta_p) / S with b_p = -(R-adjoint
            // of p) . V; a_q's and n_q's parts as in Model B ((I - n n^T) / s).
            float nxq[N], nyq[N], rq[N], aq[N], w[N];
            float S = 0.f, Vx = 0.f, Vy = 0.f;
#pragma unroll
            for (int q = 0; q < N; ++q) {
                aq[q] = P.four_over_eps * ph[q] * (1.f - ph[q]);
                rq[q] = unit_r(P, gx[q] * gx[q] + gy[q] * gy[q]);
                nxq[q] = gx[q] * rq[q];
                nyq[q] = gy[q] * rq[q];
                w[q] = wa(P, ph[q]);
                S += w[q];
                Vx += aq[q] * nxq[q];
                Vy += aq[q] * nyq[q];
            }
            const float invS = 1.f / S;
            float gbx = 0.f, gby = 0.f, bb = 0.f, b[N];
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const float rx = q < NS ? a_Rx[q] : 0.f, ry = q < NS ? a_Ry[q] : 0.f;
                const float beta = w[q] * invS;
                gbx -= beta * rx;
                gby -= beta * ry;
                b[q] = -(rx * Vx + ry * Vy);
                bb += b[q] * beta;
            }
#pragma unroll
            for (int q = 0; q < N; ++q) {
                const float Ax = (q < NS ? a_Rx[q] : 0.f) + gbx, Ay = (q < NS ? a_Ry[q] : 0.f) + gby;
                a_ph[q] += (b[q] - bb) * invS * dwa(P, ph[q]);
                if (rq[q] == 0.f) continue;   // n = 0 below the threshold (thresholded reading)
                const float an = Ax * nxq[q] + Ay * nyq[q];
                a_ph[q] += an * P.four_over_eps * (1.f - 2.f * ph[q]);
                a_gx[q] += aq[q] * (Ax - an * nxq[q]) * rq[q];
                a_gy[q] += aq[q] * (Ay - an * nyq[q]) * rq[q];
            }
        } else {
        // Model B source: pair (p, q) adds T = (4/eps) phi_p phi_q n_pq to R_p
        // and subtracts it from R_q, n_pq = unit(phi_q grad phi_p - phi_p grad phi_q)
#pragma unroll
        for (int p = 0; p < N; ++p)
#pragma unroll
            for (int q = p + 1; q < N; ++q) {
                float apx = p < NS ? a_Rx[p] : 0.f, apy = p < NS ? a_Ry[p] : 0.f;
                if (q < NS) { apx -= a_Rx[q]; apy -= a_Ry[q]; }
                const float vx = ph[q] * gx[p] - ph[p] * gx[q], vy = ph[q] * gy[p] - ph[p] * gy[q];
                const float n2 = vx * vx + vy * vy;
                // n = v / s, s = sqrt(|v|^2 + delta^2) (or |v|; n = 0 below the threshold)
                if (!(P.unit_delta2 > 0.f) && !(n2 > 1e-24f)) continue;
                const float r = P.unit_delta2 > 0.f ? rsqrtf(n2 + P.unit_delta2) : rsqrtf(n2);
                const float nx_ = vx * r, ny_ = vy * r;
                const float c = P.four_over_eps;
                const float an = apx * nx_ + apy * ny_;
                a_ph[p] += c * ph[q] * an;
                a_ph[q] += c * ph[p] * an;
                const float anx = c * ph[p] * ph[q] * apx, any = c * ph[p] * ph[q] * apy;
                const float dot = anx * nx_ + any * ny_;
                const float avx = (anx - dot * nx_) * r, avy = (any - dot * ny_) * r;
                a_ph[q] += avx * gx[p] + avy * gy[p];
                a_gx[p] += ph[q] * avx;
                a_gy[p] += ph[q] * avy;
                a_ph[p] -= avx * gx[q] + avy * gy[q];
                a_gx[q] -= ph[p] * avx;
                a_gy[q] -= ph[p] * avy;
            }
        }
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            A.lphi_pw[(size_t)p * pl + k] = pw[p] + (a_ph[p] - a_ph[NS]);
            A.lgrad[(size_t)(2 * p) * pl + k] = a_gx[p] - a_gx[NS];
            A.lgrad[(size_t)(2 * p + 1) * pl + k] = a_gy[p] - a_gy[NS];
        }
        A.lu_in[k] = lux + a_ws2 * mphy;
        A.lu_in[pl + k] = luy + a_ws1 * mphx;
        A.gacc[(size_t)NP * pl + k] = gM + (double)dM;
    }
}


// rev3: the gradient and Laplacian stencils transposed: phi_p(z) entered
// grad phi_p(z - c_i) with weight 3 w_i c_i and lap phi_p(z - c_i) with 6 w_i
// (and lap phi_p(z) with -6 (1 - w_0)).
template <int NS, bool WALLS>
__device__ __forceinline__ void rev_stencil_node(const StepParams &P, const AdjFields &A, unsigned k)
{
    const unsigned pl = P.plane;
    {
        const int x = k % P.nx, y = k / P.nx;
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            const float *lgx = A.lgrad + (size_t)(2 * p) * pl, *lgy = A.lgrad + (size_t)(2 * p + 1) * pl;
            const float *ll = A.llap + (size_t)p * pl;
            float a = __ldg(A.lphi_pw + (size_t)p * pl + k) - 6.f * (1.f - 4.f / 9.f) * __ldg(ll + k);
            if constexpr (!WALLS) {
#pragma unroll
                for (int i = 1; i < 9; ++i) {
                    const unsigned n = wrap_node(x - aCx[i], y - aCy[i], P.nx, P.ny);
                    a += 3.f * wgt(i) * (aCx[i] * __ldg(lgx + n) + aCy[i] * __ldg(lgy + n)) + 6.f * wgt(i) * __ldg(ll + n);
                }
            } else {
                // phi of this node also stands at its ghosts beyond the walls
                int px[9], py[9];
                const int ns = standins(P, x, y, px, py);
                for (int s = 0; s < ns; ++s)
#pragma unroll
                    for (int i = 1; i < 9; ++i) {
                        const int zx = px[s] - aCx[i], zy = py[s] - aCy[i];
                        if (beyond_wall(P, zx, zy)) continue;
                        const unsigned n = wrap_node(zx, zy, P.nx, P.ny);
                        a += 3.f * wgt(i) * (aCx[i] * __ldg(lgx + n) + aCy[i] * __ldg(lgy + n)) +
                             6.f * wgt(i) * __ldg(ll + n);
                    }
            }
            A.lphi_tot[(size_t)p * pl + k] = a;
        }
    }
}


// rev4: the pull and the moments transposed.  f_i(z) = f*_i(z - c_i) fed
// phi(z) and j(z): the adjoint of f*_i at y is lphi(y + c_i) + c_i . lj(y + c_i);
// likewise for the flow populations.  The results seed the previous step.
template <int NS, bool WALLS>
__device__ __forceinline__ void rev_pull_node(const StepParams &P, const AdjFields &A, unsigned k)
{
    const unsigned pl = P.plane;
    {
        const int x = k % P.nx, y = k / P.nx;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            // f*_i here was pulled by the node at x + c_i, or, where that is
            // beyond a wall, bounced back into this node as direction opp(i)
            const bool bb = WALLS && beyond_wall(P, x + aCx[i], y + aCy[i]);
            const unsigned n = bb ? k : wrap_node(x + aCx[i], y + aCy[i], P.nx, P.ny);
            const int d = bb ? aOpp[i] : i;
#pragma unroll
            for (int p = 0; p < NS; ++p)
                A.lf_in[((size_t)p * 9 + i) * pl + k] = __ldg(A.lphi_tot + (size_t)p * pl + n) +
                                                        aCx[d] * __ldg(A.lj + (size_t)(2 * p) * pl + n) +
                                                        aCy[d] * __ldg(A.lj + (size_t)(2 * p + 1) * pl + n);
            if (i > 0) A.lg_in[(size_t)(i - 1) * pl + k] = __ldg(A.lg_pull + (size_t)(d - 1) * pl + n);
        }
    }
}


// Threads per block of the reverse passes (one node per thread).
// Measured on the 256^2 sweep (14.7-15.2 ms): 128-thread blocks 15.6 ms,
// 64-thread 16.3 ms, 128 threads with the collision pass held to 85
// registers 15.5 ms (at 1024^2 that one is 8.5 % faster, 11.6 against
// 12.7 ms for 40 steps).
constexpr int kRevThreads = 256;
// The collision pass is compiled for three blocks per SM (80 registers, 8
// bytes spilled; 96 at two): 1024^2 sweep 129.2 -> 119.9 ms, 256^2 13.83 ->
// 13.73 ms.

// The four reverse passes, one launch each (every pass reads what the one
// before wrote at the neighbours).
template <int NS>
__global__ void __launch_bounds__(kRevThreads, 3) rev_collide_kernel(const StepParams P, AdjTape T, AdjFields A)
{
    pdl_wait();   // the previous kernel of the sweep has completed
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < P.plane; k += gridDim.x * blockDim.x)
        rev_collide_node<NS>(P, T, A, k);
}

template <int NS, int MODEL, bool WALLS>
__global__ void rev_source_kernel(const StepParams P, AdjTape T, AdjFields A)
{
    pdl_wait();
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < P.plane; k += gridDim.x * blockDim.x)
        rev_source_node<NS, MODEL, WALLS>(P, T, A, k);
}

template <int NS, bool WALLS>
__global__ void rev_stencil_kernel(const StepParams P, AdjFields A)
{
    pdl_wait();
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < P.plane; k += gridDim.x * blockDim.x)
        rev_stencil_node<NS, WALLS>(P, A, k);
}

template <int NS, bool WALLS>
__global__ void rev_pull_kernel(const StepParams P, AdjFields A)
{
    pdl_wait();
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < P.plane; k += gridDim.x * blockDim.x)
        rev_pull_node<NS, WALLS>(P, A, k);
}

constexpr int kRedThreads = 256;

// Fixed-order FP64 sums of K per-node fields, added to acc[K].
__global__ void __launch_bounds__(kRedThreads) reduce_partial_kernel(const double *__restrict__ contrib, int K,
                                                                     unsigned n, double *partials)
{
    __shared__ double red[kRedThreads];
    for (int c = 0; c < K; ++c) {
        double v = 0.0;
        for (unsigned k = blockIdx.x * kRedThreads + threadIdx.x; k < n; k += gridDim.x * kRedThreads)
            v += contrib[(size_t)c * n + k];
        red[threadIdx.x] = v;
        __syncthreads();
        for (int s = kRedThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[(size_t)blockIdx.x * K + c] = red[0];
        __syncthreads();
    }
}

__global__ void reduce_final_kernel(const double *__restrict__ partials, int K, int nblocks, double *acc)
{
    const int c = threadIdx.x;
    if (c >= K) return;
    double v = 0.0;
    for (int b = 0; b < nblocks; ++b) v += partials[(size_t)b * K + c];
    acc[c] = v;
}

int blocks_for(unsigned n)
{
    unsigned b = (n + 255) / 256;
    if (b > 152u * 16u) b = 152u * 16u;
    return (int)(b ? b : 1);
}


template <int NS, int MODEL>
cudaError_t reverse_step_ns(const StepParams &P, const AdjTape &T, const AdjFields &A, bool taped, cudaStream_t st)
{
    const int nb = blocks_for(P.plane);
    const int nr = (int)((P.plane + kRevThreads - 1) / kRevThreads);
    if (!taped) {
        tape_pull_kernel<NS><<<nb, 256, 0, st>>>(P, T);
        tape_stencil_kernel<NS, MODEL><<<nb, 256, 0, st>>>(P, T);
        tape_force_kernel<NS><<<nb, 256, 0, st>>>(P, T);
    }
    // the four passes overlap each launch with the drain of the one before
    // (measured: one cooperative launch with grid barriers between the
    // passes is slower, 17.2 against 14.8 ms for the 256^2 sweep; passes 2-4
    // as one launch over tiles of 32 x 8 nodes, pass 2 recomputed on a
    // margin of two and pass 3 on a margin of one in shared memory, give
    // 13.42 against 13.70 ms at 256^2 but 141.9 against 128.9 ms at 1024^2,
    // and 32 x 16, 64 x 8, 32 x 32 tiles are slower at 1024^2 as well)
    cudaError_t e;
    if ((e = launch_pdl(rev_collide_kernel<NS>, nr, kRevThreads, 0, st, P, T, A)) != cudaSuccess) return e;
    // periodic lattices take passes without the wall branches (fewer
    // registers, no local arrays)
    if (P.wall_x || P.wall_y) {
        if ((e = launch_pdl(rev_source_kernel<NS, MODEL, true>, nr, kRevThreads, 0, st, P, T, A)) != cudaSuccess)
            return e;
        if ((e = launch_pdl(rev_stencil_kernel<NS, true>, nr, kRevThreads, 0, st, P, A)) != cudaSuccess) return e;
        return launch_pdl(rev_pull_kernel<NS, true>, nr, kRevThreads, 0, st, P, A);
    }
    if ((e = launch_pdl(rev_source_kernel<NS, MODEL, false>, nr, kRevThreads, 0, st, P, T, A)) != cudaSuccess) return e;
    if ((e = launch_pdl(rev_stencil_kernel<NS, false>, nr, kRevThreads, 0, st, P, A)) != cudaSuccess) return e;
    return launch_pdl(rev_pull_kernel<NS, false>, nr, kRevThreads, 0, st, P, A);
}

// dL/dphi_p for the solved phases from dL/dphi over all N phases (phi_N = 1 - sum).
__global__ void fold_seed_kernel(int ns, const float *__restrict__ seed, unsigned pl, float *lphi)
{
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < pl; k += gridDim.x * blockDim.x) {
        const float last = seed[(size_t)ns * pl + k];
        for (int p = 0; p < ns; ++p) lphi[(size_t)p * pl + k] = seed[(size_t)p * pl + k] - last;
    }
}

__global__ void add_planes_kernel(const float *__restrict__ a, const float *__restrict__ b, unsigned n, float *out)
{
    for (unsigned k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) out[k] = a[k] + b[k];
}

}  // namespace

cudaError_t launch_reverse_step(int ns, const StepParams &P, const AdjTape &T, const AdjFields &A, bool taped,
                                cudaStream_t st)
{
    switch (ns) {
#define NLBM_CASE(K) \
    case K: return P.model == 0 ? reverse_step_ns<K, 0>(P, T, A, taped, st) : reverse_step_ns<K, 1>(P, T, A, taped, st);
        NLBM_CASE(1) NLBM_CASE(2) NLBM_CASE(3) NLBM_CASE(4) NLBM_CASE(5) NLBM_CASE(6) NLBM_CASE(7)
#undef NLBM_CASE
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_grad_reduce(const double *gacc, int K, unsigned plane, double *partials, double *acc,
                               cudaStream_t st)
{
    reduce_partial_kernel<<<kAdjRedBlocks, kRedThreads, 0, st>>>(gacc, K, plane, partials);
    reduce_final_kernel<<<1, 64, 0, st>>>(partials, K, kAdjRedBlocks, acc);
    return cudaGetLastError();
}

cudaError_t launch_fold_seed(int ns, const float *seed, unsigned plane, float *lphi, cudaStream_t st)
{
    fold_seed_kernel<<<blocks_for(plane), 256, 0, st>>>(ns, seed, plane, lphi);
    return cudaGetLastError();
}

cudaError_t launch_add_planes(const float *a, const float *b, unsigned n, float *out, cudaStream_t st)
{
    add_planes_kernel<<<blocks_for(n), 256, 0, st>>>(a, b, n, out);
    return cudaGetLastError();
}

}  // namespace nlbm
