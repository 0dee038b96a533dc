// Fields of the reverse (adjoint) step (adjoint.cu).  Every array is
// structure of arrays, [components][plane] FP32.
#pragma once

#include "nlbm_internal.cuh"

namespace nlbm {

constexpr int kAdjRedBlocks = 256;   // fixed grid: fixed FP64 summation order

// Intermediate fields of one forward step, rebuilt from its input state.
struct AdjTape {
    float *phi;    // [N-1]  phi_p (Eq. (25a))
    float *j;      // [2(N-1)] j_p = sum c_i f_i
    float *g;      // [8]    pulled flow populations g_1..g_8
    float *grad;   // [2(N-1)] grad phi_p (Eq. (27))
    float *lap;    // [N-1]  lap phi_p (Eq. (27))
    float *R;      // [2(N-1)] Model B source (Eqs. (3), (4))
    float *mphi;   // [2]    m_phi (Eq. (13))
    float *w;      // [1]    m_phi,x u_y - u_x m_phi,y (previous velocity)
    float *F;      // [2]    F_s + F_c
};

// Adjoint variables.  *_out: adjoints of this step's outputs (the seed);
// *_in: adjoints of its inputs (the seed of the previous step); the rest
// are per-step intermediates.
struct AdjFields {
    const float *lf_out;   // [9(N-1)] post-collision phase populations
    const float *lg_out;   // [8]      post-collision flow populations g_1..g_8
    const float *lphi_out; // [N-1]    phi(t) (the next step's phi_prev, and the loss)
    const float *lu_out;   // [2]      u(t)
    const float *lm_out;   // [2]      m_phi(t)
    float *lf_in, *lg_in, *lphi_in, *lu_in, *lm_in;
    float *lF;       // [2]
    float *lphi_pw;  // [N-1] pointwise part of the phi adjoint
    float *lj;       // [2(N-1)]
    float *lgrad;    // [2(N-1)]
    float *llap;     // [N-1]
    float *lR;       // [2(N-1)]
    float *lmphi;    // [2]
    float *lg_pull;  // [8]
    float *lphi_tot; // [N-1]
    double *gacc;    // [N(N-1)/2 + 1] per-node sums over the steps of dL/dsigma_pq
                     // (pair order p<q) and dL/dM, FP64
};

// Tape and reverse of one step whose input state P describes (P.fin, P.gin,
// P.phi_prev, P.uin, P.mphi); adds this step's parameter-gradient terms to
// A.gacc node by node.  taped: T already holds the step's intermediate
// fields (written by the taping forward kernel), so only the four reverse
// passes run.
cudaError_t launch_reverse_step(int ns, const StepParams &P, const AdjTape &T, const AdjFields &A, bool taped,
                                cudaStream_t st);
// acc[c] = sum over nodes of gacc[c][node], c < K, in a fixed order (FP64).
cudaError_t launch_grad_reduce(const double *gacc, int K, unsigned plane, double *partials, double *acc,
                               cudaStream_t st);
// lphi[p] = seed[p] - seed[N-1] for the N-1 solved phases.
cudaError_t launch_fold_seed(int ns, const float *seed, unsigned plane, float *lphi, cudaStream_t st);
// out = a + b over n floats.
cudaError_t launch_add_planes(const float *a, const float *b, unsigned n, float *out, cudaStream_t st);

}  // namespace nlbm
