// Internal declarations shared by the CUDA translation units of libnlbm.
//
// Lattice: D2Q9 with the velocity order of the columns of the moment matrix
// in Eq. (28): c0 = (0,0), c1 = (1,0), c2 = (0,1), c3 = (-1,0), c4 = (0,-1),
// c5 = (1,1), c6 = (-1,1), c7 = (-1,-1), c8 = (1,-1); weights 4/9, 1/9, 1/36;
// c_s^2 = 1/3 (Sec. 4).
//
// Storage (structure of arrays, one plane = nx*ny floats, row-major):
//   f  [N-1][9][plane]  post-collision phase populations (pull streaming:
//                       node x reads f*_i(x - c_i) of the previous step)
//   g  [8][plane]       post-collision flow populations g_1..g_8; g_0 is
//                       never stored: rows 1..8 of M^-1 have a zero in
//                       column 0, so g_0 feeds neither u (c_0 = 0) nor P
//                       (Eq. (25c) sums i != 0) nor any later g_i.
//   phi [N-1][plane]    phi_p of the last step (the "previous" value for the
//                       backward-Euler time derivatives of the next step)
//   u   [2][plane]      velocity of the last step (double-buffered: the next
//                       step reads it at neighbours for F_c)
//   mphi [2][plane]     m_phi of the last step
//   P   [plane]         pressure, written on request
// With 16-bit storage (bfloat16 or binary16) the moving populations are kept
// as deviations, 2 bytes each (f: phases 2q and 2q + 1 share a 32-bit word
// per direction and node, [(N-1)/2][8][plane] words, an odd last phase in
// [8][plane] 16-bit planes after them; g [8][plane]), the rest populations
// f0 [N-1][plane] in FP32, and phi and P are double-buffered: the puller adds
// w_i phi(puller, t) and 3 w_i P(source, t) back.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace nlbm {

constexpr int kMaxPhases = 8;

struct StepParams {
    int nx, ny;
    int wall_x, wall_y;
    unsigned plane;            // floats per field plane (nx*ny)
    float drho[kMaxPhases];    // rho_p - rho_N, p = 1..N-1
    float rhoN;
    float dmu[kMaxPhases];     // mu_p - mu_N
    float muN;
    float beta2[kMaxPhases][kMaxPhases];  // 2 beta_pq = 6 sigma_pq / eps (Eq. (15))
    float kap[kMaxPhases][kMaxPhases];    // -k_pq = 3 eps sigma_pq / 4 (Eq. (15))
    float four_over_eps;       // 4 / eps
    float unit_delta2;         // delta^2 of the smooth unit vector (0: thresholded reading)
    float six_over_eps;        // d beta2 / d sigma (adjoint)
    float three_eps_over_4;    // d kap / d sigma (adjoint)
    float mob;                 // M
    float s1;                  // 1 / tau_f, tau_f = 0.5 + 3 M (Eq. (20))
    float model_n;             // Model A exponent n
    int model_n_int;           // n when it is an integer in 1..8, else 0
    const float *fin;          // FP32: [N-1][9][plane]; 16-bit: deviations (see above)
    float *fout;
    const float *f0in;         // 16-bit storage only: FP32 rest populations [N-1][plane]
    float *f0out;
    const float *gin;          // FP32: [8][plane]; 16-bit: [8][plane] deviations
    float *gout;
    float *phi;                // [N-1][plane] phi of this step (FP32: in place over phi_prev)
    const float *phi_prev;     // [N-1][plane] phi of the previous step
    const float *pin;          // 16-bit storage only: P of the previous step
    const float *uin;          // [2][plane] previous step
    float *uout;               // [2][plane] this step
    float *mphi;               // [2][plane] m_phi of this step (out)
    const float *mphi_in;      // [2][plane] m_phi of the previous step (equal to mphi: updated in place)
    float *pout;               // [plane] or nullptr
    int model;                 // 0 Model A, 1 Model B (read by the ensemble kernel)
    int row_window;            // ensemble kernel: stage pulls as row windows (see step_tile)
    float *tape;               // adjoint recompute: the step's intermediate fields (launch_step_tape)
    float gx, gy;              // gravity: F_g = rho g
    int wet;                   // a y wall has a contact angle other than 90 degrees
    float wetc[2][kMaxPhases][kMaxPhases];   // (4/eps) cos theta_pq, walls y = 0 and y = ny - 1
};

// Programmatic dependent launch (the step kernels, the ensemble kernel and the
// adjoint's reverse passes): a kernel launched with launch_pdl is scheduled
// as the blocks of its
// predecessor in the stream exit, so its launch overlaps their drain.  It
// must call pdl_wait() before touching memory the predecessor reads or
// writes; the wait returns once the predecessor has completed and its writes
// are visible.  Launched without the attribute, the wait does nothing.
// (Measured: the 256^2 adjoint's reverse sweep 15.5 -> 15.0 ms as a graph,
// 20.6 -> 15.1 ms as plain launches, its forward 6.5 -> 5.5 ms; 64 lens
// simulations launched one by one 4,773 -> 5,671 MLUPS.  Releasing successors
// at the start of each kernel instead of at block exit made the adjoint's
// graph slower, 17.3 ms.)
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// One work item of the ensemble kernel: the strip of simulation `sim` that
// starts at column x0, rows [y0, y0 + ty).
struct BatchTile {
    int sim, x0, y0, ty;
};

// Launchers (defined in step_{a,b}_{f32,bf16,f16}.cu: Model A / B, FP32
// populations or 16-bit deviations).  smem bytes and grid are computed by
// the launcher; returns the launch error.
cudaError_t launch_step_a_f32(int ns, const StepParams &p, int tx, int ty, cudaStream_t st);
cudaError_t launch_step_b_f32(int ns, const StepParams &p, int tx, int ty, cudaStream_t st);
cudaError_t launch_step_a_bf16(int ns, const StepParams &p, int tx, int ty, cudaStream_t st);
cudaError_t launch_step_b_bf16(int ns, const StepParams &p, int tx, int ty, cudaStream_t st);
cudaError_t launch_step_a_f16(int ns, const StepParams &p, int tx, int ty, cudaStream_t st);
cudaError_t launch_step_b_f16(int ns, const StepParams &p, int tx, int ty, cudaStream_t st);

// The FP32 step (128-thread blocks) that also writes the step's
// intermediate fields for the adjoint to p.tape, 8 (N-1) + 13 planes in the
// order of AdjTape: phi [N-1], j [2(N-1)], pulled g [8], grad phi [2(N-1)],
// lap phi [N-1], R [2(N-1)], m_phi [2], w [1], F [2]; Model A in
// step_a_f32_tape.cu, Model B in step_b_f32_tape.cu.
cudaError_t launch_step_tape_a_f32(int ns, const StepParams &p, cudaStream_t st);
cudaError_t launch_step_tape_b_f32(int ns, const StepParams &p, cudaStream_t st);

// Ensemble of independent simulations (batch.cu): one persistent launch
// advances every simulation of the table one step; blocks take tiles from
// d_tiles through the counter d_counters[parity] and clear the other one.
cudaError_t launch_batch_step(int ns, int tx, const StepParams *d_params, const BatchTile *d_tiles,
                              int ntiles, int *d_counters, int parity, cudaStream_t st);

// Auxiliary kernels (aux_kernels.cu).
cudaError_t launch_init(int ns, const StepParams &p, cudaStream_t st);
// A state in motion (velocity.cu): p describes the state set by launch_init
// (p.phi, p.fout, p.gout, p.mphi); u0 [2][plane] the velocity, u_prev the
// velocity buffer the first step reads as its previous one, p_scratch one
// plane the first step overwrites.  FP32 storage.
cudaError_t launch_velocity_state(int ns, int model, const StepParams &p, const float *u0, float *u_prev,
                                  float *p_scratch, cudaStream_t st);
cudaError_t launch_export(int ns, const float *phi_aux, const float *u, const float *P,
                          unsigned plane, float *phi_out, float *u_out, float *p_out,
                          cudaStream_t st);
constexpr int kMassBlocks = 512;   // fixed grid: the reduction order is fixed
cudaError_t launch_phase_mass(int ns, const float *phi_aux, unsigned plane, double *partials,
                              double *mass_out, int *flag_out, cudaStream_t st);

}  // namespace nlbm
