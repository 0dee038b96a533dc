/*
 * nlbm.h -- C ABI of the GB300 (sm_103a) N-phase conservative Allen-Cahn
 * lattice Boltzmann library.
 *
 * The library advances the consistent and conservative lattice Boltzmann
 * method for immiscible N-phase flow of Zhan, Liu, Chai & Shi (arXiv
 * 2306.06983): N-1 phase-field distribution sets solving the conservative
 * Allen-Cahn equation (Sec. 2.1, Eq. (1), with the Model A source of Eq. (2)
 * or the Model B source of Eqs. (3)-(4)) and one D2Q9 set for the consistent
 * incompressible Navier-Stokes equations (Sec. 2.2, Eqs. (10)-(17)), both
 * with the moment-space MRT collision of Sec. 3-4 (Eqs. (18)-(28)).
 *
 * Conventions for every call:
 *  - All functions return an nlbm_status; none throws, none aborts.  After a
 *    non-OK status, nlbm_last_error() describes the cause.
 *  - Field arrays are single precision, structure of arrays, row-major:
 *    element (c, y, x) of a [C][ny][nx] array is at c*ny*nx + y*nx + x.
 *  - "dev_" pointers are device memory of the GPU that is current when
 *    nlbm_create() is called; "host_" pointers are host memory (pinned or
 *    pageable).  The caller owns all of them; the library never frees caller
 *    memory and keeps no pointer to it after a call returns, except the
 *    workspace given to nlbm_create().
 *  - Asynchronous calls are enqueued on the stream given to nlbm_create() and
 *    return before the GPU work finishes; calls marked "synchronizes" wait
 *    for that stream.
 *  - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef NLBM_H
#define NLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NLBM_OK = 0,
    NLBM_EINVAL = 1,     /* invalid argument or parameter set */
    NLBM_ENOMEM = 2,     /* workspace too small / host allocation failed */
    NLBM_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
    NLBM_ENOTSUP = 4,    /* valid but not supported by this build */
    NLBM_EDIVERGED = 5   /* a phase field became non-finite or left [-0.5, 1.5] */
} nlbm_status;

/* Boundary type of one lattice axis.  NLBM_BC_WALL is the half-way
 * bounce-back wall of Sec. 4 (no-flux for the phase fields, no-slip for the
 * velocity), placed half a spacing outside the first and last node; the
 * stencils of Eq. (27) see mirrored phase fields there. */
typedef enum { NLBM_BC_PERIODIC = 0, NLBM_BC_WALL = 1 } nlbm_bc;

/* Allen-Cahn source term: Model A is Eq. (2) (Lagrange multiplier with
 * exponent n), Model B is Eqs. (3)-(4) (pairwise normals). */
typedef enum { NLBM_MODEL_A = 0, NLBM_MODEL_B = 1 } nlbm_model;

/* Storage precision of the distribution functions (the arithmetic is FP32
 * in every form).  NLBM_STORE_F32 keeps every population in FP32.
 * NLBM_STORE_BF16 / NLBM_STORE_F16 keep the eight moving populations of each
 * set in 16 bits (bfloat16 / IEEE binary16, round to nearest even) as
 * deviations from a lattice-weight multiple of a field the reading node
 * knows: f_i - w_i phi_p(x + c_i) (phi of the node that pulls it, Eq. (19)'s
 * leading term) and g_i - 3 w_i P(x) (the sending node's pressure, Eq. (22)'s
 * leading term).  The rest population of each phase set stays FP32 and is
 * formed so that the values the pullers reconstruct sum to phi_p exactly (up
 * to one FP32 rounding): per-phase volume (Eq. (1)) is conserved as in FP32.
 * 16-bit storage needs an even nx (EINVAL otherwise). */
typedef enum { NLBM_STORE_F32 = 0, NLBM_STORE_BF16 = 1, NLBM_STORE_F16 = 2 } nlbm_storage;

/* The problem statement, in lattice units (dx = dt = 1, c_s^2 = 1/3). */
typedef struct nlbm_params {
    int32_t nx, ny;        /* lattice size, >= 1 each (>= 4 along a wall axis), nx ny <= 2^28 */
    int32_t bc_x, bc_y;    /* nlbm_bc per axis */
    int32_t n_phases;      /* N, 2..8; phases 1..N-1 are solved, phase N is
                              1 - sum (Sec. 4).  At large density ratios make
                              the lightest phase phase N: a three-phase lens
                              at 1000:500:1 settles that way and diverges
                              when the light phase is solved as a set */
    int32_t model;         /* nlbm_model */
    double model_a_n;      /* Model A exponent n > 0 (Eq. (2)); ignored by B */
    double eps;            /* interface thickness epsilon > 0 (Eq. (2)) */
    double mobility;       /* M > 0; tau_f = 0.5 + M / c_s^2 (Eq. (20)) */
    const double *rho;     /* [N] phase densities > 0 (Eq. (11)), host memory */
    const double *mu;      /* [N] dynamic viscosities > 0 (Eq. (12)), host */
    const double *sigma;   /* [N*N] pairwise surface tensions, symmetric,
                              zero diagonal, > 0 off it (Eq. (15)), host */
    double gx, gy;         /* gravity g: the body force F_g = rho g enters the
                              total force F = F_s + F_g + F_c (Sec. 2.2, Sec. 3);
                              finite */
    int32_t storage;       /* nlbm_storage */
    int32_t reserved;      /* must be 0 */
    double unit_delta;     /* >= 0.  Unit vectors of the sources (n_p of
                              Eq. (2), n_pq of Eq. (3)): 0 reads v/|v| as 0
                              when |v|^2 <= 1e-24 (the paper leaves v = 0
                              open); > 0 uses the smooth v / sqrt(|v|^2 +
                              delta^2), which is what a differentiated run
                              needs (see nlbm_adjoint_create) */
    const double *wall_cos;/* NULL, or [2(N-1)] host memory: wetting walls on
                              y (Sec. 4.2, n_w . grad phi_p = sum_{q != p}
                              (4/eps) phi_p phi_q cos theta_pq, n_w pointing
                              into the wall).  Entries 0..N-2 are cos theta_pN
                              (contact angle of phase p against phase N,
                              measured in phase p) of the wall at y = 0,
                              entries N-1..2N-3 those of the wall at
                              y = ny - 1; the pairwise angles follow from
                              Young's relation.  Each |cos| <= 1; nonzero
                              needs bc_y = NLBM_BC_WALL (EINVAL otherwise).
                              NULL or zeros: neutral no-flux walls.  Walls on
                              x stay neutral. */
} nlbm_params;

typedef struct nlbm_sim nlbm_sim;

/* Bytes of device workspace one simulation with these parameters needs.
 * Validates the parameters (EINVAL as nlbm_create would).  Host only, no
 * GPU call. */
nlbm_status nlbm_workspace_bytes(const nlbm_params *p, size_t *bytes);

/* Create a simulation.  dev_workspace: caller-owned device memory of at least
 * nlbm_workspace_bytes() bytes, 256-byte aligned, that must stay valid until
 * nlbm_destroy(); the library lays out the populations (two copies each, pull
 * streaming), the auxiliary fields and reduction scratch in it.
 * cuda_stream: a cudaStream_t (NULL = legacy default stream) on which every
 * later call is enqueued.  The parameters are copied; the caller may free
 * p->rho, p->mu, p->sigma, p->wall_cos afterwards.  The state is undefined until
 * nlbm_set_phi().  Errors: EINVAL (bad parameters, NULL pointers, unaligned
 * or too small workspace, odd nx with 16-bit storage, more than 2^28
 * nodes), ENOMEM (host handle allocation). */
nlbm_status nlbm_create(const nlbm_params *p, void *dev_workspace, size_t workspace_bytes,
                        void *cuda_stream, nlbm_sim **out);

/* Set the initial phase fields and reset the state to the paper's initial
 * condition: dev_phi [N-1][ny][nx] holds phases 1..N-1 (phase N = 1 - sum),
 * the fluid is at rest (u = 0, P = 0), the phase populations are the
 * equilibria w_i phi_p of Eq. (19) and the flow populations those of
 * Eq. (22) with P = 0.  Resets the step counter.  Asynchronous. */
nlbm_status nlbm_set_phi(nlbm_sim *s, const float *dev_phi);

/* Start the simulation in motion: after nlbm_set_phi() and before the first
 * step, give the fluid the velocity dev_u [2][ny][nx] (u_x plane, then u_y;
 * device memory, read before the call's work completes on the stream).  The
 * paper starts every case at rest and gives no initial state in motion; this
 * one is the equilibrium of each set at u (Eqs. (19), (22)) with
 * m = rho u + m_phi, m_phi of the initial fields (Eq. (13)), the pressure in
 * lambda_i chosen so that Eq. (25c) recovers P = 0 from these populations,
 * and the initial values as the previous values of the first step's time
 * derivatives (u(-1) = u, phi(-1) = phi(0), m_phi(-1) = m_phi(0)), so that a
 * flow in steady translation starts without a jump.  FP32 storage and no
 * wetting walls (else ENOTSUP); EINVAL after a step has been taken.  Two
 * kernel launches on the simulation's stream. */
nlbm_status nlbm_set_velocity(nlbm_sim *s, const float *dev_u);

/* As nlbm_set_phi() with host_phi [N-1][ny][nx] in host memory; the copy is
 * enqueued on the simulation's stream (synchronizes when host_phi is
 * pageable). */
nlbm_status nlbm_set_phi_host(nlbm_sim *s, const float *host_phi);

/* Advance nsteps >= 0 time steps (Sec. 3: one fused pull-stream, stencil
 * (Eq. (27)), source (Eqs. (2)-(4)), surface-tension (Eqs. (16)-(17)),
 * macroscopic (Eqs. (25)) and MRT collision (Eqs. (18)-(24), (28)) pass per
 * step).  Asynchronous; one kernel launch per step. */
nlbm_status nlbm_step(nlbm_sim *s, int64_t nsteps);

/* Macroscopic fields of the most recent step (the values the last step
 * computed before its collision; after nlbm_set_phi() and no step: the
 * initial phi, u = 0, P = 0).  dev_phi [N][ny][nx] (all N phases),
 * dev_u [2][ny][nx] (u_x then u_y, Eq. (25b)), dev_p [ny][nx] (Eq. (25c)).
 * Any pointer may be NULL.  Asynchronous. */
nlbm_status nlbm_get_moments(nlbm_sim *s, float *dev_phi, float *dev_u, float *dev_p);

/* As nlbm_get_moments() into host memory; synchronizes. */
nlbm_status nlbm_get_moments_host(nlbm_sim *s, float *host_phi, float *host_u, float *host_p);

/* Per-phase volume sum_x phi_p of the most recent step's phase fields,
 * accumulated in FP64 with a fixed reduction order (bitwise reproducible),
 * into host_mass [N].  Returns EDIVERGED (masses still written) when any
 * phi_p is non-finite or outside [-0.5, 1.5].  Synchronizes. */
nlbm_status nlbm_phase_mass(nlbm_sim *s, double *host_mass);

/* Bytes of a checkpoint of the full state (populations, auxiliary fields,
 * last moments).  Host only. */
nlbm_status nlbm_state_bytes(const nlbm_sim *s, size_t *bytes);

/* Copy the full state (populations, auxiliary fields, last moments and the
 * step counter) into / from caller device memory of nlbm_state_bytes()
 * bytes, 16-byte aligned.  Both synchronize (the step counter travels
 * through host memory).  Restore returns EINVAL if the buffer does not carry
 * the checkpoint tag written by nlbm_save(). */
nlbm_status nlbm_save(nlbm_sim *s, void *dev_dst);
nlbm_status nlbm_restore(nlbm_sim *s, const void *dev_src);

/* Wait for all work enqueued by this simulation.  Synchronizes. */
nlbm_status nlbm_synchronize(nlbm_sim *s);

/* Steps taken since nlbm_set_phi() (or the restored checkpoint). */
int64_t nlbm_steps_done(const nlbm_sim *s);

/* Number of kernels this handle has launched since creation. */
int64_t nlbm_kernel_launches(const nlbm_sim *s);

/* Tile of the fused step kernel: tx threads per block (64, 128 or 256; one
 * thread per column, each block updating a strip of tx - 4 columns) marching
 * down ty rows (>= 1), or ty = 0 (the default) to let the library cut every
 * strip into equal row chunks (at least 2 rows) so that the grid is one
 * wave of resident blocks.  EINVAL outside those values.  Takes effect on
 * the next nlbm_step(). */
nlbm_status nlbm_set_tile(nlbm_sim *s, int32_t tx, int32_t ty);
nlbm_status nlbm_get_tile(const nlbm_sim *s, int32_t *tx, int32_t *ty);

/* Tile autotuner: for every tile shape tx in {64, 128, 256} (wider strips
 * than the lattice needs are skipped) x ty in {0, 8, 12, 16, 20, 24, 32,
 * 48}, one untimed step and then steps_per_trial (>= 1) steps timed with
 * CUDA events on the simulation's stream, each trial from the state saved
 * in dev_scratch (device memory, 16-byte aligned, at least
 * nlbm_state_bytes()); keeps the fastest shape.  The result of a step does
 * not depend on the tile (every node is computed by the same code from the
 * same inputs), and the state and step counter are those of the call on
 * return; the trial launches count in nlbm_kernel_launches().  Any output
 * pointer may be NULL.  ENOMEM when the scratch is too small.
 * Synchronizes. */
nlbm_status nlbm_autotune(nlbm_sim *s, void *dev_scratch, size_t scratch_bytes, int32_t steps_per_trial,
                          int32_t *best_tx, int32_t *best_ty, float *best_ms_per_step);

/* Per-phase volume sum_x phi_p, p = 1..N, for callers that cannot allocate
 * device memory at all -- neither through this library's workspace nor their
 * own allocator: code that runs where cudaMalloc is forbidden or unsafe (a
 * real-time loop with a fixed memory budget, a plugin handed only the
 * pointers it computes on, a host callback).  The paper has no counterpart;
 * it is the reduction of nlbm_phase_mass() with its scratch moved into the
 * library.
 *   dev_phi  [n_phases-1][n_nodes] float, phases 1..N-1 (phase N = 1 - sum),
 *            e.g. the first N-1 planes written by nlbm_get_moments();
 *   dev_mass [n_phases] double, written: the volumes, FP64-accumulated in a
 *            fixed order (bitwise equal to nlbm_phase_mass() on the same
 *            fields);
 *   dev_flag [1] int32, written: 1 if any value is non-finite or outside
 *            [-0.5, 1.5], else 0.
 * The reduction's FP64 partial sums live in one file-scope device array of
 * 512 x 9 doubles (36.9 KB) that every GPU which loads the library keeps
 * until the process exits; the call allocates nothing and never calls
 * cudaMalloc or cudaFree.  n_phases must be 2..8 and n_nodes 1..2^28;
 * larger sizes are rejected with NLBM_EINVAL (and one line on stderr)
 * before any GPU work.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress, with the device current); make it
 * before any stream capture.  The address is cached per device together with
 * the context it was taken in, and looked up again when a call runs in
 * another context (a caller-created driver context, or the primary context
 * re-created after cudaDeviceReset(), which discards the array's contents
 * and may move it; after a reset the cached address is never reused unless
 * the driver hands out the same context handle again, so make the first
 * call after a reset outside stream capture too).  All calls share the array:
 * every entry the reduction reads it has first written in the same call, so
 * nothing needs clearing, but calls that overlap on the GPU (other streams,
 * other host threads) race on it -- serialise them.  Asynchronous on
 * cuda_stream (a cudaStream_t, NULL = legacy default stream). */
nlbm_status nlbm_phase_mass_noalloc(const float *dev_phi, int32_t n_phases, int64_t n_nodes,
                                    double *dev_mass, int32_t *dev_flag, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Ensembles: many independent simulations advanced together.
 *
 * Each member is the problem nlbm_create() takes (Secs. 2-4), with its own
 * lattice size, boundaries, model (A or B, any exponent n), densities,
 * viscosities, surface tensions, epsilon and mobility -- the kind of sweep
 * the paper runs case by case (the Model A exponents of Sec. 4, the lens
 * tension ratios of Sec. 4.3, Table 3).  Members share N and FP32 storage.
 * One persistent kernel launch per step advances every member: the blocks
 * resident on the GPU take (member, column strip, row chunk) tiles from a
 * table ordered largest member first.  Steps of nlbm_batch_step() are
 * replayed from a captured two-step CUDA graph when the stream is not the
 * legacy default stream.  Members never exchange data.
 * ------------------------------------------------------------------------ */
typedef struct nlbm_batch nlbm_batch;

/* Device workspace bytes for `count` (1..4096) members sims[0..count-1]
 * (validated as nlbm_workspace_bytes() does; EINVAL if N differs between
 * members, ENOTSUP for 16-bit storage).  Host only. */
nlbm_status nlbm_batch_workspace_bytes(const nlbm_params *sims, int32_t count, size_t *bytes);

/* Create an ensemble in caller-owned device memory (256-byte aligned, at
 * least nlbm_batch_workspace_bytes()); cuda_stream as for nlbm_create().
 * The member parameters are copied.  Errors as nlbm_create(). */
nlbm_status nlbm_batch_create(const nlbm_params *sims, int32_t count, void *dev_workspace,
                              size_t workspace_bytes, void *cuda_stream, nlbm_batch **out);

/* Initial phase fields of member `sim`, as nlbm_set_phi() (dev_phi
 * [N-1][ny][nx] of that member).  Asynchronous.  Does not reset the other
 * members or the ensemble's step counter. */
nlbm_status nlbm_batch_set_phi(nlbm_batch *b, int32_t sim, const float *dev_phi);

/* Advance every member nsteps >= 0 steps: one launch per step, all but the
 * last from the captured graph.  Asynchronous. */
nlbm_status nlbm_batch_step(nlbm_batch *b, int64_t nsteps);

/* Moments of member `sim` as nlbm_get_moments() (asynchronous) and its
 * per-phase volumes as nlbm_phase_mass() (synchronizes). */
nlbm_status nlbm_batch_get_moments(nlbm_batch *b, int32_t sim, float *dev_phi, float *dev_u, float *dev_p);
nlbm_status nlbm_batch_phase_mass(nlbm_batch *b, int32_t sim, double *host_mass);

/* Tile shape of the ensemble kernel: tx threads per block (64, 128, 256;
 * strips of tx - 4 columns) and ty rows per tile (>= 1, 0 = 32).  Rebuilds
 * the tile table (synchronizes).  get_tile also returns the tile count. */
nlbm_status nlbm_batch_set_tile(nlbm_batch *b, int32_t tx, int32_t ty);
nlbm_status nlbm_batch_get_tile(const nlbm_batch *b, int32_t *tx, int32_t *ty, int32_t *ntiles);

/* Bytes of all members' state (the scratch nlbm_batch_autotune() needs). */
nlbm_status nlbm_batch_state_bytes(const nlbm_batch *b, size_t *bytes);

/* Autotuner: time steps_per_trial (>= 1) ensemble steps (after one untimed
 * step) for every tile shape tx in {64, 128, 256} x ty in {8, 16, 32, 64,
 * 128} with CUDA events, restoring the state from dev_scratch (device
 * memory of at least nlbm_batch_state_bytes()) after each trial, and keep
 * the fastest.  The state and step counter are unchanged on return; any
 * output pointer may be NULL.  Synchronizes. */
nlbm_status nlbm_batch_autotune(nlbm_batch *b, void *dev_scratch, size_t scratch_bytes,
                                int32_t steps_per_trial, int32_t *best_tx, int32_t *best_ty,
                                float *best_ms_per_step);

nlbm_status nlbm_batch_synchronize(nlbm_batch *b);
int64_t nlbm_batch_steps_done(const nlbm_batch *b);
/* Kernels this ensemble has launched (graph replays count their launches). */
int64_t nlbm_batch_kernel_launches(const nlbm_batch *b);
/* Release the ensemble (not the workspace).  Safe on NULL. */
void nlbm_batch_destroy(nlbm_batch *b);
/* Text of the ensemble's last error (b may be NULL: last failed create). */
const char *nlbm_batch_last_error(const nlbm_batch *b);

/* ------------------------------------------------------------------------
 * Adjoint: gradients of a loss of the final phase fields.
 *
 * For L(phi(T)) after T steps of the problem p from phi_0, the reverse sweep
 * gives dL/dphi_0, dL/dsigma_pq (Eq. (15) tensions, through the chemical
 * potentials of Eq. (17)) and dL/dM (through tau_f, Eq. (20), and m_phi,
 * Eq. (13)).  Each step is reversed by rebuilding its intermediate fields
 * from its input state and taking the adjoint through its stages in
 * reverse order (collisions, Eqs. (18)-(24); force and macroscopic fields,
 * Eqs. (16), (25); the source, Model A Eq. (2) or Model B Eqs. (3)-(4); the
 * stencils, Eq. (27); streaming); states are checkpointed every
 * `checkpoint_every` steps and each segment is recomputed during the sweep.
 * Supported: Models A and B, periodic axes or half-way bounce-back walls
 * without wetting (all contact angles 90 degrees), gravity, FP32 storage
 * (ENOTSUP otherwise: wetting walls, 16-bit storage).  Model A's weight max(phi, 0)^n has the
 * derivative n phi^(n-1) for phi > 0 and 0 below, so with n < 1 gradients
 * through nodes where a phase tends to 0+ are unbounded.  Unit vectors
 * should use the smooth reading (p->unit_delta > 0, e.g. 1e-3): with the
 * thresholded one the step is not differentiable where v passes through 0.
 * ------------------------------------------------------------------------ */
typedef struct nlbm_adjoint nlbm_adjoint;

/* Device workspace bytes for nsteps >= 1 steps with a checkpoint every
 * checkpoint_every >= 1 steps: the simulation, ceil(nsteps / every)
 * checkpoints and every + 1 segment states of 10(N-1)+12 floats a node,
 * `every` tapes of the segment's steps (8(N-1)+13 floats a node), the
 * adjoint fields.  Host only. */
nlbm_status nlbm_adjoint_workspace_bytes(const nlbm_params *p, int32_t nsteps, int32_t checkpoint_every,
                                         size_t *bytes);

/* Create a differentiable run in caller-owned device memory (256-byte
 * aligned, at least nlbm_adjoint_workspace_bytes()); cuda_stream as for
 * nlbm_create(). */
nlbm_status nlbm_adjoint_create(const nlbm_params *p, int32_t nsteps, int32_t checkpoint_every,
                                void *dev_workspace, size_t workspace_bytes, void *cuda_stream,
                                nlbm_adjoint **out);

/* Run the nsteps forward steps from dev_phi0 [N-1][ny][nx] (as
 * nlbm_set_phi()), storing the checkpoints; write phi(T) [N][ny][nx] into
 * dev_phi_final if non-NULL.  Asynchronous. */
nlbm_status nlbm_adjoint_forward(nlbm_adjoint *a, const float *dev_phi0, float *dev_phi_final);

/* Reverse sweep after nlbm_adjoint_forward(): dev_seed [N][ny][nx] is
 * dL/dphi(T) over all N phases (phase N = 1 - sum is folded in).  Writes
 * dL/dphi_0 [N-1][ny][nx] into dev_grad_phi0 (may be NULL), dL/dsigma into
 * host_grad_sigma [N*N] (symmetric: entry (p, q) is the derivative with
 * respect to the pair's single value; may be NULL) and dL/dM into
 * *host_grad_mobility (may be NULL).  The sweep is the same launch sequence
 * on every call of a handle: on a stream other than the legacy default one,
 * the first call captures it into a CUDA graph (kernel loading and capture
 * take a while once) and later calls replay it.  Synchronizes. */
nlbm_status nlbm_adjoint_backward(nlbm_adjoint *a, const float *dev_seed, float *dev_grad_phi0,
                                  double *host_grad_sigma, double *host_grad_mobility);

/* One reverse step on its own, for losses spread over time: dev_state is a
 * step's input state [f 9(N-1), g 8, u 2, phi N-1, m_phi 2 planes] (the
 * first planes of an nlbm_save() checkpoint), dev_seed_out the adjoint of
 * its outputs [f 9(N-1), g 8, phi N-1, u 2, m_phi 2 planes]; writes the
 * adjoint of its inputs in the seed layout to dev_seed_in and this step's
 * parameter gradients to the host arrays (as nlbm_adjoint_backward()).
 * Synchronizes. */
nlbm_status nlbm_adjoint_reverse_step(nlbm_adjoint *a, const float *dev_state, const float *dev_seed_out,
                                      float *dev_seed_in, double *host_grad_sigma, double *host_grad_mobility);

/* 1 when the reverse sweep of this handle replays a captured graph. */
int32_t nlbm_adjoint_uses_graph(const nlbm_adjoint *a);
/* Kernels launched by the handle (forward, recompute and reverse). */
int64_t nlbm_adjoint_kernel_launches(const nlbm_adjoint *a);
/* Release the handle (not the workspace).  Safe on NULL. */
void nlbm_adjoint_destroy(nlbm_adjoint *a);
/* Text of the handle's last error (a may be NULL: last failed create). */
const char *nlbm_adjoint_last_error(const nlbm_adjoint *a);

/* Release the handle (not the workspace).  Safe on NULL.  Does not wait for
 * enqueued work; synchronize first if the workspace is to be reused. */
void nlbm_destroy(nlbm_sim *s);

/* Text of the last error of this handle ("" if none); s may be NULL for the
 * last error of a failed nlbm_create / nlbm_workspace_bytes on this thread. */
const char *nlbm_last_error(const nlbm_sim *s);

/* Static text of a status code. */
const char *nlbm_status_string(nlbm_status st);

#ifdef __cplusplus
}
#endif

#endif /* NLBM_H */
