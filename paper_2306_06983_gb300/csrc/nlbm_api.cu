// Host side of the C ABI declared in include/nlbm.h: parameter validation,
// workspace layout, kernel dispatch and checkpoints.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstdint>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include "../../include/nlbm.h"
#include "nlbm_internal.cuh"
#include "adjoint.cuh"

using namespace nlbm;

namespace {

thread_local char g_err[512] = "";

constexpr size_t kMaxPlane = (size_t)1 << 28;   // keeps 9 * plane in 32-bit offsets

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace layout.  FP32 storage: two copies of f [N-1][9] and g [8]
// planes, phi and P single (phi is updated in place, P written on request).
// 16-bit storage: two copies of the f deviations [N-1][8], the FP32 rest
// populations f0 [N-1], the g deviations [8], phi and P.  f[k] and g[k] are
// adjacent, so an idle f/g pair can stage N + 3 planes for host downloads.
struct Layout {
    size_t f[2], g[2], f0[2], phi[2], u[2], mphi, P[2], partials, mass, total;
    size_t fbytes, gbytes;
};

Layout make_layout(int ns, size_t plane, bool half)
{
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t es = half ? 2 : 4;
    L.fbytes = es * ns * (half ? 8 : 9) * plane;
    L.gbytes = es * 8 * plane;
    for (int k = 0; k < 2; ++k) {
        L.f[k] = take(L.fbytes);
        L.g[k] = take(L.gbytes);
    }
    for (int k = 0; k < 2; ++k) L.f0[k] = half ? take(sizeof(float) * ns * plane) : 0;
    L.phi[0] = take(sizeof(float) * ns * plane);
    L.phi[1] = half ? take(sizeof(float) * ns * plane) : L.phi[0];
    L.u[0] = take(sizeof(float) * 2 * plane);
    L.u[1] = take(sizeof(float) * 2 * plane);
    L.mphi = take(sizeof(float) * 2 * plane);
    L.P[0] = take(sizeof(float) * plane);
    L.P[1] = half ? take(sizeof(float) * plane) : L.P[0];
    L.partials = take(sizeof(double) * kMassBlocks * (ns + 2));
    L.mass = take(sizeof(double) * (ns + 2) + sizeof(int));
    L.total = off;
    return L;
}

bool is_half(int storage) { return storage == NLBM_STORE_BF16 || storage == NLBM_STORE_F16; }

void set_err(char *buf, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0.0; }

// Validates the problem statement; fills the derived kernel parameters.
nlbm_status validate(const nlbm_params *p, StepParams *kp, char *err)
{
    if (!p) { set_err(err, "params is NULL"); return NLBM_EINVAL; }
    const int N = p->n_phases;
    if (N < 2 || N > kMaxPhases) { set_err(err, "n_phases=%d outside 2..%d", N, kMaxPhases); return NLBM_EINVAL; }
    if (p->nx < 1 || p->ny < 1) { set_err(err, "lattice %dx%d is empty", p->nx, p->ny); return NLBM_EINVAL; }
    if ((p->bc_x != NLBM_BC_PERIODIC && p->bc_x != NLBM_BC_WALL) ||
        (p->bc_y != NLBM_BC_PERIODIC && p->bc_y != NLBM_BC_WALL)) {
        set_err(err, "unknown boundary type"); return NLBM_EINVAL;
    }
    if ((p->bc_x == NLBM_BC_WALL && p->nx < 4) || (p->bc_y == NLBM_BC_WALL && p->ny < 4)) {
        set_err(err, "a wall axis needs at least 4 nodes"); return NLBM_EINVAL;
    }
    if ((size_t)p->nx * (size_t)p->ny > kMaxPlane) {
        set_err(err, "lattice of %zu nodes exceeds %zu", (size_t)p->nx * p->ny, kMaxPlane);
        return NLBM_EINVAL;
    }
    if (p->model != NLBM_MODEL_A && p->model != NLBM_MODEL_B) { set_err(err, "unknown model"); return NLBM_EINVAL; }
    if (p->model == NLBM_MODEL_A && !finite_pos(p->model_a_n)) { set_err(err, "Model A exponent n must be > 0"); return NLBM_EINVAL; }
    if (!finite_pos(p->eps)) { set_err(err, "eps must be > 0"); return NLBM_EINVAL; }
    if (!finite_pos(p->mobility)) { set_err(err, "mobility must be > 0"); return NLBM_EINVAL; }
    if (!p->rho || !p->mu || !p->sigma) { set_err(err, "rho, mu and sigma must be given"); return NLBM_EINVAL; }
    for (int a = 0; a < N; ++a) {
        if (!finite_pos(p->rho[a])) { set_err(err, "rho[%d] must be > 0", a); return NLBM_EINVAL; }
        if (!finite_pos(p->mu[a])) { set_err(err, "mu[%d] must be > 0", a); return NLBM_EINVAL; }
        for (int b = 0; b < N; ++b) {
            const double s = p->sigma[a * N + b];
            if (a == b && s != 0.0) { set_err(err, "sigma[%d][%d] must be 0", a, a); return NLBM_EINVAL; }
            if (a != b && !finite_pos(s)) { set_err(err, "sigma[%d][%d] must be > 0", a, b); return NLBM_EINVAL; }
            if (s != p->sigma[b * N + a]) { set_err(err, "sigma is not symmetric at (%d,%d)", a, b); return NLBM_EINVAL; }
        }
    }
    if (p->reserved != 0) { set_err(err, "reserved must be 0"); return NLBM_EINVAL; }
    if (!std::isfinite(p->unit_delta) || p->unit_delta < 0.0) { set_err(err, "unit_delta must be >= 0"); return NLBM_EINVAL; }
    if (!std::isfinite(p->gx) || !std::isfinite(p->gy)) { set_err(err, "gravity not finite"); return NLBM_EINVAL; }
    bool wet = false;
    if (p->wall_cos) {
        for (int a = 0; a < 2 * (N - 1); ++a) {
            const double c = p->wall_cos[a];
            if (!(std::fabs(c) <= 1.0)) { set_err(err, "wall_cos[%d] must lie in [-1, 1]", a); return NLBM_EINVAL; }
            if (c != 0.0) wet = true;
        }
        if (wet && p->bc_y != NLBM_BC_WALL) { set_err(err, "wall_cos needs walls on y"); return NLBM_EINVAL; }
    }
    if (p->storage != NLBM_STORE_F32 && !is_half(p->storage)) { set_err(err, "unknown storage"); return NLBM_EINVAL; }
    if (is_half(p->storage) && (p->nx & 1)) {
        set_err(err, "16-bit storage needs an even nx (got %d)", p->nx); return NLBM_EINVAL;
    }
    if (kp) {
        memset(kp, 0, sizeof *kp);
        kp->nx = p->nx;
        kp->ny = p->ny;
        kp->wall_x = p->bc_x == NLBM_BC_WALL;
        kp->wall_y = p->bc_y == NLBM_BC_WALL;
        kp->model = p->model;
        kp->plane = (unsigned)((size_t)p->nx * p->ny);
        const double rhoN = p->rho[N - 1], muN = p->mu[N - 1];
        kp->rhoN = (float)rhoN;
        kp->muN = (float)muN;
        for (int a = 0; a < N - 1; ++a) {
            kp->drho[a] = (float)(p->rho[a] - rhoN);
            kp->dmu[a] = (float)(p->mu[a] - muN);
        }
        for (int a = 0; a < N; ++a)
            for (int b = 0; b < N; ++b) {
                const double s = p->sigma[a * N + b];
                kp->beta2[a][b] = (float)(6.0 * s / p->eps);       // 2 beta_pq, Eq. (15)
                kp->kap[a][b] = (float)(0.75 * p->eps * s);        // -k_pq, Eq. (15)
            }
        kp->four_over_eps = (float)(4.0 / p->eps);
        kp->unit_delta2 = (float)(p->unit_delta * p->unit_delta);
        kp->six_over_eps = (float)(6.0 / p->eps);
        kp->three_eps_over_4 = (float)(0.75 * p->eps);
        kp->mob = (float)p->mobility;
        kp->s1 = (float)(1.0 / (0.5 + 3.0 * p->mobility));        // Eq. (20), c_s^2 = 1/3
        kp->model_n = (float)p->model_a_n;
        kp->gx = (float)p->gx;
        kp->gy = (float)p->gy;
        // Sec. 4.2: cos theta_pq from the N-1 angles against phase N by
        // Young's relation, cos theta_qp = -cos theta_pq; stored times 4/eps
        kp->wet = wet ? 1 : 0;
        for (int w = 0; wet && w < 2; ++w) {
            const double *cn = p->wall_cos + w * (N - 1);
            for (int a = 0; a < N; ++a)
                for (int b = 0; b < N; ++b) {
                    double c = 0.0;
                    if (a != b) {
                        if (b == N - 1) c = cn[a];
                        else if (a == N - 1) c = -cn[b];
                        else c = (p->sigma[a * N + N - 1] * cn[a] - p->sigma[b * N + N - 1] * cn[b]) / p->sigma[a * N + b];
                    }
                    kp->wetc[w][a][b] = (float)(4.0 / p->eps * c);
                }
        }
        const double n = p->model_a_n;
        kp->model_n_int = (n == std::floor(n) && n >= 1.0 && n <= 8.0) ? (int)n : 0;
    }
    return NLBM_OK;
}

}  // namespace

struct nlbm_sim {
    StepParams kp;
    int N, ns, model, storage;
    size_t plane;
    cudaStream_t stream;
    char *ws;
    Layout L;
    int cur;
    int64_t steps;
    int64_t launches;
    int tx, ty;
    char err[512];
    bool half() const { return is_half(storage); }
    float *f(int k) const { return (float *)(ws + L.f[k]); }
    float *g(int k) const { return (float *)(ws + L.g[k]); }
    float *f0(int k) const { return half() ? (float *)(ws + L.f0[k]) : nullptr; }
    float *u(int k) const { return (float *)(ws + L.u[k]); }
    float *phi(int k) const { return (float *)(ws + L.phi[k]); }
    float *mphi() const { return (float *)(ws + L.mphi); }
    float *P(int k) const { return (float *)(ws + L.P[k]); }
};

namespace {

nlbm_status cuda_fail(nlbm_sim *s, cudaError_t e, const char *what)
{
    set_err(s->err, "%s: %s", what, cudaGetErrorString(e));
    return NLBM_ECUDA;
}

void default_tile(nlbm_sim *s)
{
    // 124-column strips; narrower lattices use 60-column strips, and so does
    // FP32 storage at N = 7 (2048^2: 8,562 against 8,090 MLUPS)
    s->tx = s->kp.nx > 96 && !(s->ns == 6 && s->storage == NLBM_STORE_F32) ? 128 : 64;
    s->ty = 0;
}

// Number of state bytes in a checkpoint, excluding the trailing counter.
size_t state_payload(const nlbm_sim *s)
{
    const size_t pb = sizeof(float) * s->plane;
    return s->L.fbytes + s->L.gbytes + (s->half() ? pb * s->ns : 0) + pb * (2 + s->ns + 2 + 1);
}

// Kernel parameters with the buffers of state a (input) -> b (output).
StepParams step_params(const nlbm_sim *s, int a, int b)
{
    StepParams kp = s->kp;
    kp.fin = s->f(a);
    kp.fout = s->f(b);
    kp.f0in = s->f0(a);
    kp.f0out = s->f0(b);
    kp.gin = s->g(a);
    kp.gout = s->g(b);
    kp.uin = s->u(a);
    kp.uout = s->u(b);
    kp.phi_prev = s->phi(a);
    kp.phi = s->phi(b);
    kp.mphi = s->mphi();
    kp.mphi_in = kp.mphi;
    kp.pin = s->P(a);
    kp.pout = s->P(b);
    return kp;
}

// Initial state into the buffers of state c from the phase fields in phi(c).
cudaError_t launch_initial_state(nlbm_sim *s, int c)
{
    // init writes the populations of state c; kp.uin / kp.pin name the
    // other velocity / pressure buffers, zeroed as well
    StepParams kp = step_params(s, c ^ 1, c);
    kp.phi = s->phi(c);
    return launch_init(s->ns, kp, s->stream);
}

cudaError_t launch_step(const nlbm_sim *s, const StepParams &kp)
{
    const bool a = s->model == NLBM_MODEL_A;
    switch (s->storage) {
    case NLBM_STORE_BF16: return a ? launch_step_a_bf16(s->ns, kp, s->tx, s->ty, s->stream)
                                   : launch_step_b_bf16(s->ns, kp, s->tx, s->ty, s->stream);
    case NLBM_STORE_F16: return a ? launch_step_a_f16(s->ns, kp, s->tx, s->ty, s->stream)
                                  : launch_step_b_f16(s->ns, kp, s->tx, s->ty, s->stream);
    default: return a ? launch_step_a_f32(s->ns, kp, s->tx, s->ty, s->stream)
                      : launch_step_b_f32(s->ns, kp, s->tx, s->ty, s->stream);
    }
}

}  // namespace

extern "C" {

nlbm_status nlbm_workspace_bytes(const nlbm_params *p, size_t *bytes)
{
    if (!bytes) { set_err(g_err, "bytes is NULL"); return NLBM_EINVAL; }
    nlbm_status st = validate(p, nullptr, g_err);
    if (st != NLBM_OK) return st;
    *bytes = make_layout(p->n_phases - 1, (size_t)p->nx * p->ny, is_half(p->storage)).total;
    return NLBM_OK;
}

nlbm_status nlbm_create(const nlbm_params *p, void *dev_workspace, size_t workspace_bytes,
                        void *cuda_stream, nlbm_sim **out)
{
    if (!out) { set_err(g_err, "out is NULL"); return NLBM_EINVAL; }
    *out = nullptr;
    StepParams kp;
    nlbm_status st = validate(p, &kp, g_err);
    if (st != NLBM_OK) return st;
    const int ns = p->n_phases - 1;
    const Layout L = make_layout(ns, (size_t)p->nx * p->ny, is_half(p->storage));
    if (!dev_workspace) { set_err(g_err, "workspace is NULL"); return NLBM_EINVAL; }
    if (((uintptr_t)dev_workspace & 255) != 0) { set_err(g_err, "workspace must be 256-byte aligned"); return NLBM_EINVAL; }
    if (workspace_bytes < L.total) {
        set_err(g_err, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes, L.total);
        return NLBM_ENOMEM;
    }
    nlbm_sim *s = new (std::nothrow) nlbm_sim();
    if (!s) { set_err(g_err, "host allocation failed"); return NLBM_ENOMEM; }
    s->kp = kp;
    s->N = p->n_phases;
    s->ns = ns;
    s->model = p->model;
    s->storage = p->storage;
    s->plane = (size_t)p->nx * p->ny;
    s->stream = (cudaStream_t)cuda_stream;
    s->ws = (char *)dev_workspace;
    s->L = L;
    s->cur = 0;
    s->steps = 0;
    s->launches = 0;
    s->err[0] = 0;
    default_tile(s);
    *out = s;
    return NLBM_OK;
}

nlbm_status nlbm_set_phi(nlbm_sim *s, const float *dev_phi)
{
    if (!s || !dev_phi) return NLBM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(s->phi(s->cur), dev_phi, sizeof(float) * s->ns * s->plane,
                                    cudaMemcpyDeviceToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "copy of the initial phase fields");
    e = launch_initial_state(s, s->cur);
    if (e != cudaSuccess) return cuda_fail(s, e, "init kernel");
    s->launches++;
    s->steps = 0;
    return NLBM_OK;
}

nlbm_status nlbm_set_phi_host(nlbm_sim *s, const float *host_phi)
{
    if (!s || !host_phi) return NLBM_EINVAL;
    cudaError_t e = cudaMemcpyAsync(s->phi(s->cur), host_phi, sizeof(float) * s->ns * s->plane,
                                    cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "upload of the initial phase fields");
    // the device copy in the phi planes is its own source for the init kernel
    e = launch_initial_state(s, s->cur);
    if (e != cudaSuccess) return cuda_fail(s, e, "init kernel");
    s->launches++;
    s->steps = 0;
    return NLBM_OK;
}

nlbm_status nlbm_set_velocity(nlbm_sim *s, const float *dev_u)
{
    if (!s || !dev_u) return NLBM_EINVAL;
    if (s->half()) {
        set_err(s->err, "a state in motion is set for FP32 population storage only");
        return NLBM_ENOTSUP;
    }
    if (s->kp.wet) {
        set_err(s->err, "a state in motion is not set with wetting walls");
        return NLBM_ENOTSUP;
    }
    if (s->steps != 0) {
        set_err(s->err, "set the velocity after nlbm_set_phi and before the first step");
        return NLBM_EINVAL;
    }
    const int c = s->cur;
    // the populations of state c; u(c) becomes the first step's previous
    // velocity, and the other velocity buffer holds P' until the first step
    // overwrites it
    const StepParams kp = step_params(s, c ^ 1, c);
    cudaError_t e = launch_velocity_state(s->ns, s->model, kp, dev_u, s->u(c), s->u(c ^ 1), s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "velocity initial state");
    s->launches += 2;
    return NLBM_OK;
}

nlbm_status nlbm_step(nlbm_sim *s, int64_t nsteps)
{
    if (!s || nsteps < 0) return NLBM_EINVAL;
    for (int64_t k = 0; k < nsteps; ++k) {
        const int a = s->cur, b = s->cur ^ 1;
        StepParams kp = step_params(s, a, b);
        // FP32 storage writes P on the last step of a call only; 16-bit
        // storage needs it every step (the pullers add 3 w_i P back)
        if (!s->half() && k != nsteps - 1) kp.pout = nullptr;
        cudaError_t e = launch_step(s, kp);
        if (e != cudaSuccess) return cuda_fail(s, e, "step kernel");
        s->launches++;
        s->cur = b;
        s->steps++;
    }
    return NLBM_OK;
}

nlbm_status nlbm_get_moments(nlbm_sim *s, float *dev_phi, float *dev_u, float *dev_p)
{
    if (!s) return NLBM_EINVAL;
    if (!dev_phi && !dev_u && !dev_p) return NLBM_OK;
    cudaError_t e = launch_export(s->ns, s->phi(s->cur), s->u(s->cur), s->P(s->cur), (unsigned)s->plane,
                                  dev_phi, dev_u, dev_p, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "export kernel");
    s->launches++;
    return NLBM_OK;
}

nlbm_status nlbm_get_moments_host(nlbm_sim *s, float *host_phi, float *host_u, float *host_p)
{
    if (!s) return NLBM_EINVAL;
    if (!host_phi && !host_u && !host_p) return NLBM_OK;
    // Stage through the idle population buffers (rewritten by the next
    // step): N + 3 planes fit in one f copy and the g copy after it.
    const size_t pl = s->plane, pb = sizeof(float) * pl;
    float *stage = s->f(s->cur ^ 1);
    float *sphi = stage, *su = stage + (size_t)s->N * pl, *sp = su + 2 * pl;
    cudaError_t e = launch_export(s->ns, s->phi(s->cur), s->u(s->cur), s->P(s->cur), (unsigned)pl,
                                  host_phi ? sphi : nullptr, host_u ? su : nullptr,
                                  host_p ? sp : nullptr, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "export kernel");
    s->launches++;
    if (host_phi && (e = cudaMemcpyAsync(host_phi, sphi, pb * s->N, cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess)
        return cuda_fail(s, e, "download of phi");
    if (host_u && (e = cudaMemcpyAsync(host_u, su, 2 * pb, cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess)
        return cuda_fail(s, e, "download of u");
    if (host_p && (e = cudaMemcpyAsync(host_p, sp, pb, cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess)
        return cuda_fail(s, e, "download of P");
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "synchronize");
    return NLBM_OK;
}

nlbm_status nlbm_phase_mass(nlbm_sim *s, double *host_mass)
{
    if (!s || !host_mass) return NLBM_EINVAL;
    double *partials = (double *)(s->ws + s->L.partials);
    double *mass = (double *)(s->ws + s->L.mass);
    int *flag = (int *)(mass + s->N);
    cudaError_t e = launch_phase_mass(s->ns, s->phi(s->cur), (unsigned)s->plane, partials, mass, flag, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "phase-mass kernels");
    s->launches += 2;
    double buf[kMaxPhases + 1];
    e = cudaMemcpyAsync(buf, mass, sizeof(double) * s->N + sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "download of the phase masses");
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "synchronize");
    memcpy(host_mass, buf, sizeof(double) * s->N);
    int fl = 0;
    memcpy(&fl, (const char *)buf + sizeof(double) * s->N, sizeof(int));
    if (fl) {
        set_err(s->err, "a phase field is non-finite or outside [-0.5, 1.5]");
        return NLBM_EDIVERGED;
    }
    return NLBM_OK;
}

nlbm_status nlbm_state_bytes(const nlbm_sim *s, size_t *bytes)
{
    if (!s || !bytes) return NLBM_EINVAL;
    *bytes = state_payload(s) + 16;
    return NLBM_OK;
}

nlbm_status nlbm_save(nlbm_sim *s, void *dev_dst)
{
    if (!s || !dev_dst || ((uintptr_t)dev_dst & 15)) return NLBM_EINVAL;
    char *d = (char *)dev_dst;
    const size_t pb = sizeof(float) * s->plane;
    const int c = s->cur;
    struct Part { const void *src; size_t n; } parts[] = {
        {s->f(c), s->L.fbytes}, {s->g(c), s->L.gbytes}, {s->f0(c), s->half() ? pb * s->ns : 0},
        {s->u(c), pb * 2}, {s->phi(c), pb * s->ns}, {s->mphi(), pb * 2}, {s->P(c), pb}};
    for (const Part &pt : parts) {
        if (!pt.n) continue;
        cudaError_t e = cudaMemcpyAsync(d, pt.src, pt.n, cudaMemcpyDeviceToDevice, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "checkpoint copy");
        d += pt.n;
    }
    int64_t counter[2] = {s->steps, 0x6e6c626d};   // step count and a tag
    cudaError_t e = cudaMemcpyAsync(d, counter, sizeof counter, cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "checkpoint counter");
    e = cudaStreamSynchronize(s->stream);   // counter is a host stack value
    if (e != cudaSuccess) return cuda_fail(s, e, "synchronize");
    return NLBM_OK;
}

nlbm_status nlbm_restore(nlbm_sim *s, const void *dev_src)
{
    if (!s || !dev_src || ((uintptr_t)dev_src & 15)) return NLBM_EINVAL;
    const char *d = (const char *)dev_src;
    const size_t pb = sizeof(float) * s->plane;
    s->cur = 0;
    struct Part { void *dst; size_t n; } parts[] = {
        {s->f(0), s->L.fbytes}, {s->g(0), s->L.gbytes}, {s->f0(0), s->half() ? pb * s->ns : 0},
        {s->u(0), pb * 2}, {s->phi(0), pb * s->ns}, {s->mphi(), pb * 2}, {s->P(0), pb}};
    for (const Part &pt : parts) {
        if (!pt.n) continue;
        cudaError_t e = cudaMemcpyAsync(pt.dst, d, pt.n, cudaMemcpyDeviceToDevice, s->stream);
        if (e != cudaSuccess) return cuda_fail(s, e, "restore copy");
        d += pt.n;
    }
    int64_t counter[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(counter, d, sizeof counter, cudaMemcpyDeviceToHost, s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "restore counter");
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "synchronize");
    if (counter[1] != 0x6e6c626d) {
        set_err(s->err, "checkpoint tag mismatch");
        return NLBM_EINVAL;
    }
    s->steps = counter[0];
    return NLBM_OK;
}

nlbm_status nlbm_synchronize(nlbm_sim *s)
{
    if (!s) return NLBM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_fail(s, e, "synchronize");
    return NLBM_OK;
}

int64_t nlbm_steps_done(const nlbm_sim *s) { return s ? s->steps : -1; }

int64_t nlbm_kernel_launches(const nlbm_sim *s) { return s ? s->launches : -1; }

nlbm_status nlbm_set_tile(nlbm_sim *s, int32_t tx, int32_t ty)
{
    if (!s) return NLBM_EINVAL;
    if ((tx != 64 && tx != 128 && tx != 256) || ty < 0) {
        set_err(s->err, "tile %dx%d outside tx in {64, 128, 256}, ty >= 0", tx, ty);
        return NLBM_EINVAL;
    }
    s->tx = tx;
    s->ty = ty;
    return NLBM_OK;
}

nlbm_status nlbm_get_tile(const nlbm_sim *s, int32_t *tx, int32_t *ty)
{
    if (!s || !tx || !ty) return NLBM_EINVAL;
    *tx = s->tx;
    *ty = s->ty;
    return NLBM_OK;
}

nlbm_status nlbm_autotune(nlbm_sim *s, void *dev_scratch, size_t scratch_bytes, int32_t steps_per_trial,
                          int32_t *best_tx, int32_t *best_ty, float *best_ms_per_step)
{
    if (!s || !dev_scratch || steps_per_trial < 1) return NLBM_EINVAL;
    const size_t need = state_payload(s) + 16;
    if (scratch_bytes < need) {
        set_err(s->err, "scratch of %zu bytes is smaller than the %zu of state", scratch_bytes, need);
        return NLBM_ENOMEM;
    }
    nlbm_status st = nlbm_save(s, dev_scratch);
    if (st != NLBM_OK) return st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return cuda_fail(s, e, "timing events");
    }
    static const int kTx[] = {64, 128, 256};
    static const int kTy[] = {0, 8, 12, 16, 20, 24, 32, 48};
    float best = 1e30f;
    int btx = s->tx, bty = s->ty;
    for (int tx : kTx) {
        // a strip of tx - 4 columns; skip widths the lattice cannot fill
        if (tx > 64 && (tx / 2 - 4) >= s->kp.nx) continue;
        for (int ty : kTy) {
            s->tx = tx;
            s->ty = ty;
            for (int k = 0; k <= steps_per_trial && st == NLBM_OK; ++k) {
                if (k == 1 && (e = cudaEventRecord(e0, s->stream)) != cudaSuccess) st = cuda_fail(s, e, "event");
                StepParams kp = step_params(s, s->cur, s->cur ^ 1);
                if (!s->half()) kp.pout = nullptr;
                if (st == NLBM_OK && (e = launch_step(s, kp)) != cudaSuccess) st = cuda_fail(s, e, "trial step");
                s->launches++;
                s->cur ^= 1;
            }
            float ms = 0.f;
            if (st == NLBM_OK &&
                ((e = cudaEventRecord(e1, s->stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                 (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess))
                st = cuda_fail(s, e, "trial timing");
            if (st != NLBM_OK) break;
            ms /= steps_per_trial;
            if (ms < best) {
                best = ms;
                btx = tx;
                bty = ty;
            }
            if ((st = nlbm_restore(s, dev_scratch)) != NLBM_OK) break;
        }
        if (st != NLBM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    s->tx = btx;
    s->ty = bty;
    if (st != NLBM_OK) return st;
    if (best_tx) *best_tx = btx;
    if (best_ty) *best_ty = bty;
    if (best_ms_per_step) *best_ms_per_step = best;
    return NLBM_OK;
}

void nlbm_destroy(nlbm_sim *s) { delete s; }

}  // extern "C"

// ------------------------------------------------------------------ ensembles

struct nlbm_batch {
    int count, ns;
    std::vector<nlbm_sim *> sims;
    std::vector<size_t> sim_off;         // workspace offset of each simulation
    size_t state_begin, state_end;       // span of all simulations' state
    cudaStream_t stream;
    char *ws;
    StepParams *d_params;                // [4][count]: parity 0/1 x (no P / P)
    BatchTile *d_tiles;
    size_t max_tiles;
    int ntiles;
    int *d_counters;                     // [2]
    int cur;                             // state parity shared by every simulation
    int tx, ty;
    cudaGraphExec_t graph;               // two steps (parity 0 then 1), no P output
    bool graph_ok;
    int64_t steps, launches;
    char err[512];
};

namespace {

constexpr int kBatchMaxSims = 4096;

struct BatchLayout {
    size_t params, tiles, counters, sims_begin, total;
    size_t max_tiles;
    std::vector<size_t> sim_off;
};

// Largest number of tiles any allowed tile shape gives (tx = 64, ty = 1).
size_t worst_tiles(const nlbm_params *p, int count)
{
    size_t t = 0;
    for (int k = 0; k < count; ++k) t += (size_t)((p[k].nx + 59) / 60) * (size_t)p[k].ny;
    return t;
}

nlbm_status batch_layout(const nlbm_params *p, int count, BatchLayout *B, char *err)
{
    if (!p || count < 1 || count > kBatchMaxSims) {
        set_err(err, "count=%d outside 1..%d (or params NULL)", count, kBatchMaxSims);
        return NLBM_EINVAL;
    }
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    B->max_tiles = worst_tiles(p, count);
    B->params = take(sizeof(StepParams) * 4 * (size_t)count);
    B->tiles = take(sizeof(BatchTile) * B->max_tiles);
    B->counters = take(2 * sizeof(int));
    B->sims_begin = off;
    B->sim_off.resize(count);
    for (int k = 0; k < count; ++k) {
        nlbm_status st = validate(&p[k], nullptr, err);
        if (st != NLBM_OK) {
            char tmp[512];
            snprintf(tmp, sizeof tmp, "simulation %d: %s", k, err);
            memcpy(err, tmp, sizeof tmp);
            return st;
        }
        if (p[k].n_phases != p[0].n_phases) {
            set_err(err, "simulation %d has N=%d, simulation 0 N=%d: an ensemble shares N", k,
                    p[k].n_phases, p[0].n_phases);
            return NLBM_EINVAL;
        }
        if (p[k].storage != NLBM_STORE_F32) {
            set_err(err, "simulation %d: ensembles store FP32 populations", k);
            return NLBM_ENOTSUP;
        }
        B->sim_off[k] = take(make_layout(p[k].n_phases - 1, (size_t)p[k].nx * p[k].ny, false).total);
    }
    B->total = off;
    return NLBM_OK;
}

nlbm_status batch_fail(nlbm_batch *b, cudaError_t e, const char *what)
{
    set_err(b->err, "%s: %s", what, cudaGetErrorString(e));
    return NLBM_ECUDA;
}

// Tile table for the current tile shape: every strip and row chunk of every
// simulation, the largest simulations first (so the last tiles are small).
nlbm_status build_tiles(nlbm_batch *b)
{
    const int W = b->tx - 4;
    std::vector<int> order(b->count);
    for (int k = 0; k < b->count; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
        return b->sims[a]->plane > b->sims[c]->plane;
    });
    std::vector<BatchTile> t;
    for (int k : order) {
        const nlbm_sim *s = b->sims[k];
        const int nx = s->kp.nx, ny = s->kp.ny;
        int ty = b->ty > 0 ? b->ty : 32;
        if (ty > ny) ty = ny;
        for (int y0 = 0; y0 < ny; y0 += ty)
            for (int x0 = 0; x0 < nx; x0 += W) t.push_back(BatchTile{k, x0, y0, ty});
    }
    if (t.size() > b->max_tiles) {
        set_err(b->err, "tile table of %zu entries exceeds the %zu reserved", t.size(), b->max_tiles);
        return NLBM_EINVAL;
    }
    cudaError_t e = cudaMemcpyAsync(b->d_tiles, t.data(), sizeof(BatchTile) * t.size(), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // t is a host temporary
    if (e != cudaSuccess) return batch_fail(b, e, "upload of the tile table");
    b->ntiles = (int)t.size();
    b->graph_ok = false;
    return NLBM_OK;
}

nlbm_status upload_params(nlbm_batch *b)
{
    std::vector<StepParams> h(4 * (size_t)b->count);
    for (int par = 0; par < 2; ++par)
        for (int k = 0; k < b->count; ++k) {
            StepParams kp = step_params(b->sims[k], par, par ^ 1);
            // the same condition as the single-simulation launcher's
            kp.row_window = !kp.wall_x && kp.nx % 4 == 0 &&
                            ((reinterpret_cast<uintptr_t>(kp.fin) | reinterpret_cast<uintptr_t>(kp.gin)) & 15) == 0;
            kp.pout = nullptr;
            h[(size_t)(2 * par) * b->count + k] = kp;
            kp.pout = b->sims[k]->P(0);
            h[(size_t)(2 * par + 1) * b->count + k] = kp;
        }
    cudaError_t e = cudaMemcpyAsync(b->d_params, h.data(), sizeof(StepParams) * h.size(), cudaMemcpyHostToDevice,
                                    b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "upload of the parameter blocks");
    return NLBM_OK;
}

// One step of every simulation from state parity b->cur; with_p selects the
// parameter blocks that also write P.
cudaError_t batch_launch(nlbm_batch *b, int parity, bool with_p)
{
    const StepParams *tab = b->d_params + (size_t)(2 * parity + (with_p ? 1 : 0)) * b->count;
    return launch_batch_step(b->ns, b->tx, tab, b->d_tiles, b->ntiles, b->d_counters, parity, b->stream);
}

void sync_sims(nlbm_batch *b)
{
    for (nlbm_sim *s : b->sims) {
        s->cur = b->cur;
        s->steps = b->steps;
    }
}

nlbm_status capture_graph(nlbm_batch *b)
{
    if (b->graph_ok) return NLBM_OK;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return batch_fail(b, e, "stream capture");
    cudaError_t e0 = batch_launch(b, 0, false);
    cudaError_t e1 = batch_launch(b, 1, false);
    e = cudaStreamEndCapture(b->stream, &g);
    if (e0 != cudaSuccess) e = e0;
    if (e == cudaSuccess && e1 != cudaSuccess) e = e1;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return batch_fail(b, e, "graph of two ensemble steps");
    b->graph_ok = true;
    return NLBM_OK;
}

}  // namespace

extern "C" {

nlbm_status nlbm_batch_workspace_bytes(const nlbm_params *sims, int32_t count, size_t *bytes)
{
    if (!bytes) { set_err(g_err, "bytes is NULL"); return NLBM_EINVAL; }
    BatchLayout B;
    nlbm_status st = batch_layout(sims, count, &B, g_err);
    if (st != NLBM_OK) return st;
    *bytes = B.total;
    return NLBM_OK;
}

nlbm_status nlbm_batch_create(const nlbm_params *sims, int32_t count, void *dev_workspace, size_t workspace_bytes,
                              void *cuda_stream, nlbm_batch **out)
{
    if (!out) { set_err(g_err, "out is NULL"); return NLBM_EINVAL; }
    *out = nullptr;
    BatchLayout B;
    nlbm_status st = batch_layout(sims, count, &B, g_err);
    if (st != NLBM_OK) return st;
    if (!dev_workspace || ((uintptr_t)dev_workspace & 255)) {
        set_err(g_err, "workspace must be non-NULL and 256-byte aligned");
        return NLBM_EINVAL;
    }
    if (workspace_bytes < B.total) {
        set_err(g_err, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes, B.total);
        return NLBM_ENOMEM;
    }
    nlbm_batch *b = new (std::nothrow) nlbm_batch();
    if (!b) { set_err(g_err, "host allocation failed"); return NLBM_ENOMEM; }
    b->count = count;
    b->ns = sims[0].n_phases - 1;
    b->stream = (cudaStream_t)cuda_stream;
    b->ws = (char *)dev_workspace;
    b->d_params = (StepParams *)(b->ws + B.params);
    b->d_tiles = (BatchTile *)(b->ws + B.tiles);
    b->max_tiles = B.max_tiles;
    b->d_counters = (int *)(b->ws + B.counters);
    b->sim_off = B.sim_off;
    b->state_begin = B.sims_begin;
    b->state_end = B.total;
    b->cur = 0;
    b->tx = 128;
    b->ty = 0;
    b->graph = nullptr;
    b->graph_ok = false;
    b->steps = 0;
    b->launches = 0;
    b->err[0] = 0;
    for (int k = 0; k < count; ++k) {
        nlbm_sim *s = nullptr;
        const size_t need = make_layout(b->ns, (size_t)sims[k].nx * sims[k].ny, false).total;
        st = nlbm_create(&sims[k], b->ws + B.sim_off[k], need, cuda_stream, &s);
        if (st != NLBM_OK) {
            for (nlbm_sim *q : b->sims) delete q;
            delete b;
            return st;
        }
        b->sims.push_back(s);
    }
    cudaError_t e = cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(int), b->stream);
    if (e != cudaSuccess) {
        set_err(g_err, "counter reset: %s", cudaGetErrorString(e));
        for (nlbm_sim *q : b->sims) delete q;
        delete b;
        return NLBM_ECUDA;
    }
    if ((st = upload_params(b)) != NLBM_OK || (st = build_tiles(b)) != NLBM_OK) {
        memcpy(g_err, b->err, sizeof b->err);
        for (nlbm_sim *q : b->sims) delete q;
        delete b;
        return st;
    }
    *out = b;
    return NLBM_OK;
}

nlbm_status nlbm_batch_set_phi(nlbm_batch *b, int32_t sim, const float *dev_phi)
{
    if (!b || sim < 0 || sim >= b->count || !dev_phi) return NLBM_EINVAL;
    nlbm_sim *s = b->sims[sim];
    s->cur = b->cur;
    nlbm_status st = nlbm_set_phi(s, dev_phi);
    b->launches++;
    if (st != NLBM_OK) memcpy(b->err, s->err, sizeof b->err);
    return st;
}

nlbm_status nlbm_batch_step(nlbm_batch *b, int64_t nsteps)
{
    if (!b || nsteps < 0) return NLBM_EINVAL;
    if (nsteps == 0) return NLBM_OK;
    int64_t k = 0;
    const bool use_graph = b->stream != nullptr && nsteps >= 3;
    cudaError_t e;
    if (use_graph) {
        if (b->cur == 1) {   // align to the graph's parity order
            if ((e = batch_launch(b, 1, false)) != cudaSuccess) return batch_fail(b, e, "ensemble step");
            b->launches++;
            b->cur = 0;
            ++k;
        }
        nlbm_status st = capture_graph(b);
        if (st != NLBM_OK) return st;
        for (; k + 2 < nsteps; k += 2) {
            if ((e = cudaGraphLaunch(b->graph, b->stream)) != cudaSuccess) return batch_fail(b, e, "graph launch");
            b->launches += 2;
        }
    }
    for (; k < nsteps; ++k) {
        if ((e = batch_launch(b, b->cur, k == nsteps - 1)) != cudaSuccess) return batch_fail(b, e, "ensemble step");
        b->launches++;
        b->cur ^= 1;
    }
    b->steps += nsteps;
    sync_sims(b);
    return NLBM_OK;
}

nlbm_status nlbm_batch_get_moments(nlbm_batch *b, int32_t sim, float *dev_phi, float *dev_u, float *dev_p)
{
    if (!b || sim < 0 || sim >= b->count) return NLBM_EINVAL;
    nlbm_sim *s = b->sims[sim];
    nlbm_status st = nlbm_get_moments(s, dev_phi, dev_u, dev_p);
    if (dev_phi || dev_u || dev_p) b->launches++;
    if (st != NLBM_OK) memcpy(b->err, s->err, sizeof b->err);
    return st;
}

nlbm_status nlbm_batch_phase_mass(nlbm_batch *b, int32_t sim, double *host_mass)
{
    if (!b || sim < 0 || sim >= b->count || !host_mass) return NLBM_EINVAL;
    nlbm_sim *s = b->sims[sim];
    nlbm_status st = nlbm_phase_mass(s, host_mass);
    b->launches += 2;
    if (st != NLBM_OK) memcpy(b->err, s->err, sizeof b->err);
    return st;
}

nlbm_status nlbm_batch_set_tile(nlbm_batch *b, int32_t tx, int32_t ty)
{
    if (!b) return NLBM_EINVAL;
    if ((tx != 64 && tx != 128 && tx != 256) || ty < 0) {
        set_err(b->err, "tile %dx%d outside tx in {64, 128, 256}, ty >= 0", tx, ty);
        return NLBM_EINVAL;
    }
    b->tx = tx;
    b->ty = ty;
    return build_tiles(b);
}

nlbm_status nlbm_batch_get_tile(const nlbm_batch *b, int32_t *tx, int32_t *ty, int32_t *ntiles)
{
    if (!b || !tx || !ty) return NLBM_EINVAL;
    *tx = b->tx;
    *ty = b->ty;
    if (ntiles) *ntiles = b->ntiles;
    return NLBM_OK;
}

nlbm_status nlbm_batch_state_bytes(const nlbm_batch *b, size_t *bytes)
{
    if (!b || !bytes) return NLBM_EINVAL;
    *bytes = b->state_end - b->state_begin;
    return NLBM_OK;
}

nlbm_status nlbm_batch_autotune(nlbm_batch *b, void *dev_scratch, size_t scratch_bytes, int32_t steps_per_trial,
                                int32_t *best_tx, int32_t *best_ty, float *best_ms_per_step)
{
    if (!b || !dev_scratch || steps_per_trial < 1) return NLBM_EINVAL;
    const size_t span = b->state_end - b->state_begin;
    if (scratch_bytes < span) {
        set_err(b->err, "scratch of %zu bytes is smaller than the %zu of state", scratch_bytes, span);
        return NLBM_ENOMEM;
    }
    char *state = b->ws + b->state_begin;
    const int cur0 = b->cur;
    cudaError_t e = cudaMemcpyAsync(dev_scratch, state, span, cudaMemcpyDeviceToDevice, b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "state copy");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return batch_fail(b, e, "timing events");
    }
    static const int kTx[] = {64, 128, 256};
    static const int kTy[] = {8, 16, 32, 64, 128};
    float best = 1e30f;
    int btx = b->tx, bty = b->ty;
    nlbm_status st = NLBM_OK;
    for (int tx : kTx) {
        for (int ty : kTy) {
            b->tx = tx;
            b->ty = ty;
            if ((st = build_tiles(b)) != NLBM_OK) break;
            // one untimed step, then the timed ones, from the saved state
            for (int k = 0; k <= steps_per_trial && st == NLBM_OK; ++k) {
                if (k == 1 && (e = cudaEventRecord(e0, b->stream)) != cudaSuccess) st = batch_fail(b, e, "event");
                if (st == NLBM_OK && (e = batch_launch(b, b->cur, false)) != cudaSuccess)
                    st = batch_fail(b, e, "trial step");
                b->launches++;
                b->cur ^= 1;
            }
            if (st != NLBM_OK) break;
            float ms = 0.f;
            if ((e = cudaEventRecord(e1, b->stream)) != cudaSuccess || (e = cudaEventSynchronize(e1)) != cudaSuccess ||
                (e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
                st = batch_fail(b, e, "trial timing");
                break;
            }
            ms /= steps_per_trial;
            if (ms < best) {
                best = ms;
                btx = tx;
                bty = ty;
            }
            // back to the saved state; the tile counters restart from zero
            // since the parity sequence is broken here
            b->cur = cur0;
            if ((e = cudaMemcpyAsync(state, dev_scratch, span, cudaMemcpyDeviceToDevice, b->stream)) != cudaSuccess ||
                (e = cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(int), b->stream)) != cudaSuccess) {
                st = batch_fail(b, e, "state restore");
                break;
            }
        }
        if (st != NLBM_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->cur = cur0;
    if (st == NLBM_OK) {   // state restored after the last trial
        b->tx = btx;
        b->ty = bty;
        st = build_tiles(b);
    }
    if (st == NLBM_OK && (e = cudaStreamSynchronize(b->stream)) != cudaSuccess) st = batch_fail(b, e, "synchronize");
    if (st != NLBM_OK) return st;
    if (best_tx) *best_tx = btx;
    if (best_ty) *best_ty = bty;
    if (best_ms_per_step) *best_ms_per_step = best;
    return NLBM_OK;
}

nlbm_status nlbm_batch_synchronize(nlbm_batch *b)
{
    if (!b) return NLBM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return batch_fail(b, e, "synchronize");
    return NLBM_OK;
}

int64_t nlbm_batch_steps_done(const nlbm_batch *b) { return b ? b->steps : -1; }

int64_t nlbm_batch_kernel_launches(const nlbm_batch *b) { return b ? b->launches : -1; }

void nlbm_batch_destroy(nlbm_batch *b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (nlbm_sim *s : b->sims) delete s;
    delete b;
}

const char *nlbm_batch_last_error(const nlbm_batch *b) { return b ? b->err : g_err; }

}  // extern "C"

// ------------------------------------------------------------------- adjoint

struct nlbm_adjoint {
    nlbm_sim *sim;             // forward simulation (its own workspace slice)
    int ns, N, nsteps, every, nckpt;
    size_t plane, state_floats;
    cudaStream_t stream;
    char *ws;
    float *ckpt;               // [nckpt][state]
    float *seg;                // [every + 1][state]
    float *tapes;              // [every][tape] the rebuilt segment's tapes
    AdjTape T;                 // the tape of nlbm_adjoint_reverse_step
    float *seed[2];            // two sets of step-output adjoints
    AdjFields A;               // intermediates (the seed pointers are set per step)
    double *partials, *acc;    // [kAdjRedBlocks][NP+1], [NP+1]
    float *seed_buf;           // [N][plane] copy of the caller's dL/dphi(T)
    float *grad_buf;           // [N-1][plane] dL/dphi_0
    int final_set;             // seed set holding step 1's input adjoints
    cudaGraphExec_t graph;     // the whole reverse sweep, captured on first use
    bool graph_tried;
    bool forward_done;
    char err[512];
};

namespace {

// State of a simulation between steps: f [9 NS], g [8], u [2], phi [NS],
// m_phi [2] planes (FP32 storage).
size_t adj_state_floats(int ns, size_t plane) { return plane * ((size_t)ns * 9 + 8 + 2 + ns + 2); }

// Offsets of the per-node arrays of the tape, the two seed sets and the
// intermediates, in floats per plane.
struct AdjCounts {
    int tape, seedset, inter, contrib;
};

AdjCounts adj_counts(int ns)
{
    const int np = (ns + 1) * ns / 2;
    // tape, one seed set, intermediates, per-node gradient sums (FP64: 2 floats each)
    return AdjCounts{8 * ns + 13, 10 * ns + 12, 9 * ns + 12, 2 * (np + 1)};
}

struct AdjLayout {
    size_t sim, ckpt, seg, tapes, fields, partials, acc, total;
};

nlbm_status adj_layout(const nlbm_params *p, int nsteps, int every, AdjLayout *L, char *err)
{
    nlbm_status st = validate(p, nullptr, err);
    if (st != NLBM_OK) return st;
    bool wet = false;
    for (int a = 0; p->wall_cos && a < 2 * (p->n_phases - 1); ++a) wet = wet || p->wall_cos[a] != 0.0;
    if (p->storage != NLBM_STORE_F32 || wet) {
        set_err(err, "the adjoint covers FP32 storage and walls without wetting (contact angles of 90 degrees)");
        return NLBM_ENOTSUP;
    }
    if (nsteps < 1 || every < 1) { set_err(err, "nsteps and checkpoint interval must be >= 1"); return NLBM_EINVAL; }
    const int ns = p->n_phases - 1;
    const size_t plane = (size_t)p->nx * p->ny;
    const int nckpt = (nsteps + every - 1) / every;
    const AdjCounts c = adj_counts(ns);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    L->sim = take(make_layout(ns, plane, false).total);
    L->ckpt = take(sizeof(float) * adj_state_floats(ns, plane) * nckpt);
    // a segment's states and one spare (the output of its last step), and
    // the tape of each of its steps
    const size_t seglen = (size_t)(every < nsteps ? every : nsteps);
    L->seg = take(sizeof(float) * adj_state_floats(ns, plane) * (seglen + 1));
    L->tapes = take(sizeof(float) * plane * (size_t)c.tape * seglen);
    // the FP64 per-node sums come first (8-byte alignment)
    L->fields = take(sizeof(float) * plane * (size_t)(c.contrib + c.tape + 2 * c.seedset + c.inter + 2 * ns + 1));
    L->partials = take(sizeof(double) * kAdjRedBlocks * c.contrib);
    L->acc = take(sizeof(double) * c.contrib);
    L->total = off;
    return NLBM_OK;
}

nlbm_status adj_fail(nlbm_adjoint *a, cudaError_t e, const char *what)
{
    set_err(a->err, "%s: %s", what, cudaGetErrorString(e));
    return NLBM_ECUDA;
}

// Copy the simulation's current state into / out of a packed state record.
cudaError_t adj_save_state(nlbm_adjoint *a, float *dst)
{
    nlbm_sim *s = a->sim;
    const size_t pl = a->plane, pb = sizeof(float) * pl;
    const int c = s->cur;
    struct Part { const void *src; size_t n; } parts[] = {
        {s->f(c), pb * 9 * a->ns}, {s->g(c), pb * 8}, {s->u(c), pb * 2}, {s->phi(c), pb * a->ns}, {s->mphi(), pb * 2}};
    char *d = (char *)dst;
    for (const Part &p : parts) {
        cudaError_t e = cudaMemcpyAsync(d, p.src, p.n, cudaMemcpyDeviceToDevice, a->stream);
        if (e != cudaSuccess) return e;
        d += p.n;
    }
    return cudaSuccess;
}

// Step parameters whose inputs are a packed state record.
StepParams adj_params_from_state(const nlbm_adjoint *a, const float *state)
{
    StepParams kp = a->sim->kp;
    const size_t pl = a->plane;
    kp.fin = state;
    kp.gin = state + pl * 9 * a->ns;
    kp.uin = kp.gin + pl * 8;
    kp.phi_prev = kp.uin + pl * 2;
    kp.mphi = const_cast<float *>(kp.phi_prev + pl * a->ns);
    kp.mphi_in = kp.mphi;
    return kp;
}

// Adjoint-field pointers for a step whose output adjoints are seed set so
// and input adjoints seed set si.
AdjFields adj_fields(const nlbm_adjoint *a, float *so, float *si)
{
    const size_t pl = a->plane;
    const int ns = a->ns;
    AdjFields A = a->A;
    A.lf_out = so;
    A.lg_out = so + pl * 9 * ns;
    A.lphi_out = A.lg_out + pl * 8;
    A.lu_out = A.lphi_out + pl * ns;
    A.lm_out = A.lu_out + pl * 2;
    A.lf_in = si;
    A.lg_in = si + pl * 9 * ns;
    A.lphi_in = A.lg_in + pl * 8;
    A.lu_in = A.lphi_in + pl * ns;
    A.lm_in = A.lu_in + pl * 2;
    return A;
}

// Tape k of the rebuilt segment (the field order of launch_step_tape_{a,b}_f32).
AdjTape adj_tape(const nlbm_adjoint *a, int k)
{
    const size_t pl = a->plane;
    const int ns = a->ns;
    float *b = a->tapes + pl * (size_t)adj_counts(ns).tape * k;
    AdjTape T;
    T.phi = b;
    T.j = b + pl * ns;
    T.g = b + pl * 3 * ns;
    T.grad = b + pl * (3 * ns + 8);
    T.lap = b + pl * (5 * ns + 8);
    T.R = b + pl * (6 * ns + 8);
    T.mphi = b + pl * (8 * ns + 8);
    T.w = b + pl * (8 * ns + 10);
    T.F = b + pl * (8 * ns + 11);
    return T;
}

// Kernel launches of one reverse sweep (counted, not queried).
int64_t adj_sweep_launches(const nlbm_adjoint *a)
{
    // fold + per step: one taping step kernel while the segment is rebuilt
    // and 4 reverse kernels; the phi0 sum and the two-kernel reduction
    return 1 + 5 * (int64_t)a->nsteps + 1 + 2;
}

// The reverse sweep, asynchronous and capturable: seeds from seed_buf,
// dL/dphi_0 into grad_buf, dL/dsigma and dL/dM into acc.
cudaError_t adj_backward_body(nlbm_adjoint *a)
{
    const size_t pl = a->plane, pb = sizeof(float) * pl;
    const int ns = a->ns;
    const AdjCounts c = adj_counts(ns);
    cudaError_t e;
    for (int k = 0; k < 2; ++k)
        if ((e = cudaMemsetAsync(a->seed[k], 0, pb * c.seedset, a->stream)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a->A.gacc, 0, pb * c.contrib, a->stream)) != cudaSuccess) return e;
    if ((e = launch_fold_seed(ns, a->seed_buf, (unsigned)pl, a->seed[0] + pl * (9 * ns + 8), a->stream)) != cudaSuccess)
        return e;
    int cur = 0;
    for (int k = a->nckpt - 1; k >= 0; --k) {
        const int t0 = k * a->every;
        const int len = (k + 1) * a->every <= a->nsteps ? a->every : a->nsteps - t0;
        // rebuild the segment's input states S_t0 .. S_t0+len-1 in place and,
        // with the same launches, the tape of each of its steps (the last
        // step's output state goes to the spare slot)
        if ((e = cudaMemcpyAsync(a->seg, a->ckpt + a->state_floats * k, sizeof(float) * a->state_floats,
                                 cudaMemcpyDeviceToDevice, a->stream)) != cudaSuccess)
            return e;
        for (int s = 1; s <= len; ++s) {
            const float *in = a->seg + a->state_floats * (s - 1);
            float *out = a->seg + a->state_floats * s;
            StepParams kp = adj_params_from_state(a, in);
            kp.fout = out;
            kp.gout = out + pl * 9 * ns;
            kp.uout = kp.gout + pl * 8;
            kp.phi = kp.uout + pl * 2;
            kp.mphi = kp.phi + pl * ns;   // read from the input state, written to the output
            kp.pout = nullptr;
            kp.tape = a->tapes + pl * (size_t)c.tape * (s - 1);
            if ((e = (kp.model == NLBM_MODEL_A ? launch_step_tape_a_f32 : launch_step_tape_b_f32)(ns, kp, a->stream)) !=
                cudaSuccess)
                return e;
        }
        for (int s = len - 1; s >= 0; --s) {
            const StepParams kp = adj_params_from_state(a, a->seg + a->state_floats * s);
            const AdjFields A = adj_fields(a, a->seed[cur], a->seed[cur ^ 1]);
            if ((e = launch_reverse_step(ns, kp, adj_tape(a, s), A, true, a->stream)) != cudaSuccess) return e;
            cur ^= 1;
        }
    }
    a->final_set = cur;
    // phi0 entered step 1 as its pulled phase populations (f_i = w_i phi0,
    // so the adjoint is that of phi) and as its phi_prev
    const float *lphi_in = a->seed[cur] + pl * (9 * ns + 8);
    if ((e = launch_add_planes(a->A.lphi_tot, lphi_in, (unsigned)(pl * ns), a->grad_buf, a->stream)) != cudaSuccess)
        return e;
    const int np = (ns + 1) * ns / 2;
    return launch_grad_reduce(a->A.gacc, np + 1, (unsigned)pl, a->partials, a->acc, a->stream);
}

}  // namespace

extern "C" {

nlbm_status nlbm_adjoint_workspace_bytes(const nlbm_params *p, int32_t nsteps, int32_t checkpoint_every,
                                         size_t *bytes)
{
    if (!bytes) { set_err(g_err, "bytes is NULL"); return NLBM_EINVAL; }
    AdjLayout L;
    nlbm_status st = adj_layout(p, nsteps, checkpoint_every, &L, g_err);
    if (st != NLBM_OK) return st;
    *bytes = L.total;
    return NLBM_OK;
}

nlbm_status nlbm_adjoint_create(const nlbm_params *p, int32_t nsteps, int32_t checkpoint_every, void *dev_workspace,
                                size_t workspace_bytes, void *cuda_stream, nlbm_adjoint **out)
{
    if (!out) { set_err(g_err, "out is NULL"); return NLBM_EINVAL; }
    *out = nullptr;
    AdjLayout L;
    nlbm_status st = adj_layout(p, nsteps, checkpoint_every, &L, g_err);
    if (st != NLBM_OK) return st;
    if (!dev_workspace || ((uintptr_t)dev_workspace & 255)) {
        set_err(g_err, "workspace must be non-NULL and 256-byte aligned");
        return NLBM_EINVAL;
    }
    if (workspace_bytes < L.total) {
        set_err(g_err, "workspace of %zu bytes is smaller than the %zu needed", workspace_bytes, L.total);
        return NLBM_ENOMEM;
    }
    nlbm_adjoint *a = new (std::nothrow) nlbm_adjoint();
    if (!a) { set_err(g_err, "host allocation failed"); return NLBM_ENOMEM; }
    char *ws = (char *)dev_workspace;
    st = nlbm_create(p, ws + L.sim, make_layout(p->n_phases - 1, (size_t)p->nx * p->ny, false).total, cuda_stream,
                     &a->sim);
    if (st != NLBM_OK) {
        delete a;
        return st;
    }
    a->ns = p->n_phases - 1;
    a->N = p->n_phases;
    a->nsteps = nsteps;
    a->every = checkpoint_every;
    a->nckpt = (nsteps + checkpoint_every - 1) / checkpoint_every;
    a->plane = (size_t)p->nx * p->ny;
    a->state_floats = adj_state_floats(a->ns, a->plane);
    a->stream = (cudaStream_t)cuda_stream;
    a->ws = ws;
    a->ckpt = (float *)(ws + L.ckpt);
    a->seg = (float *)(ws + L.seg);
    a->tapes = (float *)(ws + L.tapes);
    const AdjCounts c = adj_counts(a->ns);
    const size_t pl = a->plane;
    float *f = (float *)(ws + L.fields);
    auto take = [&](int planes) {
        float *q = f;
        f += (size_t)planes * pl;
        return q;
    };
    const int ns = a->ns;
    a->A.gacc = (double *)take(c.contrib);
    a->T.phi = take(ns);
    a->T.j = take(2 * ns);
    a->T.g = take(8);
    a->T.grad = take(2 * ns);
    a->T.lap = take(ns);
    a->T.R = take(2 * ns);
    a->T.mphi = take(2);
    a->T.w = take(1);
    a->T.F = take(2);
    a->seed[0] = take(c.seedset);
    a->seed[1] = take(c.seedset);
    a->A.lF = take(2);
    a->A.lphi_pw = take(ns);
    a->A.lj = take(2 * ns);
    a->A.lgrad = take(2 * ns);
    a->A.llap = take(ns);
    a->A.lR = take(2 * ns);
    a->A.lmphi = take(2);
    a->A.lg_pull = take(8);
    a->A.lphi_tot = take(ns);
    a->seed_buf = take(ns + 1);
    a->grad_buf = take(ns);
    a->partials = (double *)(ws + L.partials);
    a->acc = (double *)(ws + L.acc);
    a->final_set = 0;
    a->graph = nullptr;
    a->graph_tried = false;
    a->forward_done = false;
    a->err[0] = 0;
    *out = a;
    return NLBM_OK;
}

nlbm_status nlbm_adjoint_forward(nlbm_adjoint *a, const float *dev_phi0, float *dev_phi_final)
{
    if (!a || !dev_phi0) return NLBM_EINVAL;
    nlbm_sim *s = a->sim;
    s->cur = 0;
    nlbm_status st = nlbm_set_phi(s, dev_phi0);
    if (st != NLBM_OK) { memcpy(a->err, s->err, sizeof a->err); return st; }
    cudaError_t e;
    for (int k = 0; k < a->nckpt; ++k) {
        if ((e = adj_save_state(a, a->ckpt + a->state_floats * k)) != cudaSuccess) return adj_fail(a, e, "checkpoint");
        const int n = (k + 1) * a->every <= a->nsteps ? a->every : a->nsteps - k * a->every;
        if ((st = nlbm_step(s, n)) != NLBM_OK) { memcpy(a->err, s->err, sizeof a->err); return st; }
    }
    if (dev_phi_final && (st = nlbm_get_moments(s, dev_phi_final, nullptr, nullptr)) != NLBM_OK) {
        memcpy(a->err, s->err, sizeof a->err);
        return st;
    }
    a->forward_done = true;
    return NLBM_OK;
}

nlbm_status nlbm_adjoint_backward(nlbm_adjoint *a, const float *dev_seed, float *dev_grad_phi0,
                                  double *host_grad_sigma, double *host_grad_mobility)
{
    if (!a || !dev_seed) return NLBM_EINVAL;
    if (!a->forward_done) { set_err(a->err, "backward before forward"); return NLBM_EINVAL; }
    const size_t pl = a->plane, pb = sizeof(float) * pl;
    const int ns = a->ns, N = a->N, np = N * (N - 1) / 2;
    const AdjCounts c = adj_counts(ns);
    cudaError_t e = cudaMemcpyAsync(a->seed_buf, dev_seed, pb * N, cudaMemcpyDeviceToDevice, a->stream);
    if (e != cudaSuccess) return adj_fail(a, e, "seed copy");
    // The sweep is the same sequence of launches for every call of this
    // handle: capture it into a CUDA graph once (on a capturable stream) and
    // replay it.
    if (!a->graph && !a->graph_tried && a->stream != nullptr) {
        a->graph_tried = true;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(a->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            cudaError_t eb = adj_backward_body(a);
            cudaError_t ec = cudaStreamEndCapture(a->stream, &g);
            if (eb == cudaSuccess && ec == cudaSuccess && cudaGraphInstantiate(&a->graph, g, 0) != cudaSuccess)
                a->graph = nullptr;
            if (g) cudaGraphDestroy(g);
        }
        cudaGetLastError();   // a failed capture leaves the direct path
    }
    if (a->graph) {
        e = cudaGraphLaunch(a->graph, a->stream);
        if (e != cudaSuccess) return adj_fail(a, e, "graph launch");
    } else if ((e = adj_backward_body(a)) != cudaSuccess) {
        return adj_fail(a, e, "reverse sweep");
    }
    a->sim->launches += adj_sweep_launches(a);
    if (dev_grad_phi0 &&
        (e = cudaMemcpyAsync(dev_grad_phi0, a->grad_buf, pb * ns, cudaMemcpyDeviceToDevice, a->stream)) != cudaSuccess)
        return adj_fail(a, e, "phi0 gradient");
    double acc[kMaxPhases * kMaxPhases + 1];
    if ((e = cudaMemcpyAsync(acc, a->acc, sizeof(double) * (np + 1), cudaMemcpyDeviceToHost, a->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(a->stream)) != cudaSuccess)
        return adj_fail(a, e, "gradient download");
    (void)c;
    if (host_grad_sigma) {
        for (int i = 0; i < N * N; ++i) host_grad_sigma[i] = 0.0;
        int q = 0;
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j, ++q) host_grad_sigma[i * N + j] = host_grad_sigma[j * N + i] = acc[q];
    }
    if (host_grad_mobility) *host_grad_mobility = acc[np];
    return NLBM_OK;
}

nlbm_status nlbm_adjoint_reverse_step(nlbm_adjoint *a, const float *dev_state, const float *dev_seed_out,
                                      float *dev_seed_in, double *host_grad_sigma, double *host_grad_mobility)
{
    if (!a || !dev_state || !dev_seed_out || !dev_seed_in) return NLBM_EINVAL;
    const size_t pl = a->plane, pb = sizeof(float) * pl;
    const int ns = a->ns, N = a->N, np = N * (N - 1) / 2;
    const AdjCounts c = adj_counts(ns);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(a->seed[0], dev_seed_out, pb * c.seedset, cudaMemcpyDeviceToDevice, a->stream)) != cudaSuccess ||
        (e = cudaMemsetAsync(a->A.gacc, 0, pb * c.contrib, a->stream)) != cudaSuccess)
        return adj_fail(a, e, "seed");
    const StepParams kp = adj_params_from_state(a, dev_state);
    if ((e = launch_reverse_step(ns, kp, a->T, adj_fields(a, a->seed[0], a->seed[1]), false, a->stream)) != cudaSuccess ||
        (e = launch_grad_reduce(a->A.gacc, np + 1, (unsigned)pl, a->partials, a->acc, a->stream)) != cudaSuccess)
        return adj_fail(a, e, "reverse step");
    a->sim->launches += 9;
    double acc[kMaxPhases * kMaxPhases + 1];
    if ((e = cudaMemcpyAsync(dev_seed_in, a->seed[1], pb * c.seedset, cudaMemcpyDeviceToDevice, a->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(acc, a->acc, sizeof(double) * (np + 1), cudaMemcpyDeviceToHost, a->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(a->stream)) != cudaSuccess)
        return adj_fail(a, e, "reverse step results");
    if (host_grad_sigma) {
        for (int i = 0; i < N * N; ++i) host_grad_sigma[i] = 0.0;
        int q = 0;
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j, ++q) host_grad_sigma[i * N + j] = host_grad_sigma[j * N + i] = acc[q];
    }
    if (host_grad_mobility) *host_grad_mobility = acc[np];
    return NLBM_OK;
}

int32_t nlbm_adjoint_uses_graph(const nlbm_adjoint *a) { return a && a->graph ? 1 : 0; }

int64_t nlbm_adjoint_kernel_launches(const nlbm_adjoint *a) { return a ? a->sim->launches : -1; }

void nlbm_adjoint_destroy(nlbm_adjoint *a)
{
    if (!a) return;
    if (a->graph) cudaGraphExecDestroy(a->graph);
    nlbm_destroy(a->sim);
    delete a;
}

const char *nlbm_adjoint_last_error(const nlbm_adjoint *a) { return a ? a->err : g_err; }

}  // extern "C"

extern "C" {

const char *nlbm_last_error(const nlbm_sim *s) { return s ? s->err : g_err; }

const char *nlbm_status_string(nlbm_status st)
{
    switch (st) {
    case NLBM_OK: return "ok";
    case NLBM_EINVAL: return "invalid argument";
    case NLBM_ENOMEM: return "insufficient memory";
    case NLBM_ECUDA: return "CUDA error";
    case NLBM_ENOTSUP: return "not supported";
    case NLBM_EDIVERGED: return "diverged";
    default: return "unknown status";
    }
}

}  // extern "C"
