/*
 * nlbm_oracle.c -- plain, slow, FP64 CPU oracle for the consistent and
 * conservative lattice Boltzmann method for immiscible N-phase flow
 * (Zhan, Liu, Chai & Shi, arXiv 2306.06983).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * only the test-suite, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code, header, table or constant with the
 * CUDA library; it is written independently from the paper.
 *
 * What it computes, one time step, in the paper's order:
 *   Sec. 3, Eq. (25a)      phi_p = sum_i f_{i,p}; phi_N = 1 - sum_{p<N} phi_p
 *                          (Sec. 4: only N-1 phase equations are solved)
 *   Sec. 2.2, Eqs. (11)-(12) rho = sum rho_p phi_p, mu = sum mu_p phi_p
 *   Sec. 3, Eq. (27)       isotropic central gradient and Laplacian
 *   Sec. 2.1, Eqs. (2)-(4) Model A / Model B source R_p
 *   Sec. 2.2, Eq. (13)     m_phi = -sum_p rho_p M (grad phi_p - R_p)
 *   Sec. 2.2, Eqs. (15)-(17) chemical potential, potential-form F_s
 *   Sec. 3, text after (24) F_c = -div(m_phi u - u m_phi)/2, u lagged
 *   Sec. 3, Eqs. (25b),(25c) velocity and pressure
 *   Sec. 3, Eq. (26)       tau_g from the local mixture viscosity
 *   Sec. 3, Eqs. (18)-(20) phase-field MRT collision with source
 *   Sec. 3, Eqs. (21)-(24) flow MRT collision with forcing
 *   Sec. 4, Eq. (28)       natural moment matrix M, diagonal S, collision in
 *                          moment space  f* = f - M^-1 S M (f - f^eq)
 *                                              + M^-1 (I - S/2) M R
 *   Sec. 4                 streaming, periodic or half-way bounce-back
 *
 * The collision is evaluated literally with explicit 9x9 matrices (M is
 * inverted numerically at set-up); the equilibria and source distributions
 * are evaluated per direction from their defining formulas.
 *
 * Readings of points the paper leaves open:
 *  - Eqs. (18),(21): the collision term is the matrix product
 *    sum_j Lambda_ij (f_j - f_j^eq).
 *  - A unit vector v/|v| is taken as 0 when |v|^2 <= 1e-24.
 *  - Model B pairwise normal: quotient rule of the discrete gradients
 *    (Eq. (8), first equality), so n_pq = unit(phi_q grad phi_p - phi_p grad phi_q).
 *  - Model A weights use max(phi,0)^n.
 *  - Every u inside the force F (i.e. in F_c) is the previous step's u; all
 *    other u are the current one.  Time derivatives are backward Euler.
 *    Before the first step the fluid is at rest: u(-1) = 0, phi(-1) = phi(0),
 *    m_phi(-1) = 0 (it only ever multiplies u(-1)).
 *  - F_c,b = -1/2 sum_a d_a (m_phi,a u_b - u_a m_phi,b).
 *  - rho_0 in lambda_0 is taken as 0 (g_0 feeds no macroscopic quantity).
 *  - F_g = rho g (gravity as a body force per unit volume, Sec. 2.2).
 *  - Wall ghosts for stencils: phi mirrored, u negated (no slip), m_phi
 *    reflected (normal component negated).  At a wetting y wall (Sec. 4.2:
 *    n_w . grad phi_p = sum_{q != p} (4/eps) phi_p phi_q cos theta_pq, the
 *    pairwise angles from the N-1 given cos theta_pN by Young's relation,
 *    n_w the fluid's outward normal, pointing into the wall: an acute
 *    theta_pq makes phase p spread) the ghost row at distance k = 1, 2 is
 *    its mirror image plus (2k - 1) s_p, s_p that right-hand side at the
 *    image node, so that the difference across the wall (ghost minus first
 *    row) equals s_p; m_phi at such a ghost node is
 *    evaluated there from the ghost phase fields (Eqs. (3), (13)).  With all
 *    cos theta_pN = 0 this is the plain mirror (no-flux).
 *  - Initial state: f_i = w_i phi_p, g_i = lambda_i(P=0), u = 0, P = 0.
 *    A state that starts in motion (or_set_velocity, test cases only) takes
 *    the equilibria at the given u, with the pressure of lambda_i chosen so
 *    that Eq. (25c) recovers P = 0, and the initial values as the previous
 *    ones of the first step's time derivatives.
 *
 * Pins (tests/test_oracle_*.py) check every part of the step against what
 * the paper and the mathematics fix.  Parity unpinned: two O(dt) terms of
 * the Chapman-Enskog balance, d_t((m_phi u + u m_phi)/2) in M_2F (Eq. (24))
 * and d_t(phi_p u) in the phase-field source distribution (Eq. (19)).
 * Dropping either changes only the constant of a second-order error (the
 * uniform flow along relaxing interfaces still converges at second order),
 * so no result the paper fixes detects it; both are evaluated as printed,
 * with the explicit Euler derivative of Sec. 3.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 9
#define MAXN 8

/* Working precision.  The oracle is FP64 (the default).  Built with
 * -DORACLE_FP32 the same source runs in FP32 as a noise model: the spread
 * between the two builds is what FP32 rounding alone does to the method,
 * which sets the scale of the GPU parity tolerances.  The FP32 build is
 * never a reference value. */
#ifdef ORACLE_FP32
typedef float real;
#define RSQRT_(x) sqrtf(x)
#define RPOW_(x, y) powf(x, y)
#define RFABS_(x) fabsf(x)
#else
typedef double real;
#define RSQRT_(x) sqrt(x)
#define RPOW_(x, y) pow(x, y)
#define RFABS_(x) fabs(x)
#endif

/* D2Q9 lattice, Sec. 4: the velocity order is the column order of the
 * moment matrix in Eq. (28); c_s^2 = 1/3 with dx = dt = 1. */
static const int CX[Q] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[Q] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const real W[Q] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                            1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
static const real CS2 = 1.0 / 3.0;

typedef struct {
    int32_t nx, ny;
    int32_t n_phases;   /* N */
    int32_t model;      /* 0 = Model A (Eq. 2), 1 = Model B (Eq. 3) */
    int32_t wall_x, wall_y; /* 0 periodic, 1 half-way bounce-back walls */
    int32_t solve_all;  /* 0: N-1 LB sets (paper); 1: all N sets */
    int32_t store16;    /* noise-model build only: 0 none, 1 bfloat16, 2 binary16
                           rounding of the stored moving populations */
    double model_a_n;   /* exponent n of Model A */
    double eps;         /* interface thickness epsilon */
    double mobility;    /* M */
    double rho[MAXN];
    double mu[MAXN];    /* dynamic viscosities */
    double sigma[MAXN * MAXN];
    double unit_delta;  /* 0: unit vectors read as 0 when |v|^2 <= 1e-24; > 0: the
                           smooth reading v / sqrt(|v|^2 + delta^2) */
    double gx, gy;      /* gravity g: F_g = rho g */
    double wall_cos[2 * MAXN]; /* cos theta_pN, p < N-1, of the wall at y = 0
                           ([p]) and at y = ny - 1 ([MAXN + p]); 0 = no-flux */
} or_params;

typedef struct {
    or_params p;
    int N, L;           /* phases, LB-solved phase sets */
    size_t n;           /* nodes */
    real Mm[Q][Q], Mi[Q][Q];
    real tau_f;
    int wet;            /* a y wall with some cos theta_pN != 0 */
    real wc[2][MAXN][MAXN]; /* (4/eps) cos theta_pq of the two y walls */
    long long steps;
    /* state */
    real *f, *fn;     /* [L][Q][n] post-streaming populations, spare */
    real *g, *gn;     /* [Q][n] */
    real *phi_prev;   /* [N][n] */
    real *u_prev;     /* [2][n] */
    real *mphi_prev;  /* [2][n] */
    /* last computed macroscopic fields */
    real *phi;        /* [N][n] */
    real *u;          /* [2][n] */
    real *P;          /* [n] */
    /* per-step work fields */
    real *grad;       /* [N][2][n] */
    real *lap;        /* [N][n] */
    real *R;          /* [N][2][n] */
    real *mphi;       /* [2][n] */
    real *muphi;      /* [N][n] */
    real *F;          /* [2][n] total force */
    real *Fc;         /* [2][n] F_c alone */
    real *rho, *mu;   /* [n] */
    real *gradrho;    /* [2][n] */
} or_sim;

/* ---------------------------------------------------------------- helpers */

/* Map a coordinate onto the stored lattice.  Periodic axes wrap.  Wall axes
 * (half-way bounce-back, the wall lies half a spacing outside the first and
 * last node) mirror a ghost node onto its image; *flip is set to 1 when a
 * mirror was applied. */
static int map_coord(int c, int n, int wall, int *flip)
{
    *flip = 0;
    if (c >= 0 && c < n) return c;
    if (!wall) {
        c %= n;
        if (c < 0) c += n;
        return c;
    }
    *flip = 1;
    return c < 0 ? -1 - c : 2 * n - 1 - c;
}

static size_t nid(const or_sim *s, int x, int y) { return (size_t)y * s->p.nx + x; }

/* Kinds of ghost treatment: a scalar phase field is mirrored; the velocity
 * is negated on each mirrored axis (no slip); a flux vector is reflected
 * (its component normal to the mirrored wall is negated). */
enum { K_SCALAR = 0, K_VELOCITY = 1, K_REFLECT = 2 };

static real fetch_scalar(const or_sim *s, const real *F, int x, int y)
{
    int fx, fy;
    int xx = map_coord(x, s->p.nx, s->p.wall_x, &fx);
    int yy = map_coord(y, s->p.ny, s->p.wall_y, &fy);
    return F[nid(s, xx, yy)];
}

static void fetch_vec(const or_sim *s, const real *V, int x, int y, int kind,
                      real *vx, real *vy)
{
    int fx, fy;
    int xx = map_coord(x, s->p.nx, s->p.wall_x, &fx);
    int yy = map_coord(y, s->p.ny, s->p.wall_y, &fy);
    size_t k = nid(s, xx, yy);
    real a = V[k], b = V[s->n + k];
    if (kind == K_VELOCITY) {
        if (fx) { a = -a; b = -b; }
        if (fy) { a = -a; b = -b; }
    } else if (kind == K_REFLECT) {
        if (fx) a = -a;
        if (fy) b = -b;
    }
    *vx = a;
    *vy = b;
}

/* Phase field p at (x, y), ghosts included (the wetting ghost rows are
 * described at the top of this file). */
static real fetch_phi(const or_sim *s, int p, int x, int y)
{
    int fx, fy;
    int xx = map_coord(x, s->p.nx, s->p.wall_x, &fx);
    int yy = map_coord(y, s->p.ny, s->p.wall_y, &fy);
    size_t k = nid(s, xx, yy);
    real v = s->phi[p * s->n + k];
    if (s->wet && fy) {
        const int w = y < 0 ? 0 : 1;
        const int d = y < 0 ? -y : y - (s->p.ny - 1);
        real sp = 0;
        for (int q = 0; q < s->N; q++) sp += s->wc[w][p][q] * s->phi[q * s->n + k];
        v += (2 * d - 1) * v * sp;
    }
    return v;
}

/* Eq. (27) on phase field p (ghosts from fetch_phi). */
static void grad_phi_at(const or_sim *s, int p, int x, int y, real *gx, real *gy)
{
    real ax = 0, ay = 0;
    for (int i = 1; i < Q; i++) {
        real v = fetch_phi(s, p, x + CX[i], y + CY[i]);
        ax += W[i] * CX[i] * v;
        ay += W[i] * CY[i] * v;
    }
    *gx = ax / CS2;
    *gy = ay / CS2;
}

static real lap_phi_at(const or_sim *s, int p, int x, int y)
{
    real c0 = fetch_phi(s, p, x, y), a = 0;
    for (int i = 1; i < Q; i++) a += 2.0 * W[i] * (fetch_phi(s, p, x + CX[i], y + CY[i]) - c0);
    return a / CS2;
}

/* Sec. 3, Eq. (27): grad chi = sum_{i!=0} w_i c_i chi(x+c_i) / (c_s^2 dt). */
static void grad_at(const or_sim *s, const real *F, int x, int y, real *gx, real *gy)
{
    real ax = 0, ay = 0;
    for (int i = 1; i < Q; i++) {
        real v = fetch_scalar(s, F, x + CX[i], y + CY[i]);
        ax += W[i] * CX[i] * v;
        ay += W[i] * CY[i] * v;
    }
    *gx = ax / CS2;
    *gy = ay / CS2;
}

/* Sec. 3, Eq. (27): lap chi = sum_{i!=0} 2 w_i (chi(x+c_i) - chi(x)) / (c_s^2 dt^2). */
static real lap_at(const or_sim *s, const real *F, int x, int y)
{
    real c0 = fetch_scalar(s, F, x, y), a = 0;
    for (int i = 1; i < Q; i++) a += 2.0 * W[i] * (fetch_scalar(s, F, x + CX[i], y + CY[i]) - c0);
    return a / CS2;
}

/* Unit vector with the zero-gradient reading: 0 when |v|^2 <= 1e-24. */
static void unit(real vx, real vy, real delta, real *nx, real *ny)
{
    real n2 = vx * vx + vy * vy;
    if (delta > 0) {
        real r = RSQRT_(n2 + delta * delta);
        *nx = vx / r;
        *ny = vy / r;
    } else if (n2 > 1e-24) {
        real r = RSQRT_(n2);
        *nx = vx / r;
        *ny = vy / r;
    } else {
        *nx = 0;
        *ny = 0;
    }
}

/* Invert a 9x9 matrix by Gauss-Jordan elimination with partial pivoting. */
static int invert9(real A[Q][Q], real B[Q][Q])
{
    real T[Q][2 * Q];
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < 2 * Q; j++) T[i][j] = j < Q ? A[i][j] : (j - Q == i);
    for (int c = 0; c < Q; c++) {
        int piv = c;
        for (int r = c + 1; r < Q; r++)
            if (RFABS_(T[r][c]) > RFABS_(T[piv][c])) piv = r;
        if (RFABS_(T[piv][c]) < (real)1e-7) return -1;
        if (piv != c)
            for (int j = 0; j < 2 * Q; j++) {
                real t = T[c][j];
                T[c][j] = T[piv][j];
                T[piv][j] = t;
            }
        real d = T[c][c];
        for (int j = 0; j < 2 * Q; j++) T[c][j] /= d;
        for (int r = 0; r < Q; r++)
            if (r != c) {
                real f = T[r][c];
                if (f != 0)
                    for (int j = 0; j < 2 * Q; j++) T[r][j] -= f * T[c][j];
            }
    }
    for (int i = 0; i < Q; i++)
        for (int j = 0; j < Q; j++) B[i][j] = T[i][Q + j];
    return 0;
}

/* Sec. 4, Eq. (28): rows 1, c_x, c_y, c_x^2, c_y^2, c_x c_y, c_x^2 c_y,
 * c_x c_y^2, c_x^2 c_y^2 evaluated on the velocity set. */
static void build_M(real Mm[Q][Q])
{
    for (int i = 0; i < Q; i++) {
        real x = CX[i], y = CY[i];
        Mm[0][i] = 1;
        Mm[1][i] = x;
        Mm[2][i] = y;
        Mm[3][i] = x * x;
        Mm[4][i] = y * y;
        Mm[5][i] = x * y;
        Mm[6][i] = x * x * y;
        Mm[7][i] = x * y * y;
        Mm[8][i] = x * x * y * y;
    }
}

/* Moment-space MRT update, Sec. 4: out = f - M^-1 S M (f - feq) + M^-1 (I - S/2) M src. */
static void mrt(const or_sim *s, const real f[Q], const real feq[Q], const real src[Q],
                const real S[Q], real out[Q])
{
    real m[Q], meq[Q], ms[Q], mstar[Q];
    for (int k = 0; k < Q; k++) {
        real a = 0, b = 0, c = 0;
        for (int i = 0; i < Q; i++) {
            a += s->Mm[k][i] * f[i];
            b += s->Mm[k][i] * feq[i];
            c += s->Mm[k][i] * src[i];
        }
        m[k] = a;
        meq[k] = b;
        ms[k] = c;
    }
    for (int k = 0; k < Q; k++) mstar[k] = m[k] - S[k] * (m[k] - meq[k]) + (1.0 - 0.5 * S[k]) * ms[k];
    for (int i = 0; i < Q; i++) {
        real a = 0;
        for (int k = 0; k < Q; k++) a += s->Mi[i][k] * mstar[k];
        out[i] = a;
    }
}

/* ------------------------------------------------- pointwise model pieces */

/* Sec. 3, Eq. (19): f^eq_i = w_i phi (1 + c_i.u / c_s^2). */
void or_phase_feq(real phi, real ux, real uy, real out[Q])
{
    for (int i = 0; i < Q; i++) out[i] = W[i] * phi * (1.0 + (CX[i] * ux + CY[i] * uy) / CS2);
}

/* Sec. 3, Eq. (19): R_i = w_i [c_i . d_t(phi u) / c_s^2 + c_i . R_p]. */
void or_phase_src(real dtphiux, real dtphiuy, real Rx, real Ry, real out[Q])
{
    for (int i = 0; i < Q; i++)
        out[i] = W[i] * ((CX[i] * dtphiux + CY[i] * dtphiuy) / CS2 + CX[i] * Rx + CY[i] * Ry);
}

/* Sec. 3, Eq. (22): g^eq_i = lambda_i + w_i [c_i.(rho u)/c_s^2
 *   + (m u):(c_i c_i - c_s^2 I)/(2 c_s^4)], lambda_0 = (w_0 - 1) P/c_s^2 + rho_0,
 *   lambda_i = w_i P / c_s^2. */
void or_flow_geq(real P, real rho0, real rho, real ux, real uy, real mx, real my,
                 real out[Q])
{
    for (int i = 0; i < Q; i++) {
        real lam = i == 0 ? (W[0] - 1.0) * P / CS2 + rho0 : W[i] * P / CS2;
        real cu = CX[i] * ux + CY[i] * uy;
        real cm = CX[i] * mx + CY[i] * my;
        /* (m u):(c c - c_s^2 I) = (m.c)(u.c) - c_s^2 m.u */
        real mu2 = cm * cu - CS2 * (mx * ux + my * uy);
        out[i] = lam + W[i] * (rho * cu / CS2 + mu2 / (2.0 * CS2 * CS2));
    }
}

/* Sec. 3, Eq. (23): F_i = w_i [u.grad rho + c_i.F/c_s^2
 *   + (M_2F - c_s^2 (u.grad rho) I):(c_i c_i - c_s^2 I)/(2 c_s^4)],
 * with M_2F given as its components (xx, xy, yx, yy). */
void or_flow_force(real ugr, real Fx, real Fy, const real M2F[4], real out[Q])
{
    for (int i = 0; i < Q; i++) {
        real T[2][2] = {{M2F[0] - CS2 * ugr, M2F[1]}, {M2F[2], M2F[3] - CS2 * ugr}};
        real c[2] = {(real)CX[i], (real)CY[i]};
        real con = 0;
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) con += T[a][b] * (c[a] * c[b] - (a == b ? CS2 : 0.0));
        out[i] = W[i] * (ugr + (c[0] * Fx + c[1] * Fy) / CS2 + con / (2.0 * CS2 * CS2));
    }
}

/* g'(s) for g(s) = s^2 (1-s)^2, Sec. 2.2 below Eq. (14). */
static real gprime(real s) { return 2.0 * s * (1.0 - s) * (1.0 - 2.0 * s); }

/* Sec. 2.1, Eqs. (2)-(4): source R_p at one node for all N phases, given
 * phi[N] and grad phi[N][2]. */
static void source_at(const or_params *pp, int N, const real *phi, const real (*gp)[2],
                      real (*R)[2])
{
    const real eps = pp->eps;
    if (pp->model == 0) {
        /* Model A, Eq. (2): R_p = a_p n_p - beta_p,
         * beta_p = phi_p^n / sum_q phi_q^n * sum_q a_q n_q, a_q = 4 phi_q (1-phi_q)/eps */
        real sumw = 0, Vx = 0, Vy = 0, a[MAXN], nvx[MAXN], nvy[MAXN], w[MAXN];
        for (int q = 0; q < N; q++) {
            a[q] = 4.0 * phi[q] * (1.0 - phi[q]) / eps;
            unit(gp[q][0], gp[q][1], (real)pp->unit_delta, &nvx[q], &nvy[q]);
            w[q] = RPOW_(phi[q] > 0 ? phi[q] : (real)0, (real)pp->model_a_n);
            sumw += w[q];
            Vx += a[q] * nvx[q];
            Vy += a[q] * nvy[q];
        }
        for (int p = 0; p < N; p++) {
            real b = w[p] / sumw;
            R[p][0] = a[p] * nvx[p] - b * Vx;
            R[p][1] = a[p] * nvy[p] - b * Vy;
        }
    } else {
        /* Model B, Eqs. (3)-(4): R_p = sum_{q!=p} 4 phi_p phi_q / eps n_pq,
         * n_pq = grad phi_pq / |grad phi_pq|, phi_pq = phi_p/(phi_p+phi_q). */
        for (int p = 0; p < N; p++) {
            real rx = 0, ry = 0;
            for (int q = 0; q < N; q++) {
                if (q == p) continue;
                real vx = phi[q] * gp[p][0] - phi[p] * gp[q][0];
                real vy = phi[q] * gp[p][1] - phi[p] * gp[q][1];
                real ux, uy;
                unit(vx, vy, (real)pp->unit_delta, &ux, &uy);
                real c = 4.0 * phi[p] * phi[q] / eps;
                rx += c * ux;
                ry += c * uy;
            }
            R[p][0] = rx;
            R[p][1] = ry;
        }
    }
}

/* --------------------------------------------------------------- life cycle */

static int valid(const or_params *p)
{
#ifdef ORACLE_FP32
    if (p->store16 < 0 || p->store16 > 2) return 0;
#else
    if (p->store16 != 0) return 0;   /* the oracle proper stores exact values */
#endif
    if (p->nx < 1 || p->ny < 1 || p->n_phases < 2 || p->n_phases > MAXN) return 0;
    if ((p->wall_x && p->nx < 4) || (p->wall_y && p->ny < 4)) return 0;
    if (!(p->eps > 0) || !(p->mobility > 0)) return 0;
    if (!(p->unit_delta >= 0) || !isfinite(p->unit_delta)) return 0;
    if (!isfinite(p->gx) || !isfinite(p->gy)) return 0;
    for (int w = 0; w < 2; w++)
        for (int a = 0; a < MAXN; a++) {
            double c = p->wall_cos[w * MAXN + a];
            if (!(fabs(c) <= 1.0)) return 0;
            if (c != 0 && (!p->wall_y || a >= p->n_phases - 1)) return 0;
        }
    if (p->model != 0 && p->model != 1) return 0;
    if (p->model == 0 && !(p->model_a_n > 0)) return 0;
    for (int a = 0; a < p->n_phases; a++) {
        if (!(p->rho[a] > 0) || !(p->mu[a] > 0)) return 0;
        for (int b = 0; b < p->n_phases; b++) {
            double s = p->sigma[a * MAXN + b];
            if (a == b ? s != 0 : !(s > 0)) return 0;
            if (s != p->sigma[b * MAXN + a]) return 0;
        }
    }
    return 1;
}

void or_destroy(void *h)
{
    or_sim *s = (or_sim *)h;
    if (!s) return;
    real *bufs[] = {s->f, s->fn, s->g, s->gn, s->phi_prev, s->u_prev, s->mphi_prev, s->phi,
                      s->u, s->P, s->grad, s->lap, s->R, s->mphi, s->muphi, s->F, s->Fc, s->rho,
                      s->mu, s->gradrho};
    for (size_t i = 0; i < sizeof bufs / sizeof bufs[0]; i++) free(bufs[i]);
    free(s);
}

void *or_create(const or_params *p)
{
    if (!valid(p)) return NULL;
    or_sim *s = (or_sim *)calloc(1, sizeof(or_sim));
    if (!s) return NULL;
    s->p = *p;
    s->N = p->n_phases;
    s->L = p->solve_all ? s->N : s->N - 1;
    s->n = (size_t)p->nx * p->ny;
    /* Sec. 3, Eq. (20): M = (tau_f - 0.5) c_s^2 dt. */
    s->tau_f = 0.5 + p->mobility / CS2;
    /* Sec. 4.2: cos theta_pq from the N-1 angles against phase N (Young's
     * relation), cos theta_qp = -cos theta_pq; stored times 4/eps. */
    for (int w = 0; w < 2; w++) {
        const int N = s->N;
        const double *cn = p->wall_cos + w * MAXN;
        for (int a = 0; a < N; a++)
            for (int b = 0; b < N; b++) {
                double c = 0;
                if (a != b) {
                    if (b == N - 1) c = cn[a];
                    else if (a == N - 1) c = -cn[b];
                    else c = (p->sigma[a * MAXN + N - 1] * cn[a] - p->sigma[b * MAXN + N - 1] * cn[b]) /
                             p->sigma[a * MAXN + b];
                }
                s->wc[w][a][b] = (real)(4.0 / p->eps * c);
                if (c != 0) s->wet = 1;
            }
    }
    build_M(s->Mm);
    if (invert9(s->Mm, s->Mi)) {
        or_destroy(s);
        return NULL;
    }
    size_t n = s->n, N = s->N, L = s->L;
#define ALLOC(ptr, cnt)                                  \
    do {                                                 \
        (ptr) = (real *)calloc((cnt), sizeof(real)); \
        if (!(ptr)) {                                    \
            or_destroy(s);                               \
            return NULL;                                 \
        }                                                \
    } while (0)
    ALLOC(s->f, L * Q * n);
    ALLOC(s->fn, L * Q * n);
    ALLOC(s->g, Q * n);
    ALLOC(s->gn, Q * n);
    ALLOC(s->phi_prev, N * n);
    ALLOC(s->u_prev, 2 * n);
    ALLOC(s->mphi_prev, 2 * n);
    ALLOC(s->phi, N * n);
    ALLOC(s->u, 2 * n);
    ALLOC(s->P, n);
    ALLOC(s->grad, N * 2 * n);
    ALLOC(s->lap, N * n);
    ALLOC(s->R, N * 2 * n);
    ALLOC(s->mphi, 2 * n);
    ALLOC(s->muphi, N * n);
    ALLOC(s->F, 2 * n);
    ALLOC(s->Fc, 2 * n);
    ALLOC(s->rho, n);
    ALLOC(s->mu, n);
    ALLOC(s->gradrho, 2 * n);
#undef ALLOC
    return s;
}

/* Initial state (reading: fluid at rest): phi given for phases 1..N-1,
 * phi_N = 1 - sum; f_i = w_i phi_p; g_i = lambda_i with P = 0 and rho_0 = 0,
 * i.e. g = 0; u = 0, P = 0; the "previous" fields equal the initial ones. */
void or_set_phi(void *h, const real *phi_in)
{
    or_sim *s = (or_sim *)h;
    size_t n = s->n;
    int N = s->N;
    for (size_t k = 0; k < n; k++) {
        real sum = 0;
        for (int p = 0; p < N - 1; p++) {
            s->phi[p * n + k] = phi_in[p * n + k];
            sum += phi_in[p * n + k];
        }
        s->phi[(N - 1) * n + k] = 1.0 - sum;
    }
    for (int p = 0; p < s->L; p++)
        for (int i = 0; i < Q; i++)
            for (size_t k = 0; k < n; k++) s->f[(p * Q + i) * n + k] = W[i] * s->phi[p * n + k];
    memset(s->g, 0, Q * n * sizeof(real));
    memcpy(s->phi_prev, s->phi, N * n * sizeof(real));
    memset(s->u_prev, 0, 2 * n * sizeof(real));
    memset(s->mphi_prev, 0, 2 * n * sizeof(real));
    memset(s->u, 0, 2 * n * sizeof(real));
    memset(s->P, 0, n * sizeof(real));
    s->steps = 0;
}

/* ------------------------------------------------------------------ one step */

static void eval_fields(or_sim *s);

/* Initial velocity field u0 [2][n] for a state set by or_set_phi (test
 * cases that start in motion, such as a drop carried by a uniform flow):
 * f_i = f^eq_i(phi_p, u0) (Eq. (19)), g_i = g^eq_i (Eq. (22)) with
 * m = rho u0 + m_phi, m_phi of the initial fields (Eq. (13)), and the
 * pressure of lambda_i chosen so that Eq. (25c) recovers P = 0 from these
 * populations (it adds dt u.grad rho / 2 to the populations' own sum:
 * lambda_i takes P' = -c_s^2 u0.grad rho / (2 (1 - w_0))); the "previous"
 * values of the first step's time derivatives are the initial ones:
 * u(-1) = u0, phi(-1) = phi(0), m_phi(-1) = m_phi(0), so that a flow in
 * steady translation starts without a jump.  With u0 = 0 this is the
 * state of or_set_phi. */
void or_set_velocity(void *h, const real *u0)
{
    or_sim *s = (or_sim *)h;
    const size_t n = s->n;
    const int N = s->N;
    eval_fields(s);   /* phi, rho, grad phi, R and m_phi of f = w_i phi */
    for (size_t k = 0; k < n; k++) {
        const real ux = u0[k], uy = u0[n + k];
        for (int p = 0; p < s->L; p++) {
            real feq[Q];
            or_phase_feq(s->phi[p * n + k], ux, uy, feq);
            for (int i = 0; i < Q; i++) s->f[(p * Q + i) * n + k] = feq[i];
        }
        const real rho = s->rho[k];
        const real mx = rho * ux + s->mphi[k], my = rho * uy + s->mphi[n + k];
        const real ugr = ux * s->gradrho[k] + uy * s->gradrho[n + k];
        real geq[Q];
        or_flow_geq(-CS2 * ugr / (2.0 * (1.0 - W[0])), 0.0, rho, ux, uy, mx, my, geq);
        for (int i = 0; i < Q; i++) s->g[i * n + k] = geq[i];
        s->u[k] = s->u_prev[k] = ux;
        s->u[n + k] = s->u_prev[n + k] = uy;
        s->mphi_prev[k] = s->mphi[k];
        s->mphi_prev[n + k] = s->mphi[n + k];
        s->P[k] = 0;
    }
    memcpy(s->phi_prev, s->phi, N * n * sizeof(real));
}

#ifdef ORACLE_FP32
/* Noise model of 16-bit population storage (FP32 build only; never a
 * reference value).  A value v is rounded to nearest-even with p significant
 * bits: 8 for bfloat16 (FP32 exponent range), 11 for binary16 (normal range
 * down to 2^-14, fixed quantum 2^-24 below it). */
static real round16(real v, int mode)
{
    if (v == 0 || !isfinite(v)) return v;
    double a = fabs((double)v);
    int ex;
    frexp(a, &ex);                   /* a = m 2^ex, m in [0.5, 1) */
    int lead = ex - 1;               /* exponent of the leading bit */
    int p = mode == 1 ? 8 : 11;
    if (mode == 2 && lead < -14) lead = -14;
    double q = ldexp(1.0, lead - p + 1);
    double r = nearbyint(a / q) * q;
    return (real)copysign(r, (double)v);
}

/* Streaming with the stored moving populations rounded as deviations from
 * a lattice-weight multiple of a field the receiving side knows: f_i minus
 * w_i phi_p of the node that receives it (this step's phi), g_i minus
 * 3 w_i P of the node that sends it; the rest population keeps each node's
 * post-collision total.  Same links as the exact streaming. */
static void stream_store16(or_sim *s)
{
    static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
    const or_params *pp = &s->p;
    const int nx = pp->nx, ny = pp->ny, L = s->L;
    const size_t n = s->n;
    const int mode = pp->store16;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t k = nid(s, x, y);
            real acc[MAXN], tot[MAXN];
            for (int p = 0; p < L; p++) {
                acc[p] = 0;
                tot[p] = 0;
                for (int i = 0; i < Q; i++) tot[p] += s->f[(p * Q + i) * n + k];
            }
            for (int i = 1; i < Q; i++) {
                int tx = x + CX[i], ty = y + CY[i];
                int out_x = tx < 0 || tx >= nx, out_y = ty < 0 || ty >= ny;
                int bounce = (out_x && pp->wall_x) || (out_y && pp->wall_y);
                size_t dst;
                int di;
                if (bounce) {
                    dst = k;
                    di = OPP[i];
                } else {
                    tx = (tx % nx + nx) % nx;
                    ty = (ty % ny + ny) % ny;
                    dst = nid(s, tx, ty);
                    di = i;
                }
                for (int p = 0; p < L; p++) {
                    real base = W[i] * s->phi[p * n + dst];
                    real v = base + round16(s->f[(p * Q + i) * n + k] - base, mode);
                    s->fn[(p * Q + di) * n + dst] = v;
                    acc[p] += v;
                }
                real gb = 3 * W[i] * s->P[k];
                s->gn[di * n + dst] = gb + round16(s->g[i * n + k] - gb, mode);
            }
            for (int p = 0; p < L; p++) s->fn[(p * Q) * n + k] = tot[p] - acc[p];
            s->gn[k] = s->g[k];
        }
}
#endif

/* m_phi (Eq. (13)) at a ghost node beyond a wetting wall, evaluated there
 * from the ghost phase fields: their gradients (Eq. (27)) and sources
 * (Eqs. (2)-(4)). */
static void mphi_ghost(const or_sim *s, int x, int y, real *mx, real *my)
{
    const or_params *pp = &s->p;
    const int N = s->N;
    real ph[MAXN], gp[MAXN][2], R[MAXN][2];
    for (int p = 0; p < N; p++) {
        ph[p] = fetch_phi(s, p, x, y);
        grad_phi_at(s, p, x, y, &gp[p][0], &gp[p][1]);
    }
    source_at(pp, N, ph, (const real(*)[2])gp, R);
    real ax = 0, ay = 0;
    for (int p = 0; p < N; p++) {
        ax -= pp->rho[p] * pp->mobility * (gp[p][0] - R[p][0]);
        ay -= pp->rho[p] * pp->mobility * (gp[p][1] - R[p][1]);
    }
    *mx = ax;
    *my = ay;
}

/* The fields of the current populations f, in the paper's order: phi
 * (Eq. (25a)), rho and mu (Eqs. (11),(12)), gradients and Laplacians
 * (Eq. (27)), sources (Eqs. (2)-(4)), m_phi (Eq. (13)), chemical potentials
 * and F_s (Eqs. (15)-(17)); F holds F_s on return. */
static void eval_fields(or_sim *s)
{
    const int nx = s->p.nx, ny = s->p.ny, N = s->N, L = s->L;
    const size_t n = s->n;
    const or_params *pp = &s->p;

    /* Sec. 3, Eq. (25a): phi_p = sum_i f_{i,p}.  Sec. 4: phi_N from sum = 1
     * unless every phase is solved. */
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < (long long)n; k++) {
        real sum = 0;
        for (int p = 0; p < L; p++) {
            real a = 0;
            for (int i = 0; i < Q; i++) a += s->f[(p * Q + i) * n + k];
            s->phi[p * n + k] = a;
            sum += a;
        }
        if (L == N - 1) s->phi[(N - 1) * n + k] = 1.0 - sum;
        /* Sec. 2.2, Eqs. (11),(12) */
        real r = 0, m = 0;
        for (int p = 0; p < N; p++) {
            r += pp->rho[p] * s->phi[p * n + k];
            m += pp->mu[p] * s->phi[p * n + k];
        }
        s->rho[k] = r;
        s->mu[k] = m;
    }

    /* Sec. 3, Eq. (27): gradients and Laplacians of every phi_p, and
     * grad rho = sum_p rho_p grad phi_p (Eq. (11) is linear in phi). */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t k = nid(s, x, y);
            real grx = 0, gry = 0;
            for (int p = 0; p < N; p++) {
                real gx, gy;
                grad_phi_at(s, p, x, y, &gx, &gy);
                s->grad[(p * 2 + 0) * n + k] = gx;
                s->grad[(p * 2 + 1) * n + k] = gy;
                s->lap[p * n + k] = lap_phi_at(s, p, x, y);
                grx += pp->rho[p] * gx;
                gry += pp->rho[p] * gy;
            }
            s->gradrho[k] = grx;
            s->gradrho[n + k] = gry;
        }

    /* Sec. 2.1, Eqs. (2)-(4): sources; Sec. 2.2, Eq. (13): m_phi;
     * Sec. 2.2, Eqs. (15)-(17): chemical potentials; Eq. (16): F_s. */
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < (long long)n; k++) {
        real ph[MAXN], gp[MAXN][2], R[MAXN][2];
        for (int p = 0; p < N; p++) {
            ph[p] = s->phi[p * n + k];
            gp[p][0] = s->grad[(p * 2 + 0) * n + k];
            gp[p][1] = s->grad[(p * 2 + 1) * n + k];
        }
        source_at(pp, N, ph, (const real(*)[2])gp, R);
        real mx = 0, my = 0;
        for (int p = 0; p < N; p++) {
            s->R[(p * 2 + 0) * n + k] = R[p][0];
            s->R[(p * 2 + 1) * n + k] = R[p][1];
            mx -= pp->rho[p] * pp->mobility * (gp[p][0] - R[p][0]);
            my -= pp->rho[p] * pp->mobility * (gp[p][1] - R[p][1]);
        }
        s->mphi[k] = mx;
        s->mphi[n + k] = my;
        real fsx = 0, fsy = 0;
        for (int p = 0; p < N; p++) {
            real mu = 0;
            for (int q = 0; q < N; q++) {
                if (q == p) continue;
                real sig = pp->sigma[p * MAXN + q];
                real beta = 3.0 * sig / pp->eps;           /* Eq. (15) */
                real kpq = -3.0 * pp->eps * sig / 4.0;      /* Eq. (15) */
                mu += 2.0 * beta * (gprime(ph[p]) - gprime(ph[p] + ph[q]));
                mu -= kpq * s->lap[q * n + k];
            }
            s->muphi[p * n + k] = mu;
            fsx += mu * gp[p][0];
            fsy += mu * gp[p][1];
        }
        s->F[k] = fsx;       /* F_s now, F_c added below */
        s->F[n + k] = fsy;
    }
}

static void step_once(or_sim *s)
{
    const int nx = s->p.nx, ny = s->p.ny, N = s->N, L = s->L;
    const size_t n = s->n;
    const or_params *pp = &s->p;

    eval_fields(s);

    /* Sec. 3, text after Eq. (24): F_c = -div(m_phi u - u m_phi)/2 with the
     * lagged velocity; total force F = F_s + F_g + F_c with F_g = rho g. */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t k = nid(s, x, y);
            real div[2] = {0, 0};
            for (int i = 1; i < Q; i++) {
                real mx, my, ux, uy;
                const int yn = y + CY[i];
                if (s->wet && (yn < 0 || yn >= ny))
                    mphi_ghost(s, x + CX[i], yn, &mx, &my);
                else
                    fetch_vec(s, s->mphi, x + CX[i], yn, K_REFLECT, &mx, &my);
                fetch_vec(s, s->u_prev, x + CX[i], y + CY[i], K_VELOCITY, &ux, &uy);
                real m[2] = {mx, my}, u[2] = {ux, uy}, c[2] = {(real)CX[i], (real)CY[i]};
                for (int b = 0; b < 2; b++)
                    for (int a = 0; a < 2; a++)
                        div[b] += W[i] * c[a] * (m[a] * u[b] - u[a] * m[b]) / CS2;
            }
            s->Fc[k] = -0.5 * div[0];
            s->Fc[n + k] = -0.5 * div[1];
            s->F[k] += s->Fc[k] + s->rho[k] * pp->gx;
            s->F[n + k] += s->Fc[n + k] + s->rho[k] * pp->gy;
        }

    /* Macroscopic velocity and pressure, Eqs. (25b),(25c); collisions,
     * Eqs. (18)-(24); then streaming. */
    const real Sph[Q] = {1, 1.0 / s->tau_f, 1.0 / s->tau_f, 1, 1, 1, 1, 1, 1};
#pragma omp parallel for schedule(static)
    for (long long k = 0; k < (long long)n; k++) {
        real gk[Q];
        for (int i = 0; i < Q; i++) gk[i] = s->g[i * n + k];
        real Fx = s->F[k], Fy = s->F[n + k];
        real rho = s->rho[k];
        real jx = 0, jy = 0, sg = 0;
        for (int i = 0; i < Q; i++) {
            jx += CX[i] * gk[i];
            jy += CY[i] * gk[i];
            if (i) sg += gk[i];
        }
        /* Eq. (25b): rho u = sum c_i g_i + dt F / 2 */
        real ux = (jx + 0.5 * Fx) / rho, uy = (jy + 0.5 * Fy) / rho;
        real mphx = s->mphi[k], mphy = s->mphi[n + k];
        /* Eq. (13): m = rho u + m_phi */
        real mx = rho * ux + mphx, my = rho * uy + mphy;
        real grx = s->gradrho[k], gry = s->gradrho[n + k];
        real ugr = ux * grx + uy * gry;
        /* previous-step quantities for backward Euler */
        real upx = s->u_prev[k], upy = s->u_prev[n + k];
        real rho_p = 0;
        for (int p = 0; p < N; p++) rho_p += pp->rho[p] * s->phi_prev[p * n + k];
        real mpx = rho_p * upx + s->mphi_prev[k], mpy = rho_p * upy + s->mphi_prev[n + k];
        real mu_t = (mx * ux + my * uy), mu_prev = (mpx * upx + mpy * upy);
        real dt_mu = mu_t - mu_prev;
        /* Eq. (25c) */
        real P = CS2 / (1.0 - W[0]) *
                   (sg + 0.5 * ugr - W[0] * mu_t / (2.0 * CS2) + W[0] * 0.5 * dt_mu / (2.0 * CS2));
        s->u[k] = ux;
        s->u[n + k] = uy;
        s->P[k] = P;

        /* Phase-field collision per solved phase, Eqs. (18),(19). */
        for (int p = 0; p < L; p++) {
            real fk[Q], feq[Q], src[Q], out[Q];
            for (int i = 0; i < Q; i++) fk[i] = s->f[(p * Q + i) * n + k];
            real ph = s->phi[p * n + k], php = s->phi_prev[p * n + k];
            or_phase_feq(ph, ux, uy, feq);
            real dtx = ph * ux - php * upx, dty = ph * uy - php * upy;
            or_phase_src(dtx, dty, s->R[(p * 2 + 0) * n + k], s->R[(p * 2 + 1) * n + k], src);
            mrt(s, fk, feq, src, Sph, out);
            for (int i = 0; i < Q; i++) s->f[(p * Q + i) * n + k] = out[i]; /* post-collision */
        }

        /* Flow collision, Eqs. (21)-(24), tau_g from Eq. (26). */
        real tau_g = s->mu[k] / (rho * CS2) + 0.5;
        real s2 = 1.0 / tau_g;
        const real Sfl[Q] = {1, 1, 1, s2, s2, s2, 1, 1, 1};
        real geq[Q], Fi[Q], out[Q];
        or_flow_geq(P, 0.0, rho, ux, uy, mx, my, geq);
        /* M_2F = d_t(rho u u) + d_t((m_phi u + u m_phi)/2) + c_s^2 (u grad rho + grad rho u)
         *        + c_s^2 (u.grad rho) I, with d_t(rho u u) ~ u F + F u. */
        real u[2] = {ux, uy}, Fv[2] = {Fx, Fy}, gr[2] = {grx, gry};
        real mp[2] = {mphx, mphy}, mpp[2] = {s->mphi_prev[k], s->mphi_prev[n + k]}, up[2] = {upx, upy};
        real M2F[4];
        for (int a = 0; a < 2; a++)
            for (int b = 0; b < 2; b++) {
                real v = u[a] * Fv[b] + Fv[a] * u[b];
                v += 0.5 * (mp[a] * u[b] + u[a] * mp[b]) - 0.5 * (mpp[a] * up[b] + up[a] * mpp[b]);
                v += CS2 * (u[a] * gr[b] + gr[a] * u[b]);
                if (a == b) v += CS2 * ugr;
                M2F[a * 2 + b] = v;
            }
        or_flow_force(ugr, Fx, Fy, M2F, Fi);
        mrt(s, gk, geq, Fi, Sfl, out);
        for (int i = 0; i < Q; i++) s->g[i * n + k] = out[i];
    }

    /* Streaming, Sec. 4: f(x + c_i, t + 1) = f*(x, t); a link that leaves
     * the lattice through a wall is reflected back (half-way bounce-back). */
    static const int OPP[Q] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
#ifdef ORACLE_FP32
    if (pp->store16) stream_store16(s);
    else
#endif
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            size_t k = nid(s, x, y);
            for (int i = 0; i < Q; i++) {
                int tx = x + CX[i], ty = y + CY[i];
                int out_x = tx < 0 || tx >= nx, out_y = ty < 0 || ty >= ny;
                int bounce = (out_x && pp->wall_x) || (out_y && pp->wall_y);
                size_t dst;
                int di;
                if (bounce) {
                    dst = k;
                    di = OPP[i];
                } else {
                    tx = (tx % nx + nx) % nx;
                    ty = (ty % ny + ny) % ny;
                    dst = nid(s, tx, ty);
                    di = i;
                }
                for (int p = 0; p < L; p++) s->fn[(p * Q + di) * n + dst] = s->f[(p * Q + i) * n + k];
                s->gn[di * n + dst] = s->g[i * n + k];
            }
        }
    real *t = s->f;
    s->f = s->fn;
    s->fn = t;
    t = s->g;
    s->g = s->gn;
    s->gn = t;

    /* Store the "previous" fields for the next step's time derivatives. */
    memcpy(s->phi_prev, s->phi, N * n * sizeof(real));
    memcpy(s->u_prev, s->u, 2 * n * sizeof(real));
    memcpy(s->mphi_prev, s->mphi, 2 * n * sizeof(real));
    s->steps++;
}

void or_step(void *h, long long nsteps, int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (long long t = 0; t < nsteps; t++) step_once((or_sim *)h);
}

/* Last computed macroscopic fields: phi [N][ny][nx], u [2][ny][nx], P [ny][nx].
 * Any pointer may be NULL. */
void or_get_moments(void *h, real *phi, real *u, real *P)
{
    or_sim *s = (or_sim *)h;
    if (phi) memcpy(phi, s->phi, s->N * s->n * sizeof(real));
    if (u) memcpy(u, s->u, 2 * s->n * sizeof(real));
    if (P) memcpy(P, s->P, s->n * sizeof(real));
}

/* Per-phase mass sum_x phi_p of the last computed fields, p = 1..N. */
void or_phase_mass(void *h, real *mass)
{
    or_sim *s = (or_sim *)h;
    for (int p = 0; p < s->N; p++) {
        real a = 0;
        for (size_t k = 0; k < s->n; k++) a += s->phi[p * s->n + k];
        mass[p] = a;
    }
}

/* Intermediate fields of the last step (for inspection in tests):
 * which = 0 R [N][2][n], 1 m_phi [2][n], 2 mu_phi [N][n], 3 F [2][n],
 *         4 grad phi [N][2][n], 5 lap phi [N][n], 6 F_c [2][n]. */
void or_get_field(void *h, int which, real *out)
{
    or_sim *s = (or_sim *)h;
    size_t n = s->n, N = s->N;
    switch (which) {
    case 0: memcpy(out, s->R, N * 2 * n * sizeof(real)); break;
    case 1: memcpy(out, s->mphi, 2 * n * sizeof(real)); break;
    case 2: memcpy(out, s->muphi, N * n * sizeof(real)); break;
    case 3: memcpy(out, s->F, 2 * n * sizeof(real)); break;
    case 4: memcpy(out, s->grad, N * 2 * n * sizeof(real)); break;
    case 5: memcpy(out, s->lap, N * n * sizeof(real)); break;
    case 6: memcpy(out, s->Fc, 2 * n * sizeof(real)); break;
    default: break;
    }
}

long long or_steps_done(void *h) { return ((or_sim *)h)->steps; }

/* ----------------------------------------- field-level entry points for pins */

/* Eq. (27) applied to a standalone scalar field with the oracle's ghost
 * rules: grad -> out[2][ny][nx], lap -> out[ny][nx]. */
void or_field_grad(const real *chi, int nx, int ny, int wall_x, int wall_y, real *out)
{
    or_sim tmp;
    memset(&tmp, 0, sizeof tmp);
    tmp.p.nx = nx;
    tmp.p.ny = ny;
    tmp.p.wall_x = wall_x;
    tmp.p.wall_y = wall_y;
    tmp.n = (size_t)nx * ny;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) {
            real gx, gy;
            grad_at(&tmp, chi, x, y, &gx, &gy);
            out[nid(&tmp, x, y)] = gx;
            out[tmp.n + nid(&tmp, x, y)] = gy;
        }
}

void or_field_lap(const real *chi, int nx, int ny, int wall_x, int wall_y, real *out)
{
    or_sim tmp;
    memset(&tmp, 0, sizeof tmp);
    tmp.p.nx = nx;
    tmp.p.ny = ny;
    tmp.p.wall_x = wall_x;
    tmp.p.wall_y = wall_y;
    tmp.n = (size_t)nx * ny;
    for (int y = 0; y < ny; y++)
        for (int x = 0; x < nx; x++) out[nid(&tmp, x, y)] = lap_at(&tmp, chi, x, y);
}

/* Pointwise source of Eqs. (2)-(4) for all N phases: phi[N], grad[N][2] -> R[N][2]. */
int or_point_source(const or_params *p, const real *phi, const real *grad, real *R)
{
    if (p->n_phases < 2 || p->n_phases > MAXN) return -1;
    source_at(p, p->n_phases, phi, (const real(*)[2])grad, (real(*)[2])R);
    return 0;
}

/* Pointwise chemical potentials of Eq. (17): phi[N], lap[N] -> muphi[N]. */
int or_point_chempot(const or_params *p, const real *phi, const real *lap, real *muphi)
{
    int N = p->n_phases;
    if (N < 2 || N > MAXN) return -1;
    for (int a = 0; a < N; a++) {
        real mu = 0;
        for (int b = 0; b < N; b++) {
            if (b == a) continue;
            real sig = p->sigma[a * MAXN + b];
            mu += 2.0 * (3.0 * sig / p->eps) * (gprime(phi[a]) - gprime(phi[a] + phi[b]));
            mu -= (-3.0 * p->eps * sig / 4.0) * lap[b];
        }
        muphi[a] = mu;
    }
    return 0;
}

/* The moment matrix of Eq. (28) and its numerical inverse (row-major 9x9). */
void or_mrt_matrices(real *Mout, real *Miout)
{
    real Mm[Q][Q], Mi[Q][Q];
    build_M(Mm);
    invert9(Mm, Mi);
    memcpy(Mout, Mm, sizeof Mm);
    memcpy(Miout, Mi, sizeof Mi);
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
