// The fused per-step kernel: pull streaming, phase fields, isotropic stencils,
// Model A / Model B sources, consistent mass flux, surface tension, F_c,
// velocity, pressure and both MRT collisions in one pass over the lattice.
//
// Work decomposition.  A thread block of T threads owns a strip of T - 4
// consecutive columns and marches down TY rows; thread t always works on
// lattice column x0 - 2 + t.  The update of row r needs phi(t) on rows
// r-2..r+2 and columns +-2 (F_c differentiates m_phi, which differentiates
// phi) and m_phi on rows r-1..r+1, columns +-1, so each iteration runs three
// stages on a rolling window kept in shared memory:
//   A (row r+2): all T threads sum their pulled phase populations,
//                phi_p = sum_i f_i (Eq. (25a)); the strip's own nodes keep
//                j_p and the rounding error of that sum;
//   B (row r+1): the inner T - 2 threads compute grad phi (Eq. (27)), the
//                source R_p (Eqs. (2)-(4)) and m_phi = -M sum_p rho_p
//                (grad phi_p - R_p) (Eq. (13)); the previous step's velocity
//                of that row is staged;
//   C (row r):   the inner T - 4 threads (the strip) compute Laplacians,
//                chemical potentials and F_s (Eqs. (16)-(17)), F_c, u and P
//                (Eqs. (25b), (25c)), both collisions (Eqs. (18)-(24)), and
//                store.
// Every thread runs each stage once per row, so halo columns cost idle
// lanes, not extra passes.  The pulled populations of the next row are
// copied into shared memory asynchronously while the current rows are
// computed.  Only the 4 halo columns and 4 + 2 pre-roll rows per strip are
// computed twice; every population is read from HBM once and written once.
//
// Collision in closed form.  With the relaxation matrix of Sec. 4
// (S = diag(s0, s1, s1, s2, s2, s2, s3, s3, s4), all entries 1 except
// s1 = 1/tau_f for the phase field and s2 = 1/tau_g for the flow), every
// post-collision moment of order >= 2 of a phase set is its equilibrium plus
// half its source moment, so f* depends on the pulled f only through
// phi = sum f_i and j = sum c_i f_i.  For the flow set the pulled g enters
// through j_g, the second moments Pi and sum_{i!=0} g_i.  The inverse of the
// moment matrix of Eq. (28) is applied in closed form.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <atomic>

#include "nlbm_internal.cuh"

namespace nlbm {

__device__ __forceinline__ int map_axis(int c, int n, int wall, bool &flip)
{
    flip = false;
    if (c >= 0 && c < n) return c;
    if (!wall) {
        c %= n;
        if (c < 0) c += n;
        return c;
    }
    flip = true;                       // half-way wall: mirror image node
    return c < 0 ? -1 - c : 2 * n - 1 - c;
}

__device__ __forceinline__ int slot5(int r) { return (r + 10) % 5; }
__device__ __forceinline__ int slot3(int r) { return (r + 9) % 3; }

// Sources of the pull at node (x, y): direction i of this node comes from
// node[i] in plane dir[i] (dir[i] = i, or the opposite direction of the own
// node when the link crosses a half-way bounce-back wall).
__device__ __forceinline__ void pull_sources(const StepParams &P, int x, int y,
                                             unsigned (&node)[9], int (&dir)[9])
{
    int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1;
    bool oxm = false, oxp = false, oym = false, oyp = false;
    if (xm < 0) { if (P.wall_x) oxm = true; else xm += P.nx; }
    if (xp >= P.nx) { if (P.wall_x) oxp = true; else xp -= P.nx; }
    if (ym < 0) { if (P.wall_y) oym = true; else ym += P.ny; }
    if (yp >= P.ny) { if (P.wall_y) oyp = true; else yp -= P.ny; }
    const unsigned nx = (unsigned)P.nx;
    const unsigned self = (unsigned)y * nx + x;
    const unsigned r0 = (unsigned)y * nx, rm = (unsigned)ym * nx, rp = (unsigned)yp * nx;
    node[0] = self; dir[0] = 0;
    // f_i(x) = f*_i(x - c_i)
    if (oxm) { node[1] = self; dir[1] = 3; } else { node[1] = r0 + xm; dir[1] = 1; }
    if (oym) { node[2] = self; dir[2] = 4; } else { node[2] = rm + x; dir[2] = 2; }
    if (oxp) { node[3] = self; dir[3] = 1; } else { node[3] = r0 + xp; dir[3] = 3; }
    if (oyp) { node[4] = self; dir[4] = 2; } else { node[4] = rp + x; dir[4] = 4; }
    if (oxm || oym) { node[5] = self; dir[5] = 7; } else { node[5] = rm + xm; dir[5] = 5; }
    if (oxp || oym) { node[6] = self; dir[6] = 8; } else { node[6] = rm + xp; dir[6] = 6; }
    if (oxp || oyp) { node[7] = self; dir[7] = 5; } else { node[7] = rp + xp; dir[7] = 7; }
    if (oxm || oyp) { node[8] = self; dir[8] = 6; } else { node[8] = rp + xm; dir[8] = 8; }
}

// Error-free transformation a + b = s + e (Knuth's TwoSum, 6 flops).
__device__ __forceinline__ float two_sum(float a, float b, float &e)
{
    const float s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
    return s;
}

// Paired FP32 arithmetic.  Blackwell issues FADD2 / FMUL2 / FFMA2: one FP32
// operation on two operand pairs in a single instruction, each component
// rounded exactly as the scalar instruction (__fadd_rn, __fmul_rn,
// __fmaf_rn).  The step is bound by instruction issue, so the work done per
// phase runs on pairs of phases (p, p + 1) -- V = float2 -- and an odd last
// phase on scalars, V = float, through the same code.
__device__ __forceinline__ float vadd(float a, float b) { return a + b; }
__device__ __forceinline__ float2 vadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
// a - b as the exact product -1 * b added to a with one rounding
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
template <class V> __device__ __forceinline__ V vset(float s);
template <> __device__ __forceinline__ float vset<float>(float s) { return s; }
template <> __device__ __forceinline__ float2 vset<float2>(float s) { return make_float2(s, s); }
// Phases p (and p + 1) of a per-phase array, and back.
template <class V> __device__ __forceinline__ V vget(const float *a, int p);
template <> __device__ __forceinline__ float vget<float>(const float *a, int p) { return a[p]; }
template <> __device__ __forceinline__ float2 vget<float2>(const float *a, int p) { return make_float2(a[p], a[p + 1]); }
__device__ __forceinline__ void vput(float *a, int p, float v) { a[p] = v; }
__device__ __forceinline__ void vput(float *a, int p, float2 v) { a[p] = v.x; a[p + 1] = v.y; }
// Values of phases p (and p + 1) at offset o of shared-memory rows that are
// `stride` floats apart per phase.
template <class V> __device__ __forceinline__ V vld(const float *base, int stride, int o);
template <> __device__ __forceinline__ float vld<float>(const float *base, int, int o) { return base[o]; }
template <> __device__ __forceinline__ float2 vld<float2>(const float *base, int stride, int o)
{
    return make_float2(base[o], base[stride + o]);
}

// phi = sum_i f_i in the fixed order f_0 + f_1 + ... + f_8 (own and halo
// nodes give identical bits), and for the strip's own nodes the rounding
// error of that sum (Fast2Sum terms, exact when the running sum dominates
// each term, as the rest population does) and the first moments j.
template <class V, bool OWN>
__device__ __forceinline__ void pull_moments(const V (&f)[9], V &ph, V &plo, V &jx, V &jy)
{
    V s = f[0], e = vset<V>(0.f);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        const V t = vadd(s, f[i]);
        if (OWN) e = vadd(e, vsub(f[i], vsub(t, s)));
        s = t;
    }
    ph = s;
    if (OWN) {
        plo = e;
        jx = vadd(vadd(vsub(f[1], f[3]), vsub(f[5], f[6])), vsub(f[8], f[7]));
        jy = vsub(vadd(vsub(f[2], f[4]), vadd(f[5], f[6])), vadd(f[7], f[8]));
    }
}

// Asynchronous 4-byte global->shared copies (cp.async): the next row's
// pulled populations are in flight while the current rows are computed.
__device__ __forceinline__ void cp_async4(float *dst_smem, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// 16-byte copy (both addresses 16-byte aligned), cached in L2 only.
__device__ __forceinline__ void cp_async16(float *dst_smem, const float *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// Start the copies of the 9 (N-1) populations node (x, y) pulls into column
// col of the staging array s_F [9 (N-1)][WF].
template <int NS>
__device__ __forceinline__ void prefetch_pull(const StepParams &P, int x, int y, float *s_F, int WF,
                                              int col)
{
    unsigned node[9];
    int dir[9];
    pull_sources(P, x, y, node, dir);
    const unsigned pl = P.plane;
#pragma unroll
    for (int p = 0; p < NS; ++p) {
        const float *fp = P.fin + (size_t)p * 9 * pl;
#pragma unroll
        for (int i = 0; i < 9; ++i) cp_async4(s_F + (p * 9 + i) * WF + col, fp + (unsigned)dir[i] * pl + node[i]);
    }
}

// Phase fields of one node from its staged pulled populations (phases in
// pairs, see pull_moments).
template <class V, bool OWN>
__device__ __forceinline__ void sum_pulled_v(const float *s_F, int WF, int col, int p, float *ph, float *plo,
                                             float *jx, float *jy)
{
    V f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = vld<V>(s_F + (p * 9 + i) * WF, 9 * WF, col);
    V a, lo, x, y;
    pull_moments<V, OWN>(f, a, lo, x, y);
    vput(ph, p, a);
    if (OWN) { vput(plo, p, lo); vput(jx, p, x); vput(jy, p, y); }
}
template <int NS, bool OWN>
__device__ __forceinline__ void sum_pulled(const float *s_F, int WF, int col, float (&ph)[NS],
                                           float (&plo)[NS], float (&jx)[NS], float (&jy)[NS])
{
#pragma unroll
    for (int p = 0; p + 1 < NS; p += 2) sum_pulled_v<float2, OWN>(s_F, WF, col, p, ph, plo, jx, jy);
    if (NS & 1) sum_pulled_v<float, OWN>(s_F, WF, col, NS - 1, ph, plo, jx, jy);
}

// Row windows (FP32 storage, nx a multiple of 4, no wall across x).  Each
// warp stages the rows its 32 ring columns pull from: for every population
// plane, a window of kWin columns that starts 4 columns left of the warp's
// first node (so that it is 16-byte aligned) and covers the one-column halo
// on both sides.  Lanes 0..26 copy it in 16-byte pieces, lane 9 g + c taking
// piece c of the three directions of group g (group_dir); lane l then finds
// f_i(x - c_i) at window column 2 + l - c_ix.  Only the warp's own lanes
// read its windows, so a warp barrier orders copies and reads.
constexpr int kWin = 36;

// Direction k (0..2) of group g: g = 0 the directions with c_iy = 0
// {0, 1, 3}, g = 1 those with c_iy = +1 {2, 5, 6}, g = 2 those with
// c_iy = -1 {4, 7, 8}; groups 1 and 2 are each other's opposites in order.
__device__ __forceinline__ int group_dir(int g, int k)
{
    if (k == 0) return 2 * g;
    if (k == 1) return g == 0 ? 1 : (g == 1 ? 5 : 7);
    return g == 0 ? 3 : (g == 1 ? 6 : 8);
}

// Source row of group g for nodes of row y in [0, ny): row y - c_iy
// (wrapped on a periodic axis), or, when that row is across a half-way wall,
// row y itself with the opposite directions (the link is bounced back).
__device__ __forceinline__ void group_source(const StepParams &P, int y, int g, int &geff, unsigned &row)
{
    int ys = y - (g == 0 ? 0 : (g == 1 ? 1 : -1));
    geff = g;
    if (ys < 0 || ys >= P.ny) {
        if (P.wall_y) {
            ys = y;
            geff = 3 - g;
        } else {
            ys += ys < 0 ? P.ny : -P.ny;
        }
    }
    row = (unsigned)ys * (unsigned)P.nx;
}

// Start the copies of the phase-population windows node row y pulls:
// window slot 9 p + i of the warp holds what f_i of phase p pulls.
template <int NS>
__device__ __forceinline__ void stage_pull_rows(const StepParams &P, int y, int g, int wc, unsigned wcol,
                                                float *s_Fw)
{
    int ge;
    unsigned row;
    group_source(P, y, g, ge, row);
    const float *base = P.fin + (row + wcol);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const unsigned off = (unsigned)group_dir(ge, k) * P.plane;
        float *dst = s_Fw + group_dir(g, k) * kWin + 4 * wc;
#pragma unroll
        for (int p = 0; p < NS; ++p) cp_async16(dst + 9 * p * kWin, base + (size_t)p * 9 * P.plane + off);
    }
}

// The same for the flow populations g_1..g_8 (window slot i - 1).
__device__ __forceinline__ void stage_flow_rows(const StepParams &P, int y, int g, int wc, unsigned wcol,
                                                float *s_Gw)
{
    int ge;
    unsigned row;
    group_source(P, y, g, ge, row);
    const float *base = P.gin + (row + wcol);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (g == 0 && k == 0) continue;   // g_0 is not stored
        cp_async16(s_Gw + (group_dir(g, k) - 1) * kWin + 4 * wc,
                   base + (unsigned)(group_dir(ge, k) - 1) * P.plane);
    }
}

// Window columns a node at window column b reads f_i (or g_i) at, for a
// node row whose links with c_iy = +1 (bl) or c_iy = -1 (bh) are bounced
// back at a y wall.
struct WinCols {
    int b, c5, c6, c7, c8;   // c_0..c_4 follow from b: b, b - 1, b, b + 1, b
};
__device__ __forceinline__ WinCols win_cols(int b, bool bl, bool bh)
{
    WinCols w;
    w.b = b;
    w.c5 = bl ? w.b : w.b - 1;
    w.c6 = bl ? w.b : w.b + 1;
    w.c7 = bh ? w.b : w.b + 1;
    w.c8 = bh ? w.b : w.b - 1;
    return w;
}

// sum_pulled from the warp's windows.
template <class V, bool OWN>
__device__ __forceinline__ void sum_pulled_win_v(const float *s_Fw, const WinCols &c, int p, float *ph,
                                                 float *plo, float *jx, float *jy)
{
    const float *w = s_Fw + 9 * p * kWin;
    constexpr int S = 9 * kWin;   // next phase
    V f[9];
    f[0] = vld<V>(w, S, c.b);
    f[1] = vld<V>(w, S, kWin + c.b - 1);
    f[2] = vld<V>(w, S, 2 * kWin + c.b);
    f[3] = vld<V>(w, S, 3 * kWin + c.b + 1);
    f[4] = vld<V>(w, S, 4 * kWin + c.b);
    f[5] = vld<V>(w, S, 5 * kWin + c.c5);
    f[6] = vld<V>(w, S, 6 * kWin + c.c6);
    f[7] = vld<V>(w, S, 7 * kWin + c.c7);
    f[8] = vld<V>(w, S, 8 * kWin + c.c8);
    V a, lo, x, y;
    pull_moments<V, OWN>(f, a, lo, x, y);
    vput(ph, p, a);
    if (OWN) { vput(plo, p, lo); vput(jx, p, x); vput(jy, p, y); }
}
template <int NS, bool OWN>
__device__ __forceinline__ void sum_pulled_win(const float *s_Fw, const WinCols &c, float (&ph)[NS],
                                               float (&plo)[NS], float (&jx)[NS], float (&jy)[NS])
{
#pragma unroll
    for (int p = 0; p + 1 < NS; p += 2) sum_pulled_win_v<float2, OWN>(s_Fw, c, p, ph, plo, jx, jy);
    if (NS & 1) sum_pulled_win_v<float, OWN>(s_Fw, c, NS - 1, ph, plo, jx, jy);
}

// Phase-field collision in moment space (Eqs. (18)-(20), (28)).  With the
// relaxation rates of Sec. 4 (all 1 but s1 = 1/tau_f) the post-collision
// moments of a phase set are phi, A = (1 - s1) j_x + s1 phi u_x + (1 - s1/2)
// G_x / 3, B (the same along y), C = phi u_y / 3 + G_y / 18 and D = phi u_x / 3
// + G_x / 18 (moments c_x^2 c_y and c_x c_y^2), the second moments phi / 3,
// 0 and phi / 9 at equilibrium, with G = d_t(phi u) / c_s^2 + R_p the source
// of Eq. (19).  The coefficients are the same for every phase.
template <class V> struct CollCoef {
    V s1, c1, h1, three, k18, ux, uy, mupx, mupy, s1ux, s1uy, ux3, uy3;
    __device__ __forceinline__ CollCoef(float s1_, float ux_, float uy_, float upx_, float upy_)
    {
        s1 = vset<V>(s1_);
        c1 = vset<V>(1.f - s1_);
        h1 = vset<V>((1.f - 0.5f * s1_) * (1.f / 3.f));
        three = vset<V>(3.f);
        k18 = vset<V>(1.f / 18.f);
        ux = vset<V>(ux_);
        uy = vset<V>(uy_);
        mupx = vset<V>(-upx_);
        mupy = vset<V>(-upy_);
        s1ux = vset<V>(s1_ * ux_);
        s1uy = vset<V>(s1_ * uy_);
        ux3 = vset<V>(ux_ * (1.f / 3.f));
        uy3 = vset<V>(uy_ * (1.f / 3.f));
    }
};

template <class V>
__device__ __forceinline__ void phase_moments(V phi, V jx, V jy, V php, V Rx, V Ry, const CollCoef<V> &k, V &A,
                                              V &B, V &C, V &D)
{
    // G = d_t(phi u)/c_s^2 + R_p, backward Euler in time
    const V Gx = vfma(k.three, vfma(php, k.mupx, vmul(phi, k.ux)), Rx);
    const V Gy = vfma(k.three, vfma(php, k.mupy, vmul(phi, k.uy)), Ry);
    A = vfma(k.c1, jx, vfma(phi, k.s1ux, vmul(k.h1, Gx)));
    B = vfma(k.c1, jy, vfma(phi, k.s1uy, vmul(k.h1, Gy)));
    C = vfma(phi, k.uy3, vmul(Gy, k.k18));
    D = vfma(phi, k.ux3, vmul(Gx, k.k18));
}

__device__ __forceinline__ float vabs(float a) { return fabsf(a); }
__device__ __forceinline__ float2 vabs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float vcopysign(float a, float b) { return copysignf(a, b); }
__device__ __forceinline__ float2 vcopysign(float2 a, float2 b)
{
    return make_float2(copysignf(a.x, b.x), copysignf(a.y, b.y));
}

// Two populations c + h and c - h whose stored values sum to exactly 2c:
// big = c + |h| is rounded, and hr = big - c, c + hr = big and c - hr =
// 2c - big are exact by Sterbenz's lemma whenever |h| <= 3|c|, which holds
// away from vanishing phase fields; the sign of h picks which is which.
template <class V>
__device__ __forceinline__ void exact_pair_v(V c, V h, V &plus, V &minus)
{
    const V big = vadd(c, vabs(h));
    const V hr = vcopysign(vsub(big, c), h);
    plus = vadd(c, hr);
    minus = vsub(c, hr);
}

template <class V>
__device__ __forceinline__ V two_sum_v(V a, V b, V &e)
{
    const V s = vadd(a, b);
    const V bb = vsub(s, a);
    e = vadd(vsub(a, vsub(s, bb)), vsub(b, bb));
    return s;
}

// The nine post-collision populations f*_i = w_i phi + (moment terms) of
// one or two phases from phi, the rounding error phi_lo of the pulled sum
// and A, B, C, D.  The four +- pairs around phi/9 and phi/36 sum exactly to
// 2 phi/9 or 2 phi/36, and f*_0 = 4 phi/9 is formed as (sum_i f_i) - 5 phi/9
// with error-free subtractions, so the stored populations sum to the pulled
// ones up to one rounding (volume conservation, Eq. (1)).
template <class V>
__device__ __forceinline__ void phase_populations(V phi, V plo, V A, V B, V C, V D, V (&f)[9])
{
    const V p9 = vmul(phi, vset<V>(1.f / 9.f)), p36 = vmul(vset<V>(0.25f), p9);
    const V half = vset<V>(0.5f), quarter = vset<V>(0.25f);
    exact_pair_v(p9, vmul(half, vsub(A, D)), f[1], f[3]);
    exact_pair_v(p9, vmul(half, vsub(B, C)), f[2], f[4]);
    exact_pair_v(p36, vmul(quarter, vadd(C, D)), f[5], f[7]);
    exact_pair_v(p36, vmul(quarter, vsub(C, D)), f[6], f[8]);
    V e1, e2;
    const V a1 = two_sum_v(phi, vmul(vset<V>(-4.f), p9), e1);
    const V a2 = two_sum_v(a1, vmul(vset<V>(-1.f), p9), e2);
    f[0] = vadd(a2, vadd(vadd(e1, e2), plo));
}

// Store one value, or the values of phases p and p + 1 (`stride` floats apart).
__device__ __forceinline__ void vstore(float *a, size_t, float v) { *a = v; }
__device__ __forceinline__ void vstore(float *a, size_t stride, float2 v) { a[0] = v.x; a[stride] = v.y; }

// 1/|v| of a unit vector: with the zero-gradient reading 0 when |v|^2 <=
// 1e-24, or the smooth reading 1/sqrt(|v|^2 + delta^2) when delta2 > 0.
__device__ __forceinline__ float inv_norm(float vx, float vy, float delta2)
{
    const float n2 = vx * vx + vy * vy;
    if (delta2 > 0.f) return rsqrtf(n2 + delta2);
    return n2 > 1e-24f ? rsqrtf(n2) : 0.0f;
}

// 16-bit population storage.  The moving populations are stored as
// deviations from a lattice-weight multiple of a field the puller knows
// (f_i - w_i phi(puller), g_i - 3 w_i P(source)); the arithmetic stays FP32.
template <int ST> struct Store16;
template <> struct Store16<1> {   // bfloat16, round to nearest even
    static __device__ __forceinline__ unsigned short enc(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
    static __device__ __forceinline__ float dec(unsigned h) { return __uint_as_float(h << 16); }
};
template <> struct Store16<2> {   // IEEE binary16, round to nearest even
    static __device__ __forceinline__ unsigned short enc(float v) { return __half_as_ushort(__float2half_rn(v)); }
    static __device__ __forceinline__ float dec(unsigned h) { return __half2float(__ushort_as_half((unsigned short)h)); }
};

// Two deviations in one 32-bit word (phase 2q in the low half, 2q + 1 in
// the high half), converted together: one paired conversion rounds both to
// nearest even, exactly as two calls of Store16::enc.
template <int ST> struct Pack16;
template <> struct Pack16<1> {
    static __device__ __forceinline__ unsigned enc2(float2 v)
    {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
        return *reinterpret_cast<const unsigned *>(&h);
    }
    static __device__ __forceinline__ float2 dec2(unsigned w)
    {
        return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
    }
};
template <> struct Pack16<2> {
    static __device__ __forceinline__ unsigned enc2(float2 v)
    {
        const __half2 h = __floats2half2_rn(v.x, v.y);
        return *reinterpret_cast<const unsigned *>(&h);
    }
    static __device__ __forceinline__ float2 dec2(unsigned w)
    {
        return __half22float2(*reinterpret_cast<const __half2 *>(&w));
    }
};

// 16-bit deviation layout: phases 2q and 2q + 1 share one 32-bit word per
// direction and node, [NS/2][8][plane] words; an odd last phase follows in
// [8][plane] 16-bit planes.  i1 = direction - 1.
__device__ __forceinline__ size_t dev_word(int q, int i1, unsigned pl, unsigned k)
{
    return ((size_t)q * 8 + i1) * pl + k;
}
__device__ __forceinline__ size_t dev_tail(int NS, int i1, unsigned pl, unsigned k)
{
    return (size_t)(NS / 2) * 16 * pl + (size_t)i1 * pl + k;   // in 16-bit units
}

// Lattice weights w_i (Sec. 4) as FP32 constants; the same constants are
// used wherever a stored deviation is formed and wherever it is undone.
__device__ __forceinline__ float w_of(int i) { return i == 0 ? 4.f / 9.f : (i < 5 ? 1.f / 9.f : 1.f / 36.f); }
__device__ __forceinline__ int cx_of(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0; }
__device__ __forceinline__ int cy_of(int i) { return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0; }

// Staging of the 16-bit populations a ring node pulls.  Slots per phase: 0
// the FP32 rest population, 1..8 the moving deviations, 9 the puller's own
// phi(t).  A phase pair's word is copied whole into the slots of its even
// phase.  cp.async moves 4 bytes at least, so for an odd last phase the
// aligned word holding each 16-bit value is copied and the half is picked in
// stage A (par bit i: upper half for direction i; nx is even, so every plane
// starts on a word boundary and the half is the parity of the source node).
template <int NS>
__device__ __forceinline__ unsigned prefetch_pull16(const StepParams &P, int x, int y, float *s_F,
                                                    int WF, int col)
{
    unsigned node[9];
    int dir[9];
    pull_sources(P, x, y, node, dir);
    const unsigned pl = P.plane;
    const unsigned *w32 = (const unsigned *)P.fin;
    const char *f16 = (const char *)P.fin;
    unsigned par = 0;
#pragma unroll
    for (int i = 1; i < 9; ++i) par |= (node[i] & 1u) << i;
#pragma unroll
    for (int p = 0; p < NS; ++p) {
        cp_async4(s_F + (p * 10) * WF + col, P.f0in + (size_t)p * pl + node[0]);
        cp_async4(s_F + (p * 10 + 9) * WF + col, P.phi_prev + (size_t)p * pl + node[0]);
    }
#pragma unroll
    for (int q = 0; q < NS / 2; ++q) {
#pragma unroll
        for (int i = 1; i < 9; ++i)
            cp_async4(s_F + (2 * q * 10 + i) * WF + col, (const float *)(w32 + dev_word(q, dir[i] - 1, pl, node[i])));
    }
    if (NS & 1) {
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const size_t e = dev_tail(NS, dir[i] - 1, pl, node[i]);
            cp_async4(s_F + ((NS - 1) * 10 + i) * WF + col, (const float *)(f16 + ((e * 2) & ~(size_t)3)));
        }
    }
    return par;
}

// phi and j of one node from its staged 16-bit pull: f_i = w_i phi_own +
// dev_i (the same FP32 fma the storing node used), summed like sum_pulled.
template <int NS, int ST, bool OWN>
__device__ __forceinline__ void sum_pulled16(const float *s_F, int WF, int col, unsigned par,
                                             float (&ph)[NS], float (&plo)[NS], float (&jx)[NS],
                                             float (&jy)[NS])
{
#pragma unroll
    for (int p = 0; p + 1 < NS; p += 2) {
        const float2 own = make_float2(s_F[(p * 10 + 9) * WF + col], s_F[((p + 1) * 10 + 9) * WF + col]);
        float2 f[9];
        f[0] = make_float2(s_F[(p * 10) * WF + col], s_F[((p + 1) * 10) * WF + col]);
#pragma unroll
        for (int i = 1; i < 9; ++i)
            f[i] = vfma(vset<float2>(w_of(i)), own, Pack16<ST>::dec2(__float_as_uint(s_F[(p * 10 + i) * WF + col])));
        float2 a, lo, x, y;
        pull_moments<float2, OWN>(f, a, lo, x, y);
        vput(ph, p, a);
        if (OWN) { vput(plo, p, lo); vput(jx, p, x); vput(jy, p, y); }
    }
    if (NS & 1) {
        constexpr int p = NS - 1;
        const float own = s_F[(p * 10 + 9) * WF + col];
        float f[9];
        f[0] = s_F[(p * 10) * WF + col];
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            const unsigned wd = __float_as_uint(s_F[(p * 10 + i) * WF + col]);
            const unsigned h = ((par >> i) & 1u) ? (wd >> 16) : (wd & 0xffffu);
            f[i] = __fmaf_rn(w_of(i), own, Store16<ST>::dec(h));
        }
        float a, lo, x, y;
        pull_moments<float, OWN>(f, a, lo, x, y);
        ph[p] = a;
        if (OWN) { plo[p] = lo; jx[p] = x; jy[p] = y; }
    }
}

// Row windows of the 16-bit form (nx a multiple of 8, no wall across x).
// Deviation planes: a window of kWin16 columns starting at the 8-aligned
// column ws at or left of the warp's first source column, so lane l finds
// the value pulled along c_i at window column l + o16 - c_ix (o16 = the
// warp's first node column - ws, 2 or 6): per phase pair and direction 40
// words (10 pieces of 16 bytes), for an odd last phase 40 16-bit values (5
// pieces).  FP32 planes read at the node's own column (rest population, own
// phi) and the source pressure use the kWin windows of the FP32 form.
// Deviation pieces are copied by lanes 0..29 (group g, piece c), FP32 pieces
// by lanes 0..26.
constexpr int kWin16 = 40;

__device__ __forceinline__ void cp_async16_raw(void *dst_smem, const void *src)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst_smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

__device__ __forceinline__ unsigned wrap_col(int c, int nx)
{
    if (c < 0 || c >= nx) c = ((c % nx) + nx) % nx;
    return (unsigned)c;
}

// Copies of what node row y (ring row, image row under a y wall) pulls:
// the deviation windows s_Dw (phase pairs [NS/2][8][kWin16] words, then an
// odd last phase [8][kWin16] 16-bit values) and the rest-population and
// own-phi windows s_Ow [2 NS][kWin] (rest populations first).
template <int NS>
__device__ __forceinline__ void stage_pull_rows16(const StepParams &P, int y, int lane, int ws, int xo,
                                                  unsigned short *s_Dw, float *s_Ow)
{
    const unsigned pl = P.plane;
    if (lane < 30) {
        const int g = lane / 10, c = lane % 10;
        int ge;
        unsigned row;
        group_source(P, y, g, ge, row);
        const unsigned *w32 = (const unsigned *)P.fin;
        unsigned *dw = (unsigned *)s_Dw;
        const unsigned col4 = row + wrap_col(ws + 4 * c, P.nx);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (g == 0 && k == 0) continue;   // the rest population is FP32
            const int i1 = group_dir(ge, k) - 1, d1 = group_dir(g, k) - 1;
#pragma unroll
            for (int q = 0; q < NS / 2; ++q)
                cp_async16_raw(dw + (q * 8 + d1) * kWin16 + 4 * c, w32 + dev_word(q, i1, pl, col4));
            if ((NS & 1) && c < 5) {
                const unsigned short *f16 = (const unsigned short *)P.fin;
                cp_async16_raw(s_Dw + (NS / 2) * 16 * kWin16 + d1 * kWin16 + 8 * c,
                               f16 + dev_tail(NS, i1, pl, row + wrap_col(ws + 8 * c, P.nx)));
            }
        }
    }
    if (lane < 27) {
        const int g9 = lane / 9, c9 = lane % 9;
        const unsigned own = (unsigned)y * (unsigned)P.nx + wrap_col(xo + 4 * c9, P.nx);
#pragma unroll
        for (int m = 0; m < (2 * NS + 2) / 3; ++m) {
            const int q = g9 + 3 * m;
            if (q < 2 * NS) {
                const float *src = q < NS ? P.f0in + (size_t)q * pl : P.phi_prev + (size_t)(q - NS) * pl;
                cp_async16(s_Ow + q * kWin + 4 * c9, src + own);
            }
        }
    }
}

// Copies of what node row y (an own row) reads for its flow populations:
// the deviation windows s_Gw [8][kWin16] and the pressure of the rows
// y - 1, y, y + 1 at the source columns s_Pw [3][kWin] (the own row for a
// link bounced at a y wall).
__device__ __forceinline__ void stage_flow_rows16(const StepParams &P, int y, int lane, int ws, int xo,
                                                  unsigned short *s_Gw, float *s_Pw)
{
    if (lane < 15) {
        const int g = lane / 5, c = lane % 5;
        int ge;
        unsigned row;
        group_source(P, y, g, ge, row);
        const unsigned short *base = (const unsigned short *)P.gin + (row + wrap_col(ws + 8 * c, P.nx));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (g == 0 && k == 0) continue;   // g_0 is not stored
            cp_async16_raw(s_Gw + (group_dir(g, k) - 1) * kWin16 + 8 * c,
                           base + (unsigned)(group_dir(ge, k) - 1) * P.plane);
        }
    }
    if (lane < 27) {
        const int r9 = lane / 9, c9 = lane % 9;
        int ys = y - 1 + r9;   // sources with c_iy = +1 sit on row y - 1 (slot 0)
        if (ys < 0 || ys >= P.ny) ys = P.wall_y ? y : (ys < 0 ? ys + P.ny : ys - P.ny);
        cp_async16(s_Pw + r9 * kWin + 4 * c9, P.pin + ((unsigned)ys * (unsigned)P.nx + wrap_col(xo + 4 * c9, P.nx)));
    }
}

// sum_pulled16 from the warp's windows: f_i = w_i phi_own + dev_i (phases
// in pairs, see pull_moments).
template <class V, int NS, int ST, bool OWN>
__device__ __forceinline__ void sum_pulled16_win_v(const unsigned short *s_Dw, const float *s_Ow, int lane,
                                                   const WinCols &c, int p, float *ph, float *plo, float *jx,
                                                   float *jy)
{
    const V own = vld<V>(s_Ow + (NS + p) * kWin, kWin, 2 + lane);
    // the eight deviations: a phase pair's words, or an odd last phase's halves
    auto dev = [&](int i1, int col) -> V {
        if constexpr (sizeof(V) == 8) {
            return Pack16<ST>::dec2(((const unsigned *)s_Dw)[((p / 2) * 8 + i1) * kWin16 + col]);
        } else {
            return Store16<ST>::dec(s_Dw[(NS / 2) * 16 * kWin16 + i1 * kWin16 + col]);
        }
    };
    V f[9];
    f[0] = vld<V>(s_Ow + p * kWin, kWin, 2 + lane);
    f[1] = vfma(vset<V>(w_of(1)), own, dev(0, c.b - 1));
    f[2] = vfma(vset<V>(w_of(2)), own, dev(1, c.b));
    f[3] = vfma(vset<V>(w_of(3)), own, dev(2, c.b + 1));
    f[4] = vfma(vset<V>(w_of(4)), own, dev(3, c.b));
    f[5] = vfma(vset<V>(w_of(5)), own, dev(4, c.c5));
    f[6] = vfma(vset<V>(w_of(6)), own, dev(5, c.c6));
    f[7] = vfma(vset<V>(w_of(7)), own, dev(6, c.c7));
    f[8] = vfma(vset<V>(w_of(8)), own, dev(7, c.c8));
    V a, lo, x, y;
    pull_moments<V, OWN>(f, a, lo, x, y);
    vput(ph, p, a);
    if (OWN) { vput(plo, p, lo); vput(jx, p, x); vput(jy, p, y); }
}
template <int NS, int ST, bool OWN>
__device__ __forceinline__ void sum_pulled16_win(const unsigned short *s_Dw, const float *s_Ow, int lane,
                                                 const WinCols &c, float (&ph)[NS], float (&plo)[NS],
                                                 float (&jx)[NS], float (&jy)[NS])
{
#pragma unroll
    for (int p = 0; p + 1 < NS; p += 2)
        sum_pulled16_win_v<float2, NS, ST, OWN>(s_Dw, s_Ow, lane, c, p, ph, plo, jx, jy);
    if (NS & 1) sum_pulled16_win_v<float, NS, ST, OWN>(s_Dw, s_Ow, lane, c, NS - 1, ph, plo, jx, jy);
}

// Eq. (27) on a 3x3 window (rows south, centre, north): the isotropic
// central gradient and, with LAP, the Laplacian, for one or two phases.
template <class V, bool LAP>
__device__ __forceinline__ void grad_lap9(V sw, V s, V se, V w, V ce, V e, V nw, V n, V ne, V &gx, V &gy,
                                          V &lap)
{
    const V k3 = vset<V>(1.f / 3.f), k12 = vset<V>(1.f / 12.f);
    gx = vfma(vsub(e, w), k3, vmul(vsub(vadd(ne, se), vadd(nw, sw)), k12));
    gy = vfma(vsub(n, s), k3, vmul(vsub(vadd(ne, nw), vadd(se, sw)), k12));
    if (LAP) {
        const V ax = vadd(vadd(vsub(e, ce), vsub(w, ce)), vadd(vsub(n, ce), vsub(s, ce)));
        const V dg = vadd(vadd(vsub(ne, ce), vsub(nw, ce)), vadd(vsub(se, ce), vsub(sw, ce)));
        lap = vfma(ax, vset<V>(2.f / 3.f), vmul(dg, vset<V>(1.f / 6.f)));
    }
}

// Shared-memory rings of per-phase values (phi, j): a row of a ring holds
// [NS / 2 rounded up][W][2] floats, phases 2q and 2q + 1 side by side, so a
// phase pair is one 8-byte access.  ring_even(NS) floats per column of a row.
__host__ __device__ constexpr int ring_even(int NS) { return NS + (NS & 1); }
__device__ __forceinline__ int ring_idx(int W, int p, int c) { return ((p >> 1) * W + c) * 2 + (p & 1); }
template <class V> __device__ __forceinline__ V rld(const float *row, int W, int p, int c);
template <> __device__ __forceinline__ float rld<float>(const float *row, int W, int p, int c)
{
    return row[ring_idx(W, p, c)];
}
template <> __device__ __forceinline__ float2 rld<float2>(const float *row, int W, int p, int c)
{
    return *reinterpret_cast<const float2 *>(row + ring_idx(W, p, c));
}
__device__ __forceinline__ void rst(float *row, int W, int p, int c, float v) { row[ring_idx(W, p, c)] = v; }
__device__ __forceinline__ void rst(float *row, int W, int p, int c, float2 v)
{
    *reinterpret_cast<float2 *>(row + ring_idx(W, p, c)) = v;
}

// Phases p (and p + 1) of the 3x3 window of the phi ring at column c (rows
// sm, s0, sp of the ring).
template <class V, bool LAP>
__device__ __forceinline__ void window_v(const float *s_phi, int W, int NS, int sm, int s0, int sp, int c, int p,
                                         V &ce, V &gx, V &gy, V &lap)
{
    const int R = ring_even(NS) * W;   // floats per ring row
    const float *rm = s_phi + sm * R, *r0 = s_phi + s0 * R, *rp = s_phi + sp * R;
    ce = rld<V>(r0, W, p, c);
    grad_lap9<V, LAP>(rld<V>(rm, W, p, c - 1), rld<V>(rm, W, p, c), rld<V>(rm, W, p, c + 1), rld<V>(r0, W, p, c - 1),
                      ce, rld<V>(r0, W, p, c + 1), rld<V>(rp, W, p, c - 1), rld<V>(rp, W, p, c),
                      rld<V>(rp, W, p, c + 1), gx, gy, lap);
}

// phi, grad phi (Eq. (27)) and, with LAP, lap phi of all N phases from one
// read of the 3x3 window of the ring (phase N by phi_N = 1 - sum and
// negated sums).
template <int NS, bool LAP>
__device__ __forceinline__ void window_fields(const float *s_phi, int W, int sm, int s0, int sp, int c,
                                              float (&ph)[NS + 1], float (&gx)[NS + 1], float (&gy)[NS + 1],
                                              float (&lap)[NS + 1])
{
    float2 sph = make_float2(0.f, 0.f), sgx = sph, sgy = sph, sl = sph;
#pragma unroll
    for (int p = 0; p + 1 < NS; p += 2) {
        float2 a, x, y, l;
        window_v<float2, LAP>(s_phi, W, NS, sm, s0, sp, c, p, a, x, y, l);
        vput(ph, p, a);
        vput(gx, p, x);
        vput(gy, p, y);
        sph = vadd(sph, a);
        sgx = vadd(sgx, x);
        sgy = vadd(sgy, y);
        if (LAP) { vput(lap, p, l); sl = vadd(sl, l); }
    }
    float tph = sph.x + sph.y, tgx = sgx.x + sgx.y, tgy = sgy.x + sgy.y, tl = sl.x + sl.y;
    if (NS & 1) {
        float a, x, y, l;
        window_v<float, LAP>(s_phi, W, NS, sm, s0, sp, c, NS - 1, a, x, y, l);
        ph[NS - 1] = a;
        gx[NS - 1] = x;
        gy[NS - 1] = y;
        tph += a;
        tgx += x;
        tgy += y;
        if (LAP) { lap[NS - 1] = l; tl += l; }
    }
    ph[NS] = 1.f - tph;
    gx[NS] = -tgx;
    gy[NS] = -tgy;
    if (LAP) lap[NS] = -tl;
}

template <int NS>
__device__ __forceinline__ void window_grad(const float *s_phi, int W, int sm, int s0, int sp,
                                            int c, float (&ph)[NS + 1], float (&gx)[NS + 1],
                                            float (&gy)[NS + 1])
{
    float lap[NS + 1];
    window_fields<NS, false>(s_phi, W, sm, s0, sp, c, ph, gx, gy, lap);
}

template <int NS>
__device__ __forceinline__ void window_grad_lap(const float *s_phi, int W, int sm, int s0, int sp,
                                                int c, float (&ph)[NS + 1], float (&gx)[NS + 1],
                                                float (&gy)[NS + 1], float (&lap)[NS + 1])
{
    window_fields<NS, true>(s_phi, W, sm, s0, sp, c, ph, gx, gy, lap);
}

// 1/|v| from |v|^2, as inv_norm.
__device__ __forceinline__ float inv_norm2(float n2, float delta2)
{
    if (delta2 > 0.f) return rsqrtf(n2 + delta2);
    return n2 > 1e-24f ? rsqrtf(n2) : 0.0f;
}

// Model A weight max(phi, 0)^n (integer n by multiplication).
__device__ __forceinline__ float model_a_weight(const StepParams &P, float ph)
{
    const float pc = fmaxf(ph, 0.f);
    if (P.model_n_int == 1) return pc;
    if (P.model_n_int == 2) return pc * pc;
    if (P.model_n_int > 2) {
        float wq = pc;
        for (int k = 1; k < P.model_n_int; ++k) wq *= pc;
        return wq;
    }
    return powf(pc, P.model_n);
}

// Source R_p of the solved phases (Eqs. (2)-(4)).
template <int NS, int MODEL>
__device__ __forceinline__ void source_terms(const StepParams &P, const float (&ph)[NS + 1],
                                             const float (&gx)[NS + 1], const float (&gy)[NS + 1],
                                             float (&Rx)[NS], float (&Ry)[NS])
{
    constexpr int N = NS + 1;
    if (MODEL == 0) {
        // Model A, Eq. (2): R_p = a_p n_p - phi_p^n / sum_q phi_q^n * sum_q a_q n_q
        float anx[N], any[N], w[N];
        float2 S2 = make_float2(0.f, 0.f), V2x = S2, V2y = S2;
#pragma unroll
        for (int q = 0; q + 1 < N; q += 2) {
            const float2 f = vget<float2>(ph, q);
            const float2 a = vmul(vmul(vset<float2>(P.four_over_eps), f), vsub(vset<float2>(1.f), f));
            const float2 r = make_float2(inv_norm(gx[q], gy[q], P.unit_delta2), inv_norm(gx[q + 1], gy[q + 1], P.unit_delta2));
            const float2 ar = vmul(a, r);
            const float2 nx2 = vmul(ar, vget<float2>(gx, q)), ny2 = vmul(ar, vget<float2>(gy, q));
            vput(anx, q, nx2);
            vput(any, q, ny2);
            const float2 wq = make_float2(model_a_weight(P, f.x), model_a_weight(P, f.y));
            vput(w, q, wq);
            S2 = vadd(S2, wq);
            V2x = vadd(V2x, nx2);
            V2y = vadd(V2y, ny2);
        }
        float S = S2.x + S2.y, Vx = V2x.x + V2x.y, Vy = V2y.x + V2y.y;
        if (N & 1) {
            const int q = N - 1;
            const float a = P.four_over_eps * ph[q] * (1.f - ph[q]);
            const float ar = a * inv_norm(gx[q], gy[q], P.unit_delta2);
            anx[q] = ar * gx[q];
            any[q] = ar * gy[q];
            w[q] = model_a_weight(P, ph[q]);
            S += w[q];
            Vx += anx[q];
            Vy += any[q];
        }
        const float invS = 1.f / S;
        const float2 Vx2 = vset<float2>(Vx), Vy2 = vset<float2>(Vy), iS2 = vset<float2>(-invS);
#pragma unroll
        for (int p = 0; p + 1 < NS; p += 2) {
            const float2 b = vmul(vget<float2>(w, p), iS2);   // -beta weight
            vput(Rx, p, vfma(b, Vx2, vget<float2>(anx, p)));
            vput(Ry, p, vfma(b, Vy2, vget<float2>(any, p)));
        }
        if (NS & 1) {
            const float b = w[NS - 1] * invS;
            Rx[NS - 1] = anx[NS - 1] - b * Vx;
            Ry[NS - 1] = any[NS - 1] - b * Vy;
        }
    } else {
        // Model B, Eqs. (3)-(4): R_p = sum_{q!=p} 4 phi_p phi_q / eps n_pq,
        // n_pq = unit(phi_q grad phi_p - phi_p grad phi_q), n_qp = -n_pq.
        // The partners q of phase p are taken two at a time.
#pragma unroll
        for (int p = 0; p < NS; ++p) { Rx[p] = 0.f; Ry[p] = 0.f; }
#pragma unroll
        for (int p = 0; p < N; ++p) {
            const float2 kp = vset<float2>(-(P.four_over_eps * ph[p]));
            const float2 gxp = vset<float2>(gx[p]), gyp = vset<float2>(gy[p]), mp = vset<float2>(-ph[p]);
            int q = p + 1;
#pragma unroll
            for (; q + 1 < N; q += 2) {
                const float2 phq = vget<float2>(ph, q);
                const float2 vx = vfma(phq, gxp, vmul(mp, vget<float2>(gx, q)));
                const float2 vy = vfma(phq, gyp, vmul(mp, vget<float2>(gy, q)));
                const float2 n2 = vfma(vx, vx, vmul(vy, vy));
                // cn = -4 phi_p phi_q / eps / |v|
                const float2 cn = vmul(vmul(kp, phq), make_float2(inv_norm2(n2.x, P.unit_delta2),
                                                                  inv_norm2(n2.y, P.unit_delta2)));
                if (p < NS) {
                    Rx[p] = __fmaf_rn(-cn.x, vx.x, Rx[p]);
                    Ry[p] = __fmaf_rn(-cn.x, vy.x, Ry[p]);
                    Rx[p] = __fmaf_rn(-cn.y, vx.y, Rx[p]);
                    Ry[p] = __fmaf_rn(-cn.y, vy.y, Ry[p]);
                }
                if (q + 1 < NS) {
                    vput(Rx, q, vfma(cn, vx, vget<float2>(Rx, q)));
                    vput(Ry, q, vfma(cn, vy, vget<float2>(Ry, q)));
                } else if (q < NS) {
                    Rx[q] = __fmaf_rn(cn.x, vx.x, Rx[q]);
                    Ry[q] = __fmaf_rn(cn.x, vy.x, Ry[q]);
                }
            }
            if (q < N) {
                const float vx = ph[q] * gx[p] - ph[p] * gx[q];
                const float vy = ph[q] * gy[p] - ph[p] * gy[q];
                const float c = P.four_over_eps * ph[p] * ph[q] * inv_norm(vx, vy, P.unit_delta2);
                if (p < NS) { Rx[p] += c * vx; Ry[p] += c * vy; }
                if (q < NS) { Rx[q] -= c * vx; Ry[q] -= c * vy; }
            }
        }
    }
}

// Consistent mass flux, Eq. (13), with phase N eliminated:
// m_phi = -M sum_{p<N} (rho_p - rho_N) (grad phi_p - R_p).
template <int NS>
__device__ __forceinline__ void mass_flux(const StepParams &P, const float (&gx)[NS + 1],
                                          const float (&gy)[NS + 1], const float (&Rx)[NS],
                                          const float (&Ry)[NS], float &mx, float &my)
{
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int p = 0; p < NS; ++p) {
        ax += P.drho[p] * (gx[p] - Rx[p]);
        ay += P.drho[p] * (gy[p] - Ry[p]);
    }
    mx = -P.mob * ax;
    my = -P.mob * ay;
}

// One tile of the fused step: the strip of columns [x0, x0 + T - 4) marching
// rows [y0, y0 + TY) of the simulation described by P.  smem is the dynamic
// shared memory of the block (step_smem_bytes gives its size).  VEC: the
// pulled populations are staged as row windows (nx a multiple of 4, of 8
// with 16-bit storage, 16-byte aligned planes, no wall across x);
// otherwise every ring thread copies the values its node pulls, 4 bytes at
// a time.
template <int NS, int MODEL, int T, int ST, bool VEC = false, bool TAPE = false>
__device__ __forceinline__ void step_tile(const StepParams &P, const int x0, const int y0, const int TY,
                                          float *smem)
{
    constexpr int N = NS + 1;
    constexpr bool V32 = VEC && ST == 0, V16 = VEC && ST != 0;
    static_assert(!TAPE || ST == 0, "the adjoint tape is written by the FP32 form");
    // Thread t owns ring column t, lattice column x0 - 2 + t: every thread
    // pulls one phase field in stage A, the inner T - 2 compute m_phi in
    // stage B and the inner T - 4 (the strip) complete their node in stage
    // C, so no warp runs a stage twice for halo nodes.
    constexpr int W = T - 4;                 // strip width
    constexpr int NE = ring_even(NS);       // phases per ring row, rounded up to pairs
    float *s_phi = smem;                     // [5][NE/2][T][2] phi(t) rows r-2..r+2 (see ring_idx)
    float *s_w = s_phi + 5 * NE * T;         // [3][T]       w = m_phi,x u_y - u_x m_phi,y, rows r-1..r+1
    float *s_j = s_w + 3 * T;                // [3][3][NE/2][T][2] j_x, j_y, phi_lo of own nodes
    float *s_F = s_j + 9 * NE * T;           // [9NS][T]     staged pulled f of the next row
                                             // ([10NS][T] with 16-bit storage, see prefetch_pull16;
                                             // VEC: [T/32][9NS][kWin] row windows)
    float *s_G = s_F + (T / 32) * 9 * NS * kWin;   // VEC: [2][T/32][8][kWin] g windows of two rows
    // VEC with 16-bit storage: [T/32][8NS][kWin16] deviation and [T/32][2NS][kWin]
    // rest-population / own-phi windows, then per row parity [T/32][8][kWin16] g
    // deviations and [T/32][3][kWin] pressure rows
    unsigned short *s_D16 = (unsigned short *)s_F;
    float *s_O16 = (float *)(s_D16 + (T / 32) * 8 * NS * kWin16);
    unsigned short *s_G16 = (unsigned short *)(s_O16 + (T / 32) * 2 * NS * kWin);
    float *s_P16 = (float *)(s_G16 + 2 * (T / 32) * 8 * kWin16);

    const int t = threadIdx.x;
    const int We = min(W, P.nx - x0), TYe = min(TY, P.ny - y0);
    const bool in_ring = t < We + 4;             // phi needed here
    const bool in_flux = t >= 1 && t < We + 3;   // m_phi needed here
    const bool own = t >= 2 && t < We + 2;       // node updated here
    const unsigned pl = P.plane;
    const int nx = P.nx;
    bool xflip = false;
    const int xc = in_ring ? map_axis(x0 - 2 + t, nx, P.wall_x, xflip) : 0;
    const int xg = x0 - 2 + t;                   // lattice x of an own node

    unsigned par_next = 0, par_cur = 0;   // halves of the staged 16-bit words
    // VEC: this lane's window piece and direction group, the (wrapped)
    // lattice column of that piece, and the warp's windows.
    const int lane = t & 31, wc = lane % 9, wg = lane / 9, warp = t >> 5;
    const bool copier = V32 ? (lane < 27 && 32 * warp < We + 4) : (V16 && 32 * warp < We + 4);
    unsigned wcol = 0;
    if constexpr (V32) {
        int c = x0 - 4 + 32 * warp + 4 * wc;
        if (c < 0 || c >= nx) c = ((c % nx) + nx) % nx;   // periodic x: a piece never straddles the edge
        wcol = (unsigned)c;
    }
    float *s_Fw = s_F + warp * 9 * NS * kWin;
    float *s_Gw = s_G + warp * 8 * kWin;   // + (row & 1) * (T / 32) * 8 * kWin
    // 16-bit windows of this warp: first column of the deviation windows (ws),
    // of the FP32 windows (xo), and the window column of lane 0's node (o16)
    const int xo = x0 - 4 + 32 * warp, ws = ((x0 - 3 + 32 * warp) >> 3) * 8, o16 = x0 - 2 + 32 * warp - ws;
    unsigned short *s_Dw = s_D16 + warp * 8 * NS * kWin16;
    float *s_Ow = s_O16 + warp * 2 * NS * kWin;
    // The pulled populations of row r+1 are copied into shared memory
    // (cp.async) while rows r..r-2 are computed.  Without VEC each thread
    // only reads the slots it filled itself; with VEC the warp barrier after
    // the wait makes the warp's windows visible to all its lanes.
    {
        bool yflip;
        const int ya = map_axis(y0 - 2, P.ny, P.wall_y, yflip);
        if constexpr (V32) {
            if (copier) stage_pull_rows<NS>(P, ya, wg, wc, wcol, s_Fw);
        } else if constexpr (V16) {
            if (copier) stage_pull_rows16<NS>(P, ya, lane, ws, xo, s_Dw, s_Ow);
        } else if (in_ring) {
            if constexpr (ST == 0) prefetch_pull<NS>(P, xc, ya, s_F, T, t);
            else par_next = prefetch_pull16<NS>(P, xc, ya, s_F, T, t);
        }
        cp_async_commit();
    }
    // Values a thread hands from stage B of one row to stage C of the same
    // row one iteration later (c: row being completed, n: next row), and the
    // previous-step velocity loaded one iteration ahead of stage B.
    float Rcx[NS], Rcy[NS], Rnx[NS], Rny[NS];   // sources R_p
#pragma unroll
    for (int p = 0; p < NS; ++p) { Rcx[p] = Rcy[p] = Rnx[p] = Rny[p] = 0.f; }
    float Mcx = 0.f, Mcy = 0.f, Mnx = 0.f, Mny = 0.f;   // m_phi(t)
    // FP32 storage: phi, grad phi and lap phi of the row stage B evaluated
    // (Eq. (27)); stage C of the same row reuses them instead of reading the
    // window again (16-bit storage reads the window there anyway)
    float PHc[NS], GXc[NS], GYc[NS], LPc[NS], PHn[NS], GXn[NS], GYn[NS], LPn[NS];
#pragma unroll
    for (int p = 0; p < NS; ++p) PHc[p] = GXc[p] = GYc[p] = LPc[p] = PHn[p] = GXn[p] = GYn[p] = LPn[p] = 0.f;
    float Ucx = 0.f, Ucy = 0.f, Unx = 0.f, Uny = 0.f;   // u(t-1) of the own node
    float ub_x = 0.f, ub_y = 0.f;                       // u(t-1) for stage B of this iteration
    float ub_s = 1.f;                                   // its sign: -1 on a no-slip ghost node

    // ring slots of row ra (5-row phi ring, 3-row rings), advanced each iteration
    int a5 = slot5(y0 - 2), a3 = slot3(y0 - 2);
    for (int it = 0; it < TYe + 4; ++it) {
        const int ra = y0 - 2 + it;
        const int a5m1 = a5 == 0 ? 4 : a5 - 1, a5m2 = a5 >= 2 ? a5 - 2 : a5 + 3, a5m3 = a5 >= 3 ? a5 - 3 : a5 + 2;
        const int a3m1 = a3 == 0 ? 2 : a3 - 1, a3m2 = a3 >= 2 ? a3 - 2 : a3 + 1;
        // stage-C inputs of row ra - 2, requested before stages A and B
        // (loaded raw; anything computed from them waits until stage C, so
        // that the loads overlap stages A and B)
        float g[9], php[NS], mpx = 0.f, mpy = 0.f;
        float gps[9];             // 16-bit storage: P of the source node
        unsigned short gq[9];     // 16-bit storage: stored deviation
        unsigned node = 0;
        const bool do_c = it >= 4 && own;
        if (do_c) {
            const int y = ra - 2;
            unsigned gnode[9];
            int gdir[9];
            if constexpr (!VEC) pull_sources(P, xg, y, gnode, gdir);
#pragma unroll
            for (int i = 1; i < 9; ++i) {
                if constexpr (VEC) {
                    // staged as a row window, read in stage C
                } else if constexpr (ST == 0) {
                    g[i] = __ldg(P.gin + (unsigned)(gdir[i] - 1) * pl + gnode[i]);
                } else {
                    const unsigned short *g16 = (const unsigned short *)P.gin;
                    gq[i] = __ldg(g16 + (unsigned)(gdir[i] - 1) * pl + gnode[i]);
                    gps[i] = __ldg(P.pin + gnode[i]);
                }
            }
            node = (unsigned)y * nx + xg;
#pragma unroll
            for (int p = 0; p < NS; ++p) php[p] = P.phi_prev[(size_t)p * pl + node];
            mpx = P.mphi_in[node];
            mpy = P.mphi_in[pl + node];
        }
        // previous-step velocity of row ra, used by stage B of the next iteration
        // (the ghost sign is applied where the value is used, so that no
        // instruction here waits for these loads)
        float ua_x = 0.f, ua_y = 0.f, ua_s = 1.f;
        if (in_ring && it >= 1 && it + 1 < TYe + 4) {
            bool yflip;
            const int yv = map_axis(ra, P.ny, P.wall_y, yflip);
            const unsigned k = (unsigned)yv * nx + xc;
            ua_x = __ldg(P.uin + k);
            ua_y = __ldg(P.uin + pl + k);
            if (xflip != yflip) ua_s = -1.f;   // no-slip ghost: u = -u(image)
        }
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");   // this row's pulled f landed
        if constexpr (VEC) __syncwarp();
        par_cur = par_next;
        // ---------------------------------------------------- stage A
        if (in_ring) {
            float ph[NS], plo[NS], jx[NS], jy[NS];
            if constexpr (VEC) {
                bool yflip;
                const int yi = map_axis(ra, P.ny, P.wall_y, yflip);
                const bool bl = P.wall_y && yi == 0, bh = P.wall_y && yi == P.ny - 1;
                if constexpr (V32) sum_pulled_win<NS, true>(s_Fw, win_cols(2 + lane, bl, bh), ph, plo, jx, jy);
                else sum_pulled16_win<NS, ST, true>(s_Dw, s_Ow, lane, win_cols(lane + o16, bl, bh), ph, plo, jx, jy);
            } else if constexpr (ST == 0) {
                sum_pulled<NS, true>(s_F, T, t, ph, plo, jx, jy);
            } else {
                sum_pulled16<NS, ST, true>(s_F, T, t, par_cur, ph, plo, jx, jy);
            }
            if (P.wet && (ra < 0 || ra >= P.ny)) {
                // ghost row beyond a wetting wall (Sec. 4.2): its mirror image
                // plus (2k - 1) s_p, s_p = phi_p sum_q (4/eps) cos theta_pq phi_q
                // at the image node, so that the difference across the wall
                // is s_p (n_w pointing into the wall)
                const int w = ra < 0 ? 0 : 1;
                const float k2 = (float)(2 * (ra < 0 ? -ra : ra - (P.ny - 1)) - 1);
                float phN = 1.f;
#pragma unroll
                for (int p = 0; p < NS; ++p) phN -= ph[p];
                float sp[NS];
#pragma unroll
                for (int p = 0; p < NS; ++p) {
                    float a = P.wetc[w][p][NS] * phN;
#pragma unroll
                    for (int q = 0; q < NS; ++q) a += P.wetc[w][p][q] * ph[q];
                    sp[p] = ph[p] * a;
                }
#pragma unroll
                for (int p = 0; p < NS; ++p) ph[p] += k2 * sp[p];
            }
            float *prow = s_phi + a5 * NE * T;
#pragma unroll
            for (int p = 0; p + 1 < NS; p += 2) rst(prow, T, p, t, vget<float2>(ph, p));
            if (NS & 1) rst(prow, T, NS - 1, t, ph[NS - 1]);
            if (own && ra >= y0 && ra < y0 + TYe) {
                float *jrow = s_j + a3 * 3 * NE * T;   // j_x, then j_y, then phi_lo rows
#pragma unroll
                for (int p = 0; p + 1 < NS; p += 2) {
                    rst(jrow, T, p, t, vget<float2>(jx, p));
                    rst(jrow + NE * T, T, p, t, vget<float2>(jy, p));
                    rst(jrow + 2 * NE * T, T, p, t, vget<float2>(plo, p));
                }
                if (NS & 1) {
                    rst(jrow, T, NS - 1, t, jx[NS - 1]);
                    rst(jrow + NE * T, T, NS - 1, t, jy[NS - 1]);
                    rst(jrow + 2 * NE * T, T, NS - 1, t, plo[NS - 1]);
                }
            }
            if (!VEC && it + 1 < TYe + 4) {
                bool yflip;
                const int yn = map_axis(ra + 1, P.ny, P.wall_y, yflip);
                if constexpr (ST == 0) prefetch_pull<NS>(P, xc, yn, s_F, T, t);
                else par_next = prefetch_pull16<NS>(P, xc, yn, s_F, T, t);
            }
        }
        if constexpr (VEC) {
            __syncwarp();   // every lane of the warp has read its windows of row ra
            if (copier) {
                if (it + 1 < TYe + 4) {
                    bool yflip;
                    const int yn = map_axis(ra + 1, P.ny, P.wall_y, yflip);
                    if constexpr (V32) stage_pull_rows<NS>(P, yn, wg, wc, wcol, s_Fw);
                    else stage_pull_rows16<NS>(P, yn, lane, ws, xo, s_Dw, s_Ow);
                }
                // g of the row stage C completes next iteration
                const int yg = ra - 1;
                if (it >= 3 && yg < y0 + TYe) {
                    if constexpr (V32) {
                        stage_flow_rows(P, yg, wg, wc, wcol, s_Gw + (yg & 1) * (T / 32) * 8 * kWin);
                    } else {
                        const int b = (yg & 1) * (T / 32) + warp;
                        stage_flow_rows16(P, yg, lane, ws, xo, s_G16 + b * 8 * kWin16, s_P16 + b * 3 * kWin);
                    }
                }
            }
        }
        cp_async_commit();
        __syncthreads();
        // ---------------------------------------------------- stage B
        if (it >= 2) {
            const int s3 = a3m1;   // row rb = ra - 1
            if (in_flux) {
                float ph[N], gx[N], gy[N], Rx[NS], Ry[NS], mx, my;
                if constexpr (ST == 0) {
                    float lap[N];
                    window_grad_lap<NS>(s_phi, T, a5m2, a5m1, a5, t, ph, gx, gy, lap);
#pragma unroll
                    for (int p = 0; p < NS; ++p) { PHn[p] = ph[p]; GXn[p] = gx[p]; GYn[p] = gy[p]; LPn[p] = lap[p]; }
                } else {
                    window_grad<NS>(s_phi, T, a5m2, a5m1, a5, t, ph, gx, gy);
                }
                source_terms<NS, MODEL>(P, ph, gx, gy, Rx, Ry);
                mass_flux<NS>(P, gx, gy, Rx, Ry, mx, my);
                s_w[s3 * T + t] = ub_s * (mx * ub_y - ub_x * my);
#pragma unroll
                for (int p = 0; p < NS; ++p) { Rnx[p] = Rx[p]; Rny[p] = Ry[p]; }
                Mnx = mx;
                Mny = my;
                Unx = ub_x;
                Uny = ub_y;
            }
        }
        __syncthreads();
        // ---------------------------------------------------- stage C
        if (do_c) {
            const int y = ra - 2;
            const int sm = a5m3, s0 = a5m2, sp = a5m1;
            float ph[N], gx[N], gy[N], lap[N];
            if constexpr (ST == 0) {
                float sph = 0.f, sgx = 0.f, sgy = 0.f, sl = 0.f;
#pragma unroll
                for (int p = 0; p < NS; ++p) {
                    ph[p] = PHc[p];
                    gx[p] = GXc[p];
                    gy[p] = GYc[p];
                    lap[p] = LPc[p];
                    sph += ph[p];
                    sgx += gx[p];
                    sgy += gy[p];
                    sl += lap[p];
                }
                ph[NS] = 1.f - sph;
                gx[NS] = -sgx;
                gy[NS] = -sgy;
                lap[NS] = -sl;
            } else {
                window_grad_lap<NS>(s_phi, T, sm, s0, sp, t, ph, gx, gy, lap);
            }

            // mixture density, viscosity and grad rho (Eqs. (11),(12))
            float rho = P.rhoN, mu = P.muN, grx = 0.f, gry = 0.f;
#pragma unroll
            for (int p = 0; p < NS; ++p) {
                rho += P.drho[p] * ph[p];
                mu += P.dmu[p] * ph[p];
                grx += P.drho[p] * gx[p];
                gry += P.drho[p] * gy[p];
            }

            // chemical potentials (Eq. (17)) and F_s = sum_p mu_p grad phi_p
            // (Eq. (16)); the partners q of phase p two at a time
            float gp[N], muph[N];
            {
                const float2 one = vset<float2>(1.f), two = vset<float2>(2.f);
#pragma unroll
                for (int p = 0; p + 1 < N; p += 2) {
                    const float2 f = vget<float2>(ph, p);
                    vput(gp, p, vmul(vmul(vmul(two, f), vsub(one, f)), vfma(vset<float2>(-2.f), f, one)));
                }
                if (N & 1) gp[N - 1] = 2.f * ph[N - 1] * (1.f - ph[N - 1]) * (1.f - 2.f * ph[N - 1]);
#pragma unroll
                for (int p = 0; p < N; ++p) muph[p] = 0.f;
#pragma unroll
                for (int p = 0; p < N; ++p) {
                    const float2 php2 = vset<float2>(ph[p]), gpp = vset<float2>(gp[p]), lpp = vset<float2>(lap[p]);
                    int q = p + 1;
#pragma unroll
                    for (; q + 1 < N; q += 2) {
                        const float2 sq = vadd(php2, vget<float2>(ph, q));
                        const float2 G = vmul(vmul(vmul(two, sq), vsub(one, sq)), vfma(vset<float2>(-2.f), sq, one));
                        const float2 b = make_float2(P.beta2[p][q], P.beta2[p][q + 1]);
                        const float2 k = make_float2(P.kap[p][q], P.kap[p][q + 1]);
                        // mu_p accumulates its terms in the order q, q + 1
                        // (the pairwise sum keeps the cancellation of
                        // g'(phi_p) - g'(phi_p + phi_q) where phase q is
                        // nearly absent; the adjoint's gradients depend on it)
                        const float2 tp = vfma(b, vsub(gpp, G), vmul(k, vget<float2>(lap, q)));
                        muph[p] += tp.x;
                        muph[p] += tp.y;
                        vput(muph, q, vadd(vget<float2>(muph, q), vfma(b, vsub(vget<float2>(gp, q), G), vmul(k, lpp))));
                    }
                    if (q < N) {
                        const float sq = ph[p] + ph[q];
                        const float G = 2.f * sq * (1.f - sq) * (1.f - 2.f * sq);
                        const float b = P.beta2[p][q], k = P.kap[p][q];
                        muph[p] += b * (gp[p] - G) + k * lap[q];
                        muph[q] += b * (gp[q] - G) + k * lap[p];
                    }
                }
            }
            float Fx = 0.f, Fy = 0.f;
#pragma unroll
            for (int p = 0; p < NS; ++p) {
                const float d = muph[p] - muph[NS];
                Fx += d * gx[p];
                Fy += d * gy[p];
            }

            // F_c = -div(m_phi u - u m_phi)/2 with the previous velocity:
            // with w = m_x u_y - u_x m_y, F_c = (d_y w / 2, -d_x w / 2).
            {
                const float *wm = s_w + a3 * T + t;
                const float *w0 = s_w + a3m2 * T + t;
                const float *wp = s_w + a3m1 * T + t;
                const float wsw = wm[-1], ws = wm[0], wse = wm[1];
                const float ww = w0[-1], we = w0[1];
                const float wnw = wp[-1], wn = wp[0], wne = wp[1];
                const float dxw = (we - ww) * (1.f / 3.f) + ((wne + wse) - (wnw + wsw)) * (1.f / 12.f);
                const float dyw = (wn - ws) * (1.f / 3.f) + ((wne + wnw) - (wse + wsw)) * (1.f / 12.f);
                Fx += 0.5f * dyw;
                Fy -= 0.5f * dxw;
            }
            // gravity: F_g = rho g (total force F = F_s + F_g + F_c)
            Fx += rho * P.gx;
            Fy += rho * P.gy;

            // macroscopic velocity (Eq. (25b)) and mass flux (Eq. (13))
            if constexpr (V16) {
                const int b = (y & 1) * (T / 32) + warp;
                const unsigned short *gd = s_G16 + b * 8 * kWin16;
                const float *pw = s_P16 + b * 3 * kWin;   // rows y - 1, y, y + 1
                const bool bl = P.wall_y && y == 0, bh = P.wall_y && y == P.ny - 1;
                const WinCols wd = win_cols(lane + o16, bl, bh), wp = win_cols(2 + lane, bl, bh);
                gq[1] = gd[wd.b - 1];
                gq[2] = gd[kWin16 + wd.b];
                gq[3] = gd[2 * kWin16 + wd.b + 1];
                gq[4] = gd[3 * kWin16 + wd.b];
                gq[5] = gd[4 * kWin16 + wd.c5];
                gq[6] = gd[5 * kWin16 + wd.c6];
                gq[7] = gd[6 * kWin16 + wd.c7];
                gq[8] = gd[7 * kWin16 + wd.c8];
                gps[1] = pw[kWin + wp.b - 1];
                gps[2] = pw[(bl ? kWin : 0) + wp.b];
                gps[3] = pw[kWin + wp.b + 1];
                gps[4] = pw[(bh ? kWin : 2 * kWin) + wp.b];
                gps[5] = pw[(bl ? kWin : 0) + wp.c5];
                gps[6] = pw[(bl ? kWin : 0) + wp.c6];
                gps[7] = pw[(bh ? kWin : 2 * kWin) + wp.c7];
                gps[8] = pw[(bh ? kWin : 2 * kWin) + wp.c8];
            }
            if constexpr (V32) {
                const float *gw = s_Gw + (y & 1) * (T / 32) * 8 * kWin;
                const WinCols wcl = win_cols(2 + lane, P.wall_y && y == 0, P.wall_y && y == P.ny - 1);
                g[1] = gw[wcl.b - 1];
                g[2] = gw[kWin + wcl.b];
                g[3] = gw[2 * kWin + wcl.b + 1];
                g[4] = gw[3 * kWin + wcl.b];
                g[5] = gw[4 * kWin + wcl.c5];
                g[6] = gw[5 * kWin + wcl.c6];
                g[7] = gw[6 * kWin + wcl.c7];
                g[8] = gw[7 * kWin + wcl.c8];
            }
            if constexpr (ST != 0) {
                // g_i = 3 w_i P(source) + stored deviation
#pragma unroll
                for (int i = 1; i < 9; ++i) g[i] = __fmaf_rn(3.f * w_of(i), gps[i], Store16<ST>::dec(gq[i]));
            }
            const float sg = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
            const float jgx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
            const float jgy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
            const float d58 = (g[5] + g[6]) + (g[7] + g[8]);
            const float Pxx = (g[1] + g[3]) + d58;
            const float Pyy = (g[2] + g[4]) + d58;
            const float Pxy = (g[5] - g[6]) + (g[7] - g[8]);
            const float inv_rho = 1.f / rho;
            const float2 uv = vmul(vfma(vset<float2>(0.5f), make_float2(Fx, Fy), make_float2(jgx, jgy)),
                                   vset<float2>(inv_rho));
            const float ux = uv.x, uy = uv.y;
            const float mphx = Mcx, mphy = Mcy;
            const float upx = Ucx, upy = Ucy;
            const float2 mv = vfma(vset<float2>(rho), uv, make_float2(mphx, mphy));
            const float mx = mv.x, my = mv.y;
            const float ugr = ux * grx + uy * gry;
            float rho_prev = P.rhoN;
#pragma unroll
            for (int p = 0; p < NS; ++p) rho_prev += P.drho[p] * php[p];
            const float mu_t = mx * ux + my * uy;
            const float mu_prev = (rho_prev * upx + mpx) * upx + (rho_prev * upy + mpy) * upy;
            // Eq. (25c): P = c_s^2/(1-w0) [sum_{i!=0} g_i + u.grad rho/2
            //   - w0 m.u/(2 c_s^2) + w0 d_t(m.u)/(4 c_s^2)], c_s^2 = 1/3, w0 = 4/9
            const float Pr = 0.6f * (sg + 0.5f * ugr - (2.f / 3.f) * mu_t + (1.f / 3.f) * (mu_t - mu_prev));

            // phase-field collisions, Eqs. (18),(19) in moment space
            const int s3 = a3m2;
            // links of this node that end in a wall: their population comes
            // back to this node (half-way bounce-back)
            const bool bxl = P.wall_x && xg == 0, bxh = P.wall_x && xg == nx - 1;
            const bool byl = P.wall_y && y == 0, byh = P.wall_y && y == P.ny - 1;
            auto bounce = [&](int j) {
                return (cx_of(j) < 0 && bxl) || (cx_of(j) > 0 && bxh) || (cy_of(j) < 0 && byl) ||
                       (cy_of(j) > 0 && byh);
            };
            (void)bounce;
            const CollCoef<float2> k2(P.s1, ux, uy, upx, upy);
            const CollCoef<float> k1(P.s1, ux, uy, upx, upy);
            const float *sjx = s_j + s3 * 3 * NE * T, *sjy = sjx + NE * T, *slo = sjy + NE * T;
            auto collide = [&](auto tag, const auto &k, int p) {
                using V = decltype(tag);
                V A, B, C, D;
                phase_moments<V>(vget<V>(ph, p), rld<V>(sjx, T, p, t), rld<V>(sjy, T, p, t), vget<V>(php, p),
                                 vget<V>(Rcx, p), vget<V>(Rcy, p), k, A, B, C, D);
                if constexpr (ST == 0) {
                    V fo[9];
                    phase_populations<V>(vget<V>(ph, p), rld<V>(slo, T, p, t), A, B, C, D, fo);
#pragma unroll
                    for (int i = 0; i < 9; ++i) vstore(P.fout + ((size_t)p * 9 + i) * pl + node, 9 * (size_t)pl, fo[i]);
                } else {
                    // f*_j = w_j phi + h_j; stored: dev_j = f*_j - w_j phi(puller
                    // of j), rounded to 16 bits (a phase pair's two deviations
                    // in one word).  The rest population (FP32) is what makes
                    // the nine values the pullers reconstruct sum to phi.
                    const V phi = vget<V>(ph, p);
                    const V h1 = vmul(vset<V>(0.5f), vsub(A, D)), h2 = vmul(vset<V>(0.5f), vsub(B, C));
                    const V h5 = vmul(vset<V>(0.25f), vadd(C, D)), h6 = vmul(vset<V>(0.25f), vsub(C, D));
                    const V zero = vset<V>(0.f);
                    const V hdev[9] = {zero, h1, h2, vsub(zero, h1), vsub(zero, h2), h5, h6, vsub(zero, h5),
                                       vsub(zero, h6)};
                    V r[9];
#pragma unroll
                    for (int j = 1; j < 9; ++j) {
                        const int sl = cy_of(j) > 0 ? sp : (cy_of(j) < 0 ? sm : s0);
                        const V base = bounce(j) ? phi : rld<V>(s_phi + sl * NE * T, T, p, t + cx_of(j));
                        const V dev = vfma(vset<V>(w_of(j)), vsub(phi, base), hdev[j]);
                        if constexpr (sizeof(V) == 8) {
                            const unsigned wd = Pack16<ST>::enc2(dev);
                            ((unsigned *)P.fout)[dev_word(p / 2, j - 1, pl, node)] = wd;
                            r[j] = vfma(vset<V>(w_of(j)), base, Pack16<ST>::dec2(wd));
                        } else {
                            const unsigned short q = Store16<ST>::enc(dev);
                            ((unsigned short *)P.fout)[dev_tail(NS, j - 1, pl, node)] = q;
                            r[j] = __fmaf_rn(w_of(j), base, Store16<ST>::dec(q));
                        }
                    }
                    V e13, e24, e57, e68, ea, eb, es, e0;
                    const V s13 = two_sum_v(r[1], r[3], e13), s24 = two_sum_v(r[2], r[4], e24);
                    const V s57 = two_sum_v(r[5], r[7], e57), s68 = two_sum_v(r[6], r[8], e68);
                    const V sa = two_sum_v(s13, s24, ea), sb = two_sum_v(s57, s68, eb);
                    const V S = two_sum_v(sa, sb, es);
                    const V E = vadd(vadd(vadd(e13, e24), vadd(e57, e68)), vadd(vadd(ea, eb), es));
                    const V a0 = two_sum_v(phi, vsub(zero, S), e0);
                    const V plo = rld<V>(slo, T, p, t);
                    vstore(P.f0out + (size_t)p * pl + node, (size_t)pl, vadd(a0, vsub(vadd(e0, plo), E)));
                }
                vstore(P.phi + (size_t)p * pl + node, (size_t)pl, vget<V>(ph, p));
            };
#pragma unroll
            for (int p = 0; p + 1 < NS; p += 2) collide(float2(), k2, p);
            if (NS & 1) collide(0.f, k1, NS - 1);

            // flow collision, Eqs. (21)-(24), tau_g from Eq. (26)
            {
                // (x, y) pairs: diagonal second moments (xx, yy), first
                // moments, and (m7, m6) = (rho u_x, rho u_y)/3 + (F_x, F_y)/6
                const float s2r = 2.f * rho / (6.f * mu + rho);   // 1/tau_g, tau_g = 3 mu/rho + 1/2
                const float c2 = 1.f - s2r, h2 = 1.f - 0.5f * s2r;
                const float2 u2 = make_float2(ux, uy), F2 = make_float2(Fx, Fy), gr2 = make_float2(grx, gry);
                const float2 Qd = vmul(make_float2(mx, my), u2);   // (Qxx, Qyy)
                const float Qxy = 0.5f * (mx * uy + my * ux);
                const float2 dQd = vsub(vmul(make_float2(mphx, mphy), u2), vmul(make_float2(mpx, mpy), make_float2(upx, upy)));
                const float dQxy = 0.5f * ((mphx * uy + mphy * ux) - (mpx * upy + mpy * upx));
                const float2 Md = vadd(vfma(vset<float2>(2.f / 3.f), vmul(u2, gr2), vfma(vset<float2>(2.f), vmul(u2, F2), dQd)),
                                       vset<float2>((1.f / 3.f) * ugr));   // (Mxx, Myy)
                const float Mxy = ux * Fy + Fx * uy + dQxy + (1.f / 3.f) * (ux * gry + grx * uy);
                const float2 m12 = vadd(make_float2(jgx, jgy), F2);
                const float2 m34 = vfma(vset<float2>(c2), make_float2(Pxx, Pyy),
                                        vfma(vset<float2>(s2r), vadd(vset<float2>(Pr), Qd), vmul(vset<float2>(h2), Md)));
                const float m5 = c2 * Pxy + s2r * Qxy + h2 * Mxy;
                const float2 m76 = vfma(vset<float2>(rho * (1.f / 3.f)), u2, vmul(F2, vset<float2>(1.f / 6.f)));
                const float m6 = m76.y, m7 = m76.x;
                const float m8 = (Pr + Qd.x + Qd.y) * (1.f / 3.f) + (Md.x + Md.y) * (1.f / 6.f) - ugr * (1.f / 18.f);
                const float2 h34 = vsub(m34, vset<float2>(m8));
                const float2 gs12 = vmul(vset<float2>(0.5f), vadd(vsub(m12, m76), h34));
                const float2 gs34 = vmul(vset<float2>(0.5f), vadd(vsub(m76, m12), h34));
                const float gs[9] = {0.f, gs12.x, gs12.y, gs34.x, gs34.y,
                                     0.25f * ((m5 + m6) + (m7 + m8)),
                                     0.25f * ((m6 - m5) + (m8 - m7)),
                                     0.25f * ((m5 - m6) + (m8 - m7)),
                                     0.25f * ((m7 - m5) + (m8 - m6))};
                if constexpr (ST == 0) {
                    float *go = P.gout + node;
#pragma unroll
                    for (int i = 1; i < 9; ++i) go[(i - 1) * pl] = gs[i];
                } else {
                    // stored: g*_i - 3 w_i P of this node (the puller adds it back)
                    unsigned short *go = (unsigned short *)P.gout + node;
#pragma unroll
                    for (int i = 1; i < 9; ++i) go[(size_t)(i - 1) * pl] = Store16<ST>::enc(__fmaf_rn(-3.f * w_of(i), Pr, gs[i]));
                }
            }
            P.uout[node] = ux;
            P.uout[pl + node] = uy;
            P.mphi[node] = mphx;
            P.mphi[pl + node] = mphy;
            if (P.pout) P.pout[node] = Pr;
            if constexpr (TAPE) {
                // the intermediate fields of this step at this node, for the
                // adjoint: phi, j, pulled g, grad phi, lap phi, R, m_phi, w, F
                float *tp = P.tape + node;
#pragma unroll
                for (int p = 0; p < NS; ++p) {
                    tp[(size_t)p * pl] = ph[p];
                    tp[(size_t)(NS + 2 * p) * pl] = rld<float>(sjx, T, p, t);
                    tp[(size_t)(NS + 2 * p + 1) * pl] = rld<float>(sjy, T, p, t);
                    tp[(size_t)(3 * NS + 8 + 2 * p) * pl] = gx[p];
                    tp[(size_t)(3 * NS + 9 + 2 * p) * pl] = gy[p];
                    tp[(size_t)(5 * NS + 8 + p) * pl] = lap[p];
                    tp[(size_t)(6 * NS + 8 + 2 * p) * pl] = Rcx[p];
                    tp[(size_t)(6 * NS + 9 + 2 * p) * pl] = Rcy[p];
                }
#pragma unroll
                for (int i = 1; i < 9; ++i) tp[(size_t)(3 * NS + i - 1) * pl] = g[i];
                tp[(size_t)(8 * NS + 8) * pl] = mphx;
                tp[(size_t)(8 * NS + 9) * pl] = mphy;
                tp[(size_t)(8 * NS + 10) * pl] = s_w[a3m2 * T + t];
                tp[(size_t)(8 * NS + 11) * pl] = Fx;
                tp[(size_t)(8 * NS + 12) * pl] = Fy;
            }
        }
#pragma unroll
        for (int p = 0; p < NS; ++p) {
            Rcx[p] = Rnx[p];
            Rcy[p] = Rny[p];
            PHc[p] = PHn[p];
            GXc[p] = GXn[p];
            GYc[p] = GYn[p];
            LPc[p] = LPn[p];
        }
        Mcx = Mnx;
        Mcy = Mny;
        Ucx = Unx;
        Ucy = Uny;
        ub_x = ua_x;
        ub_y = ua_y;
        ub_s = ua_s;
        a5 = a5 == 4 ? 0 : a5 + 1;
        a3 = a3 == 2 ? 0 : a3 + 1;
    }
}

// Dynamic shared memory of step_tile: phi ring, w ring, own-node j ring and
// the staging rows (9 slots per phase, 10 with 16-bit storage; VEC: the
// warps' pull windows and two rows of flow windows).
template <int NS, int T, int ST, bool VEC = false>
constexpr size_t step_smem_bytes()
{
    constexpr size_t rings = (size_t)T * (14 * ring_even(NS) + 3);   // phi, w and j rings (floats)
    if (VEC && ST == 0) return sizeof(float) * (rings + (size_t)(T / 32) * kWin * (9 * NS + 16));
    if (VEC)   // 16-bit deviation windows (2 bytes a value) and FP32 windows
        return sizeof(float) * rings +
               (size_t)(T / 32) * (2 * kWin16 * (8 * NS + 16) + sizeof(float) * kWin * (2 * NS + 6));
    return sizeof(float) * (rings + (size_t)T * (ST == 0 ? 9 : 10) * NS);
}

// Blocks per SM the step kernel is compiled for.  FP32 storage: three of 128
// threads (up to 170 registers a thread; measured: the throughput is flat
// between 12 and 16 resident warps and falls when the registers are squeezed
// to fit more); from N = 7 on the row windows leave shared memory for two
// blocks of 128 (or four of 64), so the registers may grow to 255 (2048^2
// N = 7: 6,602 -> 8,562 MLUPS with 64-thread blocks).  16-bit storage: four
// of 128 (128 registers), or as many as the shared memory of a block leaves
// room for (from N = 6 on).
template <int NS, int T, int ST, bool VEC>
constexpr int step_min_blocks()
{
    if (ST == 0) return (NS >= 6 && VEC ? 256 : 384) / T;   // measured best at N = 7, 8 (255 registers)
    constexpr size_t smem = step_smem_bytes<NS, T, ST, VEC>();
    constexpr int by_smem = (int)((228u * 1024u) / (smem + 1024u));
    constexpr int want = 512 / T;
    return by_smem < 1 ? 1 : (by_smem < want ? by_smem : want);
}

// Grid: one block per (strip, row chunk), strips of T - 4 columns, strip
// index fastest.  TY > 0: chunks of TY rows; TY = 0: chunk k of `chunks`
// covers rows [k ny / chunks, (k + 1) ny / chunks).
template <int NS, int MODEL, int T, int ST, bool VEC, bool TAPE = false>
__global__ void __launch_bounds__(T, (step_min_blocks<NS, T, ST, VEC>()))
    step_kernel(const StepParams P, const int TY, const int chunks, const int strips)
{
    extern __shared__ __align__(16) float smem[];
    pdl_wait();   // launched with launch_pdl
    const int s = blockIdx.x % strips, k = blockIdx.x / strips;
    int y0, ty;
    if (TY > 0) {
        y0 = k * TY;
        ty = TY;
    } else {
        y0 = (int)((long long)k * P.ny / chunks);
        ty = (int)((long long)(k + 1) * P.ny / chunks) - y0;
    }
    if (ty <= 0 || y0 >= P.ny) return;
    step_tile<NS, MODEL, T, ST, VEC, TAPE>(P, s * (T - 4), y0, ty, smem);
}

// Resident blocks of one kernel variant on device dev (the dynamic
// shared-memory limit, a per-device function attribute, is set on first use).
template <int NS, int MODEL, int T, int ST, bool VEC, bool TAPE = false>
cudaError_t variant_slots(int dev, int *out)
{
    constexpr size_t smem = step_smem_bytes<NS, T, ST, VEC>();
    // resident blocks per device, 0 until configured (threads that race here
    // compute and store the same value)
    static std::atomic<int> slots[64];
    int n = slots[dev].load(std::memory_order_acquire);
    if (!n) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel<NS, MODEL, T, ST, VEC, TAPE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_kernel<NS, MODEL, T, ST, VEC, TAPE>, T, smem);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        n = per_sm * sms > 0 ? per_sm * sms : 1;
        slots[dev].store(n, std::memory_order_release);
    }
    *out = n;
    return cudaSuccess;
}

template <int NS, int MODEL, int T, int ST, bool VEC, bool TAPE = false>
cudaError_t launch_step_variant(const StepParams &p, int ty, int nslots, cudaStream_t st)
{
    constexpr size_t smem = step_smem_bytes<NS, T, ST, VEC>();
    const int strips = (p.nx + T - 5) / (T - 4);
    int chunks;
    if (ty > 0) {
        chunks = (p.ny + ty - 1) / ty;
    } else {
        // Automatic march length: as many row chunks per strip as there are
        // resident-block slots per strip (one full wave), chunks of at least
        // 2 rows.  On a lattice too small to fill the GPU, short chunks put
        // more SMs to work although each repeats the 4 + 2 pre-roll rows
        // (measured: 256^2 N=5 at 2 rows 3,188 MLUPS, at 16 rows 1,675).
        // Every chunk, of a narrow last strip too, gets the same rows: a
        // block's time per row hardly depends on how many of its warps hold
        // ring columns.
        chunks = nslots / strips;
        const int maxc = p.ny / 2 > 1 ? p.ny / 2 : 1;
        if (chunks > maxc) chunks = maxc;
        if (chunks < 1) chunks = 1;
        ty = 0;
    }
    const long long blocks = (long long)strips * chunks;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    return launch_pdl(step_kernel<NS, MODEL, T, ST, VEC, TAPE>, dim3((unsigned)blocks), dim3(T), smem, st, p, ty,
                      chunks, strips);
}

// Row windows need nx a multiple of 4 (of 8 with 16-bit storage: rows and
// planes start on 16-byte boundaries), 16-byte aligned arrays and no wall
// across x (a wall bounces single columns back, which a window cannot
// express); they are used whenever they apply, even where their larger
// shared memory leaves fewer blocks resident (N = 7: two blocks per SM
// with windows against three with per-node pulls, and the windows are
// faster).
template <int NS, int MODEL, int T, int ST, bool TAPE = false>
cudaError_t launch_step_nst(const StepParams &p, int ty, cudaStream_t st)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    {
        uintptr_t a = reinterpret_cast<uintptr_t>(p.fin) | reinterpret_cast<uintptr_t>(p.gin);
        if (ST != 0)
            a |= reinterpret_cast<uintptr_t>(p.f0in) | reinterpret_cast<uintptr_t>(p.phi_prev) |
                 reinterpret_cast<uintptr_t>(p.pin);
        const bool vec = !p.wall_x && p.nx % (ST == 0 ? 4 : 8) == 0 && (a & 15) == 0;
        if (vec) {
            int win = 0;
            if ((e = variant_slots<NS, MODEL, T, ST, true, TAPE>(dev, &win)) != cudaSuccess) return e;
            return launch_step_variant<NS, MODEL, T, ST, true, TAPE>(p, ty, win, st);
        }
    }
    int plain = 0;
    if ((e = variant_slots<NS, MODEL, T, ST, false, TAPE>(dev, &plain)) != cudaSuccess) return e;
    return launch_step_variant<NS, MODEL, T, ST, false, TAPE>(p, ty, plain, st);
}

template <int NS, int MODEL, int ST>
cudaError_t launch_step_ns(const StepParams &p, int tx, int ty, cudaStream_t st)
{
    switch (tx) {
    case 64: return launch_step_nst<NS, MODEL, 64, ST>(p, ty, st);
    case 128: return launch_step_nst<NS, MODEL, 128, ST>(p, ty, st);
    case 256: return launch_step_nst<NS, MODEL, 256, ST>(p, ty, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int MODEL, int ST>
cudaError_t launch_step_model(int ns, const StepParams &p, int tx, int ty, cudaStream_t st)
{
    switch (ns) {
    case 1: return launch_step_ns<1, MODEL, ST>(p, tx, ty, st);
    case 2: return launch_step_ns<2, MODEL, ST>(p, tx, ty, st);
    case 3: return launch_step_ns<3, MODEL, ST>(p, tx, ty, st);
    case 4: return launch_step_ns<4, MODEL, ST>(p, tx, ty, st);
    case 5: return launch_step_ns<5, MODEL, ST>(p, tx, ty, st);
    case 6: return launch_step_ns<6, MODEL, ST>(p, tx, ty, st);
    case 7: return launch_step_ns<7, MODEL, ST>(p, tx, ty, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace nlbm
