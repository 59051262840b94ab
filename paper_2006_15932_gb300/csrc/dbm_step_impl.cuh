// dbm_step_impl.cuh -- the fused per-timestep update of the D2V16 DBM.
//
// One thread owns two horizontally adjacent cells (x0, y), (x0+1, y) and
// computes (section "Discrete Boltzmann model" and section "Numerical
// simulation" of arXiv 2006.15932):
//   1. species moments n^s, n^s u^s, E^s = sum f (v.v + eta^2) by ring sums;
//   2. mixture u, T for which the collision conserves momentum and energy
//      (the energy-minus-kinetic subtraction of T in FP64);
//   3. the one-step Arrhenius rate and the post-reaction n^s*, T*;
//   4. the merged equilibrium f^eq,tot = M^-1 [f-hat(n*, u, T*)
//      + f-hat(n, u^dag, T^s) - f-hat(n, u^s, T^s)], so that
//      Omega + R + G = (f^eq,tot - f) / tau (Eqs. CollisionTerm,
//      ReactionTerm, ForceTerm: f^eq is linear in f-hat).  M^-1 is applied
//      in the symmetry-adapted basis of D2V16 (see below);
//   5. the NND flux differences of v_i . grad f along x (faces shared by
//      the two cells) and y;
//   6. the forward-Euler update, stored as a pair to the other buffer with
//      the ghost images the boundary conditions ask for.
// The inputs come from a Tile policy: straight from global memory (k_step)
// or from a shared-memory tile that one TMA bulk copy filled (k_step_tma).
//
// Symmetry-adapted equilibrium.  Each ring of four velocities splits into
// a ring mean A, a vector part (E_x, E_y on the axis rings, G_x, G_y on the
// diagonal rings) and a quadrupole part (B ~ x^2 - y^2 on the axis rings,
// H ~ xy on the diagonal rings):
//   axis ring:     f(+x) = A + Ex + B, f(+y) = A + Ey - B,
//                  f(-x) = A - Ex + B, f(-y) = A - Ey - B;
//   diagonal ring: f(s_x v, s_y v) = A + s_x Gx + s_y Gy + s_x s_y H.
// The 16 moment relations f-hat = M f then decouple into independent
// systems: the ring means from (f1, f4, f5+f7, f14+f16), the two B from
// (f5-f7, f14-f16), the two H from (f6, f15), the x vector parts from
// (f2, f8, f10, f12) and the y vector parts from (f3, f9, f13, f11) with
// the same 4x4 matrix (f-hat indices 1-based as printed): 56 multiply-adds
// instead of 256.  The host inverts these blocks in FP64 to correct
// rounding and checks that they reproduce the full M^-1.
//
// Exact conservation.  The block coefficients are rounded to the working
// precision, so the computed equilibrium would miss its mass, momentum and
// energy by a fixed relative amount (~1e-7 in FP32) in every collision, a
// bias that accumulates over the steps.  After the block solve the
// equilibrium's own mass, energy and momenta are measured and the residuals
// are put back along the block columns that carry them (one projection
// step), which leaves only unbiased rounding.
#pragma once
#include <cuda.h>

#include "dbm_consts.h"
#include "dbm_device.cuh"

namespace dbm {

template <typename real>
struct Vec2;
template <>
struct Vec2<float> {
    using t = float2;
};
template <>
struct Vec2<double> {
    using t = double2;
};

// Pairs of cells straight from global memory (read-only path).
template <typename real>
struct GlobalTile {
    using R2 = typename Vec2<real>::t;
    const real *base;  // plane 0, row y + GY, column x0 + GX
    long long P;       // plane stride
    long long py;      // row stride
    __device__ __forceinline__ R2 ld(int p, int dx, int dy) const
    {
        return __ldg(reinterpret_cast<const R2 *>(base + p * P + dy * py + dx));
    }
};

// Pairs of cells from a shared-memory tile [plane][row][column].
template <typename real>
struct SmemTile {
    using R2 = typename Vec2<real>::t;
    const real *base;  // plane 0, this thread's row and first column
    int P, py;
    __device__ __forceinline__ R2 ld(int p, int dx, int dy) const
    {
        return *reinterpret_cast<const R2 *>(base + p * P + dy * py + dx);
    }
};

// The 16 combinations of f-hat that feed the symmetry blocks, for one cell:
// c[0..3] ring-mean system, c[4..5] B system, c[6..7] H system,
// c[8..11] x-vector system, c[12..15] y-vector system.
template <typename real>
__device__ __forceinline__ void fhat_blocks(real n, real ux, real uy, real th, real dpi, real c[16])
{
    const real xx = ux * ux, yy = uy * uy, u2 = xx + yy;
    const real a2 = (dpi + real(2)) * th + u2;  // (D+I+2) T/m + u.u
    const real a4 = (dpi + real(4)) * th + u2;  // (D+I+4) T/m + u.u
    const real nux = n * ux, nuy = n * uy, nxy = nux * uy, nd = n * (xx - yy);
    c[0] = n;                                  // f1
    c[1] = n * (dpi * th + u2);                // f4
    c[2] = n * (real(2) * th + u2);            // f5 + f7
    c[3] = n * (real(2) * a2 * th + u2 * a4);  // f14 + f16
    c[4] = nd;                                 // f5 - f7
    c[5] = nd * a4;                            // f14 - f16
    c[6] = nxy;                                // f6
    c[7] = nxy * a4;                           // f15
    c[8] = nux;                                // f2
    c[9] = nux * a2;                           // f8
    c[10] = nux * (real(3) * th + xx);         // f10
    c[11] = nux * (th + yy);                   // f12
    c[12] = nuy;                               // f3
    c[13] = nuy * a2;                          // f9
    c[14] = nuy * (real(3) * th + yy);         // f13
    c[15] = nuy * (th + xx);                   // f11
}

// Solve the symmetry blocks (out: ring means A[4], B[2], H[2], X[4], Y[4])
// and project the result onto exact mass, energy and momentum.
template <typename real, int S>
__device__ __forceinline__ void solve_blocks(const StepConsts<real, S> &k, int s, const real c[16],
                                             real o[16])
{
#pragma unroll
    for (int r = 0; r < 4; ++r)
        o[r] = k.eqA[s][r][0] * c[0] + k.eqA[s][r][1] * c[1] + k.eqA[s][r][2] * c[2] +
               k.eqA[s][r][3] * c[3];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        o[4 + r] = k.eqB[s][r][0] * c[4] + k.eqB[s][r][1] * c[5];
        o[6 + r] = k.eqH[s][r][0] * c[6] + k.eqH[s][r][1] * c[7];
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        o[8 + r] = k.eqX[s][r][0] * c[8] + k.eqX[s][r][1] * c[9] + k.eqX[s][r][2] * c[10] +
                   k.eqX[s][r][3] * c[11];
        o[12 + r] = k.eqX[s][r][0] * c[12] + k.eqX[s][r][1] * c[13] + k.eqX[s][r][2] * c[14] +
                    k.eqX[s][r][3] * c[15];
    }
    // residual mass (sum f = 4 sum A), energy (sum q f = 4 sum q_r A_r) and
    // momenta (sum v f = sum w_r v_r X_r) of the computed equilibrium
    const real dm = c[0] - real(4) * ((o[0] + o[1]) + (o[2] + o[3]));
    const real de = c[1] - (k.q4[s][0] * o[0] + k.q4[s][1] * o[1] + k.q4[s][2] * o[2] + k.q4[s][3] * o[3]);
    const real dx = c[8] - (k.wv[s][0] * o[8] + k.wv[s][1] * o[9] + k.wv[s][2] * o[10] + k.wv[s][3] * o[11]);
    const real dy =
        c[12] - (k.wv[s][0] * o[12] + k.wv[s][1] * o[13] + k.wv[s][2] * o[14] + k.wv[s][3] * o[15]);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        o[r] += k.eqA[s][r][0] * dm + k.eqA[s][r][1] * de;
        o[8 + r] += k.eqX[s][r][0] * dx;
        o[12 + r] += k.eqX[s][r][0] * dy;
    }
}

// f^eq of velocity i from the block solution o (see the header comment).
template <typename real>
__device__ __forceinline__ real feq_of(int i, const real o[16])
{
    const int r = i >> 2, k = i & 3;
    const real A = o[r], X = o[8 + r], Y = o[12 + r];
    if ((r & 1) == 0) {  // axis ring: B = o[4 + r/2]
        const real B = o[4 + (r >> 1)];
        return k == 0 ? (A + B) + X : k == 1 ? (A - B) + Y : k == 2 ? (A + B) - X : (A - B) - Y;
    }
    const real H = o[6 + (r >> 1)];  // diagonal ring
    return k == 0 ? (A + H) + (X + Y) : k == 1 ? (A - H) + (Y - X) : k == 2 ? (A + H) - (X + Y)
                                                                          : (A - H) - (Y - X);
}

// NND flux differences along x for the two cells x0, x0+1 from
// f[x0-2 .. x0+3] = l0, l1, c0, c1, r0, r1: (H_{j+1/2} - H_{j-1/2}) / c for
// both cells, with H/c = f_j + mm(.,.)/2 (c > 0) or f_{j+1} - mm(.,.)/2
// (c < 0).  The face between the two cells is computed once.
template <typename real>
__device__ __forceinline__ void nnd_x_pair(int sgn, real l0, real l1, real c0, real c1, real r0, real r1,
                                           real &o0, real &o1)
{
    if (sgn > 0) {
        const real dm32 = l1 - l0, dm12 = c0 - l1, dp12 = c1 - c0, dp32 = r0 - c1;
        const real hm = l1 + real(0.5) * minmod(dm32, dm12);  // face x0 - 1/2
        const real h0 = c0 + real(0.5) * minmod(dm12, dp12);  // face x0 + 1/2
        const real hp = c1 + real(0.5) * minmod(dp12, dp32);  // face x0 + 3/2
        o0 = h0 - hm;
        o1 = hp - h0;
    } else {
        const real dm12 = c0 - l1, dp12 = c1 - c0, dp32 = r0 - c1, dp52 = r1 - r0;
        const real hm = c0 - real(0.5) * minmod(dm12, dp12);  // face x0 - 1/2
        const real h0 = c1 - real(0.5) * minmod(dp12, dp32);  // face x0 + 1/2
        const real hp = r0 - real(0.5) * minmod(dp32, dp52);  // face x0 + 3/2
        o0 = h0 - hm;
        o1 = hp - h0;
    }
}

// Ghost-image bitmask of interior index k on an axis of n cells: bit j set
// when ghost index {-2, -1, n, n+1}[j] takes its value from cell k.
__device__ __forceinline__ unsigned ghost_mask(int k, int n, int bc)
{
    unsigned m = 0;
    if (bc == DBM_BC_PERIODIC) {
        if ((((-2 % n) + n) % n) == k) m |= 1u;
        if ((((-1 % n) + n) % n) == k) m |= 2u;
        if ((n % n) == k) m |= 4u;
        if (((n + 1) % n) == k) m |= 8u;
    } else {
        if (k == 0) m |= 3u;
        if (k == n - 1) m |= 12u;
    }
    return m;
}

__device__ __forceinline__ int ghost_index(int j, int n) { return j < 2 ? j - 2 : n + (j - 2); }

template <typename real>
__device__ __forceinline__ void store_images(real *pl, int x, int y, int nx, int ny, int pitch,
                                             unsigned mx, unsigned my, real v)
{
    for (int j = 0; j < 4; ++j) {
        if (mx & (1u << j)) pl[(long long)(y + GY) * pitch + (ghost_index(j, nx) + GX)] = v;
        if (my & (1u << j)) pl[(long long)(ghost_index(j, ny) + GY) * pitch + (x + GX)] = v;
    }
}

// Mixture temperature T = (W - (u.u) w) / wd of one cell, with the
// cancelling subtraction in FP64 (W = sum lam E, w = sum lam n,
// wd = sum kap n: the weights under which the update conserves momentum and
// energy exactly).
__device__ __forceinline__ float mixture_T(float W, float w, float wd, float ux, float uy, double &Td)
{
    const float u2 = ux * ux + uy * uy;
    const double num = (double)W - (double)u2 * (double)w;
    const float T = (float)num / wd;
    Td = (double)T;
    return T;
}

// Where the pair sits: interior coordinates, whether the second cell
// exists, and the ghost images its values must also be written to.
struct Site {
    int x0, y;
    bool two, images;
    unsigned mx0, mx1, my;
    long long cell;  // element offset of (x0, y) in a plane
};

// Output of the FP32 state: f^{n+1} as a pair, plus ghost images.
template <typename real>
struct StateOut {
    using R2 = typename Vec2<real>::t;
    real *f;  // plane 0 of the output buffer
    long long P;
    int nx, ny, pitch;
    __device__ __forceinline__ void put(const Site &w, int p, real g0, real g1, real, real) const
    {
        real *pl = f + (long long)p * P;
        if (w.two) {
            R2 v;
            v.x = g0;
            v.y = g1;
            __stcs(reinterpret_cast<R2 *>(pl + w.cell), v);  // streamed: not re-read this step
        } else {
            __stcs(pl + w.cell, g0);
        }
        if (w.images) {
            store_images(pl, w.x0, w.y, nx, ny, pitch, w.mx0, w.my, g0);
            if (w.two) store_images(pl, w.x0 + 1, w.y, nx, ny, pitch, w.mx1, w.my, g1);
        }
    }
    __device__ __forceinline__ void put_n(const Site &, int, real, real) const {}
    __device__ __forceinline__ void put_mix(const Site &, real, real, real, real, real, real) const {}
};

// The whole update of the cell pair (x0, y), (x0+1, y).
template <typename real, int S, class Tile, class Out>
__device__ __forceinline__ void step_pair(const StepConsts<real, S> &c, const Tile &t, int x0, int y,
                                          const Out &out, unsigned *__restrict__ flag)
{
    using R2 = typename Vec2<real>::t;
    const bool two = x0 + 1 < c.nx;
    const long long P = c.plane;
    const long long cell = (long long)(y + GY) * c.pitch + (x0 + GX);

    // 1. species moments of both cells, by ring sums
    real n0[S], n1[S], cap0 = 0, cap1 = 0;
    real nf0 = 0, nf1 = 0, no0 = 0, no1 = 0;  // fuel and oxidiser densities
    real w0 = 0, w1 = 0, wx0 = 0, wx1 = 0, wy0 = 0, wy1 = 0, we0 = 0, we1 = 0, wd0 = 0, wd1 = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        real sn0 = 0, sn1 = 0, sx0 = 0, sx1 = 0, sy0 = 0, sy1 = 0, se0 = 0, se1 = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            real rs0 = 0, rs1 = 0, rx0 = 0, rx1 = 0, ry0 = 0, ry1 = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = 4 * r + k;
                const R2 f = t.ld(s * Q + i, 0, 0);
                rs0 += f.x;
                rs1 += f.y;
                if (dir_x(i) > 0) { rx0 += f.x; rx1 += f.y; }
                if (dir_x(i) < 0) { rx0 -= f.x; rx1 -= f.y; }
                if (dir_y(i) > 0) { ry0 += f.x; ry1 += f.y; }
                if (dir_y(i) < 0) { ry0 -= f.x; ry1 -= f.y; }
            }
            sn0 += rs0;
            sn1 += rs1;
            sx0 += c.vr[s][r] * rx0;
            sx1 += c.vr[s][r] * rx1;
            sy0 += c.vr[s][r] * ry0;
            sy1 += c.vr[s][r] * ry1;
            se0 += c.qr[s][r] * rs0;
            se1 += c.qr[s][r] * rs1;
        }
        n0[s] = sn0;
        n1[s] = sn1;
        if (s == c.fuel) { nf0 = sn0; nf1 = sn1; }  // no runtime-indexed register array
        if (s == c.oxid) { no0 = sn0; no1 = sn1; }
        const real lh = c.lam_h[s], ll = c.lam_l[s], kh = c.kap_h[s], kl = c.kap_l[s];
        w0 += lh * sn0 + ll * sn0;
        w1 += lh * sn1 + ll * sn1;
        wx0 += lh * sx0 + ll * sx0;
        wx1 += lh * sx1 + ll * sx1;
        wy0 += lh * sy0 + ll * sy0;
        wy1 += lh * sy1 + ll * sy1;
        we0 += lh * se0 + ll * se0;
        we1 += lh * se1 + ll * se1;
        wd0 += kh * sn0 + kl * sn0;
        wd1 += kh * sn1 + kl * sn1;
        cap0 += c.dpi[s] * sn0;
        cap1 += c.dpi[s] * sn1;
    }

    // 2. mixture velocity and temperature
    const real ux0 = wx0 / w0, uy0 = wy0 / w0, ux1 = wx1 / w1, uy1 = wy1 / w1;
    double T0d, T1d;
    const real T0 = mixture_T(we0, w0, wd0, ux0, uy0, T0d);
    const real T1 = mixture_T(we1, w1, wd1, ux1, uy1, T1d);

    unsigned bad = 0;
    real a0 = 0, a1 = 0;  // sum_s |n^s| of both cells
#pragma unroll
    for (int s = 0; s < S; ++s) {
        a0 += fabs(n0[s]);
        a1 += fabs(n1[s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (!(n0[s] >= real(-1e-6) * a0) || !(n1[s] >= real(-1e-6) * a1)) bad |= DBM_HEALTH_DENSITY;
    if (!(a0 > real(0)) || !(a1 > real(0))) bad |= DBM_HEALTH_DENSITY;
    if (!(T0 > real(0)) || !(T1 > real(0))) bad |= DBM_HEALTH_TEMPERATURE;
    if (!isfinite(T0 + T1 + ux0 + uy0 + ux1 + uy1)) bad |= DBM_HEALTH_NONFINITE;

    // 3. reaction: omega_ov and T' (state after a time tau^s), FP64
    double om0 = 0.0, om1 = 0.0, dT0 = 0.0, dT1 = 0.0;
    if (c.has_reaction) {
        om0 = c.k_ov * (double)nf0 * (double)no0 * exp(-c.Ea_over_R / T0d);
        om1 = c.k_ov * (double)nf1 * (double)no1 * exp(-c.Ea_over_R / T1d);
        dT0 = (c.Qheat - 0.5 * T0d * c.src) * om0 / (0.5 * (double)cap0);
        dT1 = (c.Qheat - 0.5 * T1d * c.src) * om1 / (0.5 * (double)cap1);
    }

    Site w;
    w.x0 = x0;
    w.y = y;
    w.two = two;
    w.mx0 = ghost_mask(x0, c.nx, c.bc_x);
    w.mx1 = two ? ghost_mask(x0 + 1, c.nx, c.bc_x) : 0u;
    w.my = ghost_mask(y, c.ny, c.bc_y);
    w.images = (w.mx0 | w.mx1 | w.my) != 0u;
    w.cell = cell;
    out.put_mix(w, ux0, uy0, T0, ux1, uy1, T1);

#pragma unroll 1
    for (int s = 0; s < S; ++s) {
        // centres of this species, both cells
        real f0[Q], f1[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R2 v = t.ld(s * Q + i, 0, 0);
            f0[i] = v.x;
            f1[i] = v.y;
        }
        // 4. merged equilibrium moments of both cells
        real cb0[16], cb1[16];
        real ns0 = 0, ns1 = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            ns0 += f0[i];
            ns1 += f1[i];
        }
        out.put_n(w, s, ns0, ns1);
        {
            real nr0 = ns0, nr1 = ns1;
            real Ts0 = T0, Ts1 = T1;
            if (c.has_reaction) {
                const double e0 = (double)ns0 + c.tau_a[s] * om0, e1 = (double)ns1 + c.tau_a[s] * om1;
                if (e0 < -1e-6 * (double)a0 || e1 < -1e-6 * (double)a1) bad |= DBM_HEALTH_NSTAR;
                nr0 = (real)e0;
                nr1 = (real)e1;
                Ts0 = (real)(T0d + c.tau_d[s] * dT0);
                Ts1 = (real)(T1d + c.tau_d[s] * dT1);
            }
            fhat_blocks<real>(nr0, ux0, uy0, Ts0 * c.inv_m[s], c.dpi[s], cb0);
            fhat_blocks<real>(nr1, ux1, uy1, Ts1 * c.inv_m[s], c.dpi[s], cb1);
            if (c.has_force) {
                // species velocity and temperature from this species' moments
                real jx0 = 0, jx1 = 0, jy0 = 0, jy1 = 0, e0 = 0, e1 = 0;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const real vx = dir_x(i) * c.vr[s][i >> 2], vy = dir_y(i) * c.vr[s][i >> 2];
                    jx0 += vx * f0[i];
                    jx1 += vx * f1[i];
                    jy0 += vy * f0[i];
                    jy1 += vy * f1[i];
                    e0 += c.qr[s][i >> 2] * f0[i];
                    e1 += c.qr[s][i >> 2] * f1[i];
                }
                real g[16], h[16];
                if (ns0 != real(0)) {  // an absent species feels no force
                    const real usx = jx0 / ns0, usy = jy0 / ns0;
                    const real th = (e0 / ns0 - (usx * usx + usy * usy)) / c.dpi[s];
                    fhat_blocks<real>(ns0, usx + c.accel_x * c.tau[s], usy + c.accel_y * c.tau[s], th,
                                      c.dpi[s], g);
                    fhat_blocks<real>(ns0, usx, usy, th, c.dpi[s], h);
#pragma unroll
                    for (int k = 0; k < 16; ++k) cb0[k] += g[k] - h[k];
                }
                if (ns1 != real(0)) {
                    const real usx = jx1 / ns1, usy = jy1 / ns1;
                    const real th = (e1 / ns1 - (usx * usx + usy * usy)) / c.dpi[s];
                    fhat_blocks<real>(ns1, usx + c.accel_x * c.tau[s], usy + c.accel_y * c.tau[s], th,
                                      c.dpi[s], g);
                    fhat_blocks<real>(ns1, usx, usy, th, c.dpi[s], h);
#pragma unroll
                    for (int k = 0; k < 16; ++k) cb1[k] += g[k] - h[k];
                }
            }
        }
        real o0[16], o1[16];
        solve_blocks<real, S>(c, s, cb0, o0);
        solve_blocks<real, S>(c, s, cb1, o1);
        const real dtt = c.dt_tau[s];

#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int p = s * Q + i;
            const int r = i >> 2;
            real d0 = 0, d1 = 0;  // dt * v . grad f of both cells
            // 5. NND advection
            if (dir_x(i) != 0) {
                const R2 L = t.ld(p, -2, 0), Rr = t.ld(p, 2, 0);
                real e0, e1;
                nnd_x_pair<real>(dir_x(i), L.x, L.y, f0[i], f1[i], Rr.x, Rr.y, e0, e1);
                const real cx = dir_x(i) * c.cdx[s][r];
                d0 += cx * e0;
                d1 += cx * e1;
            }
            if (dir_y(i) > 0) {
                const R2 m2 = t.ld(p, 0, -2), m1 = t.ld(p, 0, -1), p1 = t.ld(p, 0, 1);
                const real cy = c.cdy[s][r];
                d0 += cy * nnd_diff_pos(m2.x, m1.x, f0[i], p1.x);
                d1 += cy * nnd_diff_pos(m2.y, m1.y, f1[i], p1.y);
            } else if (dir_y(i) < 0) {
                const R2 m1 = t.ld(p, 0, -1), p1 = t.ld(p, 0, 1), p2 = t.ld(p, 0, 2);
                const real cy = c.cdy[s][r];
                d0 -= cy * nnd_diff_neg(m1.x, f0[i], p1.x, p2.x);
                d1 -= cy * nnd_diff_neg(m1.y, f1[i], p1.y, p2.y);
            }
            // 6. forward Euler: f + dt/tau (f^eq,tot - f) - dt v . grad f
            const real e0 = feq_of<real>(i, o0), e1 = feq_of<real>(i, o1);
            const real g0 = f0[i] + dtt * (e0 - f0[i]) - d0;
            const real g1 = f1[i] + dtt * (e1 - f1[i]) - d1;
            out.put(w, p, g0, g1, e0, e1);
        }
    }
    if (bad) raise_flag(flag, bad);
}

// Generic kernel: inputs from global memory through the read-only path.
template <typename real, int S>
__global__ void __launch_bounds__(256, 2)
    k_step(const __grid_constant__ StepConsts<real, S> c, const real *__restrict__ fin,
           real *__restrict__ fout, unsigned *__restrict__ flag)
{
    const int x0 = 2 * (blockIdx.x * blockDim.x + threadIdx.x);
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x0 >= c.nx || y >= c.ny) return;
    GlobalTile<real> t;
    t.base = fin + (long long)(y + GY) * c.pitch + (x0 + GX);
    t.P = c.plane;
    t.py = c.pitch;
    StateOut<real> o{fout, c.plane, c.nx, c.ny, c.pitch};
    step_pair<real, S>(c, t, x0, y, o, flag);
}

// ---------------------------------------------------------------------------
// TMA-staged kernel: one CTA steps a TX x TY tile of cells.  One thread
// issues a single cp.async.bulk.tensor copy of the tile plus its radius-2
// halo (all 16 S planes, columns x0-4 .. x0+TX+3 so that the copy starts on
// a 16-byte boundary) into shared memory, completing on an mbarrier; every
// thread then reads its stencil from shared memory.
// ---------------------------------------------------------------------------

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}

// Wait on phase `parity` of an mbarrier with an iteration limit; returns
// false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long long limit)
{
    for (long long it = 0; it < limit; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

constexpr long long TMA_WAIT_LIMIT = 1LL << 22;  // try_wait polls (each may suspend ~us)

template <typename real, int S, int TX, int TY>
__global__ void __launch_bounds__((TX / 2) * TY, 2)
    k_step_tma(const __grid_constant__ StepConsts<real, S> c, const __grid_constant__ CUtensorMap tmap,
               real *__restrict__ fout, unsigned *__restrict__ flag)
{
    constexpr int BX = TX + 8, BY = TY + 4, NP = S * Q;
    constexpr unsigned BYTES = (unsigned)(BX * BY * NP * sizeof(real));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    real *tile = reinterpret_cast<real *>(smem_raw);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool leader = tx == 0 && ty == 0;
    const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY;
    const unsigned b = smem_u32(&bar);
    if (leader) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (leader) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(BYTES) : "memory");
        // box origin: column (bx0 + GX) - 4 = bx0, row (by0 + GY) - 2 = by0, plane 0
        asm volatile(
            "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
            " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(tile)),
            "l"(reinterpret_cast<unsigned long long>(&tmap)), "r"(bx0), "r"(by0), "r"(0), "r"(b)
            : "memory");
    }
    if (!mbar_wait(b, 0, TMA_WAIT_LIMIT)) {
        // the copy did not land: report, give it one more bounded wait so
        // that no copy is left writing into this block's shared memory, leave
        if (leader) raise_flag(flag, DBM_HEALTH_TIMEOUT);
        mbar_wait(b, 0, TMA_WAIT_LIMIT);
        return;
    }
    const int x0 = bx0 + 2 * tx, y = by0 + ty;
    if (x0 >= c.nx || y >= c.ny) return;
    SmemTile<real> t;
    t.base = tile + (ty + 2) * BX + (2 * tx + 4);
    t.P = BY * BX;
    t.py = BX;
    StateOut<real> o{fout, c.plane, c.nx, c.ny, c.pitch};
    step_pair<real, S>(c, t, x0, y, o, flag);
}

template <typename real, int S>
int launch_step_t(dbm_handle *h, const void *fin, void *fout, cudaStream_t st)
{
    StepConsts<real, S> c;
    fill_step_consts<real, S>(h, c);
    dim3 block(32, 8);
    dim3 grid((h->p.nx + 63) / 64, (h->p.ny + 7) / 8);
    k_step<real, S><<<grid, block, 0, st>>>(c, (const real *)fin, (real *)fout, (unsigned *)h->scratch);
    return set_cuda_error(h, cudaGetLastError(), "step kernel launch");
}

template <typename real, int S, int TX, int TY>
int launch_step_tma_t(dbm_handle *h, const CUtensorMap *tmap, void *fout, cudaStream_t st)
{
    constexpr size_t smem = (size_t)(TX + 8) * (TY + 4) * S * Q * sizeof(real);
    static bool attr_set = false;  // per instantiation, set once per process
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_step_tma<real, S, TX, TY>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return set_cuda_error(h, e, "TMA step kernel shared-memory attribute");
        attr_set = true;
    }
    StepConsts<real, S> c;
    fill_step_consts<real, S>(h, c);
    dim3 block(TX / 2, TY);
    dim3 grid((h->p.nx + TX - 1) / TX, (h->p.ny + TY - 1) / TY);
    k_step_tma<real, S, TX, TY><<<grid, block, smem, st>>>(c, *tmap, (real *)fout, (unsigned *)h->scratch);
    return set_cuda_error(h, cudaGetLastError(), "TMA step kernel launch");
}

}  // namespace dbm
