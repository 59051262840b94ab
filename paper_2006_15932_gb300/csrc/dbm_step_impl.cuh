// dbm_step_impl.cuh -- the fused per-timestep update of the D2V16 DBM (FP32).
//
// One thread owns one cell, or two adjacent cells of a row (packed FP32x2
// arithmetic, see below), and computes (section "Discrete Boltzmann model"
// and section "Numerical simulation" of arXiv 2006.15932):
//   1. species moments n^s, n^s u^s, E^s = sum f (v.v + eta^2) by ring sums;
//   2. mixture u, T for which the collision conserves momentum and energy
//      (the energy-minus-kinetic subtraction of T in float-float);
//   3. the one-step Arrhenius rate and the post-reaction n^s*, T*;
//   4. the merged equilibrium f^eq,tot = M^-1 [f-hat(n*, u, T*)
//      + f-hat(n, u^dag, T^s) - f-hat(n, u^s, T^s)], so that
//      Omega + R + G = (f^eq,tot - f) / tau (Eqs. CollisionTerm,
//      ReactionTerm, ForceTerm: f^eq is linear in f-hat).  M^-1 is applied
//      in the symmetry-adapted basis of D2V16 (see below);
//   5. the NND flux differences of v_i . grad f along x and y;
//   6. the forward-Euler update, stored to the other buffer, then the ghost
//      images the boundary conditions ask for (edge cells only).
// The inputs come from a Tile policy: straight from global memory (k_step)
// or from a shared-memory tile that one TMA bulk copy filled (k_step_tma,
// one cell or a pair of cells per thread);
// the outputs go through an Out policy (FP32 state, or the BF16-deviation
// state of dbm_bf16.cuh).
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

#include <type_traits>

#include "dbm_consts.h"
#include "dbm_device.cuh"

namespace dbm {

// ---------------------------------------------------------------------------
// Arithmetic of one cell (float) or of two adjacent cells at once (float2:
// the packed FP32x2 add/sub/mul/fma instructions of sm_100 and later, one
// instruction for both cells, each half rounded like the scalar operation).
// Every operation of the step is an explicitly rounded one, so the compiler
// does not regroup it.  The code also never passes a product to an add or a
// subtract (a multiply-add is written as an FMA, and a difference of two
// products as an FMA chain): the backend may fuse a packed multiply into a
// following packed add despite the .rn modifier (measured: x*y - z*w comes
// out as fma(x, y, -(z*w))), never a scalar one.  With that rule the
// generic, TMA-staged, two-cell and batched kernels produce the same bits
// for a cell.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float vmm(float a, float b) { return minmod(a, b); }

// The packed operations are written as PTX with an explicit .rn rounding,
// which keeps the front end from contracting them; the backend can still
// fuse a packed multiply into a following packed add (see above), which the
// step avoids by never passing a product to an add or a subtract.
__device__ __forceinline__ unsigned long long vpk(float2 a)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
    return r;
}
__device__ __forceinline__ float2 vupk(unsigned long long r)
{
    float2 o;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(o.x), "=f"(o.y) : "l"(r));
    return o;
}
__device__ __forceinline__ float2 vadd(float2 a, float2 b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(vpk(a)), "l"(vpk(b)));
    return vupk(r);
}
__device__ __forceinline__ float2 vsub(float2 a, float2 b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(vpk(a)), "l"(vpk(b)));
    return vupk(r);
}
__device__ __forceinline__ float2 vmul(float2 a, float2 b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(vpk(a)), "l"(vpk(b)));
    return vupk(r);
}
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(vpk(a)), "l"(vpk(b)), "l"(vpk(c)));
    return vupk(r);
}
__device__ __forceinline__ float2 vmm(float2 a, float2 b) { return make_float2(minmod(a.x, b.x), minmod(a.y, b.y)); }

// Per-cell access to a value: n cells, broadcast, lane j.
template <class V>
struct Lanes;
template <>
struct Lanes<float> {
    static constexpr int n = 1;
    __device__ static float bc(float a) { return a; }
    __device__ static float get(float v, int) { return v; }
    __device__ static void set(float &v, int, float a) { v = a; }
};
template <>
struct Lanes<float2> {
    static constexpr int n = 2;
    __device__ static float2 bc(float a) { return make_float2(a, a); }
    __device__ static float get(float2 v, int j) { return j ? v.y : v.x; }
    __device__ static void set(float2 &v, int j, float a)
    {
        if (j)
            v.y = a;
        else
            v.x = a;
    }
};
template <class V>
__device__ __forceinline__ V bc(float a)
{
    return Lanes<V>::bc(a);
}

// Stencil values of one cell straight from global memory (read-only path).
struct GlobalTile {
    using V = float;
    const float *base;  // plane 0, row y + GY, column x + GX
    long long P;        // plane stride
    long long py;       // row stride
    const float *lo;    // checked builds: the buffer and its extent
    long long n;
    unsigned *flag;
    __device__ __forceinline__ float ld(int p, int dx, int dy) const
    {
        const float *q = base + p * P + dy * py + dx;
        if (!in_bounds(q - lo, n, flag)) return 0.0f;
        return __ldg(q);
    }
};

// Stencil values of one cell from a shared-memory tile [plane][row][column].
struct SmemTile {
    using V = float;
    const float *base;  // plane 0, this thread's row and column
    int P, py;
    const float *lo;  // checked builds: the tile and its extent (floats)
    int n;
    unsigned *flag;
    __device__ __forceinline__ float ld(int p, int dx, int dy) const
    {
        const float *q = base + p * P + dy * py + dx;
        if (!in_bounds(q - lo, n, flag)) return 0.0f;
        return *q;
    }
};

// Stencil values of the cells (x, y) and (x + 1, y) from a shared-memory
// tile: ld(p, dx, dy) = (f(x + dx, y + dy), f(x + 1 + dx, y + dy)) of plane
// p.  x is even in the tile, so an even dx is one aligned 64-bit load.
struct SmemTile2 {
    using V = float2;
    const float *base;  // plane 0, this thread's row, its first column
    int P, py;
    const float *lo;  // checked builds: the tile and its extent (floats)
    int n;
    unsigned *flag;
    __device__ __forceinline__ float2 ld(int p, int dx, int dy) const
    {
        const float *q = base + p * P + dy * py + dx;
        if (!in_bounds(q - lo, n - 1, flag)) return make_float2(0.0f, 0.0f);
        if (dx & 1) return make_float2(q[0], q[1]);
        return *reinterpret_cast<const float2 *>(q);
    }
};

// A tile that passes through shared memory one species at a time
// (StagedTile2, the species-staged step) declares kStaged; step_cell then
// brackets the reads of each species with acquire / release and reads
// through view(k, s), the buffer of use k.  Other tiles hold every species
// at once and are read as they are.
template <class T, class = void>
struct is_staged : std::false_type {
};
template <class T>
struct is_staged<T, std::void_t<decltype(T::kStaged)>> : std::true_type {
};

template <class Tile>
__device__ __forceinline__ decltype(auto) stage_view(const Tile &t, int k, int s)
{
    if constexpr (is_staged<Tile>::value)
        return t.view(k, s);
    else
        return (t);
}

// The 16 combinations of f-hat that feed the symmetry blocks, for one cell:
// c[0..3] ring-mean system, c[4..5] B system, c[6..7] H system,
// c[8..11] x-vector system, c[12..15] y-vector system.  Each is returned as
// two factors, c[k] = L[k] R[k], so that a caller can fold the last product
// into a multiply-add.
template <class V>
__device__ __forceinline__ void fhat_factors(V n, V ux, V uy, V th, float dpi, V L[16], V R[16])
{
    const V xx = vmul(ux, ux), yy = vmul(uy, uy), u2 = vfma(ux, ux, yy);
    const V a2 = vfma(bc<V>(dpi + 2.0f), th, u2);  // (D+I+2) T/m + u.u
    const V a4 = vfma(bc<V>(dpi + 4.0f), th, u2);  // (D+I+4) T/m + u.u
    const V nux = vmul(n, ux), nuy = vmul(n, uy), nxy = vmul(nux, uy);
    const V q = vfma(vmul(bc<V>(-1.0f), uy), uy, xx);  // ux^2 - uy^2
    L[0] = n, R[0] = bc<V>(1.0f);                         // f1
    L[1] = n, R[1] = vfma(bc<V>(dpi), th, u2);            // f4
    L[2] = n, R[2] = vfma(bc<V>(2.0f), th, u2);           // f5 + f7
    L[3] = n, R[3] = vfma(vadd(a2, a2), th, vmul(u2, a4)); // f14 + f16
    L[4] = n, R[4] = q;                                   // f5 - f7
    L[5] = vmul(n, q), R[5] = a4;                         // f14 - f16
    L[6] = nux, R[6] = uy;                                // f6
    L[7] = nxy, R[7] = a4;                                // f15
    L[8] = n, R[8] = ux;                                  // f2
    L[9] = nux, R[9] = a2;                                // f8
    L[10] = nux, R[10] = vfma(bc<V>(3.0f), th, xx);       // f10
    L[11] = nux, R[11] = vfma(uy, uy, th);                // f12
    L[12] = n, R[12] = uy;                                // f3
    L[13] = nuy, R[13] = a2;                              // f9
    L[14] = nuy, R[14] = vfma(bc<V>(3.0f), th, yy);       // f13
    L[15] = nuy, R[15] = vfma(ux, ux, th);                // f11
}

template <class V>
__device__ __forceinline__ void fhat_blocks(V n, V ux, V uy, V th, float dpi, V c[16])
{
    V L[16], R[16];
    fhat_factors<V>(n, ux, uy, th, dpi, L, R);
#pragma unroll
    for (int k = 0; k < 16; ++k) c[k] = k == 0 ? n : vmul(L[k], R[k]);
}

// k0 c0 + k1 c1 + k2 c2 + k3 c3, accumulated left to right.
template <class V>
__device__ __forceinline__ V dot4(const float k[4], V c0, V c1, V c2, V c3)
{
    return vfma(bc<V>(k[3]), c3, vfma(bc<V>(k[2]), c2, vfma(bc<V>(k[1]), c1, vmul(bc<V>(k[0]), c0))));
}

// t - (k0 c0 + k1 c1 + k2 c2 + k3 c3) as a chain of multiply-adds from t.
template <class V>
__device__ __forceinline__ V resid4(const float k[4], V c0, V c1, V c2, V c3, V t)
{
    return vfma(bc<V>(-k[3]), c3, vfma(bc<V>(-k[2]), c2, vfma(bc<V>(-k[1]), c1, vfma(bc<V>(-k[0]), c0, t))));
}

__device__ __forceinline__ float sr_uniform(unsigned h, int k);
__device__ __forceinline__ float ff_prod(float a, float b, float &e);
__device__ __forceinline__ float ff_sum(float a, float b, float &e);
__device__ __forceinline__ float sr_ff(float hi, float lo, float u);

// Solve the symmetry blocks (out: ring means A[4], B[2], H[2], X[4], Y[4])
// and project the result onto exact mass, energy and momentum.  With SR the
// projected ring means, which carry the equilibrium's mass and energy, are
// formed exactly (float-float) and rounded stochastically (random numbers
// kb..kb+3 of the cell hashes h): a round-to-nearest result misses the mass
// target by a rounding error that follows the slowly varying macroscopic
// state, and so adds up over the steps instead of averaging out.
template <class V, class K, bool SR = false>
__device__ __forceinline__ void solve_blocks(const K &k, int s, const V c[16], V o[16], const unsigned *h = nullptr,
                                             int kb = 0)
{
#pragma unroll
    for (int r = 0; r < 4; ++r) o[r] = dot4<V>(k.eqA[s][r], c[0], c[1], c[2], c[3]);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        o[4 + r] = vfma(bc<V>(k.eqB[s][r][1]), c[5], vmul(bc<V>(k.eqB[s][r][0]), c[4]));
        o[6 + r] = vfma(bc<V>(k.eqH[s][r][1]), c[7], vmul(bc<V>(k.eqH[s][r][0]), c[6]));
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        o[8 + r] = dot4<V>(k.eqX[s][r], c[8], c[9], c[10], c[11]);
        o[12 + r] = dot4<V>(k.eqX[s][r], c[12], c[13], c[14], c[15]);
    }
    // residual mass (sum f = 4 sum A), energy (sum q f = 4 sum q_r A_r) and
    // momenta (sum v f = sum w_r v_r X_r) of the computed equilibrium
    const V dm = vfma(bc<V>(-4.0f), vadd(vadd(o[0], o[1]), vadd(o[2], o[3])), c[0]);
    const V de = resid4<V>(k.q4[s], o[0], o[1], o[2], o[3], c[1]);
    const V dx = resid4<V>(k.wv[s], o[8], o[9], o[10], o[11], c[8]);
    const V dy = resid4<V>(k.wv[s], o[12], o[13], o[14], o[15], c[12]);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if constexpr (SR) {
            using L = Lanes<V>;
#pragma unroll
            for (int j = 0; j < L::n; ++j) {
                // o + eqA0 dm + eqA1 de = s + (e3 + e4) + (e1 + e2) exactly
                float e1, e2, e3, e4;
                const float p1 = ff_prod(k.eqA[s][r][0], L::get(dm, j), e1);
                const float p2 = ff_prod(k.eqA[s][r][1], L::get(de, j), e2);
                const float s1 = ff_sum(ff_sum(L::get(o[r], j), p1, e3), p2, e4);
                L::set(o[r], j, sr_ff(s1, __fadd_rn(__fadd_rn(e3, e4), __fadd_rn(e1, e2)), sr_uniform(h[j], kb + r)));
            }
        } else {
            o[r] = vfma(bc<V>(k.eqA[s][r][1]), de, vfma(bc<V>(k.eqA[s][r][0]), dm, o[r]));
        }
        o[8 + r] = vfma(bc<V>(k.eqX[s][r][0]), dx, o[8 + r]);
        o[12 + r] = vfma(bc<V>(k.eqX[s][r][0]), dy, o[12 + r]);
    }
}

// f^eq of velocity i from the block solution o (see the header comment).
template <class V>
__device__ __forceinline__ V feq_of(int i, const V o[16])
{
    const int r = i >> 2, k = i & 3;
    const V A = o[r], X = o[8 + r], Y = o[12 + r];
    if ((r & 1) == 0) {  // axis ring: B = o[4 + r/2]
        const V B = o[4 + (r >> 1)];
        return k == 0 ? vadd(vadd(A, B), X) : k == 1 ? vadd(vsub(A, B), Y) : k == 2 ? vsub(vadd(A, B), X)
                                                                                   : vsub(vsub(A, B), Y);
    }
    const V H = o[6 + (r >> 1)];  // diagonal ring
    return k == 0   ? vadd(vadd(A, H), vadd(X, Y))
           : k == 1 ? vadd(vsub(A, H), vsub(Y, X))
           : k == 2 ? vsub(vadd(A, H), vadd(X, Y))
                    : vsub(vsub(A, H), vsub(Y, X));
}

// NND flux difference along one axis for a velocity component of sign
// `sgn` (+1 or -1): (H_{j+1/2} - H_{j-1/2}) / c, from f_{j-2..j+2}.
//   c > 0: H_{j+1/2} = c [f_j + mm(f_j - f_{j-1}, f_{j+1} - f_j)/2]
//   c < 0: H_{j+1/2} = c [f_{j+1} - mm(f_{j+1} - f_j, f_{j+2} - f_{j+1})/2]
template <class V>
__device__ __forceinline__ V nnd_diff_pos(V fm2, V fm1, V f0, V fp1)
{
    const V d0 = vsub(fm1, fm2), d1 = vsub(f0, fm1), d2 = vsub(fp1, f0);
    return vfma(bc<V>(0.5f), vsub(vmm(d1, d2), vmm(d0, d1)), d1);
}
template <class V>
__device__ __forceinline__ V nnd_diff_neg(V fm1, V f0, V fp1, V fp2)
{
    const V d1 = vsub(f0, fm1), d2 = vsub(fp1, f0), d3 = vsub(fp2, fp1);
    return vfma(bc<V>(-0.5f), vsub(vmm(d2, d3), vmm(d1, d2)), d2);
}

// The same x-direction flux differences for the pair of cells (x, x + 1),
// from the two aligned 64-bit loads a = (f_{x-2}, f_{x-1}) and
// b = (f_{x+2}, f_{x+3}) and the pair's own values c = (f_x, f_{x+1}): the
// odd shifts are assembled from registers, and the limiter of the face
// between the two cells is evaluated once (the second cell's left-face
// minmod is the first cell's right-face minmod, with the same operands), so
// the result is bitwise that of nnd_diff_pos / nnd_diff_neg.
__device__ __forceinline__ float2 nnd_diff_pos_pair(float2 a, float2 c, float2 b)
{
    const float2 fm1 = make_float2(a.y, c.x), fp1 = make_float2(c.y, b.x);
    const float2 d0 = vsub(fm1, a), d1 = vsub(c, fm1), d2 = vsub(fp1, c);
    const float2 m12 = vmm(d1, d2);
    const float2 m01 = make_float2(minmod(d0.x, d1.x), m12.x);
    return vfma(bc<float2>(0.5f), vsub(m12, m01), d1);
}
__device__ __forceinline__ float2 nnd_diff_neg_pair(float2 a, float2 c, float2 b)
{
    const float2 fm1 = make_float2(a.y, c.x), fp1 = make_float2(c.y, b.x);
    const float2 d1 = vsub(c, fm1), d2 = vsub(fp1, c), d3 = vsub(b, fp1);
    const float2 m23 = vmm(d2, d3);
    const float2 m12 = make_float2(minmod(d1.x, d2.x), m23.x);
    return vfma(bc<float2>(-0.5f), vsub(m23, m12), d2);
}

// Ghost-image bitmask of interior index k on an axis of n cells: bit j set
// when ghost index {-2, -1, n, n+1}[j] takes its value from cell k.
__device__ __forceinline__ unsigned ghost_mask(int k, int n, int bc)
{
    unsigned m = 0;
    if (bc == DBM_BC_PERIODIC) {
        // sources (-2, -1, n, n+1) mod n, without a division: n-2, n-1, 0, 1
        // for n >= 2 and 0 for every ghost when n == 1
        const bool one = n == 1;
        if (k == (one ? 0 : n - 2)) m |= 1u;
        if (k == n - 1) m |= 2u;
        if (k == 0) m |= 4u;
        if (k == (one ? 0 : 1)) m |= 8u;
    } else {
        if (k == 0) m |= 3u;
        if (k == n - 1) m |= 12u;
    }
    return m;
}

__device__ __forceinline__ int ghost_index(int j, int n) { return j < 2 ? j - 2 : n + (j - 2); }

template <typename T>
__device__ __forceinline__ void store_images(T *pl, int x, int y, int nx, int ny, int pitch, unsigned mx,
                                             unsigned my, T v)
{
    for (int j = 0; j < 4; ++j) {
        if (mx & (1u << j)) pl[(long long)(y + GY) * pitch + (ghost_index(j, nx) + GX)] = v;
        if (my & (1u << j)) pl[(long long)(ghost_index(j, ny) + GY) * pitch + (x + GX)] = v;
    }
}

// Mixture temperature T = (W - (u.u) w) / wd of one cell (W = sum lam E,
// w = sum lam n, wd = sum kap n: the weights under which the update
// conserves momentum and energy exactly).  The cancelling subtraction is
// carried in float-float: the product (u.u) w = p + pe exactly (FMA) and
// W - p = s + se exactly (Knuth's two-sum), so the numerator is as accurate
// as an FP64 evaluation while every operation stays on the FP32 pipes.  The
// _rn intrinsics keep the compiler from contracting these steps.
__device__ __forceinline__ void mixture_T_num(float W, float w, float ux, float uy, float &hi, float &lo)
{
    const float u2 = __fmaf_rn(ux, ux, __fmul_rn(uy, uy));
    const float p = __fmul_rn(u2, w);
    const float pe = fmaf(u2, w, -p);
    const float s = __fsub_rn(W, p);
    const float bb = __fsub_rn(s, W);
    const float se = __fadd_rn(__fsub_rn(W, __fsub_rn(s, bb)), __fsub_rn(-p, bb));
    hi = s;
    lo = __fsub_rn(se, pe);
}
// The same numerator with u.u itself carried exactly (error-free products
// and sum): the stochastic mode's energy targets use the exact u.u, and the
// temperature has to see the same value, else each cell's collision moves
// energy by (u.u - RN(u.u)) w, whose sign is systematic.
__device__ __forceinline__ void mixture_T_num_exact(float W, float w, float ux, float uy, float &hi, float &lo)
{
    float xl, yl, e1, pe, se;
    const float x2 = ff_prod(ux, ux, xl), y2 = ff_prod(uy, uy, yl);
    const float u2 = ff_sum(x2, y2, e1);  // u.u = u2 + (e1 + xl + yl)
    const float u2l = __fadd_rn(e1, __fadd_rn(xl, yl));
    const float p = ff_prod(u2, w, pe);
    hi = ff_sum(W, -p, se);  // W - u2 w = hi + se - pe
    lo = __fsub_rn(__fsub_rn(se, pe), __fmul_rn(u2l, w));
}
__device__ __forceinline__ float mixture_T(float W, float w, float wd, float ux, float uy)
{
    float hi, lo;
    mixture_T_num(W, w, ux, uy, hi, lo);
    return __fadd_rn(hi, lo) / wd;
}

// Stochastic rounding (dbm_params.rounding = DBM_ROUND_STOCHASTIC).  The
// exact value is s + e with s its round-to-nearest float; the result is the
// float neighbour of s on e's side with probability |e| / (spacing of the
// floats there), else s, so that its expectation is exactly s + e.  u is
// uniform in [0, 1).  Zero, infinite and NaN s are returned as they are.
__device__ __forceinline__ float sr_finish(float s, float e, float u)
{
    if (e == 0.0f || s == 0.0f) return s;
    const int away = (e > 0.0f) == (s > 0.0f) ? 1 : -1;  // one step away from zero, or towards it
    const float nb = __int_as_float(__float_as_int(s) + away);
    const float gap = fabsf(__fsub_rn(nb, s));
    return fabsf(e) > __fmul_rn(u, gap) ? nb : s;
}
// a + b rounded stochastically: s + e = a + b exactly (Knuth's two-sum).
__device__ __forceinline__ float sr_add(float a, float b, float u)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return sr_finish(s, e, u);
}
// a double rounded stochastically to float (x - s is exact in double).
__device__ __forceinline__ float sr_round(double x, float u)
{
    const float s = __double2float_rn(x);
    return sr_finish(s, __double2float_rn(x - (double)s), u);
}
// Error-free transformations on the FP32 pipes: a b = p + e (FMA residual)
// and a + b = s + e (Knuth's two-sum), exactly.
__device__ __forceinline__ float ff_prod(float a, float b, float &e)
{
    const float p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
    return p;
}
__device__ __forceinline__ float ff_sum(float a, float b, float &e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}
// hi + lo rounded stochastically; renormalised first, so that the head is
// the round-to-nearest value and the tail its rounding error.
__device__ __forceinline__ float sr_ff(float hi, float lo, float u)
{
    float e;
    const float s = ff_sum(hi, lo, e);
    return sr_finish(s, e, u);
}
// c + a b rounded stochastically.
__device__ __forceinline__ float sr_fma(float a, float b, float c, float u)
{
    float pe, se;
    const float s = ff_sum(c, ff_prod(a, b, pe), se);
    return sr_ff(s, __fadd_rn(se, pe), u);
}
// The k-th uniform number in [0, 1) of a cell whose hash is h: the hash
// of a golden-ratio Weyl sequence from h, top 24 bits.  A rounding's
// residual depends on earlier roundings of the same cell (the store on the
// temperature), so the numbers of one cell are hashed one by one rather
// than taken as fixed shifts of the first, which would make a later number
// a function of an earlier one.
__device__ __forceinline__ float sr_uniform(unsigned h, int k)
{
    return __uint2float_rz(mix32(h + (unsigned)k * 0x9e3779b9u) >> 8) * 0x1p-24f;
}

// Mixture u, T of one cell (reading R1 of the collision's conservation)
// and the species densities, evaluated in double from the stored floats
// of the tile (dbm_params.thermo = DBM_THERMO_FP64): ring sums, species
// moments, weighted sums, u = sum lam j / sum lam n and
// T = (sum lam E - u.u sum lam n) / sum kap n.  Lane j of the tile's values.
template <int S, class Tile, class X>
__device__ __forceinline__ void moments_fp64(const X &xa, const Tile &t, int j, double n64[S], double &ux,
                                             double &uy, double &T, double &cap)
{
    using L = Lanes<typename Tile::V>;
    double w = 0.0, wx = 0.0, wy = 0.0, we = 0.0, wd = 0.0;
    cap = 0.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        double sn = 0.0, sx = 0.0, sy = 0.0, se = 0.0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const double f0 = L::get(t.ld(s * Q + 4 * r, 0, 0), j), f1 = L::get(t.ld(s * Q + 4 * r + 1, 0, 0), j);
            const double f2 = L::get(t.ld(s * Q + 4 * r + 2, 0, 0), j), f3 = L::get(t.ld(s * Q + 4 * r + 3, 0, 0), j);
            const double rs = (f0 + f2) + (f1 + f3);
            double rx, ry;
            if ((r & 1) == 0) {
                rx = f0 - f2;
                ry = f1 - f3;
            } else {
                const double a = f0 - f2, b = f3 - f1;
                rx = a + b;
                ry = a - b;
            }
            sn += rs;
            sx = fma(xa.vr[s][r], rx, sx);
            sy = fma(xa.vr[s][r], ry, sy);
            se = fma(xa.qr[s][r], rs, se);
        }
        n64[s] = sn;
        w = fma(xa.lam[s], sn, w);
        wx = fma(xa.lam[s], sx, wx);
        wy = fma(xa.lam[s], sy, wy);
        we = fma(xa.lam[s], se, we);
        wd = fma(xa.kap[s], sn, wd);
        cap = fma(xa.dpi[s], sn, cap);
    }
    ux = wx / w;
    uy = wy / w;
    T = (we - fma(ux, ux, uy * uy) * w) / wd;
}

// Where the cell sits and which ghost images its values must also reach.
struct Site {
    int x, y;
    unsigned mx, my;
    long long cell;  // element offset of (x, y) in a plane
    bool two;        // two cells per thread: (x + 1, y) is inside the domain
};

// Output of the FP32 state: f^{n+1}, and the ghost images of a species
// after all 16 of its values are stored (the thread re-reads its own
// stores: no registers held across the species loop).  One cell per thread.
struct StateOut {
    static constexpr bool kNoImages = false;
    float *f;  // plane 0 of the output buffer
    long long P;
    int nx, ny, pitch;
    long long n;  // checked builds: elements of the buffer
    unsigned *flag;
    __device__ __forceinline__ void put(const Site &w, int p, float g, float) const
    {
        const long long i = (long long)p * P + w.cell;
        if (in_bounds(i, n, flag)) __stcs(f + i, g);  // streamed: not re-read this step
    }
    __device__ __forceinline__ void put_n(const Site &, int, float) const {}
    __device__ __forceinline__ void put_mix(const Site &, float, float, float) const {}
    __device__ __forceinline__ void images(const Site &w, int s) const
    {
        for (int i = 0; i < Q; ++i) {
            float *pl = f + (long long)(s * Q + i) * P;
            // ghost images lie within rows -2 .. ny+1 and columns -2 .. nx+1
            if (in_bounds((long long)(s * Q + i) * P + (long long)(ny + 1 + GY) * pitch + (nx + 1 + GX), n, flag))
                store_images(pl, w.x, w.y, nx, ny, pitch, w.mx, w.my, pl[w.cell]);
        }
    }
    __device__ __forceinline__ void images_mix(const Site &) const {}
};

// Output of the TMA-staged FP32 steps: f^{n+1} only, one or two cells per
// thread.  These kernels never read the stored ghost cells (a tile at the
// domain boundary takes its halo from the interior, halo_fill), so they
// do not write them either.
struct StateOutNoImages {
    static constexpr bool kNoImages = true;
    float *f;  // plane 0 of the output buffer
    long long P;
    long long n;  // checked builds: elements of the buffer
    unsigned *flag;
    __device__ __forceinline__ void put(const Site &w, int p, float g, float) const
    {
        const long long i = (long long)p * P + w.cell;
        if (in_bounds(i, n, flag)) __stcs(f + i, g);
    }
    __device__ __forceinline__ void put(const Site &w, int p, float2 g, float2) const
    {
        const long long i = (long long)p * P + w.cell;
        if (!in_bounds(i, n - (w.two ? 1 : 0), flag)) return;
        float *q = f + i;  // x even: 8-byte aligned
        if (w.two)
            __stcs(reinterpret_cast<float2 *>(q), g);
        else
            __stcs(q, g.x);
    }
    template <class V>
    __device__ __forceinline__ void put_n(const Site &, int, V) const
    {
    }
    template <class V>
    __device__ __forceinline__ void put_mix(const Site &, V, V, V) const
    {
    }
    __device__ __forceinline__ void images(const Site &, int) const {}
    __device__ __forceinline__ void images_mix(const Site &) const {}
};

// The ring order the moment sums below are written for (D2V16 definition):
// axis rings +x, +y, -x, -y; diagonal rings (+,+), (-,+), (-,-), (+,-).
static_assert(dir_x(0) == 1 && dir_y(1) == 1 && dir_x(2) == -1 && dir_y(3) == -1 && dir_y(0) == 0 &&
                  dir_x(1) == 0 && dir_x(4) == 1 && dir_y(4) == 1 && dir_x(5) == -1 && dir_y(5) == 1 &&
                  dir_x(6) == -1 && dir_y(6) == -1 && dir_x(7) == 1 && dir_y(7) == -1,
              "D2V16 ring order");

// The whole update of cell (x, y), or of the cells (x, y) and (x + 1, y)
// when the tile delivers pairs (Tile::V = float2; `two` false when x + 1 is
// outside the domain: that half is computed but neither stored nor checked).
// `c` supplies the constants the cell uses many times (equilibrium blocks,
// ring speeds, weights, advection numbers); `g` the ones it uses once or
// twice (grid geometry and boundaries, reaction and force).  The
// single-problem kernels pass the same parameter block twice; the batched
// kernel passes the launch's shared constants as `c`, so that they stay
// constant-bank operands, and each instance's own block as `g`.
template <int S, class K, class G, class Tile, class Out, class X = NoAcc>
__device__ __forceinline__ void step_cell(const K &c, const G &g, const Tile &t, int x, int y, bool two,
                                          const Out &out, unsigned *__restrict__ flag, const X &xa = X{})
{
    using V = typename Tile::V;
    using L = Lanes<V>;
    static_assert(L::n == 1 || Out::kNoImages, "ghost images are written one cell per thread");
    // arithmetic options (AccConsts): run-time switches of the option kernel
    bool t64 = false, sr = false;
    if constexpr (X::on) {
        t64 = xa.thermo64 != 0;
        sr = xa.stochastic != 0;
    }

    constexpr bool kStaged = is_staged<Tile>::value;
    static_assert(!(kStaged && X::on), "the arithmetic options read every species at once");

    // 1. species moments, by ring sums
    V n[S], nf = bc<V>(0.0f), no = bc<V>(0.0f), cap, w, wx, wy, we, wd;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        if constexpr (kStaged) t.acquire(s);
        const auto &ts = stage_view(t, s, s);
        V sn, sx, sy, se;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const V f0 = ts.ld(s * Q + 4 * r, 0, 0), f1 = ts.ld(s * Q + 4 * r + 1, 0, 0);
            const V f2 = ts.ld(s * Q + 4 * r + 2, 0, 0), f3 = ts.ld(s * Q + 4 * r + 3, 0, 0);
            const V rs = vadd(vadd(f0, f2), vadd(f1, f3));
            V rx, ry;
            if ((r & 1) == 0) {
                rx = vsub(f0, f2);
                ry = vsub(f1, f3);
            } else {
                const V a = vsub(f0, f2), b = vsub(f3, f1);
                rx = vadd(a, b);
                ry = vsub(a, b);
            }
            if (r == 0) {
                sn = rs;
                sx = vmul(bc<V>(c.vr[s][0]), rx);
                sy = vmul(bc<V>(c.vr[s][0]), ry);
                se = vmul(bc<V>(c.qr[s][0]), rs);
            } else {
                sn = vadd(sn, rs);
                sx = vfma(bc<V>(c.vr[s][r]), rx, sx);
                sy = vfma(bc<V>(c.vr[s][r]), ry, sy);
                se = vfma(bc<V>(c.qr[s][r]), rs, se);
            }
        }
        if constexpr (kStaged) t.release(s);
        n[s] = sn;
        if (s == g.fuel) nf = sn;  // selects, no runtime-indexed register array
        if (s == g.oxid) no = sn;
        const V lh = bc<V>(c.lam_h[s]), ll = bc<V>(c.lam_l[s]), kh = bc<V>(c.kap_h[s]), kl = bc<V>(c.kap_l[s]);
        const V ws = vfma(lh, sn, vmul(ll, sn)), wxs = vfma(lh, sx, vmul(ll, sx));
        const V wys = vfma(lh, sy, vmul(ll, sy)), wes = vfma(lh, se, vmul(ll, se));
        const V wds = vfma(kh, sn, vmul(kl, sn));
        if (s == 0) {
            w = ws, wx = wxs, wy = wys, we = wes, wd = wds;
            cap = vmul(bc<V>(c.dpi[0]), sn);
        } else {
            w = vadd(w, ws), wx = vadd(wx, wxs), wy = vadd(wy, wys), we = vadd(we, wes), wd = vadd(wd, wds);
            cap = vfma(bc<V>(c.dpi[s]), sn, cap);
        }
    }

    // 2. mixture velocity and temperature (per cell: division, float-float T)
    V rw, T;
#pragma unroll
    for (int j = 0; j < L::n; ++j) L::set(rw, j, 1.0f / L::get(w, j));
    V ux = vmul(wx, rw), uy = vmul(wy, rw);
#pragma unroll
    for (int j = 0; j < L::n; ++j)
        L::set(T, j, mixture_T(L::get(we, j), L::get(w, j), L::get(wd, j), L::get(ux, j), L::get(uy, j)));
    // DBM_THERMO_FP64: n^s, u and T from double sums replace the float ones
    double n64[S][L::n], T64[L::n], cap64[L::n], om64[L::n], dT64[L::n];
    unsigned hcell[L::n];  // per-cell hash of the stochastic rounding
    if constexpr (X::on) {
#pragma unroll
        for (int j = 0; j < L::n; ++j) hcell[j] = mix32((unsigned)(y * g.nx + x + j) * 0x9e3779b9u ^ xa.seed);
    }
    if constexpr (X::on) {
        if (t64) {
#pragma unroll
            for (int j = 0; j < L::n; ++j) {
                double nl[S], u0, u1, Tj, cp;
                moments_fp64<S>(xa, t, j, nl, u0, u1, Tj, cp);
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    n64[s][j] = nl[s];
                    L::set(n[s], j, __double2float_rn(nl[s]));
                }
                T64[j] = Tj;
                cap64[j] = cp;
                L::set(ux, j, __double2float_rn(u0));
                L::set(uy, j, __double2float_rn(u1));
                L::set(T, j, __double2float_rn(Tj));
            }
        }
        // stochastic rounding: the mixture T, from which every species'
        // equilibrium energy follows, rounded without bias (the double T, or
        // the quotient of the float-float numerator with its remainder)
        if (sr) {
#pragma unroll
            for (int j = 0; j < L::n; ++j) {
                if (t64) {
                    L::set(T, j, sr_round(T64[j], sr_uniform(hcell[j], 0)));
                } else {
                    float nh, nl;
                    mixture_T_num_exact(L::get(we, j), L::get(w, j), L::get(ux, j), L::get(uy, j), nh, nl);
                    const float wdj = L::get(wd, j);
                    const float q = __fadd_rn(nh, nl) / wdj;
                    const float r = __fadd_rn(__fmaf_rn(-q, wdj, nh), nl);  // (nh + nl) - q wd
                    L::set(T, j, sr_ff(q, r / wdj, sr_uniform(hcell[j], 0)));
                }
            }
        }
    }

    unsigned bad = 0;
    V a;  // sum_s |n^s|
#pragma unroll
    for (int j = 0; j < L::n; ++j) {
        float aj = 0.0f;
#pragma unroll
        for (int s = 0; s < S; ++s) aj += fabsf(L::get(n[s], j));
        L::set(a, j, aj);
        if (j == 0 || two) {
#pragma unroll
            for (int s = 0; s < S; ++s)
                if (!(L::get(n[s], j) >= -1e-6f * aj)) bad |= DBM_HEALTH_DENSITY;
            if (!(aj > 0.0f)) bad |= DBM_HEALTH_DENSITY;
            if (!(L::get(T, j) > 0.0f)) bad |= DBM_HEALTH_TEMPERATURE;
            if (!isfinite(L::get(T, j) + L::get(ux, j) + L::get(uy, j))) bad |= DBM_HEALTH_NONFINITE;
        }
    }

    // 3. reaction: omega_ov and T' (state after a time tau^s)
    V om = bc<V>(0.0f), dT = bc<V>(0.0f);
    if constexpr (X::on) {
        if (t64 && g.has_reaction) {  // the Arrhenius rate and T' in double
#pragma unroll
            for (int j = 0; j < L::n; ++j) {
                double nF = 0.0, nO = 0.0;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    if (s == g.fuel) nF = n64[s][j];
                    if (s == g.oxid) nO = n64[s][j];
                }
                const double Tj = T64[j];
                om64[j] = xa.k_ov * nF * nO * exp(-xa.Ea_over_R / Tj);
                dT64[j] = (xa.Qheat - 0.5 * Tj * xa.src) * om64[j] / (0.5 * cap64[j]);
            }
        }
    }
    if (g.has_reaction && !t64) {
#pragma unroll
        for (int j = 0; j < L::n; ++j) {
            const float Tj = L::get(T, j);
            const float omj = g.k_ov * L::get(nf, j) * L::get(no, j) * expf(-g.Ea_over_R / Tj);
            L::set(om, j, omj);
            L::set(dT, j,
                   __fmul_rn(__fsub_rn(g.Qheat, __fmul_rn(__fmul_rn(0.5f, Tj), g.src)), omj) /
                       __fmul_rn(0.5f, L::get(cap, j)));
        }
    }

    Site w_;
    w_.x = x;
    w_.y = y;
    w_.two = two;
    constexpr bool kImages = !Out::kNoImages;
    w_.mx = kImages ? ghost_mask(x, g.nx, g.bc_x) : 0u;
    w_.my = kImages ? ghost_mask(y, g.ny, g.bc_y) : 0u;
    w_.cell = (long long)(y + GY) * g.pitch + (x + GX);
    const bool images = kImages && (w_.mx | w_.my) != 0u;
    out.put_mix(w_, ux, uy, T);

    // the species loop is unrolled up to three species: the constants of each
    // species then index the constant bank directly (measured 6-8 % faster
    // for one to three species; the four-species generic kernel ran 30 %
    // slower unrolled)
#pragma unroll(S <= 3 ? S : 1)
    for (int s = 0; s < S; ++s) {
        if constexpr (kStaged) t.acquire(S + s);
        const auto &ts = stage_view(t, S + s, s);
        V f0[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f0[i] = ts.ld(s * Q + i, 0, 0);
        // species density from step 1 (selected, not indexed)
        V ns = n[0];
#pragma unroll
        for (int j = 1; j < S; ++j)
            if (s == j) ns = n[j];
        out.put_n(w_, s, ns);
        // 4. merged equilibrium moments
        V cb[16];
        {
            V nr = ns, Ts = T;
            if (g.has_reaction) {
                nr = vfma(bc<V>(g.tau_a[s]), om, ns);
                Ts = vfma(bc<V>(g.tau_d[s]), dT, T);
                if constexpr (X::on) {
                    if (t64 || sr) {
#pragma unroll
                        for (int j = 0; j < L::n; ++j) {
                            const float un = sr_uniform(hcell[j], S * Q + 1 + s);
                            const float uT = sr_uniform(hcell[j], S * Q + 1 + S + s);
                            if (t64) {
                                double n_s = 0.0;
#pragma unroll
                                for (int q = 0; q < S; ++q)
                                    if (q == s) n_s = n64[q][j];
                                const double nd = fma(xa.tau_a[s], om64[j], n_s);
                                const double Td = fma(xa.tau_d[s], dT64[j], T64[j]);
                                L::set(nr, j, sr ? sr_round(nd, un) : __double2float_rn(nd));
                                L::set(Ts, j, sr ? sr_round(Td, uT) : __double2float_rn(Td));
                            } else {  // n + tau a omega and T + tau T' exactly, then rounded
                                L::set(nr, j, sr_fma(g.tau_a[s], L::get(om, j), L::get(ns, j), un));
                                L::set(Ts, j, sr_fma(g.tau_d[s], L::get(dT, j), L::get(T, j), uT));
                            }
                        }
                    }
                }
#pragma unroll
                for (int j = 0; j < L::n; ++j)
                    if ((j == 0 || two) && L::get(nr, j) < -1e-6f * L::get(a, j)) bad |= DBM_HEALTH_NSTAR;
            }
            fhat_blocks<V>(nr, ux, uy, vmul(Ts, bc<V>(c.inv_m[s])), c.dpi[s], cb);
            if constexpr (X::on) {
                if (sr) {  // the energy target n* ((D+I) T*/m + u.u) formed in float-float, rounded without bias
#pragma unroll
                    for (int j = 0; j < L::n; ++j) {
                        float thl, al, xl, yl, e1, e2, cl;
                        const float th = ff_prod(L::get(Ts, j), c.inv_m[s], thl);  // T*/m
                        const float a1 = ff_prod(c.dpi[s], th, al);
                        const float x2 = ff_prod(L::get(ux, j), L::get(ux, j), xl);
                        const float y2 = ff_prod(L::get(uy, j), L::get(uy, j), yl);
                        const float u2 = ff_sum(x2, y2, e1);
                        const float r1 = ff_sum(a1, u2, e2);  // (D+I) T*/m + u.u = r1 + r1l
                        const float r1l = __fadd_rn(__fadd_rn(e2, __fmaf_rn(c.dpi[s], thl, al)),
                                                    __fadd_rn(e1, __fadd_rn(xl, yl)));
                        const float nrj = L::get(nr, j);
                        const float c1 = ff_prod(nrj, r1, cl);
                        L::set(cb[1], j, sr_ff(c1, __fmaf_rn(nrj, r1l, cl), sr_uniform(hcell[j], S * Q + 1 + 6 * S + s)));
                    }
                }
            }
            bool present = false;  // an absent species feels no force
#pragma unroll
            for (int j = 0; j < L::n; ++j) present |= L::get(ns, j) != 0.0f;
            if (g.has_force && present) {
                V jx, jy, e;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const float v = c.vr[s][i >> 2];
                    e = i == 0 ? vmul(bc<V>(c.qr[s][0]), f0[0]) : vfma(bc<V>(c.qr[s][i >> 2]), f0[i], e);
                    if (dir_x(i) != 0) jx = i == 0 ? vmul(bc<V>(dir_x(i) * v), f0[i]) : vfma(bc<V>(dir_x(i) * v), f0[i], jx);
                    if (dir_y(i) != 0) jy = i == 1 ? vmul(bc<V>(dir_y(i) * v), f0[i]) : vfma(bc<V>(dir_y(i) * v), f0[i], jy);
                }
                V usx, usy, th;
#pragma unroll
                for (int j = 0; j < L::n; ++j) {
                    const float nsj = L::get(ns, j);
                    const float ux_s = L::get(jx, j) / nsj, uy_s = L::get(jy, j) / nsj;
                    L::set(usx, j, ux_s);
                    L::set(usy, j, uy_s);
                    L::set(th, j, __fsub_rn(L::get(e, j) / nsj, __fmaf_rn(ux_s, ux_s, __fmul_rn(uy_s, uy_s))) / c.dpi[s]);
                }
                // cb += f-hat(u-dagger) - f-hat(u^s), each term one multiply-add
                // (the second at -n^s, which negates every f-hat exactly)
                V Ld[16], Rd[16], Ls[16], Rs[16];
                fhat_factors<V>(ns, vfma(bc<V>(g.accel_x), bc<V>(c.tau[s]), usx),
                                vfma(bc<V>(g.accel_y), bc<V>(c.tau[s]), usy), th, c.dpi[s], Ld, Rd);
                fhat_factors<V>(vmul(bc<V>(-1.0f), ns), usx, usy, th, c.dpi[s], Ls, Rs);
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    V sum = vfma(Ls[k], Rs[k], vfma(Ld[k], Rd[k], cb[k]));
#pragma unroll
                    for (int j = 0; j < L::n; ++j)
                        if (L::get(ns, j) == 0.0f) L::set(sum, j, L::get(cb[k], j));
                    cb[k] = sum;
                }
            }
        }
        V o[16];
        bool done = false;
        if constexpr (X::on) {
            if (sr) {
                solve_blocks<V, K, true>(c, s, cb, o, hcell, S * Q + 1 + 2 * S + 4 * s);
                done = true;
            }
        }
        if (!done) solve_blocks<V>(c, s, cb, o);
        const V dtt = bc<V>(c.dt_tau[s]);

#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int p = s * Q + i, r = i >> 2;
            // 6. forward Euler: f + dt/tau (f^eq,tot - f) - dt v . grad f,
            // with the 5. NND advection terms of x and y each applied as one
            // fused multiply-add (no product is left for the compiler to fuse)
            const V e = feq_of<V>(i, o);
            if constexpr (X::on) {
                if (sr) {  // the increment, then one stochastically rounded sum
                    V d = vmul(dtt, vsub(e, f0[i]));
                    if (dir_x(i) > 0)
                        d = vfma(bc<V>(-c.cdx[s][r]), nnd_diff_pos<V>(ts.ld(p, -2, 0), ts.ld(p, -1, 0), f0[i], ts.ld(p, 1, 0)),
                                 d);
                    else if (dir_x(i) < 0)
                        d = vfma(bc<V>(c.cdx[s][r]), nnd_diff_neg<V>(ts.ld(p, -1, 0), f0[i], ts.ld(p, 1, 0), ts.ld(p, 2, 0)),
                                 d);
                    if (dir_y(i) > 0)
                        d = vfma(bc<V>(-c.cdy[s][r]), nnd_diff_pos<V>(ts.ld(p, 0, -2), ts.ld(p, 0, -1), f0[i], ts.ld(p, 0, 1)),
                                 d);
                    else if (dir_y(i) < 0)
                        d = vfma(bc<V>(c.cdy[s][r]), nnd_diff_neg<V>(ts.ld(p, 0, -1), f0[i], ts.ld(p, 0, 1), ts.ld(p, 0, 2)),
                                 d);
                    V f1;
#pragma unroll
                    for (int j = 0; j < L::n; ++j)
                        L::set(f1, j, sr_add(L::get(f0[i], j), L::get(d, j), sr_uniform(hcell[j], p + 1)));
                    out.put(w_, p, f1, e);
                    continue;
                }
            }
            V f1 = vfma(dtt, vsub(e, f0[i]), f0[i]);
            if constexpr (L::n == 2) {
                if (dir_x(i) != 0) {
                    const V a = ts.ld(p, -2, 0), b = ts.ld(p, 2, 0);
                    if (dir_x(i) > 0)
                        f1 = vfma(bc<V>(-c.cdx[s][r]), nnd_diff_pos_pair(a, f0[i], b), f1);
                    else
                        f1 = vfma(bc<V>(c.cdx[s][r]), nnd_diff_neg_pair(a, f0[i], b), f1);
                }
            } else if (dir_x(i) > 0) {
                f1 = vfma(bc<V>(-c.cdx[s][r]), nnd_diff_pos<V>(ts.ld(p, -2, 0), ts.ld(p, -1, 0), f0[i], ts.ld(p, 1, 0)),
                          f1);
            } else if (dir_x(i) < 0) {
                f1 = vfma(bc<V>(c.cdx[s][r]), nnd_diff_neg<V>(ts.ld(p, -1, 0), f0[i], ts.ld(p, 1, 0), ts.ld(p, 2, 0)),
                          f1);
            }
            if (dir_y(i) > 0)
                f1 = vfma(bc<V>(-c.cdy[s][r]), nnd_diff_pos<V>(ts.ld(p, 0, -2), ts.ld(p, 0, -1), f0[i], ts.ld(p, 0, 1)),
                          f1);
            else if (dir_y(i) < 0)
                f1 = vfma(bc<V>(c.cdy[s][r]), nnd_diff_neg<V>(ts.ld(p, 0, -1), f0[i], ts.ld(p, 0, 1), ts.ld(p, 0, 2)),
                          f1);
            out.put(w_, p, f1, e);
        }
        if (images) out.images(w_, s);
        if constexpr (kStaged) t.release(S + s);
    }
    if (images) out.images_mix(w_);
    if (bad) raise_flag(flag, bad);
}

// Generic kernel: inputs from global memory through the read-only path.
template <int S>
__global__ void __launch_bounds__(256)
    k_step(const __grid_constant__ StepConsts<float, S> c, const float *__restrict__ fin, float *__restrict__ fout,
           unsigned *__restrict__ flag)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= c.nx || y >= c.ny) return;
    GlobalTile t;
    t.base = fin + (long long)(y + GY) * c.pitch + (x + GX);
    t.P = c.plane;
    t.py = c.pitch;
    t.lo = fin;
    t.n = (long long)S * Q * c.plane;
    t.flag = flag;
    StateOut o{fout, c.plane, c.nx, c.ny, c.pitch, (long long)S * Q * c.plane, flag};
    step_cell<S>(c, c, t, x, y, true, o, flag);
}

// ---------------------------------------------------------------------------
// TMA-staged kernel: one CTA steps a TX x TY tile of cells, CW (1 or 2)
// adjacent cells of a row per thread.  One thread issues a single
// cp.async.bulk.tensor copy of the tile plus its radius-2 halo (all 16 S
// planes, columns x0-4 .. x0+TX+3 so that the copy starts on a 16-byte
// boundary) into shared memory, completing on an mbarrier; every thread then
// reads its stencil from shared memory.
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

constexpr long long TMA_WAIT_LIMIT = TMA_WAIT_POLLS;  // drain wait: try_wait polls (each may suspend ~us)

// Issue the tile copy (leader thread): box origin column bx0 (= bx0 + GX - 4),
// row by0 (= by0 + GY - 2), plane z.
__device__ __forceinline__ void tma_tile_load(float *tile, unsigned long long tmap, int bx0, int by0,
                                              unsigned bar, unsigned bytes, int z = 0)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(tile)),
        "l"(tmap), "r"(bx0), "r"(by0), "r"(z), "r"(bar)
        : "memory");
}

// Source index of ghost index g (one of -2, -1, n, n + 1) on an axis of n
// cells: the periodic image or the outflow edge cell.
__device__ __forceinline__ int halo_source(int g, int n, int bc)
{
    if (bc != DBM_BC_PERIODIC) return min(max(g, 0), n - 1);
    if (n >= 2) return g < 0 ? g + n : g - n;
    return 0;  // one cell: every image is that cell
}

// Halo of a tile that touches the domain boundary, taken from the interior
// of the input state (periodic: the wrapped cells; outflow: the edge cell)
// instead of from stored ghost cells.  The tile holds global columns
// bx0-4 .. bx0+TX+3 and rows by0-2 .. by0+TY+1 of all NP planes; only the
// cross-shaped stencil reaches into the halo, so the x halo is needed in the
// tile's interior rows and the y halo in its interior columns: interior
// cells span columns bx0 .. x_hi-1 and rows by0 .. y_hi-1, their stencil
// reads columns bx0-2 .. x_hi+1 and rows by0-2 .. y_hi+1, so only the ghost
// columns {-2, -1, nx, nx+1} and rows {-2, -1, ny, ny+1} inside those
// ranges are filled (tile column = x - bx0 + 4 stays within 2 .. TX+5, tile
// row = y - by0 + 2 within 0 .. TY+3).
//
// The input buffer is only read by the step, so a boundary tile loads its
// halo values into registers before it waits for its tile copy (halo_load)
// and stores them into the tile once the copy has landed (halo_store): the
// load latency overlaps the copy instead of following it.  Work items of a
// side are (plane, row or column, ghost index j of 2) with compile-time
// extents; thread tid takes items tid, tid + NT, ... into fixed registers.
template <int NP, int TX, int TY, int NT>
struct HaloRegs {
    static constexpr int XI = 2 * TY * NP, YI = 2 * TX * NP;  // items of one x side, one y side
    static constexpr int XK = (XI + NT - 1) / NT, YK = (YI + NT - 1) / NT;
    float x[2][XK], y[2][YK];
};

// Which ghost layers a tile needs: 2 columns left, `right` (0..2) columns
// right, 2 rows on top, `bottom` rows at the bottom; false for an interior
// tile (uniform over the CTA).
struct HaloSides {
    int left, right, top, bottom, x_hi, y_hi;
    __device__ __forceinline__ bool any() const { return left + right + top + bottom != 0; }
};

template <int TX, int TY>
__device__ __forceinline__ HaloSides halo_sides(int bx0, int by0, int nx, int ny)
{
    HaloSides h;
    h.x_hi = min(bx0 + TX, nx);
    h.y_hi = min(by0 + TY, ny);
    h.left = bx0 == 0 ? 2 : 0;
    h.top = by0 == 0 ? 2 : 0;
    h.right = min(max(h.x_hi - nx + 2, 0), 2);
    h.bottom = min(max(h.y_hi - ny + 2, 0), 2);
    return h;
}

template <int NP, int TX, int TY, int NT>
__device__ __forceinline__ void halo_load(HaloRegs<NP, TX, TY, NT> &hr, const HaloSides &hs,
                                          const float *__restrict__ fin, int bx0, int by0, int nx, int ny,
                                          int pitch, long long plane, int bc_x, int bc_y, int tid, unsigned *flag)
{
    using H = HaloRegs<NP, TX, TY, NT>;
    const long long base = (long long)GY * pitch + GX;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int need = side == 0 ? hs.left : hs.right;
        if (need == 0) continue;
#pragma unroll
        for (int k = 0; k < H::XK; ++k) {
            const int it = tid + k * NT;
            const int j = it & 1, r = (it >> 1) % TY, p = (it >> 1) / TY;
            const int y = by0 + r;
            if (it < H::XI && j < need && y < hs.y_hi) {
                const int xs = halo_source(side == 0 ? j - 2 : nx + j, nx, bc_x);
                const long long i = p * plane + base + (long long)y * pitch + xs;
                if (in_bounds(i, NP * plane, flag)) hr.x[side][k] = fin[i];
            }
        }
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int need = side == 0 ? hs.top : hs.bottom;
        if (need == 0) continue;
#pragma unroll
        for (int k = 0; k < H::YK; ++k) {
            const int it = tid + k * NT;
            const int c = it % TX, j = (it / TX) & 1, p = it / (2 * TX);
            const int x = bx0 + c;
            if (it < H::YI && j < need && x < hs.x_hi) {
                const int ys = halo_source(side == 0 ? j - 2 : ny + j, ny, bc_y);
                const long long i = p * plane + base + (long long)ys * pitch + x;
                if (in_bounds(i, NP * plane, flag)) hr.y[side][k] = fin[i];
            }
        }
    }
}

// The halo of a boundary tile straight from the input into the tile, then
// a barrier (the same items as halo_load / halo_store, without holding them
// in registers: for kernels whose boundary tiles are rare, where the extra
// registers would cost every tile).  All threads of the CTA call this for a
// boundary tile.
template <int NP, int TX, int TY, int NT>
__device__ __forceinline__ void halo_fill(const HaloSides &hs, float *tile, const float *__restrict__ fin, int bx0,
                                          int by0, int nx, int ny, int pitch, long long plane, int bc_x, int bc_y,
                                          int tid, unsigned *flag)
{
    using H = HaloRegs<NP, TX, TY, NT>;
    constexpr int BX = TX + 8, PS = (TY + 4) * BX;
    const long long base = (long long)GY * pitch + GX;
    for (int side = 0; side < 2; ++side) {
        const int need = side == 0 ? hs.left : hs.right;
        if (need == 0) continue;
        for (int it = tid; it < H::XI; it += NT) {
            const int j = it & 1, r = (it >> 1) % TY, p = (it >> 1) / TY;
            const int y = by0 + r;
            if (j >= need || y >= hs.y_hi) continue;
            const int xg = side == 0 ? j - 2 : nx + j;
            const long long i = p * plane + base + (long long)y * pitch + halo_source(xg, nx, bc_x);
            const int t = p * PS + (r + 2) * BX + (xg - bx0 + 4);
            if (in_bounds(i, NP * plane, flag) && in_bounds(t, NP * PS, flag)) tile[t] = fin[i];
        }
    }
    for (int side = 0; side < 2; ++side) {
        const int need = side == 0 ? hs.top : hs.bottom;
        if (need == 0) continue;
        for (int it = tid; it < H::YI; it += NT) {
            const int c = it % TX, j = (it / TX) & 1, p = it / (2 * TX);
            const int x = bx0 + c;
            if (j >= need || x >= hs.x_hi) continue;
            const int yg = side == 0 ? j - 2 : ny + j;
            const long long i = p * plane + base + (long long)halo_source(yg, ny, bc_y) * pitch + x;
            const int t = p * PS + (yg - by0 + 2) * BX + (c + 4);
            if (in_bounds(i, NP * plane, flag) && in_bounds(t, NP * PS, flag)) tile[t] = fin[i];
        }
    }
    __syncthreads();
}

// Store the values halo_load fetched into the tile, then a barrier.  All
// threads of the CTA call this for a boundary tile.
template <int NP, int TX, int TY, int NT>
__device__ __forceinline__ void halo_store(const HaloRegs<NP, TX, TY, NT> &hr, const HaloSides &hs, float *tile,
                                           int bx0, int by0, int nx, int ny, int tid, unsigned *flag)
{
    using H = HaloRegs<NP, TX, TY, NT>;
    constexpr int BX = TX + 8, PS = (TY + 4) * BX;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int need = side == 0 ? hs.left : hs.right;
        if (need == 0) continue;
#pragma unroll
        for (int k = 0; k < H::XK; ++k) {
            const int it = tid + k * NT;
            const int j = it & 1, r = (it >> 1) % TY, p = (it >> 1) / TY;
            if (it < H::XI && j < need && by0 + r < hs.y_hi) {
                const int xg = side == 0 ? j - 2 : nx + j;
                const int t = p * PS + (r + 2) * BX + (xg - bx0 + 4);
                if (in_bounds(t, NP * PS, flag)) tile[t] = hr.x[side][k];
            }
        }
    }
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        const int need = side == 0 ? hs.top : hs.bottom;
        if (need == 0) continue;
#pragma unroll
        for (int k = 0; k < H::YK; ++k) {
            const int it = tid + k * NT;
            const int c = it % TX, j = (it / TX) & 1, p = it / (2 * TX);
            if (it < H::YI && j < need && bx0 + c < hs.x_hi) {
                const int yg = side == 0 ? j - 2 : ny + j;
                const int t = p * PS + (yg - by0 + 2) * BX + (c + 4);
                if (in_bounds(t, NP * PS, flag)) tile[t] = hr.y[side][k];
            }
        }
    }
    __syncthreads();
}

// X: NoAcc for the default arithmetic, AccConsts<S> for the kernel with the
// thermo and rounding options.
template <int S, int TX, int TY, int CW, class X>
__global__ void __launch_bounds__(TX / CW * TY, tma_ctas_per_sm(S, TX, TY))
    k_step_tma(const __grid_constant__ StepConsts<float, S> c, const __grid_constant__ CUtensorMap tmap,
               const float *__restrict__ fin, float *__restrict__ fout, unsigned *__restrict__ flag,
               const __grid_constant__ X xa)
{
    static_assert(CW == 1 || CW == 2, "one or two cells per thread");
    constexpr int BX = TX + 8, BY = TY + 4, NP = S * Q, NT = TX / CW * TY;
    constexpr unsigned BYTES = (unsigned)(BX * BY * NP * sizeof(float));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    float *tile = reinterpret_cast<float *>(smem_raw);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const bool leader = tx == 0 && ty == 0;
    const int bx0 = blockIdx.x * TX, by0 = blockIdx.y * TY;
    const unsigned b = smem_u32(&bar);
    if (leader) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    if (leader) tma_tile_load(tile, reinterpret_cast<unsigned long long>(&tmap), bx0, by0, b, BYTES);
    const int tid = ty * (TX / CW) + tx;
    const HaloSides hs = halo_sides<TX, TY>(bx0, by0, c.nx, c.ny);
    const bool ok = mbar_wait(b, 0, c.wait_polls);
    if (__syncthreads_or(!ok)) {
        // the copy did not land: report, give it one more bounded wait so
        // that no copy is left writing into this block's shared memory, and
        // leave together
        if (leader) raise_flag(flag, DBM_HEALTH_TIMEOUT);
        mbar_wait(b, 0, TMA_WAIT_LIMIT);
        return;
    }
    if (hs.any())
        halo_fill<NP, TX, TY, NT>(hs, tile, fin, bx0, by0, c.nx, c.ny, c.pitch, c.plane, c.bc_x, c.bc_y, tid, flag);
    const int x = bx0 + CW * tx, y = by0 + ty;
    if (x >= c.nx || y >= c.ny) return;
    StateOutNoImages o{fout, c.plane, (long long)NP * c.plane, flag};
    const float *base = tile + (ty + 2) * BX + (CW * tx + 4);
    if constexpr (CW == 2) {
        const SmemTile2 t{base, BY * BX, BX, tile, NP * BY * BX, flag};
        step_cell<S>(c, c, t, x, y, x + 1 < c.nx, o, flag, xa);
    } else {
        const SmemTile t{base, BY * BX, BX, tile, NP * BY * BX, flag};
        step_cell<S>(c, c, t, x, y, true, o, flag, xa);
    }
}

template <int S>
int launch_step_t(dbm_handle *h, const void *fin, void *fout, cudaStream_t st)
{
    StepConsts<float, S> c;
    fill_step_consts<float, S>(h, c);
    dim3 block(64, 4);
    dim3 grid((h->p.nx + 63) / 64, (h->p.ny + 3) / 4);
    k_step<S><<<grid, block, 0, st>>>(c, (const float *)fin, (float *)fout, (unsigned *)h->scratch);
    return set_cuda_error(h, cudaGetLastError(), "step kernel launch");
}

// ACC: the kernel with the thermo and rounding options (AccConsts).
template <int S, int TX, int TY, int CW, bool ACC>
int launch_step_tma_t(dbm_handle *h, const CUtensorMap *tmap, const void *fin, void *fout, cudaStream_t st)
{
    using X = typename std::conditional<ACC, AccConsts<S>, NoAcc>::type;
    constexpr size_t smem = (size_t)(TX + 8) * (TY + 4) * S * Q * sizeof(float);
    static bool attr_set = false;  // per instantiation, set once per process
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_step_tma<S, TX, TY, CW, X>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return set_cuda_error(h, e, "TMA step kernel shared-memory attribute");
        attr_set = true;
    }
    StepConsts<float, S> c;
    fill_step_consts<float, S>(h, c);
    X xa{};
    if constexpr (ACC) fill_acc_consts<S>(h, c, xa);
    dim3 block(TX / CW, TY);
    dim3 grid((h->p.nx + TX - 1) / TX, (h->p.ny + TY - 1) / TY);
    k_step_tma<S, TX, TY, CW, X><<<grid, block, smem, st>>>(c, *tmap, (const float *)fin, (float *)fout,
                                                              (unsigned *)h->scratch, xa);
    return set_cuda_error(h, cudaGetLastError(), "TMA step kernel launch");
}


// ---------------------------------------------------------------------------
// The species-staged step.  The tile and its radius-2 halo pass through
// shared memory one species at a time, in two buffers that each hold the Q
// planes of one species (BX x BY cells), so the shared memory of a CTA does
// not grow with the species count: three and more species run two cells per
// thread at two CTAs per SM (the all-species tile of three species in pairs
// would hold one).  Each species is copied twice per tile: for its moment
// sums only its TX x TY own cells (a second descriptor, an interior box; no
// halo), for its update the tile and its halo.  Use k = 0 .. 2S-1 takes
// species k mod S from buffer k & 1,
// whose mbarrier completes its phase k >> 1 with that copy; while a use is
// computed the copy of the next one is in flight, and once every thread is
// done with a buffer (the barrier in release) the leader refills it for use
// k + 2.  A tile at the domain boundary fills each copy's halo from the
// interior of the input (halo_fill on that species' planes).
//
// Waits are bounded.  The first one takes c.wait_polls polls (a test can
// make it run out); a wait that runs out raises DBM_HEALTH_TIMEOUT, and the
// first one then waits once more, with the full limit.  A thread whose wait
// ran out for good stops waiting, the leader stops issuing copies, and at
// the end the leader waits (bounded) for the copies it left in flight.
template <int S, int TX, int TY>
struct StagedTile2 {
    static constexpr bool kStaged = true;
    static constexpr int BX = TX + 8, BY = TY + 4, PS = BX * BY, NT = TX / 2 * TY;
    static constexpr int PI = TX * TY;  // plane of an interior copy
    static constexpr unsigned BYTES = (unsigned)(PS * Q * sizeof(float));
    static constexpr unsigned BYTES_IN = (unsigned)(PI * Q * sizeof(float));
    using V = float2;
    float *buf;         // buffer 0 (buffer 1 follows at Q * PS)
    const float *cell;  // buffer 0, plane 0, this thread's row and first column
    const float *own;   // the same cells in the interior layout [plane][TY][TX]
    unsigned long long tmap, tmap_in;  // tile + halo box; interior box
    unsigned bar0;      // mbarrier of buffer 0 (buffer 1: bar0 + 8)
    const float *fin;
    int bx0, by0, nx, ny, pitch, bc_x, bc_y, wait_polls;
    long long plane;
    unsigned *flag;
    mutable int failed_at;  // the use whose wait ran out for good; 2S: none

    // view of use k: plane s * Q + i of species s read from buffer k & 1
    // (interior layout for the moment sums, k < S)
    __device__ __forceinline__ SmemTile2 view(int k, int s) const
    {
        if (k < S) return SmemTile2{own + (k & 1) * Q * PS - s * Q * PI, PI, TX, buf, 2 * Q * PS, flag};
        return SmemTile2{cell + ((k & 1) - s) * Q * PS, PS, BX, buf, 2 * Q * PS, flag};
    }
    __device__ __forceinline__ static bool leader() { return threadIdx.x == 0 && threadIdx.y == 0; }
    // leader: the copy of use k into its buffer
    __device__ __forceinline__ void issue(int k) const
    {
        if (k < S)  // interior box: origin at the tile's first cell
            tma_tile_load(buf + (k & 1) * Q * PS, tmap_in, bx0 + GX, by0 + GY, bar0 + 8u * (k & 1), BYTES_IN, k * Q);
        else
            tma_tile_load(buf + (k & 1) * Q * PS, tmap, bx0, by0, bar0 + 8u * (k & 1), BYTES, (k - S) * Q);
    }
    __device__ __forceinline__ void acquire(int k) const
    {
        if (failed_at == 2 * S) {
            const unsigned bar = bar0 + 8u * (k & 1), par = (k >> 1) & 1;
            bool ok = mbar_wait(bar, par, k == 0 ? wait_polls : TMA_WAIT_LIMIT);
            if (!ok) {
                raise_flag(flag, DBM_HEALTH_TIMEOUT);
                if (k == 0) ok = mbar_wait(bar, par, TMA_WAIT_LIMIT);
                if (!ok) failed_at = k;
            }
        }
        const HaloSides hs = halo_sides<TX, TY>(bx0, by0, nx, ny);
        if (k >= S && hs.any())
            halo_fill<Q, TX, TY, NT>(hs, buf + (k & 1) * Q * PS, fin + (long long)(k % S) * Q * plane, bx0, by0,
                                     nx, ny, pitch, plane, bc_x, bc_y, threadIdx.y * (TX / 2) + threadIdx.x, flag);
    }
    __device__ __forceinline__ void release(int k) const
    {
        __syncthreads();  // every thread is done with buffer k & 1
        if (k + 2 < 2 * S && leader() && failed_at == 2 * S) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(k + 2);
        }
    }
    // leader, after the last use: wait for the copies left in flight by a
    // wait that ran out (use failed_at and the one after it)
    __device__ __forceinline__ void drain() const
    {
        if (!leader() || failed_at == 2 * S) return;
        for (int k = failed_at; k < 2 * S && k <= failed_at + 1; ++k)
            mbar_wait(bar0 + 8u * (k & 1), (k >> 1) & 1, TMA_WAIT_LIMIT);
    }
};

constexpr int staged_ctas_per_sm(int TX, int TY)
{
    const int by_smem = (227 * 1024) / (2 * (TX + 8) * (TY + 4) * Q * 4 + 1024);
    return by_smem > 4 ? 4 : by_smem < 1 ? 1 : by_smem;
}

// Output of the species-staged kernel.  Its barriers are CTA-wide and sit
// inside the step, so every thread runs the whole step, in the same order
// of barrier instructions: a thread whose cells lie outside the domain (the
// ragged edge of a tile) computes on the in-range shared-memory values at
// its position and stores nothing.
struct StagedOut : StateOutNoImages {
    bool live;
    template <class G>
    __device__ __forceinline__ void put(const Site &w, int p, G g, G e) const
    {
        if (live) StateOutNoImages::put(w, p, g, e);
    }
};

template <int S, int TX, int TY>
__global__ void __launch_bounds__(TX / 2 * TY, staged_ctas_per_sm(TX, TY))
    k_step_staged(const __grid_constant__ StepConsts<float, S> c, const __grid_constant__ CUtensorMap tmap,
                  const __grid_constant__ CUtensorMap tmap_in, const float *__restrict__ fin,
                  float *__restrict__ fout, unsigned *__restrict__ flag)
{
    static_assert(S >= 2 && TX % 8 == 0, "two or more species; 16-byte aligned tile columns");
    using T = StagedTile2<S, TX, TY>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bars[2];
    float *buf = reinterpret_cast<float *>(smem_raw);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const unsigned b0 = smem_u32(&bars[0]);
    if (T::leader()) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b0 + 8u) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    __syncthreads();
    const T t{buf,
              buf + (ty + 2) * T::BX + (2 * tx + 4),
              buf + ty * TX + 2 * tx,
              reinterpret_cast<unsigned long long>(&tmap),
              reinterpret_cast<unsigned long long>(&tmap_in),
              b0,
              fin,
              (int)blockIdx.x * TX,
              (int)blockIdx.y * TY,
              c.nx,
              c.ny,
              c.pitch,
              c.bc_x,
              c.bc_y,
              c.wait_polls,
              c.plane,
              flag,
              2 * S};
    if (T::leader()) {
        t.issue(0);
        t.issue(1);
    }
    // every thread steps (see StagedOut); one outside the domain stores
    // nothing and sends its health bits to a sink
    __shared__ unsigned health_sink;
    const int x = t.bx0 + 2 * tx, y = t.by0 + ty;
    const bool live = x < c.nx && y < c.ny;
    const StagedOut o{{fout, c.plane, (long long)S * Q * c.plane, flag}, live};
    step_cell<S>(c, c, t, x, y, live && x + 1 < c.nx, o, live ? flag : &health_sink);
    t.drain();
}

template <int S, int TX, int TY>
int launch_step_staged_t(dbm_handle *h, const CUtensorMap *tmap, const CUtensorMap *tmap_in, const void *fin,
                         void *fout, cudaStream_t st)
{
    constexpr size_t smem = (size_t)2 * (TX + 8) * (TY + 4) * Q * sizeof(float);
    static bool attr_set = false;  // per instantiation, set once per process
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_step_staged<S, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return set_cuda_error(h, e, "staged step kernel shared-memory attribute");
        attr_set = true;
    }
    StepConsts<float, S> c;
    fill_step_consts<float, S>(h, c);
    dim3 block(TX / 2, TY);
    dim3 grid((h->p.nx + TX - 1) / TX, (h->p.ny + TY - 1) / TY);
    k_step_staged<S, TX, TY><<<grid, block, smem, st>>>(c, *tmap, *tmap_in, (const float *)fin, (float *)fout,
                                                         (unsigned *)h->scratch);
    return set_cuda_error(h, cudaGetLastError(), "staged step kernel launch");
}

}  // namespace dbm
