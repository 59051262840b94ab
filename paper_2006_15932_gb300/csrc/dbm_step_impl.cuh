// dbm_step_impl.cuh -- the fused per-timestep update of the D2V16 DBM (FP32).
//
// One thread owns one cell and computes (section "Discrete Boltzmann model"
// and section "Numerical simulation" of arXiv 2006.15932):
//   1. species moments n^s, n^s u^s, E^s = sum f (v.v + eta^2) by ring sums;
//   2. mixture u, T for which the collision conserves momentum and energy
//      (the energy-minus-kinetic subtraction of T in FP64);
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
// or from a shared-memory tile that one TMA bulk copy filled (k_step_tma);
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

#include "dbm_consts.h"
#include "dbm_device.cuh"

namespace dbm {

// Stencil values of one cell straight from global memory (read-only path).
struct GlobalTile {
    const float *base;  // plane 0, row y + GY, column x + GX
    long long P;        // plane stride
    long long py;       // row stride
    __device__ __forceinline__ float ld(int p, int dx, int dy) const { return __ldg(base + p * P + dy * py + dx); }
};

// Stencil values of one cell from a shared-memory tile [plane][row][column].
struct SmemTile {
    const float *base;  // plane 0, this thread's row and column
    int P, py;
    __device__ __forceinline__ float ld(int p, int dx, int dy) const { return base[p * P + dy * py + dx]; }
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
template <typename real, class K>
__device__ __forceinline__ void solve_blocks(const K &k, int s, const real c[16], real o[16])
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
__device__ __forceinline__ float mixture_T(float W, float w, float wd, float ux, float uy)
{
    const float u2 = ux * ux + uy * uy;
    const float p = __fmul_rn(u2, w);
    const float pe = fmaf(u2, w, -p);
    const float s = __fsub_rn(W, p);
    const float bb = __fsub_rn(s, W);
    const float se = __fadd_rn(__fsub_rn(W, __fsub_rn(s, bb)), __fsub_rn(-p, bb));
    return __fadd_rn(s, __fsub_rn(se, pe)) / wd;
}

// Where the cell sits and which ghost images its values must also reach.
struct Site {
    int x, y;
    unsigned mx, my;
    long long cell;  // element offset of (x, y) in a plane
};

// Output of the FP32 state: f^{n+1}, and the ghost images of a species
// after all 16 of its values are stored (the thread re-reads its own
// stores: no registers held across the species loop).
struct StateOut {
    static constexpr bool kNoImages = false;
    float *f;  // plane 0 of the output buffer
    long long P;
    int nx, ny, pitch;
    __device__ __forceinline__ void put(const Site &w, int p, float g, float) const
    {
        __stcs(f + (long long)p * P + w.cell, g);  // streamed: not re-read this step
    }
    __device__ __forceinline__ void put_n(const Site &, int, float) const {}
    __device__ __forceinline__ void put_mix(const Site &, float, float, float) const {}
    __device__ __forceinline__ void images(const Site &w, int s) const
    {
        for (int i = 0; i < Q; ++i) {
            float *pl = f + (long long)(s * Q + i) * P;
            store_images(pl, w.x, w.y, nx, ny, pitch, w.mx, w.my, pl[w.cell]);
        }
    }
    __device__ __forceinline__ void images_mix(const Site &) const {}
};

// Output of the TMA-staged FP32 steps: f^{n+1} only.  These kernels never
// read the stored ghost cells (a tile at the domain boundary takes its halo
// from the interior, fill_tile_halo), so they do not write them either.
struct StateOutNoImages {
    static constexpr bool kNoImages = true;
    float *f;  // plane 0 of the output buffer
    long long P;
    __device__ __forceinline__ void put(const Site &w, int p, float g, float) const
    {
        __stcs(f + (long long)p * P + w.cell, g);
    }
    __device__ __forceinline__ void put_n(const Site &, int, float) const {}
    __device__ __forceinline__ void put_mix(const Site &, float, float, float) const {}
    __device__ __forceinline__ void images(const Site &, int) const {}
    __device__ __forceinline__ void images_mix(const Site &) const {}
};

// The whole update of cell (x, y).  `c` supplies the constants the cell
// uses many times (equilibrium blocks, ring speeds, weights, advection
// numbers); `g` the ones it uses once or twice (grid geometry and
// boundaries, reaction and force).  The single-problem kernels pass the same
// parameter block twice; the batched kernel passes the launch's shared
// constants as `c`, so that they stay constant-bank operands, and each
// instance's own block as `g`.
template <int S, class K, class G, class Tile, class Out>
__device__ __forceinline__ void step_cell(const K &c, const G &g, const Tile &t, int x, int y, const Out &out,
                                          unsigned *__restrict__ flag)
{
    // 1. species moments, by ring sums
    float n[S], cap = 0, nf = 0, no = 0;
    float w = 0, wx = 0, wy = 0, we = 0, wd = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        float sn = 0, sx = 0, sy = 0, se = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float rs = 0, rx = 0, ry = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = 4 * r + k;
                const float f = t.ld(s * Q + i, 0, 0);
                rs += f;
                if (dir_x(i) > 0) rx += f;
                if (dir_x(i) < 0) rx -= f;
                if (dir_y(i) > 0) ry += f;
                if (dir_y(i) < 0) ry -= f;
            }
            sn += rs;
            sx += c.vr[s][r] * rx;
            sy += c.vr[s][r] * ry;
            se += c.qr[s][r] * rs;
        }
        n[s] = sn;
        if (s == g.fuel) nf = sn;  // selects, no runtime-indexed register array
        if (s == g.oxid) no = sn;
        const float lh = c.lam_h[s], ll = c.lam_l[s], kh = c.kap_h[s], kl = c.kap_l[s];
        w += lh * sn + ll * sn;
        wx += lh * sx + ll * sx;
        wy += lh * sy + ll * sy;
        we += lh * se + ll * se;
        wd += kh * sn + kl * sn;
        cap += c.dpi[s] * sn;
    }

    // 2. mixture velocity and temperature
    const float rw = 1.0f / w;
    const float ux = wx * rw, uy = wy * rw;
    const float T = mixture_T(we, w, wd, ux, uy);

    unsigned bad = 0;
    float a = 0;  // sum_s |n^s|
#pragma unroll
    for (int s = 0; s < S; ++s) a += fabsf(n[s]);
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (!(n[s] >= -1e-6f * a)) bad |= DBM_HEALTH_DENSITY;
    if (!(a > 0.0f)) bad |= DBM_HEALTH_DENSITY;
    if (!(T > 0.0f)) bad |= DBM_HEALTH_TEMPERATURE;
    if (!isfinite(T + ux + uy)) bad |= DBM_HEALTH_NONFINITE;

    // 3. reaction: omega_ov and T' (state after a time tau^s)
    float om = 0.0f, dT = 0.0f;
    if (g.has_reaction) {
        om = g.k_ov * nf * no * expf(-g.Ea_over_R / T);
        dT = (g.Qheat - 0.5f * T * g.src) * om / (0.5f * cap);
    }

    Site w_;
    w_.x = x;
    w_.y = y;
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
        float f0[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f0[i] = t.ld(s * Q + i, 0, 0);
        // species density from step 1 (selected, not indexed)
        float ns = n[0];
#pragma unroll
        for (int j = 1; j < S; ++j)
            if (s == j) ns = n[j];
        out.put_n(w_, s, ns);
        // 4. merged equilibrium moments
        float cb[16];
        {
            float nr = ns, Ts = T;
            if (g.has_reaction) {
                nr = ns + g.tau_a[s] * om;
                if (nr < -1e-6f * a) bad |= DBM_HEALTH_NSTAR;
                Ts = T + g.tau_d[s] * dT;
            }
            fhat_blocks<float>(nr, ux, uy, Ts * c.inv_m[s], c.dpi[s], cb);
            if (g.has_force && ns != 0.0f) {  // an absent species feels no force
                float jx = 0, jy = 0, e = 0;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    const float v = c.vr[s][i >> 2];
                    jx += (dir_x(i) * v) * f0[i];
                    jy += (dir_y(i) * v) * f0[i];
                    e += c.qr[s][i >> 2] * f0[i];
                }
                const float usx = jx / ns, usy = jy / ns;
                const float th = (e / ns - (usx * usx + usy * usy)) / c.dpi[s];
                float fd[16], fs[16];  // f-hat at u-dagger and at u^s
                fhat_blocks<float>(ns, usx + g.accel_x * c.tau[s], usy + g.accel_y * c.tau[s], th, c.dpi[s], fd);
                fhat_blocks<float>(ns, usx, usy, th, c.dpi[s], fs);
#pragma unroll
                for (int k = 0; k < 16; ++k) cb[k] += fd[k] - fs[k];
            }
        }
        float o[16];
        solve_blocks<float>(c, s, cb, o);
        const float dtt = c.dt_tau[s];

#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int p = s * Q + i, r = i >> 2;
            float d = 0;  // dt v . grad f
            // 5. NND advection
            if (dir_x(i) > 0)
                d += c.cdx[s][r] * nnd_diff_pos(t.ld(p, -2, 0), t.ld(p, -1, 0), f0[i], t.ld(p, 1, 0));
            else if (dir_x(i) < 0)
                d -= c.cdx[s][r] * nnd_diff_neg(t.ld(p, -1, 0), f0[i], t.ld(p, 1, 0), t.ld(p, 2, 0));
            if (dir_y(i) > 0)
                d += c.cdy[s][r] * nnd_diff_pos(t.ld(p, 0, -2), t.ld(p, 0, -1), f0[i], t.ld(p, 0, 1));
            else if (dir_y(i) < 0)
                d -= c.cdy[s][r] * nnd_diff_neg(t.ld(p, 0, -1), f0[i], t.ld(p, 0, 1), t.ld(p, 0, 2));
            // 6. forward Euler: f + dt/tau (f^eq,tot - f) - dt v . grad f
            const float e = feq_of<float>(i, o);
            const float f1 = f0[i] + dtt * (e - f0[i]) - d;
            out.put(w_, p, f1, e);
        }
        if (images) out.images(w_, s);
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
    StateOut o{fout, c.plane, c.nx, c.ny, c.pitch};
    step_cell<S>(c, c, t, x, y, o, flag);
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

// Issue the tile copy (leader thread): box origin column bx0 (= bx0 + GX - 4),
// row by0 (= by0 + GY - 2), plane 0.
__device__ __forceinline__ void tma_tile_load(float *tile, unsigned long long tmap, int bx0, int by0,
                                              unsigned bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(tile)),
        "l"(tmap), "r"(bx0), "r"(by0), "r"(0), "r"(bar)
        : "memory");
}

// Halo of a tile that touches the domain boundary, taken from the interior
// of the input state (periodic: the wrapped cells; outflow: the edge cell)
// instead of from stored ghost cells.  The tile holds global columns
// bx0-4 .. bx0+TX+3 and rows by0-2 .. by0+TY+1 of all NP planes; only the
// cross-shaped stencil reaches into the halo, so the x halo is needed in the
// tile's interior rows and the y halo in its interior columns.  All threads
// of the CTA call this (it ends with a barrier when it wrote anything).
template <int NP, int TX, int TY>
__device__ __forceinline__ void fill_tile_halo(float *tile, const float *__restrict__ fin, int bx0, int by0, int nx,
                                               int ny, int pitch, long long plane, int bc_x, int bc_y, int tid,
                                               int nthr)
{
    constexpr int BX = TX + 8, PS = (TY + 4) * BX;
    // interior cells of the tile: columns bx0 .. x_hi-1, rows by0 .. y_hi-1;
    // their stencil reads columns bx0-2 .. x_hi+1 and rows by0-2 .. y_hi+1,
    // so only the ghost columns {-2, -1, nx, nx+1} and rows {-2, -1, ny,
    // ny+1} inside those ranges are filled (tile column = x - bx0 + 4 stays
    // within 2 .. TX+5, tile row = y - by0 + 2 within 0 .. TY+3)
    const int x_hi = min(bx0 + TX, nx), y_hi = min(by0 + TY, ny);
    const int left = bx0 == 0 ? 2 : 0, right = min(max(x_hi - nx + 2, 0), 2);
    const int top = by0 == 0 ? 2 : 0, bottom = min(max(y_hi - ny + 2, 0), 2);
    if (left + right + top + bottom == 0) return;  // uniform over the CTA
    // x halo, rows by0 .. y_hi-1
    const int ncx = left + right, rows = y_hi - by0;
    const int nxi = ncx * rows * NP;
    for (int it = tid; it < nxi; it += nthr) {
        const int cidx = it % ncx, r = (it / ncx) % rows, p = it / (ncx * rows);
        const int xg = cidx < left ? cidx - 2 : nx + (cidx - left);
        const int xs = bc_x == DBM_BC_PERIODIC ? ((xg % nx) + nx) % nx : min(max(xg, 0), nx - 1);
        const int y = by0 + r;
        tile[p * PS + (y - by0 + 2) * BX + (xg - bx0 + 4)] =
            fin[(long long)p * plane + (long long)(y + GY) * pitch + (xs + GX)];
    }
    // y halo, columns bx0 .. x_hi-1
    const int nry = top + bottom, cols = x_hi - bx0;
    const int nyi = nry * cols * NP;
    for (int it = tid; it < nyi; it += nthr) {
        const int c = it % cols, ridx = (it / cols) % nry, p = it / (cols * nry);
        const int yg = ridx < top ? ridx - 2 : ny + (ridx - top);
        const int ys = bc_y == DBM_BC_PERIODIC ? ((yg % ny) + ny) % ny : min(max(yg, 0), ny - 1);
        const int x = bx0 + c;
        tile[p * PS + (yg - by0 + 2) * BX + (x - bx0 + 4)] =
            fin[(long long)p * plane + (long long)(ys + GY) * pitch + (x + GX)];
    }
    __syncthreads();
}

template <int S, int TX, int TY>
__global__ void __launch_bounds__(TX *TY, tma_ctas_per_sm(S, TX, TY))
    k_step_tma(const __grid_constant__ StepConsts<float, S> c, const __grid_constant__ CUtensorMap tmap,
               const float *__restrict__ fin, float *__restrict__ fout, unsigned *__restrict__ flag)
{
    constexpr int BX = TX + 8, BY = TY + 4, NP = S * Q;
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
    const bool ok = mbar_wait(b, 0, TMA_WAIT_LIMIT);
    if (__syncthreads_or(!ok)) {
        // the copy did not land: report, give it one more bounded wait so
        // that no copy is left writing into this block's shared memory, and
        // leave together
        if (leader) raise_flag(flag, DBM_HEALTH_TIMEOUT);
        mbar_wait(b, 0, TMA_WAIT_LIMIT);
        return;
    }
    fill_tile_halo<NP, TX, TY>(tile, fin, bx0, by0, c.nx, c.ny, c.pitch, c.plane, c.bc_x, c.bc_y, ty * TX + tx,
                               TX * TY);
    const int x = bx0 + tx, y = by0 + ty;
    if (x >= c.nx || y >= c.ny) return;
    SmemTile t;
    t.base = tile + (ty + 2) * BX + (tx + 4);
    t.P = BY * BX;
    t.py = BX;
    StateOutNoImages o{fout, c.plane};
    step_cell<S>(c, c, t, x, y, o, flag);
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

template <int S, int TX, int TY>
int launch_step_tma_t(dbm_handle *h, const CUtensorMap *tmap, const void *fin, void *fout, cudaStream_t st)
{
    constexpr size_t smem = (size_t)(TX + 8) * (TY + 4) * S * Q * sizeof(float);
    static bool attr_set = false;  // per instantiation, set once per process
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_step_tma<S, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return set_cuda_error(h, e, "TMA step kernel shared-memory attribute");
        attr_set = true;
    }
    StepConsts<float, S> c;
    fill_step_consts<float, S>(h, c);
    dim3 block(TX, TY);
    dim3 grid((h->p.nx + TX - 1) / TX, (h->p.ny + TY - 1) / TY);
    k_step_tma<S, TX, TY><<<grid, block, smem, st>>>(c, *tmap, (const float *)fin, (float *)fout,
                                                       (unsigned *)h->scratch);
    return set_cuda_error(h, cudaGetLastError(), "TMA step kernel launch");
}

}  // namespace dbm
