// dbm_aux_impl.cuh -- kernels of the initialisation, state transfer and
// FP64 output calls of the D2V16 DBM (f = f^eq from macroscopic fields, the
// macroscopic fields, the nonequilibrium moments of Eqs. Delta2, Delta31,
// Delta3, Delta42, the conserved totals), and their launches for one species
// count S.  dbm_aux_s<S>.cu instantiates the launches per S so that the
// units compile in parallel; dbm_aux.cu dispatches on S.
#pragma once
#include <stdio.h>

#include "dbm_bf16.cuh"

namespace dbm {

// f = f^eq(rho^s / m^s, u, T), computed in FP64 and rounded to `real`.
template <typename real, int S>
__global__ void __launch_bounds__(256)
    k_set_state(const __grid_constant__ OutConsts<S> c, real *__restrict__ f,
                const double *__restrict__ rho_s, const double *__restrict__ ux,
                const double *__restrict__ uy, const double *__restrict__ T)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= c.nx || y >= c.ny) return;
    const long long N = (long long)c.nx * c.ny;
    const long long d = (long long)y * c.nx + x;
    const long long cell = (long long)(y + GY) * c.pitch + (x + GX);
    const Images im = cell_images(x, y, c.nx, c.ny, c.bc_x, c.bc_y);
    const double u_x = ux[d], u_y = uy[d], t = T[d];
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
        double fh[Q];
        fhat16<double>(rho_s[s * N + d] / c.m[s], u_x, u_y, t / c.m[s], c.dpi[s], fh);
        for (int i = 0; i < Q; ++i) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) v += c.cinv[s][i][k] * fh[k];
            store_with_images(f + (s * Q + i) * c.plane, cell, x, y, c.pitch, im, (real)v);
        }
    }
}

// 1 / m^s in FP64, for the conversion of the FP64 input fields.
template <int S>
struct InvMass {
    double v[S];
};

// FP32 storage: f = f^eq(rho^s / m^s, u, T) by the step kernel's own FP32
// symmetry-block solve (with its projection onto exact mass, momentum and
// energy): the state starts as the equilibrium the FP32 step itself builds,
// at a fraction of the cost of the FP64 matrix product (a few float ulps
// from the correctly rounded FP64 equilibrium).
template <int S>
__global__ void __launch_bounds__(256)
    k_set_state_blocks(const __grid_constant__ StepConsts<float, S> c, float *__restrict__ f,
                       const double *__restrict__ rho_s, const double *__restrict__ ux,
                       const double *__restrict__ uy, const double *__restrict__ T, const __grid_constant__ InvMass<S> im_d)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= c.nx || y >= c.ny) return;
    const long long N = (long long)c.nx * c.ny;
    const long long d = (long long)y * c.nx + x;
    const long long cell = (long long)(y + GY) * c.pitch + (x + GX);
    const Images im = cell_images(x, y, c.nx, c.ny, c.bc_x, c.bc_y);
    const float u_x = (float)ux[d], u_y = (float)uy[d];
    const double t = T[d];
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
        float cb[16], o[16];
        fhat_blocks<float>((float)(rho_s[s * N + d] * im_d.v[s]), u_x, u_y, (float)(t * im_d.v[s]), c.dpi[s], cb);
        solve_blocks<float>(c, s, cb, o);
        for (int i = 0; i < Q; ++i)
            store_with_images(f + (s * Q + i) * c.plane, cell, x, y, c.pitch, im, feq_of<float>(i, o));
    }
}

// Source of f for the output kernels: a plain FP64 or FP32 state buffer
// (the BF16-deviation state has BfSrc, which rebuilds f).
template <typename real>
struct PlainSrc {
    const real *f;
    long long plane;
    __device__ __forceinline__ void load16(int s, long long cell, double v[Q]) const
    {
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = (double)f[(s * Q + i) * plane + cell];
    }
    __device__ __forceinline__ void load16f(int s, long long cell, float v[Q]) const
    {
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = (float)f[(s * Q + i) * plane + cell];
    }
};

// Species moments of one cell in FP64: n, j = sum f v, E = sum f (v.v+eta^2).
template <int S, class Src>
__device__ __forceinline__ void cell_moments(const OutConsts<S> &c, const Src &src, long long cell,
                                             double n[S], double jx[S], double jy[S], double en[S])
{
#pragma unroll
    for (int s = 0; s < S; ++s) {
        double sn = 0, sx = 0, sy = 0, se = 0;
        double fv[Q];
        src.load16(s, cell, fv);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double v = fv[i];
            const int r = i >> 2;
            sn += v;
            sx += dir_x(i) * c.vr[s][r] * v;
            sy += dir_y(i) * c.vr[s][r] * v;
            se += c.qr[s][r] * v;
        }
        n[s] = sn;
        jx[s] = sx;
        jy[s] = sy;
        en[s] = se;
    }
}

template <int S>
__device__ __forceinline__ void cell_mixture(const OutConsts<S> &c, const double n[S],
                                             const double jx[S], const double jy[S],
                                             const double en[S], double &ux, double &uy, double &T)
{
    double w = 0, wx = 0, wy = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        w += c.m[s] * n[s] * c.inv_tau[s];
        wx += c.m[s] * jx[s] * c.inv_tau[s];
        wy += c.m[s] * jy[s] * c.inv_tau[s];
    }
    ux = wx / w;
    uy = wy / w;
    const double u2 = ux * ux + uy * uy;
    double num = 0, den = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        num += (c.m[s] * en[s] - c.m[s] * n[s] * u2) * c.inv_tau[s];
        den += n[s] * c.dpi[s] * c.inv_tau[s];
    }
    T = num / den;
}

template <int S, class Src>
__global__ void __launch_bounds__(256)
    k_moments(const __grid_constant__ OutConsts<S> c, const __grid_constant__ Src src,
              double *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= c.nx || y >= c.ny) return;
    const long long N = (long long)c.nx * c.ny;
    const long long d = (long long)y * c.nx + x;
    const long long cell = (long long)(y + GY) * c.pitch + (x + GX);
    double n[S], jx[S], jy[S], en[S];
    cell_moments<S>(c, src, cell, n, jx, jy, en);
    double rho = 0, ntot = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        // an absent species (n = 0) reports zero velocity and temperature
        const bool here = n[s] != 0.0;
        const double usx = here ? jx[s] / n[s] : 0.0, usy = here ? jy[s] / n[s] : 0.0;
        out[(4 * s + 0) * N + d] = n[s];
        out[(4 * s + 1) * N + d] = usx;
        out[(4 * s + 2) * N + d] = usy;
        out[(4 * s + 3) * N + d] =
            here ? c.m[s] * (en[s] / n[s] - (usx * usx + usy * usy)) / c.dpi[s] : 0.0;
        rho += c.m[s] * n[s];
        ntot += n[s];
    }
    double ux, uy, T;
    cell_mixture<S>(c, n, jx, jy, en, ux, uy, T);
    out[(4 * S + 0) * N + d] = rho;
    out[(4 * S + 1) * N + d] = ux;
    out[(4 * S + 2) * N + d] = uy;
    out[(4 * S + 3) * N + d] = T;
    out[(4 * S + 4) * N + d] = ntot * T;
}

// The macroscopic fields of a float state (DBM_FP32 or DBM_BF16DEV), in
// float arithmetic, stored as FP64: the state carries float precision, and
// on this GPU the FP64 evaluation of k_moments is bound by the FP64 pipe (8 ms
// for 4096^2 cells against 0.6 ms for the memory traffic).  Species sums by
// rings as in the step; the mixture temperature's cancelling subtraction in
// float-float (mixture_T); u^s and T^s from n^s, j^s, E^s with one fused
// multiply-add each.  Relative error a few float ulps of each field.
template <int S, class Src>
__global__ void __launch_bounds__(256)
    k_moments_f32(const __grid_constant__ OutConsts<S> c, const __grid_constant__ Src src,
                  double *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= c.nx || y >= c.ny) return;
    const long long N = (long long)c.nx * c.ny;
    const long long d = (long long)y * c.nx + x;
    const long long cell = (long long)(y + GY) * c.pitch + (x + GX);
    float rho = 0.0f, ntot = 0.0f, w = 0.0f, wx = 0.0f, wy = 0.0f, we = 0.0f, wd = 0.0f;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        float f[Q];
        src.load16f(s, cell, f);
        float sn = 0.0f, sx = 0.0f, sy = 0.0f, se = 0.0f;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const float f0 = f[4 * r], f1 = f[4 * r + 1], f2 = f[4 * r + 2], f3 = f[4 * r + 3];
            const float rs = (f0 + f2) + (f1 + f3);
            float rx, ry;
            if ((r & 1) == 0) {
                rx = f0 - f2;
                ry = f1 - f3;
            } else {
                const float a = f0 - f2, b = f3 - f1;
                rx = a + b;
                ry = a - b;
            }
            const float v = (float)c.vr[s][r];
            sn += rs;
            sx = fmaf(v, rx, sx);
            sy = fmaf(v, ry, sy);
            se = fmaf((float)c.qr[s][r], rs, se);
        }
        const bool here = sn != 0.0f;  // an absent species reports zero velocity and temperature
        const float rn = here ? 1.0f / sn : 0.0f;
        const float usx = sx * rn, usy = sy * rn;
        const float ts = here ? (float)c.m[s] * fmaf(-usx, usx, fmaf(-usy, usy, se * rn)) / (float)c.dpi[s] : 0.0f;
        out[(4 * s + 0) * N + d] = sn;
        out[(4 * s + 1) * N + d] = usx;
        out[(4 * s + 2) * N + d] = usy;
        out[(4 * s + 3) * N + d] = ts;
        const float m = (float)c.m[s], lam = (float)(c.m[s] * c.inv_tau[s]);
        const float kap = (float)(c.dpi[s] * c.inv_tau[s]);
        rho = fmaf(m, sn, rho);
        ntot += sn;
        w = fmaf(lam, sn, w);
        wx = fmaf(lam, sx, wx);
        wy = fmaf(lam, sy, wy);
        we = fmaf(lam, se, we);
        wd = fmaf(kap, sn, wd);
    }
    const float rw = 1.0f / w, ux = wx * rw, uy = wy * rw;
    const float T = mixture_T(we, w, wd, ux, uy);
    out[(4 * S + 0) * N + d] = rho;
    out[(4 * S + 1) * N + d] = ux;
    out[(4 * S + 2) * N + d] = uy;
    out[(4 * S + 3) * N + d] = T;
    out[(4 * S + 4) * N + d] = (double)ntot * (double)T;
}

template <int S, class Src>
__global__ void __launch_bounds__(128)
    k_noneq(const __grid_constant__ OutConsts<S> c, const __grid_constant__ Src src,
            double *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= c.nx || y >= c.ny) return;
    const long long N = (long long)c.nx * c.ny;
    const long long d = (long long)y * c.nx + x;
    const long long cell = (long long)(y + GY) * c.pitch + (x + GX);
    double n[S], jx[S], jy[S], en[S];
    cell_moments<S>(c, src, cell, n, jx, jy, en);
    double ux, uy, T;
    cell_mixture<S>(c, n, jx, jy, en, ux, uy, T);
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
        double fh[Q];
        fhat16<double>(n[s], ux, uy, T / c.m[s], c.dpi[s], fh);
        double acc[20];
#pragma unroll
        for (int k = 0; k < 20; ++k) acc[k] = 0.0;
        const double m = c.m[s];
        double fc[Q];
        src.load16(s, cell, fc);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            double feq = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) feq += c.cinv[s][i][k] * fh[k];
            const int r = i >> 2;
            const double vx = dir_x(i) * c.vr[s][r], vy = dir_y(i) * c.vr[s][r];
            const double q = c.qr[s][r];
            const double fv = fc[i];
            const double dm = m * (fv - feq), mf = 0.5 * m * fv, me = 0.5 * m * feq;
            acc[0] += dm * vx * vx;
            acc[1] += dm * vx * vy;
            acc[2] += dm * vy * vy;
            acc[3] += dm * q * vx;
            acc[4] += dm * q * vy;
            acc[5] += dm * vx * vx * vx;
            acc[6] += dm * vx * vx * vy;
            acc[7] += dm * vx * vy * vy;
            acc[8] += dm * vy * vy * vy;
            acc[9] += dm * q * vx * vx;
            acc[10] += dm * q * vx * vy;
            acc[11] += dm * q * vy * vy;
            acc[12] += mf * vx * vx;
            acc[13] += mf * vy * vy;
            acc[14] += me * vx * vx;
            acc[15] += me * vy * vy;
            acc[16] += mf * q * vx;
            acc[17] += mf * q * vy;
            acc[18] += me * q * vx;
            acc[19] += me * q * vy;
        }
#pragma unroll
        for (int k = 0; k < 20; ++k) out[(20 * s + k) * N + d] = acc[k];
    }
}

// Conserved totals: each block sums a fixed, strided subset of cells in a
// fixed order and reduces them by a fixed tree; the final kernel adds the
// block partials in block order.  The result is independent of timing.
template <int S, class Src>
__global__ void __launch_bounds__(256)
    k_cons_partial(const __grid_constant__ OutConsts<S> c, const __grid_constant__ Src src,
                   double *__restrict__ partial)
{
    constexpr int K = S + 4;
    __shared__ double red[K][256];
    double acc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = 0.0;
    const long long N = (long long)c.nx * c.ny;
    for (long long d = (long long)blockIdx.x * blockDim.x + threadIdx.x; d < N;
         d += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(d % c.nx), y = (int)(d / c.nx);
        const long long cell = (long long)(y + GY) * c.pitch + (x + GX);
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const double m = c.m[s];
            double fv[Q];
            src.load16(s, cell, fv);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const double v = fv[i];
                const int r = i >> 2;
                acc[s] += m * v;
                acc[S] += m * v * (dir_x(i) * c.vr[s][r]);
                acc[S + 1] += m * v * (dir_y(i) * c.vr[s][r]);
                acc[S + 2] += 0.5 * m * v * c.qr[s][r];
                if (c.has_reaction && s == c.fuel) acc[S + 3] += c.Qheat * v / c.abs_a_fuel;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) red[k][threadIdx.x] = acc[k];
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < K; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < K) partial[blockIdx.x * K + threadIdx.x] = red[threadIdx.x][0];
}

static __global__ void k_cons_final(const double *__restrict__ partial, int nblocks, int K,
                             double *__restrict__ out)
{
    const int k = threadIdx.x;
    if (k >= K) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[b * K + k];
    out[k] = s;
}

inline dim3 cell_grid(const dbm_handle *h, dim3 block)
{
    return dim3((h->p.nx + block.x - 1) / block.x, (h->p.ny + block.y - 1) / block.y);
}

template <typename real, int S>
inline void set_state_t(dbm_handle *h, void *f, const double *rho_s, const double *ux,
                        const double *uy, const double *T, cudaStream_t st)
{
    dim3 b(32, 8);
    if (sizeof(real) == 4) {
        StepConsts<float, S> c;
        fill_step_consts<float, S>(h, c);
        InvMass<S> im;
        for (int s = 0; s < S; ++s) im.v[s] = 1.0 / h->p.sp[s].m;
        k_set_state_blocks<S><<<cell_grid(h, b), b, 0, st>>>(c, (float *)f, rho_s, ux, uy, T, im);
        return;
    }
    OutConsts<S> c;
    fill_out_consts<S>(h, c);
    k_set_state<real, S><<<cell_grid(h, b), b, 0, st>>>(c, (real *)f, rho_s, ux, uy, T);
}

// The source of f for a state buffer of this handle's precision.
template <typename real, int S>
inline PlainSrc<real> plain_src(const dbm_handle *h, const void *f)
{
    return PlainSrc<real>{(const real *)f, h->lay.plane};
}
template <int S>
inline BfSrc<S> bf_src(const dbm_handle *h, const void *f)
{
    BfSrc<S> b;
    fill_step_consts<float, S>(h, b.k);
    b.st = bf_state(h, (void *)f);
    return b;
}

template <int S, class Src>
inline void moments_t(dbm_handle *h, const Src &src, double *out, cudaStream_t st)
{
    OutConsts<S> c;
    fill_out_consts<S>(h, c);
    dim3 b(32, 8);
    if (h->p.precision == DBM_FP64)
        k_moments<S, Src><<<cell_grid(h, b), b, 0, st>>>(c, src, out);
    else
        k_moments_f32<S, Src><<<cell_grid(h, b), b, 0, st>>>(c, src, out);
}

template <int S, class Src>
inline void noneq_t(dbm_handle *h, const Src &src, double *out, cudaStream_t st)
{
    OutConsts<S> c;
    fill_out_consts<S>(h, c);
    dim3 b(32, 4);
    k_noneq<S, Src><<<cell_grid(h, b), b, 0, st>>>(c, src, out);
}

template <int S, class Src>
inline void cons_t(dbm_handle *h, const Src &src, double *partial, double *out, cudaStream_t st)
{
    OutConsts<S> c;
    fill_out_consts<S>(h, c);
    k_cons_partial<S, Src><<<CONS_BLOCKS, 256, 0, st>>>(c, src, partial);
    k_cons_final<<<1, 32, 0, st>>>(partial, CONS_BLOCKS, S + 4, out);
}


// The launches of one species count, dispatching on the handle's precision
// (the BF16-deviation state exists for S <= 4).
template <int S>
void aux_set_state(dbm_handle *h, void *f, const double *rho_s, const double *ux, const double *uy, const double *T,
                   cudaStream_t st)
{
    if (h->p.precision == DBM_FP64)
        set_state_t<double, S>(h, f, rho_s, ux, uy, T, st);
    else
        set_state_t<float, S>(h, f, rho_s, ux, uy, T, st);
}

template <int S>
void aux_moments(dbm_handle *h, const void *f, double *out, cudaStream_t st)
{
    if (h->p.precision == DBM_FP64) {
        moments_t<S>(h, plain_src<double, S>(h, f), out, st);
    } else if (h->p.precision == DBM_FP32) {
        moments_t<S>(h, plain_src<float, S>(h, f), out, st);
    } else if constexpr (S <= 4) {
        moments_t<S>(h, bf_src<S>(h, f), out, st);
    }
}

template <int S>
void aux_noneq(dbm_handle *h, const void *f, double *out, cudaStream_t st)
{
    if (h->p.precision == DBM_FP64) {
        noneq_t<S>(h, plain_src<double, S>(h, f), out, st);
    } else if (h->p.precision == DBM_FP32) {
        noneq_t<S>(h, plain_src<float, S>(h, f), out, st);
    } else if constexpr (S <= 4) {
        noneq_t<S>(h, bf_src<S>(h, f), out, st);
    }
}

template <int S>
void aux_cons(dbm_handle *h, const void *f, double *partial, double *out, cudaStream_t st)
{
    if (h->p.precision == DBM_FP64) {
        cons_t<S>(h, plain_src<double, S>(h, f), partial, out, st);
    } else if (h->p.precision == DBM_FP32) {
        cons_t<S>(h, plain_src<float, S>(h, f), partial, out, st);
    } else if constexpr (S <= 4) {
        cons_t<S>(h, bf_src<S>(h, f), partial, out, st);
    }
}

}  // namespace dbm
