// dbm_aux.cu -- initialisation, raw state transfer and FP64 output kernels
// of the D2V16 DBM: f = f^eq from macroscopic fields, checkpoint load/read,
// the macroscopic fields, the nonequilibrium moments (Eqs. Delta2, Delta31,
// Delta3, Delta42) and the conserved totals.
#include <stdio.h>

#include <mutex>

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

template <typename real>
__global__ void __launch_bounds__(256)
    k_set_f(real *__restrict__ f, const double *__restrict__ src, int nplanes, int nx, int ny,
            int pitch, long long plane, int bc_x, int bc_y)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long N = (long long)nx * ny;
    const long long d = (long long)y * nx + x;
    const long long cell = (long long)(y + GY) * pitch + (x + GX);
    const Images im = cell_images(x, y, nx, ny, bc_x, bc_y);
    for (int p = 0; p < nplanes; ++p)
        store_with_images(f + p * plane, cell, x, y, pitch, im, (real)src[p * N + d]);
}

template <typename real>
__global__ void __launch_bounds__(256)
    k_get_f(const real *__restrict__ f, double *__restrict__ dst, int nplanes, int nx, int ny,
            int pitch, long long plane)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long N = (long long)nx * ny;
    const long long d = (long long)y * nx + x;
    const long long cell = (long long)(y + GY) * pitch + (x + GX);
    for (int p = 0; p < nplanes; ++p) dst[p * N + d] = (double)f[p * plane + cell];
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

__global__ void k_cons_final(const double *__restrict__ partial, int nblocks, int K,
                             double *__restrict__ out)
{
    const int k = threadIdx.x;
    if (k >= K) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += partial[b * K + k];
    out[k] = s;
}

static dim3 cell_grid(const dbm_handle *h, dim3 block)
{
    return dim3((h->p.nx + block.x - 1) / block.x, (h->p.ny + block.y - 1) / block.y);
}

// ---------------------------------------------------------------------------
// launchers (dispatch on precision and S)
// ---------------------------------------------------------------------------

#define DBM_DISPATCH_S(S_, CALL)             \
    switch (S_) {                            \
    case 1: { constexpr int S = 1; CALL; } break; \
    case 2: { constexpr int S = 2; CALL; } break; \
    case 3: { constexpr int S = 3; CALL; } break; \
    case 4: { constexpr int S = 4; CALL; } break; \
    case 5: { constexpr int S = 5; CALL; } break; \
    case 6: { constexpr int S = 6; CALL; } break; \
    case 7: { constexpr int S = 7; CALL; } break; \
    case 8: { constexpr int S = 8; CALL; } break; \
    default: return DBM_ERR_INVALID;         \
    }

#define DBM_DISPATCH_BF(S_, CALL)            \
    switch (S_) {                            \
    case 1: { constexpr int S = 1; CALL; } break; \
    case 2: { constexpr int S = 2; CALL; } break; \
    case 3: { constexpr int S = 3; CALL; } break; \
    case 4: { constexpr int S = 4; CALL; } break; \
    default: return DBM_ERR_INVALID;         \
    }

template <typename real, int S>
static void set_state_t(dbm_handle *h, void *f, const double *rho_s, const double *ux,
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

int launch_set_state(dbm_handle *h, void *f, const double *rho_s, const double *ux,
                     const double *uy, const double *T, cudaStream_t st)
{
    if (h->p.precision == DBM_FP64) {
        DBM_DISPATCH_S(h->p.nspecies, (set_state_t<double, S>(h, f, rho_s, ux, uy, T, st)));
    } else if (h->p.precision == DBM_FP32) {
        DBM_DISPATCH_S(h->p.nspecies, (set_state_t<float, S>(h, f, rho_s, ux, uy, T, st)));
    } else {
        return launch_set_state_bf16(h, f, rho_s, ux, uy, T, st);
    }
    return set_cuda_error(h, cudaGetLastError(), "set_state kernel launch");
}

int launch_set_f(dbm_handle *h, void *f, const double *src, cudaStream_t st)
{
    dim3 b(32, 8);
    const int np = h->p.nspecies * Q;
    if (h->p.precision == DBM_FP64)
        k_set_f<double><<<cell_grid(h, b), b, 0, st>>>((double *)f, src, np, h->p.nx, h->p.ny,
                                                       h->lay.pitch, h->lay.plane, h->p.bc_x, h->p.bc_y);
    else if (h->p.precision == DBM_FP32)
        k_set_f<float><<<cell_grid(h, b), b, 0, st>>>((float *)f, src, np, h->p.nx, h->p.ny,
                                                      h->lay.pitch, h->lay.plane, h->p.bc_x, h->p.bc_y);
    else
        return launch_set_f_bf16(h, f, src, st);
    return set_cuda_error(h, cudaGetLastError(), "set_f kernel launch");
}

int launch_get_f(dbm_handle *h, const void *f, double *dst, cudaStream_t st)
{
    dim3 b(32, 8);
    const int np = h->p.nspecies * Q;
    if (h->p.precision == DBM_FP64)
        k_get_f<double><<<cell_grid(h, b), b, 0, st>>>((const double *)f, dst, np, h->p.nx, h->p.ny,
                                                       h->lay.pitch, h->lay.plane);
    else if (h->p.precision == DBM_FP32)
        k_get_f<float><<<cell_grid(h, b), b, 0, st>>>((const float *)f, dst, np, h->p.nx, h->p.ny,
                                                      h->lay.pitch, h->lay.plane);
    else
        return launch_get_f_bf16(h, f, dst, st);
    return set_cuda_error(h, cudaGetLastError(), "get_f kernel launch");
}

// The source of f for a state buffer of this handle's precision.
template <typename real, int S>
static PlainSrc<real> plain_src(const dbm_handle *h, const void *f)
{
    return PlainSrc<real>{(const real *)f, h->lay.plane};
}
template <int S>
static BfSrc<S> bf_src(const dbm_handle *h, const void *f)
{
    BfSrc<S> b;
    fill_step_consts<float, S>(h, b.k);
    b.st = bf_state(h, (void *)f);
    return b;
}

template <int S, class Src>
static void moments_t(dbm_handle *h, const Src &src, double *out, cudaStream_t st)
{
    OutConsts<S> c;
    fill_out_consts<S>(h, c);
    dim3 b(32, 8);
    if (h->p.precision == DBM_FP64)
        k_moments<S, Src><<<cell_grid(h, b), b, 0, st>>>(c, src, out);
    else
        k_moments_f32<S, Src><<<cell_grid(h, b), b, 0, st>>>(c, src, out);
}

int launch_moments(dbm_handle *h, const void *f, double *out, cudaStream_t st)
{
    if (h->p.precision == DBM_FP64) {
        DBM_DISPATCH_S(h->p.nspecies, (moments_t<S>(h, plain_src<double, S>(h, f), out, st)));
    } else if (h->p.precision == DBM_FP32) {
        DBM_DISPATCH_S(h->p.nspecies, (moments_t<S>(h, plain_src<float, S>(h, f), out, st)));
    } else {
        DBM_DISPATCH_BF(h->p.nspecies, (moments_t<S>(h, bf_src<S>(h, f), out, st)));
    }
    return set_cuda_error(h, cudaGetLastError(), "moments kernel launch");
}

template <int S, class Src>
static void noneq_t(dbm_handle *h, const Src &src, double *out, cudaStream_t st)
{
    OutConsts<S> c;
    fill_out_consts<S>(h, c);
    dim3 b(32, 4);
    k_noneq<S, Src><<<cell_grid(h, b), b, 0, st>>>(c, src, out);
}

int launch_noneq(dbm_handle *h, const void *f, double *out, cudaStream_t st)
{
    if (h->p.precision == DBM_FP64) {
        DBM_DISPATCH_S(h->p.nspecies, (noneq_t<S>(h, plain_src<double, S>(h, f), out, st)));
    } else if (h->p.precision == DBM_FP32) {
        DBM_DISPATCH_S(h->p.nspecies, (noneq_t<S>(h, plain_src<float, S>(h, f), out, st)));
    } else {
        DBM_DISPATCH_BF(h->p.nspecies, (noneq_t<S>(h, bf_src<S>(h, f), out, st)));
    }
    return set_cuda_error(h, cudaGetLastError(), "nonequilibrium kernel launch");
}

template <int S, class Src>
static void cons_t(dbm_handle *h, const Src &src, double *partial, double *out, cudaStream_t st)
{
    OutConsts<S> c;
    fill_out_consts<S>(h, c);
    k_cons_partial<S, Src><<<CONS_BLOCKS, 256, 0, st>>>(c, src, partial);
    k_cons_final<<<1, 32, 0, st>>>(partial, CONS_BLOCKS, S + 4, out);
}

// Conserved totals into `out` with the block partials in `partial`.
static int conservation_into(dbm_handle *h, const void *f, double *partial, double *out, cudaStream_t st)
{
    if (h->p.precision == DBM_FP64) {
        DBM_DISPATCH_S(h->p.nspecies, (cons_t<S>(h, plain_src<double, S>(h, f), partial, out, st)));
    } else if (h->p.precision == DBM_FP32) {
        DBM_DISPATCH_S(h->p.nspecies, (cons_t<S>(h, plain_src<float, S>(h, f), partial, out, st)));
    } else {
        DBM_DISPATCH_BF(h->p.nspecies, (cons_t<S>(h, bf_src<S>(h, f), partial, out, st)));
    }
    return DBM_OK;
}

int launch_conservation(dbm_handle *h, const void *f, double *out, cudaStream_t st)
{
    double *partial = (double *)((char *)h->scratch + SCRATCH_HEAD);
    const int rc = conservation_into(h, f, partial, out, st);
    if (rc) return rc;
    return set_cuda_error(h, cudaGetLastError(), "conservation kernel launch");
}

// ---------------------------------------------------------------------------
// Conserved totals without a caller-provided scratch buffer.
//
// Some callers cannot allocate device memory at the point where they need
// the totals (for example a plug-in that runs inside a host application
// which owns all of the GPU's memory and forbids further allocations).  For
// them the block partials of the reduction live in this file-scope device
// array instead of the caller's scratch buffer.  Every GPU that loads the
// library holds the array until the process exits.  Host code must not
// pass the array's name to a kernel (on the host it is only a stand-in):
// its device address is looked up once per device with cudaGetSymbolAddress
// and cached.
// ---------------------------------------------------------------------------

static __device__ __align__(256) double g_noalloc_partials[DBM_NOALLOC_SCRATCH_DOUBLES];

static const int NOALLOC_MAX_DEVICES = 64;
static double *g_noalloc_addr[NOALLOC_MAX_DEVICES];
static std::mutex g_noalloc_mutex;

// Device address of g_noalloc_partials on the current device (looked up on
// the first call per device, with that device current).
static int noalloc_scratch(dbm_handle *h, double **out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(h, e, "conservation_noalloc: current device");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        snprintf(h->err, sizeof(h->err),
                 "conservation_noalloc: device ordinal %d outside the %d devices whose array address is cached", dev,
                 NOALLOC_MAX_DEVICES);
        return DBM_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_partials);
        if (e != cudaSuccess) return set_cuda_error(h, e, "conservation_noalloc: cudaGetSymbolAddress");
        g_noalloc_addr[dev] = (double *)ptr;
    }
    *out = g_noalloc_addr[dev];
    return DBM_OK;
}

int launch_conservation_noalloc(dbm_handle *h, const void *f, double *out, cudaStream_t st)
{
    const size_t need = (size_t)CONS_BLOCKS * (h->p.nspecies + 4);
    if (need > DBM_NOALLOC_SCRATCH_DOUBLES) return DBM_ERR_INVALID;
    double *partial = nullptr;
    int rc = noalloc_scratch(h, &partial);
    if (rc) return rc;
    // every block overwrites all of its partials, so nothing needs clearing
    rc = conservation_into(h, f, partial, out, st);
    if (rc) return rc;
    return set_cuda_error(h, cudaGetLastError(), "conservation_noalloc kernel launch");
}

}  // namespace dbm
