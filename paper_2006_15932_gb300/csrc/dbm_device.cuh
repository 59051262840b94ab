// dbm_device.cuh -- device building blocks of the D2V16 DBM step:
// the equilibrium moments f-hat, the minmod limiter of the NND scheme and
// the ghost-image bookkeeping of the boundary conditions.  The NND flux
// differences are in dbm_step_impl.cuh.
#pragma once

#include "dbm_internal.h"

namespace dbm {

// f-hat_1..16 of the moment relations (section "Discrete Boltzmann model",
// the f-hat list restating Eqs. relation1..relation7) at (n, u, theta = T/m)
// with dpi = D + I.  Factored for the GPU; the same polynomials as printed.
template <typename real>
__device__ __forceinline__ void fhat16(real n, real ux, real uy, real th, real dpi, real fh[Q])
{
    const real u2 = ux * ux + uy * uy;
    const real a2 = (dpi + real(2)) * th + u2;  // (D+I+2) T/m + u.u
    const real a4 = (dpi + real(4)) * th + u2;  // (D+I+4) T/m + u.u
    const real nux = n * ux, nuy = n * uy;
    const real xx = ux * ux, yy = uy * uy;
    fh[0] = n;
    fh[1] = nux;
    fh[2] = nuy;
    fh[3] = n * (dpi * th + u2);
    fh[4] = n * (th + xx);
    fh[5] = nux * uy;
    fh[6] = n * (th + yy);
    fh[7] = nux * a2;
    fh[8] = nuy * a2;
    fh[9] = nux * (real(3) * th + xx);
    fh[10] = nuy * (th + xx);
    fh[11] = nux * (th + yy);
    fh[12] = nuy * (real(3) * th + yy);
    fh[13] = n * (a2 * th + xx * a4);
    fh[14] = nux * uy * a4;
    fh[15] = n * (a2 * th + yy * a4);
}

// minmod(a, b): the argument of smaller magnitude when both have the same
// sign, else 0 (limiter of the NND scheme).
__device__ __forceinline__ double minmod(double a, double b)
{
    const double s = copysign(1.0, a);
    return s * fmax(fmin(fabs(a), s * b), 0.0);
}
__device__ __forceinline__ float minmod(float a, float b)
{
    // t = min(|a|, |b|) carrying the sign (sgn a) xor (sgn b): positive
    // exactly when a and b agree in sign
    float t;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(t) : "f"(a), "f"(b));
    return copysignf(fmaxf(t, 0.0f), a);
}

// Ghost images of interior index k along an axis of n cells: the ghost
// indices g in {-2, -1, n, n+1} whose source cell is k (periodic wrap, or
// the edge cell for outflow).  Returns the count (0..4) and the indices.
__device__ __forceinline__ int ghost_images(int k, int n, int bc, int g[4])
{
    int cnt = 0;
    const int cand[4] = {-2, -1, n, n + 1};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = cand[j];
        int src;
        if (bc == DBM_BC_PERIODIC)
            src = ((c % n) + n) % n;
        else
            src = c < 0 ? 0 : n - 1;
        if (src == k) g[cnt++] = c;
    }
    return cnt;
}

struct Images {
    int gx[4], gy[4];
    int ngx, ngy;
};

__device__ __forceinline__ Images cell_images(int x, int y, int nx, int ny, int bc_x, int bc_y)
{
    Images im;
    im.ngx = ghost_images(x, nx, bc_x, im.gx);
    im.ngy = ghost_images(y, ny, bc_y, im.gy);
    return im;
}

// Store v at interior cell (x, y) of plane base `pl` and at its ghost images.
template <typename T>
__device__ __forceinline__ void store_with_images(T *pl, long long cell, int x, int y, int pitch,
                                                  const Images &im, T v)
{
    pl[cell] = v;
    for (int j = 0; j < im.ngx; ++j) pl[(long long)(y + GY) * pitch + (im.gx[j] + GX)] = v;
    for (int j = 0; j < im.ngy; ++j) pl[(long long)(im.gy[j] + GY) * pitch + (x + GX)] = v;
}

__device__ __forceinline__ void raise_flag(unsigned *flag, unsigned bits)
{
    if (bits) atomicOr(flag, bits);
}

// Checked builds (-DDBM_CHECKED, a debugging aid that stands in for a
// memory checker): every index into a shared-memory tile, a state buffer or
// a ghost image is compared with the extent of what it addresses; one
// outside it raises DBM_HEALTH_BOUNDS and the access is skipped (a load
// gives 0).  The default build compiles the checks away.
__device__ __forceinline__ bool in_bounds(long long i, long long n, unsigned *flag)
{
#ifdef DBM_CHECKED
    if (i >= 0 && i < n) return true;
    raise_flag(flag, DBM_HEALTH_BOUNDS);
    return false;
#else
    return true;
#endif
}

}  // namespace dbm
