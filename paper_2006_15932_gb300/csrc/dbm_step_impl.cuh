// dbm_step_impl.cuh -- the fused per-timestep update of the D2V16 DBM.
//
// One thread owns one cell and, in one pass, computes (section "Discrete
// Boltzmann model" and section "Numerical simulation" of arXiv 2006.15932):
//   1. species moments n^s, n^s u^s, E^s = sum f (v.v + eta^2);
//   2. mixture u, T for which the collision conserves momentum and energy;
//   3. the one-step Arrhenius rate and the post-reaction n^s*, T*;
//   4. the merged equilibrium f^eq,tot = M^-1 [f-hat(n*, u, T*)
//      + f-hat(n, u^dag, T^s) - f-hat(n, u^s, T^s)], so that
//      Omega + R + G = (f^eq,tot - f) / tau (Eqs. CollisionTerm,
//      ReactionTerm, ForceTerm: f^eq is linear in f-hat);
//   5. the NND flux differences of v_i . grad f along x and y;
//   6. the forward-Euler update, stored to the other buffer together with
//      the ghost images the boundary conditions ask for.
#pragma once
#include "dbm_consts.h"
#include "dbm_device.cuh"

namespace dbm {

template <typename real, int S>
__global__ void __launch_bounds__(256)
    k_step(const __grid_constant__ StepConsts<real, S> c, const real *__restrict__ fin,
           real *__restrict__ fout, unsigned *__restrict__ flag)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= c.nx || y >= c.ny) return;
    const long long P = c.plane;
    const long long cell = (long long)(y + GY) * c.pitch + (x + GX);

    // 1. species moments, by ring sums
    real n[S], jx[S], jy[S], en[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        real sn = 0, sx = 0, sy = 0, se = 0;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            real rs = 0, rx = 0, ry = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int i = 4 * r + k;
                const real f = fin[(s * Q + i) * P + cell];
                rs += f;
                rx += dir_x(i) * f;
                ry += dir_y(i) * f;
            }
            sn += rs;
            sx += c.vr[s][r] * rx;
            sy += c.vr[s][r] * ry;
            se += c.qr[s][r] * rs;
        }
        n[s] = sn;
        jx[s] = sx;
        jy[s] = sy;
        en[s] = se;
    }

    // 2. mixture velocity and temperature (temperature always in FP64)
    real w = 0, wx = 0, wy = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const real mt = c.m[s] * c.inv_tau[s];
        w += mt * n[s];
        wx += mt * jx[s];
        wy += mt * jy[s];
    }
    const real ux = wx / w, uy = wy / w;
    const double u2 = (double)ux * (double)ux + (double)uy * (double)uy;
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        num += (c.m_d[s] * (double)en[s] - c.m_d[s] * (double)n[s] * u2) * c.inv_tau_d[s];
        den += (double)n[s] * c.dpi_d[s] * c.inv_tau_d[s];
    }
    const double Td = num / den;

    // health: a species may be absent (n = 0) or slightly negative from
    // numerical diffusion; flag densities below -1e-6 of the mixture
    unsigned bad = 0;
    real nabs = 0;
#pragma unroll
    for (int s = 0; s < S; ++s) nabs += fabs(n[s]);
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (!(n[s] >= real(-1e-6) * nabs)) bad |= DBM_HEALTH_DENSITY;
    if (!(nabs > real(0))) bad |= DBM_HEALTH_DENSITY;
    if (!(Td > 0.0)) bad |= DBM_HEALTH_TEMPERATURE;
    if (!isfinite(Td) || !isfinite((double)ux) || !isfinite((double)uy)) bad |= DBM_HEALTH_NONFINITE;

    // 3. reaction: omega_ov and T' (reading: state after a time tau^s)
    double omega = 0.0, dTdt = 0.0;
    if (c.has_reaction) {
        const double nf = (double)n[c.fuel], no = (double)n[c.oxid];
        omega = c.k_ov * nf * no * exp(-c.Ea_over_R / Td);
        double src = 0.0, cap = 0.0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            src += c.dpi_d[s] * c.a_d[s];
            cap += (double)n[s] * c.dpi_d[s];
        }
        dTdt = (c.Qheat - 0.5 * Td * src) * omega / (0.5 * cap);
    }

    const Images im = cell_images(x, y, c.nx, c.ny, c.bc_x, c.bc_y);

#pragma unroll
    for (int s = 0; s < S; ++s) {
        // 4. merged equilibrium moments
        real fh[Q];
        real ns = n[s];
        double Ts = Td;
        if (c.has_reaction) {
            const double nstar = (double)n[s] + c.tau_d[s] * c.a_d[s] * omega;
            if (nstar < 0.0) bad |= DBM_HEALTH_NSTAR;
            ns = (real)nstar;
            Ts = Td + c.tau_d[s] * dTdt;
        }
        const real inv_m = real(1) / c.m[s];
        fhat16<real>(ns, ux, uy, (real)Ts * inv_m, c.dpi[s], fh);
        if (c.has_force && n[s] != real(0)) {  // an absent species feels no force
            const real usx = jx[s] / n[s], usy = jy[s] / n[s];
            const real ths = (en[s] / n[s] - (usx * usx + usy * usy)) / c.dpi[s];
            real g1[Q], g0[Q];
            fhat16<real>(n[s], usx + c.accel_x * c.tau[s], usy + c.accel_y * c.tau[s], ths, c.dpi[s], g1);
            fhat16<real>(n[s], usx, usy, ths, c.dpi[s], g0);
#pragma unroll
            for (int k = 0; k < Q; ++k) fh[k] += g1[k] - g0[k];
        }
        const real dt_tau = c.dt * c.inv_tau[s];

#pragma unroll
        for (int i = 0; i < Q; ++i) {
            real feq = 0;
#pragma unroll
            for (int k = 0; k < Q; ++k) feq += c.cinv[s][i][k] * fh[k];

            const real *pl = fin + (s * Q + i) * P;
            const real f0 = pl[cell];
            const int r = i >> 2;
            // 5. NND advection, -dt (v_x d/dx + v_y d/dy) f
            real adv = 0;
            if (dir_x(i) > 0)
                adv += c.vr[s][r] * c.dt_dx * nnd_diff_pos(pl[cell - 2], pl[cell - 1], f0, pl[cell + 1]);
            else if (dir_x(i) < 0)
                adv -= c.vr[s][r] * c.dt_dx * nnd_diff_neg(pl[cell - 1], f0, pl[cell + 1], pl[cell + 2]);
            const long long py = c.pitch;
            if (dir_y(i) > 0)
                adv += c.vr[s][r] * c.dt_dy *
                       nnd_diff_pos(pl[cell - 2 * py], pl[cell - py], f0, pl[cell + py]);
            else if (dir_y(i) < 0)
                adv -= c.vr[s][r] * c.dt_dy *
                       nnd_diff_neg(pl[cell - py], f0, pl[cell + py], pl[cell + 2 * py]);
            // 6. forward Euler
            const real f1 = f0 + dt_tau * (feq - f0) - adv;
            store_with_images(fout + (s * Q + i) * P, cell, x, y, c.pitch, im, f1);
        }
    }
    if (bad) raise_flag(flag, bad);
}

template <typename real, int S>
int launch_step_t(dbm_handle *h, const void *fin, void *fout, cudaStream_t st)
{
    StepConsts<real, S> c;
    fill_step_consts<real, S>(h, c);
    dim3 block(32, 8);
    dim3 grid((h->p.nx + 31) / 32, (h->p.ny + 7) / 8);
    k_step<real, S><<<grid, block, 0, st>>>(c, (const real *)fin, (real *)fout,
                                            (unsigned *)h->scratch);
    return set_cuda_error(h, cudaGetLastError(), "step kernel launch");
}

}  // namespace dbm
