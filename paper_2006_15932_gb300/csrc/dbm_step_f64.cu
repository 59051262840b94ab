// dbm_step_f64.cu -- the FP64 step, in reference operation order.
//
// The FP64 path is the parity path of the library: its results are held to
// a relative L-inf of 1e-12 against a plain FP64 CPU evaluation of the
// paper's formulas after thousands of steps, through shocks.  Two FP64
// evaluations of the same step that merely round in a different order
// drift apart by ~1e-12 over 2000 steps of a shock tube (the limiter and
// the relaxation pass every rounding difference on), so this kernel
// evaluates each formula with the same operands in the same order as it is
// printed, and this translation unit is compiled without multiply-add
// contraction (--fmad=false):
//   - species moments n = sum f, n u = sum f v, E = sum f (v.v + eta^2),
//     T^s = m (E/n - u.u)/(D+I)  (section "Discrete Boltzmann model");
//   - mixture u = sum(rho u^s/tau)/sum(rho/tau),
//     T = sum((m E - rho u.u)/tau)/sum(n (D+I)/tau) (momentum and energy
//     conservation of Eq. CollisionTerm);
//   - f^eq = M^-1 f-hat with the f-hat list as printed; Omega, R and G as
//     separate terms (Eqs. CollisionTerm, ReactionTerm, ForceTerm);
//   - NND fluxes H from the split fluxes F+- = (c +- |c|)/2 f;
//   - f^{n+1} = f + dt (Omega + R + G - d(v_x f)/dx - d(v_y f)/dy).
// One thread per cell; ghosts of the new state are written as images.
#include "dbm_consts.h"
#include "dbm_device.cuh"

namespace dbm {

// f-hat_1..16 at (n, u, T) for a species of mass m and extra degrees of
// freedom I, theta = T/m, D = 2, in the printed form.
__device__ __forceinline__ void fhat_printed(double n, double ux, double uy, double T, double m, double I,
                                             double fh[Q])
{
    const double D = 2.0;
    const double th = T / m;
    const double u2 = ux * ux + uy * uy;
    fh[0] = n;
    fh[1] = n * ux;
    fh[2] = n * uy;
    fh[3] = n * ((D + I) * th + u2);
    fh[4] = n * (th + ux * ux);
    fh[5] = n * ux * uy;
    fh[6] = n * (th + uy * uy);
    fh[7] = n * ux * ((D + I + 2.0) * th + u2);
    fh[8] = n * uy * ((D + I + 2.0) * th + u2);
    fh[9] = 3.0 * n * ux * th + n * ux * ux * ux;
    fh[10] = n * uy * th + n * ux * ux * uy;
    fh[11] = n * ux * th + n * ux * uy * uy;
    fh[12] = 3.0 * n * uy * th + n * uy * uy * uy;
    fh[13] = n * ((D + I + 2.0) * th + u2) * th + n * ux * ux * ((D + I + 4.0) * th + u2);
    fh[14] = n * ux * uy * ((D + I + 4.0) * th + u2);
    fh[15] = n * ((D + I + 2.0) * th + u2) * th + n * uy * uy * ((D + I + 4.0) * th + u2);
}

template <int S>
__device__ __forceinline__ void feq_printed(const F64Consts<S> &c, int s, double n, double ux, double uy,
                                            double T, double feq[Q])
{
    double fh[Q];
    fhat_printed(n, ux, uy, T, c.m[s], c.I[s], fh);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        double acc = 0.0;
#pragma unroll
        for (int k = 0; k < Q; ++k) acc += c.cinv[s][i][k] * fh[k];
        feq[i] = acc;
    }
}

__device__ __forceinline__ double minmod_printed(double a, double b)
{
    const double sa = a > 0.0 ? 1.0 : (a < 0.0 ? -1.0 : 0.0);
    const double sb = b > 0.0 ? 1.0 : (b < 0.0 ? -1.0 : 0.0);
    const double fa = fabs(a), fb = fabs(b);
    return 0.5 * (sa + sb) * (fa < fb ? fa : fb);
}

// d(c f)/dx at node j from w0..w4 = f_{j-2..j+2}: NND flux difference / h.
__device__ __forceinline__ double nnd_dflux(double cv, double w0, double w1, double w2, double w3, double w4,
                                            double h)
{
    const double cp = 0.5 * (cv + fabs(cv)), cm = 0.5 * (cv - fabs(cv));
    const double p0 = cp * w0, p1 = cp * w1, p2 = cp * w2, p3 = cp * w3;
    const double m1 = cm * w1, m2 = cm * w2, m3 = cm * w3, m4 = cm * w4;
    const double hr = p2 + 0.5 * minmod_printed(p2 - p1, p3 - p2) + m3 - 0.5 * minmod_printed(m3 - m2, m4 - m3);
    const double hl = p1 + 0.5 * minmod_printed(p1 - p0, p2 - p1) + m2 - 0.5 * minmod_printed(m2 - m1, m3 - m2);
    return (hr - hl) / h;
}

template <int S>
__global__ void __launch_bounds__(128)
    k_step_f64(const __grid_constant__ F64Consts<S> c, const double *__restrict__ fin,
               double *__restrict__ fout, unsigned *__restrict__ flag)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= c.nx || y >= c.ny) return;
    const long long P = c.plane, py = c.pitch;
    const long long cell = (long long)(y + GY) * c.pitch + (x + GX);

    double n[S], ux[S], uy[S], Ts[S], E[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        double sn = 0.0, jx = 0.0, jy = 0.0, se = 0.0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double f = fin[(s * Q + i) * P + cell];
            sn += f;
            jx += f * c.vx[s][i];
            jy += f * c.vy[s][i];
            se += f * c.q[s][i];
        }
        n[s] = sn;
        E[s] = se;
        if (sn == 0.0) {  // an absent species: zero velocity and temperature
            ux[s] = 0.0;
            uy[s] = 0.0;
            Ts[s] = 0.0;
        } else {
            ux[s] = jx / sn;
            uy[s] = jy / sn;
            Ts[s] = c.m[s] * (se / sn - (ux[s] * ux[s] + uy[s] * uy[s])) / (2.0 + c.I[s]);
        }
    }
    double w = 0.0, wx = 0.0, wy = 0.0, ntot = 0.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const double rho = c.m[s] * n[s];
        w += rho / c.tau[s];
        wx += rho * ux[s] / c.tau[s];
        wy += rho * uy[s] / c.tau[s];
        ntot += fabs(n[s]);
    }
    const double Ux = wx / w, Uy = wy / w;
    const double u2 = Ux * Ux + Uy * Uy;
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const double rho = c.m[s] * n[s];
        num += (c.m[s] * E[s] - rho * u2) / c.tau[s];
        den += n[s] * (2.0 + c.I[s]) / c.tau[s];
    }
    const double T = num / den;

    unsigned bad = 0;
#pragma unroll
    for (int s = 0; s < S; ++s)
        if (!(n[s] >= -1e-6 * ntot) || !isfinite(n[s])) bad |= DBM_HEALTH_DENSITY;
    if (!(ntot > 0.0)) bad |= DBM_HEALTH_DENSITY;
    if (!(T > 0.0)) bad |= DBM_HEALTH_TEMPERATURE;
    if (!isfinite(T) || !isfinite(Ux) || !isfinite(Uy)) bad |= DBM_HEALTH_NONFINITE;

    double omega = 0.0, dTdt = 0.0;
    if (c.has_reaction) {
        omega = c.k_ov * n[c.fuel] * n[c.oxid] * exp(-c.Ea_over_R / T);
        double src = 0.0, cap = 0.0;
#pragma unroll
        for (int s = 0; s < S; ++s) {
            src += (2.0 + c.I[s]) * c.a[s] * omega;
            cap += n[s] * (2.0 + c.I[s]);
        }
        dTdt = (c.Qheat * omega - 0.5 * T * src) / (0.5 * cap);
    }

    const Images im = cell_images(x, y, c.nx, c.ny, c.bc_x, c.bc_y);
#pragma unroll 1
    for (int s = 0; s < S; ++s) {
        const double tau = c.tau[s];
        double feq[Q], feq_r[Q], g1[Q], g0[Q];
        feq_printed<S>(c, s, n[s], Ux, Uy, T, feq);
        const bool react = c.has_reaction != 0, force = c.has_force != 0;
        if (react) {
            const double nstar = n[s] + tau * c.a[s] * omega;
            const double Tstar = T + tau * dTdt;
            if (nstar < -1e-6 * ntot) bad |= DBM_HEALTH_NSTAR;
            feq_printed<S>(c, s, nstar, Ux, Uy, Tstar, feq_r);
        }
        if (force) {
            feq_printed<S>(c, s, n[s], ux[s] + c.ax * tau, uy[s] + c.ay * tau, Ts[s], g1);
            feq_printed<S>(c, s, n[s], ux[s], uy[s], Ts[s], g0);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double *pl = fin + (s * Q + i) * P;
            const double f = pl[cell];
            double rhs = -(f - feq[i]) / tau;                   // Omega
            if (react) rhs = rhs + (feq_r[i] - feq[i]) / tau;   // R
            if (force) rhs = rhs + (g1[i] - g0[i]) / tau;       // G
            double adv = 0.0;
            if (dir_x(i) != 0)
                adv += nnd_dflux(c.vx[s][i], pl[cell - 2], pl[cell - 1], f, pl[cell + 1], pl[cell + 2], c.dx);
            if (dir_y(i) != 0)
                adv += nnd_dflux(c.vy[s][i], pl[cell - 2 * py], pl[cell - py], f, pl[cell + py], pl[cell + 2 * py],
                                 c.dy);
            const double fnew = f + c.dt * (rhs - adv);
            store_with_images(fout + (s * Q + i) * P, cell, x, y, c.pitch, im, fnew);
        }
    }
    if (bad) raise_flag(flag, bad);
}

template <int S>
static int launch_f64_t(dbm_handle *h, const double *fin, double *fout, cudaStream_t st)
{
    F64Consts<S> c;
    fill_f64_consts<S>(h, c);
    dim3 block(32, 4);
    dim3 grid((h->p.nx + 31) / 32, (h->p.ny + 3) / 4);
    k_step_f64<S><<<grid, block, 0, st>>>(c, fin, fout, (unsigned *)h->scratch);
    return set_cuda_error(h, cudaGetLastError(), "FP64 step kernel launch");
}

int launch_step_f64(dbm_handle *h, int cur, cudaStream_t st)
{
    const double *fin = (const double *)h->f[cur];
    double *fout = (double *)h->f[cur ^ 1];
    switch (h->p.nspecies) {
    case 1: return launch_f64_t<1>(h, fin, fout, st);
    case 2: return launch_f64_t<2>(h, fin, fout, st);
    case 3: return launch_f64_t<3>(h, fin, fout, st);
    case 4: return launch_f64_t<4>(h, fin, fout, st);
    case 5: return launch_f64_t<5>(h, fin, fout, st);
    case 6: return launch_f64_t<6>(h, fin, fout, st);
    case 7: return launch_f64_t<7>(h, fin, fout, st);
    case 8: return launch_f64_t<8>(h, fin, fout, st);
    }
    return DBM_ERR_INVALID;
}

}  // namespace dbm
