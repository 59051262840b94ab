// dbm_consts.h -- fill the kernel-parameter blocks from a validated handle.
#pragma once

#include <math.h>
#include <string.h>

#include "dbm_internal.h"

namespace dbm {

// v.v + eta^2 of ring r: |v|^2 = v_r^2 on the axis rings, 2 v_r^2 on the
// diagonal rings.
inline double ring_q(const dbm_species &sp, int r)
{
    const double v2 = sp.v[r] * sp.v[r] * ((r & 1) ? 2.0 : 1.0);
    return v2 + sp.eta[r] * sp.eta[r];
}

template <typename real, int S>
void fill_step_consts(const dbm_handle *h, StepConsts<real, S> &c)
{
    memset(&c, 0, sizeof(c));
    const dbm_params &p = h->p;
    double src = 0.0;
    for (int s = 0; s < S; ++s) {
        const dbm_species &sp = p.sp[s];
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
                c.eqA[s][a][b] = (real)h->eqA[s][a][b];
                c.eqX[s][a][b] = (real)h->eqX[s][a][b];
            }
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
                c.eqB[s][a][b] = (real)h->eqB[s][a][b];
                c.eqH[s][a][b] = (real)h->eqH[s][a][b];
            }
        for (int r = 0; r < 4; ++r) {
            c.vr[s][r] = (real)sp.v[r];
            c.qr[s][r] = (real)ring_q(sp, r);
            c.q4[s][r] = (real)(4.0 * ring_q(sp, r));
            c.wv[s][r] = (real)(((r & 1) ? 4.0 : 2.0) * sp.v[r]);
            c.cdx[s][r] = (real)(sp.v[r] * p.dt / p.dx);
            c.cdy[s][r] = (real)(sp.v[r] * p.dt / p.dy);
        }
        c.dpi[s] = (real)(2.0 + sp.I);
        c.inv_m[s] = (real)(1.0 / sp.m);
        c.tau[s] = (real)sp.tau;
        c.dt_tau[s] = (real)(p.dt / sp.tau);
        // exact products of the constants as stored (errors ~1e-16), split so
        // that no rounding of a constant biases the mixture u and T
        const double lam = sp.m * (double)c.dt_tau[s];
        const double kap = lam * (double)c.dpi[s] * (double)c.inv_m[s];
        c.lam_h[s] = (real)lam;
        c.lam_l[s] = (real)(lam - (double)c.lam_h[s]);
        c.kap_h[s] = (real)kap;
        c.kap_l[s] = (real)(kap - (double)c.kap_h[s]);
        c.tau_d[s] = (real)sp.tau;
        c.tau_a[s] = (real)(sp.tau * sp.a_stoich);
        src += (2.0 + sp.I) * sp.a_stoich;
    }
    c.accel_x = (real)p.accel[0];
    c.accel_y = (real)p.accel[1];
    c.k_ov = (real)p.k_ov;
    c.Ea_over_R = (real)p.Ea_over_R;
    c.Qheat = (real)p.Q;
    c.src = (real)src;
    c.fuel = p.fuel;
    c.oxid = p.oxidizer;
    c.has_reaction = p.k_ov != 0.0;
    c.has_force = p.accel[0] != 0.0 || p.accel[1] != 0.0;
    c.nx = p.nx;
    c.ny = p.ny;
    c.pitch = h->lay.pitch;
    c.bc_x = p.bc_x;
    c.bc_y = p.bc_y;
    c.wait_polls = p.wait_polls == 0 ? TMA_WAIT_POLLS : p.wait_polls < 0 ? 0 : p.wait_polls;
    c.plane = h->lay.plane;
}

// Integer hash "lowbias32" (C. Wellons' hash-prospector: xor-shift /
// multiply rounds with its published constants); seeds and random numbers
// of the stochastic rounding.
__host__ __device__ inline unsigned mix32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <int S>
void fill_acc_consts(const dbm_handle *h, const StepConsts<float, S> &c, AccConsts<S> &a)
{
    memset(&a, 0, sizeof(a));
    const dbm_params &p = h->p;
    a.thermo64 = p.thermo == DBM_THERMO_FP64;
    a.stochastic = p.rounding == DBM_ROUND_STOCHASTIC;
    a.seed = mix32((unsigned)h->steps * 0x9e3779b9u + 0x632be5abu) ^ mix32((unsigned)(h->steps >> 32));
    double src = 0.0;
    for (int s = 0; s < S; ++s) {
        for (int r = 0; r < 4; ++r) {
            a.vr[s][r] = (double)c.vr[s][r];
            a.qr[s][r] = (double)c.qr[s][r];
        }
        // the weights of the float step as exact doubles (lam_h + lam_l)
        a.lam[s] = (double)c.lam_h[s] + (double)c.lam_l[s];
        a.kap[s] = (double)c.kap_h[s] + (double)c.kap_l[s];
        a.dpi[s] = (double)c.dpi[s];
        a.tau_a[s] = p.sp[s].tau * p.sp[s].a_stoich;
        a.tau_d[s] = p.sp[s].tau;
        src += (2.0 + p.sp[s].I) * p.sp[s].a_stoich;
    }
    a.k_ov = p.k_ov;
    a.Ea_over_R = p.Ea_over_R;
    a.Qheat = p.Q;
    a.src = src;
}

template <int S>
void fill_out_consts(const dbm_handle *h, OutConsts<S> &c)
{
    memset(&c, 0, sizeof(c));
    const dbm_params &p = h->p;
    for (int s = 0; s < S; ++s) {
        const dbm_species &sp = p.sp[s];
        for (int i = 0; i < Q; ++i)
            for (int k = 0; k < Q; ++k) c.cinv[s][i][k] = h->cinv[s][i][k];
        for (int r = 0; r < 4; ++r) {
            c.vr[s][r] = sp.v[r];
            c.qr[s][r] = ring_q(sp, r);
            c.eta[s][r] = sp.eta[r];
        }
        c.m[s] = sp.m;
        c.inv_tau[s] = 1.0 / sp.tau;
        c.dpi[s] = 2.0 + sp.I;
        c.a[s] = sp.a_stoich;
    }
    c.has_reaction = p.k_ov != 0.0;
    c.fuel = p.fuel;
    c.Qheat = p.Q;
    c.abs_a_fuel = c.has_reaction ? fabs(p.sp[p.fuel].a_stoich) : 1.0;
    c.nx = p.nx;
    c.ny = p.ny;
    c.pitch = h->lay.pitch;
    c.bc_x = p.bc_x;
    c.bc_y = p.bc_y;
    c.plane = h->lay.plane;
}

}  // namespace dbm

namespace dbm {

template <int S>
void fill_f64_consts(const dbm_handle *h, F64Consts<S> &c)
{
    memset(&c, 0, sizeof(c));
    const dbm_params &p = h->p;
    for (int s = 0; s < S; ++s) {
        const dbm_species &sp = p.sp[s];
        for (int i = 0; i < Q; ++i) {
            for (int k = 0; k < Q; ++k) c.cinv[s][i][k] = h->cinv[s][i][k];
            const double x = dir_x(i) * sp.v[i >> 2], y = dir_y(i) * sp.v[i >> 2], e = sp.eta[i >> 2];
            c.vx[s][i] = x;
            c.vy[s][i] = y;
            c.q[s][i] = x * x + y * y + e * e;  // host code is built without contraction
        }
        c.m[s] = sp.m;
        c.I[s] = sp.I;
        c.tau[s] = sp.tau;
        c.a[s] = sp.a_stoich;
    }
    c.dt = p.dt;
    c.dx = p.dx;
    c.dy = p.dy;
    c.ax = p.accel[0];
    c.ay = p.accel[1];
    c.k_ov = p.k_ov;
    c.Ea_over_R = p.Ea_over_R;
    c.Qheat = p.Q;
    c.fuel = p.fuel;
    c.oxid = p.oxidizer;
    c.has_reaction = p.k_ov != 0.0;
    c.has_force = p.accel[0] != 0.0 || p.accel[1] != 0.0;
    c.nx = p.nx;
    c.ny = p.ny;
    c.pitch = h->lay.pitch;
    c.bc_x = p.bc_x;
    c.bc_y = p.bc_y;
    c.plane = h->lay.plane;
}

}  // namespace dbm
