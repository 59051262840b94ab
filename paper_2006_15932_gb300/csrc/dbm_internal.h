// dbm_internal.h -- internal declarations shared by the library's
// translation units: the handle, the kernel-parameter blocks and the
// launchers.  Not part of the public ABI (include/dbm.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dbm.h"

namespace dbm {

constexpr int Q = 16;
constexpr int GX = 4;  // ghost columns left of the interior (2 used; 4 keep rows 16-byte aligned)
constexpr int GY = 2;  // ghost rows above and below the interior
constexpr int CONS_BLOCKS = 512;          // fixed grid of the conservation reduction
constexpr size_t SCRATCH_HEAD = 256;      // health flag area at the start of scratch

// Direction of velocity i inside its ring: rings a, c (i/4 even) lie on the
// axes, rings b, d (i/4 odd) on the diagonals (D2V16 definition).
__host__ __device__ constexpr int dir_x(int i)
{
    return ((i >> 2) & 1) ? ((i & 3) == 0 || (i & 3) == 3 ? 1 : -1)
                          : ((i & 3) == 0 ? 1 : ((i & 3) == 2 ? -1 : 0));
}
__host__ __device__ constexpr int dir_y(int i)
{
    return ((i >> 2) & 1) ? ((i & 3) < 2 ? 1 : -1)
                          : ((i & 3) == 1 ? 1 : ((i & 3) == 3 ? -1 : 0));
}

// Kernel parameters of the fused step, one block per launch (passed by
// value as a __grid_constant__; up to 32 KB of parameters are allowed).
template <typename real, int S>
struct StepConsts {
    real cinv[S][Q][Q];  // M^-1 of each species, row i = velocity, column k = moment
    real vr[S][4];       // ring speeds v_a..v_d
    real qr[S][4];       // v.v + eta^2 of each ring
    real m[S], inv_tau[S], dpi[S], tau[S], a[S];
    real dt, dt_dx, dt_dy;
    real accel_x, accel_y;
    double m_d[S], inv_tau_d[S], dpi_d[S], tau_d[S], a_d[S];
    double k_ov, Ea_over_R, Qheat;
    int fuel, oxid;
    int has_reaction, has_force;
    int nx, ny, pitch, bc_x, bc_y;
    long long plane;
};

// Kernel parameters of the FP64 output / initialisation kernels.
template <int S>
struct OutConsts {
    double cinv[S][Q][Q];
    double vr[S][4], qr[S][4], eta[S][4];
    double m[S], inv_tau[S], dpi[S], a[S];
    double Qheat, abs_a_fuel;
    int fuel, has_reaction;
    int nx, ny, pitch, bc_x, bc_y;
    long long plane;
};

}  // namespace dbm

struct dbm_handle {
    dbm_params p;
    double cinv[DBM_MAX_SPECIES][16][16];  // host FP64 M^-1 per species
    dbm_layout lay;
    void *f[2];
    int cur;
    void *scratch;
    int bound;
    long long steps;
    char err[512];
};

namespace dbm {

// Launchers; each returns DBM_OK or DBM_ERR_CUDA (message in h->err).
int launch_step(dbm_handle *h, const void *fin, void *fout, cudaStream_t st);
int launch_set_state(dbm_handle *h, void *f, const double *rho_s, const double *ux,
                     const double *uy, const double *T, cudaStream_t st);
int launch_set_f(dbm_handle *h, void *f, const double *src, cudaStream_t st);
int launch_get_f(dbm_handle *h, const void *f, double *dst, cudaStream_t st);
int launch_moments(dbm_handle *h, const void *f, double *out, cudaStream_t st);
int launch_noneq(dbm_handle *h, const void *f, double *out, cudaStream_t st);
int launch_conservation(dbm_handle *h, const void *f, double *out, cudaStream_t st);

template <typename real, int S>
void fill_step_consts(const dbm_handle *h, StepConsts<real, S> &c);
template <int S>
void fill_out_consts(const dbm_handle *h, OutConsts<S> &c);

int set_cuda_error(dbm_handle *h, cudaError_t e, const char *what);

}  // namespace dbm
