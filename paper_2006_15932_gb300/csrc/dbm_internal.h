// dbm_internal.h -- internal declarations shared by the library's
// translation units: the handle, the kernel-parameter blocks and the
// launchers.  Not part of the public ABI (include/dbm.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dbm.h"

namespace dbm {

constexpr int Q = 16;
constexpr int GX = 4;  // ghost columns left of the interior (2 used; 4 keep rows 16-byte aligned)
constexpr int GY = 2;  // ghost rows above and below the interior
constexpr int CONS_BLOCKS = 512;          // fixed grid of the conservation reduction
constexpr size_t SCRATCH_HEAD = 256;      // health flag area at the start of scratch
// polls of an mbarrier wait for a tile copy before it gives up (each poll
// may suspend the thread for a while); the first wait of a step can be
// shortened per handle (dbm_params.wait_polls), the drain wait cannot
constexpr int TMA_WAIT_POLLS = 1 << 22;

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
// eqA..eqX are the symmetry blocks of M^-1 (see dbm_step_impl.cuh).
template <typename real, int S>
struct StepConsts {
    real eqA[S][4][4];   // ring means      <- (f1, f4, f5+f7, f14+f16)
    real eqB[S][2][2];   // axis B (a, c)   <- (f5-f7, f14-f16)
    real eqH[S][2][2];   // diag H (b, d)   <- (f6, f15)
    real eqX[S][4][4];   // vector parts    <- (f2, f8, f10, f12) / (f3, f9, f13, f11)
    real vr[S][4];       // ring speeds v_a..v_d
    real qr[S][4];       // v.v + eta^2 of each ring
    real q4[S][4];       // 4 (v.v + eta^2): energy of a unit ring mean
    real wv[S][4];       // 2 v_r (axis) or 4 v_r (diagonal): momentum of a unit vector part
    real cdx[S][4], cdy[S][4];  // v_r dt/dx, v_r dt/dy
    // mixture weights as hi + lo pairs of the exact products of the constants
    // the kernel applies: lam = m dt_tau (momentum/energy weight of a species
    // in an update), kap = lam dpi inv_m (its heat capacity weight)
    real lam_h[S], lam_l[S], kap_h[S], kap_l[S];
    real dpi[S], inv_m[S], tau[S], dt_tau[S];
    real accel_x, accel_y;
    real tau_d[S], tau_a[S];  // tau^s, tau^s a^s
    real k_ov, Ea_over_R, Qheat, src;  // src = sum_s (D+I^s) a^s
    int fuel, oxid;
    int has_reaction, has_force;
    int nx, ny, pitch, bc_x, bc_y;
    int wait_polls;  // polls of the first wait for the tile copy (TMA-staged steps)
    long long plane;
};

// Extra kernel parameters of the FP32 step with its arithmetic options
// (dbm_params.thermo, dbm_params.rounding): the run-time switches, the
// seed of the stochastic rounding for this launch, and the constants of the
// FP64 moment and rate evaluation (the float constants of StepConsts
// widened, so that both evaluations use the same discrete velocities and
// weights).  NoAcc stands in for it in the default kernels.
template <int S>
struct AccConsts {
    static constexpr bool on = true;
    int thermo64;    // DBM_THERMO_FP64
    int stochastic;  // DBM_ROUND_STOCHASTIC
    unsigned seed;   // per launch: hash of the handle's step count
    double vr[S][4], qr[S][4];  // ring speeds and v.v + eta^2, as the float step uses them
    double lam[S], kap[S];      // mixture weights m dt_tau and lam dpi / m
    double dpi[S], tau_a[S], tau_d[S];
    double k_ov, Ea_over_R, Qheat, src;
};
struct NoAcc {
    static constexpr bool on = false;
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
    CUtensorMap tmap[2];  // TMA descriptors of the two bound state buffers
    CUtensorMap tmap_in[2];  // the same with an interior box (species-staged moment sums)
    int tma_ok;           // the TMA-staged step kernel can run
    int tma_tx, tma_ty;   // its tile (cells) and cells per thread (1 or 2),
    int tma_cw;           // fixed at dbm_bind
    int tma_staged;       // the species-staged step (one species per copy)
    double cinv[DBM_MAX_SPECIES][16][16];  // host FP64 M^-1 per species
    double eqA[DBM_MAX_SPECIES][4][4];     // symmetry blocks of M^-1
    double eqB[DBM_MAX_SPECIES][2][2];
    double eqH[DBM_MAX_SPECIES][2][2];
    double eqX[DBM_MAX_SPECIES][4][4];
    dbm_layout lay;
    void *f[2];
    int cur;
    void *scratch;
    int bound;
    long long steps;
    char err[512];
};

namespace dbm {

// Tile of the TMA-staged FP32 step, by species count, and the cells a
// thread updates (CW: 1, or 2 adjacent cells of a row with packed FP32x2
// arithmetic).  One cell per thread: 64 x 4 cells for one species (4 CTAs of
// 256 threads per SM), 32 x 8 for three (92 KB of shared memory, two CTAs),
// 32 x 6 for four (102 KB, two CTAs of 192 threads; 29.4 G/s on 2048 x 2048
// against 22.3 G/s for the generic kernel; 32x4, 64x4, 32x2, 32x3 and 64x2
// were slower).  Measured fastest among 32x16, 32x12, 32x10, 32x9, 32x8,
// 32x7, 32x6, 32x5, 32x4, 40x8, 48x6, 64x8, 64x6, 64x5, 64x4, 128x4 and
// others on 4096 x 4096 (two species) and 4096 x 2048 (one) grids: more
// resident CTAs per SM hide each CTA's wait for its tile.  For three species
// 64 x 4 is 3 % faster on 2048 x 2048 but 10 % slower on the 1024 x 256
// reactive gas, whose halo re-reads (2.25x against 1.9x) come from L2.  Two
// species: 32 x 7 with one cell per thread (56 KB, four CTAs of 224
// threads), and on large grids two cells per thread on PAIR_TX x PAIR_TY =
// 64 x 8 cells (110 KB, two CTAs of 256 threads): one thread per cell runs
// 812 instructions per species-cell and is issue-bound; pairs run 528, and
// the taller tile keeps 16 warps per SM (on 4096 x 4096: 42.0 G/s against
// 37.7; pairs on 64 x 4, 64 x 6 and 64 x 7 gave 39.6, 36.1 and 39.9).  With
// fewer CTAs per wave the pair tile loses on small grids (KH, G/s, pairs
// against one cell: 256^2 6.6 / 8.9, 512^2 17.6 / 21.8, 768^2 21.6 / 24.9,
// 1024^2 26.6 / 28.7, 1536^2 33.7 / 32.9, 2048^2 37.8 / 35.1), so pairs run
// from PAIR_MIN_TILES tiles up.  Three species in pairs hold half the warps
// per SM and ran slower (64 x 4 and 32 x 8: 12.4 and 15.5 G/s against 21.4
// on the 1024 x 256 reactive gas, 25.2 and 26.6 against 31.2 on 2048 x 1024).
constexpr int tma_tile_x(int S) { return S == 1 ? 64 : 32; }
constexpr int tma_tile_y(int S) { return S == 1 ? 4 : S == 2 ? 7 : S == 3 ? 8 : 6; }
constexpr int PAIR_TX = 64, PAIR_TY = 8;
// The species-staged step (two cells per thread, the tile passing through
// shared memory one species at a time in two buffers; k_step_staged): its
// tile, 64 x 8 cells in two buffers of 55 KB, two CTAs of 256 threads per
// SM.  A build may set another with -DDBM_STAGED_TX=.. -DDBM_STAGED_TY=..
// (TX a multiple of 8).
#ifndef DBM_STAGED_TX
#define DBM_STAGED_TX 64
#endif
#ifndef DBM_STAGED_TY
#define DBM_STAGED_TY 8
#endif
constexpr int STAGED_TX = DBM_STAGED_TX, STAGED_TY = DBM_STAGED_TY;
constexpr long long PAIR_MIN_TILES = 4096;

// CTAs of a TX x TY tile kernel that fit on one SM at once, limited by
// shared memory (the tile plus halo of 16 S float planes, and 1 KB reserved
// per CTA) and by registers (at least 64 per cell: 64 per thread for one
// cell per thread, 128 for two), at most four: the minimum-blocks bound of
// the kernel's __launch_bounds__.
constexpr int tma_ctas_per_sm(int S, int TX, int TY)
{
    const int by_smem = (227 * 1024) / ((TX + 8) * (TY + 4) * S * 64 + 1152);
    const int by_regs = 65536 / (TX * TY * 64);
    const int n = by_smem < by_regs ? by_smem : by_regs;
    return n > 4 ? 4 : n < 1 ? 1 : n;
}

// Launchers; each returns DBM_OK or DBM_ERR_CUDA (message in h->err).
int launch_step(dbm_handle *h, int cur, cudaStream_t st);
int make_tensor_maps(dbm_handle *h);
int launch_set_state(dbm_handle *h, void *f, const double *rho_s, const double *ux,
                     const double *uy, const double *T, cudaStream_t st);
int launch_set_f(dbm_handle *h, void *f, const double *src, cudaStream_t st);
int launch_get_f(dbm_handle *h, const void *f, double *dst, cudaStream_t st);
int launch_moments(dbm_handle *h, const void *f, double *out, cudaStream_t st);
int launch_noneq(dbm_handle *h, const void *f, double *out, cudaStream_t st);
int launch_conservation(dbm_handle *h, const void *f, double *out, cudaStream_t st);
int launch_conservation_noalloc(dbm_handle *h, const void *f, double *out, cudaStream_t st);

template <typename real, int S>
void fill_step_consts(const dbm_handle *h, StepConsts<real, S> &c);
template <int S>
void fill_acc_consts(const dbm_handle *h, const StepConsts<float, S> &c, AccConsts<S> &a);
// the FP32 step runs the kernel with the arithmetic options
inline bool uses_acc(const dbm_params &p)
{
    return p.precision == DBM_FP32 && (p.thermo != DBM_THERMO_FLOATFLOAT || p.rounding != DBM_ROUND_NEAREST);
}
template <int S>
void fill_out_consts(const dbm_handle *h, OutConsts<S> &c);

int set_cuda_error(dbm_handle *h, cudaError_t e, const char *what);

}  // namespace dbm

namespace dbm {

// Kernel parameters of the FP64 reference-order step (dbm_step_f64.cu):
// per-velocity constants so that every product is formed as in the
// plain restatement of the paper (same operands, same order).
template <int S>
struct F64Consts {
    double cinv[S][Q][Q];
    double vx[S][Q], vy[S][Q], q[S][Q];  // q = vx*vx + vy*vy + eta*eta
    double m[S], I[S], tau[S], a[S];
    double dt, dx, dy, ax, ay;
    double k_ov, Ea_over_R, Qheat;
    int fuel, oxid, has_reaction, has_force;
    int nx, ny, pitch, bc_x, bc_y;
    long long plane;
};

template <int S>
void fill_f64_consts(const dbm_handle *h, F64Consts<S> &c);
int launch_step_f64(dbm_handle *h, int cur, cudaStream_t st);
int launch_step_bf16(dbm_handle *h, int cur, cudaStream_t st);
int launch_set_state_bf16(dbm_handle *h, void *f, const double *rho_s, const double *ux, const double *uy,
                          const double *T, cudaStream_t st);
int launch_set_f_bf16(dbm_handle *h, void *f, const double *src, cudaStream_t st);
int launch_get_f_bf16(dbm_handle *h, const void *f, double *dst, cudaStream_t st);

}  // namespace dbm
