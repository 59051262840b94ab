// dbm_api.cu -- host side of the C ABI declared in include/dbm.h:
// parameter validation, the FP64 host inversion of the D2V16 moment matrix
// M (section "Discrete Boltzmann model": f^eq = M^-1 f-hat), buffer
// geometry, binding, and the enqueueing of the device kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include "dbm_internal.h"

namespace dbm {

static int fail(dbm_handle *h, int code, const char *fmt, ...)
{
    if (h) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(h->err, sizeof(h->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int set_cuda_error(dbm_handle *h, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return DBM_OK;
    return fail(h, DBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Row k of M for velocity (x, y) with internal speed eta: the moment
// monomials 1, v_x, v_y, q, v_x^2, v_x v_y, v_y^2, q v_x, q v_y, v_x^3,
// v_x^2 v_y, v_x v_y^2, v_y^3, q v_x^2, q v_x v_y, q v_y^2 with
// q = v.v + eta^2 (the M_9 row is q v_y).
static void build_moment_matrix(const dbm_species &sp, double M[Q][Q])
{
    for (int i = 0; i < Q; ++i) {
        const int r = i >> 2;
        const double x = dir_x(i) * sp.v[r], y = dir_y(i) * sp.v[r];
        const double q = x * x + y * y + sp.eta[r] * sp.eta[r];
        const double col[Q] = {1.0,       x,         y,         q,         x * x,     x * y,
                               y * y,     q * x,     q * y,     x * x * x, x * x * y, x * y * y,
                               y * y * y, q * x * x, q * x * y, q * y * y};
        for (int k = 0; k < Q; ++k) M[k][i] = col[k];
    }
}

// LU factorisation with partial pivoting (Doolittle, in place) of the
// n x n row-major A, then A^-1 column by column from forward and back
// substitution.  Returns 0, or -1 when a pivot vanishes.
static int lu_inverse_n(const double *A, double *Ainv, int n)
{
    double LU[Q * Q];
    int perm[Q];
    memcpy(LU, A, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(LU[k * n + k]);
        for (int r = k + 1; r < n; ++r)
            if (fabs(LU[r * n + k]) > best) {
                best = fabs(LU[r * n + k]);
                piv = r;
            }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (int c = 0; c < n; ++c) {
                const double t = LU[k * n + c];
                LU[k * n + c] = LU[piv * n + c];
                LU[piv * n + c] = t;
            }
            const int t = perm[k];
            perm[k] = perm[piv];
            perm[piv] = t;
        }
        for (int r = k + 1; r < n; ++r) {
            LU[r * n + k] /= LU[k * n + k];
            const double l = LU[r * n + k];
            for (int c = k + 1; c < n; ++c) LU[r * n + c] -= l * LU[k * n + c];
        }
    }
    for (int col = 0; col < n; ++col) {
        double z[Q];
        for (int r = 0; r < n; ++r) {  // L z = P e_col
            double s = (perm[r] == col) ? 1.0 : 0.0;
            for (int c = 0; c < r; ++c) s -= LU[r * n + c] * z[c];
            z[r] = s;
        }
        for (int r = n - 1; r >= 0; --r) {  // U x = z
            double s = z[r];
            for (int c = r + 1; c < n; ++c) s -= LU[r * n + c] * Ainv[c * n + col];
            Ainv[r * n + col] = s / LU[r * n + r];
        }
    }
    return 0;
}

// Compensated dot product c - sum_k a[k] b[k*stride], k < n (Ogita-Rump-Oishi
// "Dot2": error-free products via fma and error-free sums), as accurate as
// if accumulated in twice the working precision.
static double residual_dot2(double c, const double *a, const double *b, int stride, int n)
{
    double s = c, err = 0.0;
    for (int k = 0; k < n; ++k) {
        const double p = -a[k] * b[k * stride];
        const double pe = fma(-a[k], b[k * stride], -p);
        const double t = s + p;
        const double z = t - s;
        err += ((s - (t - z)) + (p - z)) + pe;
        s = t;
    }
    return s + err;
}

// Refinement X <- X + X (I - A X) with the residual from residual_dot2:
// the error of X squares at each pass, so X becomes the inverse of A
// rounded correctly to double (ties aside).  Exact conservation by
// f^eq = M^-1 f-hat needs this: a few ulps of error in M^-1 bias the mass,
// momentum and energy of every collision the same way, and that bias
// accumulates step after step.
static void refine_inverse_n(const double *A, double *X, int n, int passes)
{
    for (int it = 0; it < passes; ++it) {
        double R[Q * Q], Xn[Q * Q];
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c)
                R[r * n + c] = residual_dot2(r == c ? 1.0 : 0.0, A + r * n, X + c, n, n);
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c) {
                double d = 0.0;
                for (int k = 0; k < n; ++k) d += X[r * n + k] * R[k * n + c];
                Xn[r * n + c] = X[r * n + c] + d;
            }
        memcpy(X, Xn, sizeof(double) * n * n);
    }
}

static int inverse_refined(const double *A, double *X, int n)
{
    if (lu_inverse_n(A, X, n) != 0) return -1;
    refine_inverse_n(A, X, n, 3);
    return 0;
}

// The symmetry blocks of M (see dbm_step_impl.cuh): with ring means A_r,
// axis quadrupoles B_a, B_c, diagonal quadrupoles H_b, H_d and vector parts
// (E on axis rings, G on diagonal rings) as unknowns, the moment relations
// read
//   (f1, f4, f5+f7, f14+f16) = bA (A_a, A_b, A_c, A_d)
//   (f5-f7, f14-f16)         = bB (B_a, B_c)
//   (f6, f15)                = bH (H_b, H_d)
//   (f2, f8, f10, f12)       = bX (E_xa, G_xb, E_xc, G_xd)   (and y alike)
// with entries from the ring sums of the monomials (4 velocities per ring;
// |v|^2 = v^2 on axis rings and 2 v^2 on diagonal rings).
static int symmetry_blocks(const dbm_species &sp, double iA[16], double iB[4], double iH[4],
                           double iX[16])
{
    double v[4], q[4], w[4];
    for (int r = 0; r < 4; ++r) {
        v[r] = sp.v[r];
        const double v2 = v[r] * v[r] * ((r & 1) ? 2.0 : 1.0);
        q[r] = v2 + sp.eta[r] * sp.eta[r];
        w[r] = (r & 1) ? 4.0 : 2.0;  // weight of the vector part in a ring sum
    }
    double bA[16], bB[4], bH[4], bX[16];
    for (int r = 0; r < 4; ++r) {
        const double g = (r & 1) ? 8.0 : 4.0;  // sum over the ring of v_x^2 + v_y^2 per unit v^2
        bA[0 * 4 + r] = 4.0;
        bA[1 * 4 + r] = 4.0 * q[r];
        bA[2 * 4 + r] = g * v[r] * v[r];
        bA[3 * 4 + r] = g * q[r] * v[r] * v[r];
        bX[0 * 4 + r] = w[r] * v[r];
        bX[1 * 4 + r] = w[r] * q[r] * v[r];
        bX[2 * 4 + r] = w[r] * v[r] * v[r] * v[r];
        bX[3 * 4 + r] = (r & 1) ? 4.0 * v[r] * v[r] * v[r] : 0.0;
    }
    for (int j = 0; j < 2; ++j) {
        const int ra = 2 * j, rb = 2 * j + 1;
        bB[0 * 2 + j] = 4.0 * v[ra] * v[ra];
        bB[1 * 2 + j] = 4.0 * q[ra] * v[ra] * v[ra];
        bH[0 * 2 + j] = 4.0 * v[rb] * v[rb];
        bH[1 * 2 + j] = 4.0 * q[rb] * v[rb] * v[rb];
    }
    if (inverse_refined(bA, iA, 4) || inverse_refined(bB, iB, 2) || inverse_refined(bH, iH, 2) ||
        inverse_refined(bX, iX, 4))
        return -1;
    return 0;
}

// f^eq of all 16 velocities from the blocks, for unit moment vectors:
// column k of the matrix the kernels apply, to compare with M^-1.
static void blocks_to_matrix(const double iA[16], const double iB[4], const double iH[4],
                             const double iX[16], double out[Q][Q])
{
    for (int k = 0; k < Q; ++k) {
        double fh[Q] = {0};
        fh[k] = 1.0;
        const double cA[4] = {fh[0], fh[3], fh[4] + fh[6], fh[13] + fh[15]};
        const double cB[2] = {fh[4] - fh[6], fh[13] - fh[15]};
        const double cH[2] = {fh[5], fh[14]};
        const double cX[4] = {fh[1], fh[7], fh[9], fh[11]};
        const double cY[4] = {fh[2], fh[8], fh[12], fh[10]};
        double A[4], B[2], H[2], X[4], Y[4];
        for (int r = 0; r < 4; ++r) {
            A[r] = X[r] = Y[r] = 0.0;
            for (int j = 0; j < 4; ++j) {
                A[r] += iA[r * 4 + j] * cA[j];
                X[r] += iX[r * 4 + j] * cX[j];
                Y[r] += iX[r * 4 + j] * cY[j];
            }
        }
        for (int r = 0; r < 2; ++r) {
            B[r] = iB[r * 2] * cB[0] + iB[r * 2 + 1] * cB[1];
            H[r] = iH[r * 2] * cH[0] + iH[r * 2 + 1] * cH[1];
        }
        for (int r = 0; r < 4; ++r) {
            const int i = 4 * r;
            if ((r & 1) == 0) {
                const double b = B[r >> 1];
                out[i + 0][k] = A[r] + X[r] + b;
                out[i + 1][k] = A[r] + Y[r] - b;
                out[i + 2][k] = A[r] - X[r] + b;
                out[i + 3][k] = A[r] - Y[r] - b;
            } else {
                const double hq = H[r >> 1];
                out[i + 0][k] = A[r] + X[r] + Y[r] + hq;
                out[i + 1][k] = A[r] - X[r] + Y[r] - hq;
                out[i + 2][k] = A[r] - X[r] - Y[r] + hq;
                out[i + 3][k] = A[r] + X[r] - Y[r] - hq;
            }
        }
    }
}

static double norm_inf(const double A[Q][Q])
{
    double best = 0.0;
    for (int r = 0; r < Q; ++r) {
        double s = 0.0;
        for (int c = 0; c < Q; ++c) s += fabs(A[r][c]);
        if (s > best) best = s;
    }
    return best;
}

static int validate(dbm_handle *h, const dbm_params &p)
{
    if (p.nspecies < 1 || p.nspecies > DBM_MAX_SPECIES)
        return fail(h, DBM_ERR_INVALID, "nspecies=%d outside 1..%d", p.nspecies, DBM_MAX_SPECIES);
    if (p.nx < 1 || p.ny < 1) return fail(h, DBM_ERR_INVALID, "grid %dx%d must be >= 1x1", p.nx, p.ny);
    if ((long long)p.nx * p.ny > (1LL << 31))
        return fail(h, DBM_ERR_INVALID, "grid %dx%d exceeds 2^31 cells", p.nx, p.ny);
    if (!(p.dx > 0) || !(p.dy > 0) || !(p.dt > 0))
        return fail(h, DBM_ERR_INVALID, "dx, dy, dt must be > 0");
    for (int a = 0; a < 2; ++a) {
        const int bc = a ? p.bc_y : p.bc_x;
        if (bc != DBM_BC_PERIODIC && bc != DBM_BC_OUTFLOW)
            return fail(h, DBM_ERR_INVALID, "unknown boundary condition %d", bc);
    }
    if (p.precision != DBM_FP64 && p.precision != DBM_FP32 && p.precision != DBM_BF16DEV)
        return fail(h, DBM_ERR_INVALID, "unknown precision %d", p.precision);
    if (p.step_kernel < DBM_KERNEL_AUTO || p.step_kernel > DBM_KERNEL_TMA_STAGED)
        return fail(h, DBM_ERR_INVALID, "unknown step kernel %d", p.step_kernel);
    const bool options = p.thermo != DBM_THERMO_FLOATFLOAT || p.rounding != DBM_ROUND_NEAREST;
    if (p.step_kernel == DBM_KERNEL_TMA_PAIR &&
        (p.precision != DBM_FP32 || p.nspecies < 2 || (p.nspecies > 2 && options)))
        return fail(h, DBM_ERR_INVALID,
                    "the two-cells-per-thread step is built for FP32 with two or more species "
                    "(with the thermo or rounding option: two species)");
    if (p.step_kernel == DBM_KERNEL_TMA_STAGED && (p.precision != DBM_FP32 || p.nspecies < 2 || options))
        return fail(h, DBM_ERR_INVALID,
                    "the species-staged step is built for FP32 with two or more species, without the thermo "
                    "and rounding options");
    if (p.step_kernel == DBM_KERNEL_TMA_CELL && p.nspecies > 4)
        return fail(h, DBM_ERR_INVALID, "the one-cell TMA-staged step is built for up to four species");
    const bool tma_kind = p.step_kernel != DBM_KERNEL_AUTO && p.step_kernel != DBM_KERNEL_GENERIC;
    if (p.precision == DBM_BF16DEV &&
        (p.nspecies > 4 || p.k_ov != 0.0 || p.accel[0] != 0.0 || p.accel[1] != 0.0 || tma_kind))
        return fail(h, DBM_ERR_INVALID,
                    "BF16DEV storage is built for up to 4 species without reaction or force "
                    "(its reference equilibrium is that of the stored moments)");
    if (p.thermo != DBM_THERMO_FLOATFLOAT && p.thermo != DBM_THERMO_FP64)
        return fail(h, DBM_ERR_INVALID, "unknown thermo option %d", p.thermo);
    if (p.rounding != DBM_ROUND_NEAREST && p.rounding != DBM_ROUND_STOCHASTIC)
        return fail(h, DBM_ERR_INVALID, "unknown rounding option %d", p.rounding);
    if ((p.thermo != DBM_THERMO_FLOATFLOAT || p.rounding != DBM_ROUND_NEAREST) &&
        (p.precision != DBM_FP32 || p.nspecies > 4 || p.step_kernel == DBM_KERNEL_GENERIC))
        return fail(h, DBM_ERR_INVALID,
                    "the thermo and rounding options are built for the TMA-staged FP32 step (up to 4 species)");
    if (!isfinite(p.accel[0]) || !isfinite(p.accel[1]))
        return fail(h, DBM_ERR_INVALID, "acceleration must be finite");
    double vmax = 0.0;
    for (int s = 0; s < p.nspecies; ++s) {
        const dbm_species &sp = p.sp[s];
        if (!(sp.m > 0) || !(sp.tau > 0) || !(sp.I >= 0))
            return fail(h, DBM_ERR_INVALID, "species %d: need m > 0, tau > 0, I >= 0", s);
        for (int r = 0; r < 4; ++r) {
            if (!(sp.v[r] > 0) || !isfinite(sp.v[r]))
                return fail(h, DBM_ERR_INVALID, "species %d: ring speed v[%d] must be > 0", s, r);
            if (!(sp.eta[r] >= 0) || !isfinite(sp.eta[r]))
                return fail(h, DBM_ERR_INVALID, "species %d: eta[%d] must be >= 0", s, r);
            if (sp.v[r] > vmax) vmax = sp.v[r];
        }
        if (!(p.dt < 2.0 * sp.tau))
            return fail(h, DBM_ERR_STABILITY, "species %d: dt=%g >= 2 tau=%g (unstable relaxation)", s,
                        p.dt, 2.0 * sp.tau);
    }
    const double cfl = vmax * p.dt / fmin(p.dx, p.dy);
    if (cfl > 0.5) return fail(h, DBM_ERR_STABILITY, "CFL number %g > 0.5", cfl);
    if (p.k_ov != 0.0) {
        if (!(p.k_ov > 0) || !isfinite(p.k_ov) || !isfinite(p.Ea_over_R) || !isfinite(p.Q))
            return fail(h, DBM_ERR_INVALID, "reaction constants must be finite, k_ov > 0");
        if (p.fuel < 0 || p.fuel >= p.nspecies || p.oxidizer < 0 || p.oxidizer >= p.nspecies)
            return fail(h, DBM_ERR_INVALID, "fuel/oxidizer index out of range");
        if (p.sp[p.fuel].a_stoich == 0.0)
            return fail(h, DBM_ERR_INVALID, "fuel must have a nonzero stoichiometric coefficient");
        double sum = 0.0, mag = 0.0;
        for (int s = 0; s < p.nspecies; ++s) {
            sum += p.sp[s].a_stoich * p.sp[s].m;
            mag += fabs(p.sp[s].a_stoich * p.sp[s].m);
        }
        if (fabs(sum) > 1e-12 * mag)
            return fail(h, DBM_ERR_INVALID, "sum_s a^s m^s = %g: the reaction does not conserve mass", sum);
    }
    return DBM_OK;
}

static void compute_layout(dbm_handle *h)
{
    const dbm_params &p = h->p;
    dbm_layout &L = h->lay;
    memset(&L, 0, sizeof(L));
    L.gx = GX;
    L.gy = GY;
    L.pitch = ((GX + p.nx + 4) + 31) / 32 * 32;  // room for the pair loads at x0+2, x0+3
    L.rows = p.ny + 2 * GY;
    L.plane = (long long)L.pitch * L.rows;
    const size_t nplanes = (size_t)p.nspecies * Q;
    if (p.precision == DBM_FP64) {
        L.elem_bytes = 8;
        L.bytes = nplanes * L.plane * 8;
    } else if (p.precision == DBM_FP32) {
        L.elem_bytes = 4;
        L.bytes = nplanes * L.plane * 4;
    } else {
        L.elem_bytes = 2;
        L.moments_offset = (nplanes * L.plane * 2 + 255) / 256 * 256;
        L.bytes = L.moments_offset + (size_t)(p.nspecies + 3) * L.plane * 4;
    }
}

}  // namespace dbm

using namespace dbm;

static thread_local char g_init_error[512];

extern "C" {

const char *dbm_init_error(void) { return g_init_error; }

int dbm_init(const dbm_params *params, dbm_handle **out)
{
    if (!params || !out) return DBM_ERR_INVALID;
    *out = nullptr;
    dbm_handle *h = (dbm_handle *)calloc(1, sizeof(dbm_handle));
    if (!h) return DBM_ERR_INVALID;
    h->p = *params;
    int rc = validate(h, h->p);
    if (rc == DBM_OK) {
        for (int s = 0; s < h->p.nspecies && rc == DBM_OK; ++s) {
            double M[Q][Q], Mi[Q][Q];
            build_moment_matrix(h->p.sp[s], M);
            if (inverse_refined(&M[0][0], &Mi[0][0], Q) != 0) {
                rc = fail(h, DBM_ERR_SINGULAR, "species %d: moment matrix M is singular", s);
                break;
            }
            // condition number of the row-equilibrated matrix D M (D scales each
            // row to unit max-norm), independent of the unit of velocity
            double rowmax[Q], DM[Q][Q], MiD[Q][Q];
            for (int r = 0; r < Q; ++r) {
                rowmax[r] = 0.0;
                for (int c = 0; c < Q; ++c) rowmax[r] = fmax(rowmax[r], fabs(M[r][c]));
            }
            for (int r = 0; r < Q; ++r)
                for (int c = 0; c < Q; ++c) {
                    DM[r][c] = M[r][c] / rowmax[r];
                    MiD[r][c] = Mi[r][c] * rowmax[c];
                }
            const double cond = norm_inf(DM) * norm_inf(MiD);
            // round trip M M^-1 = I
            double res = 0.0;
            for (int r = 0; r < Q; ++r)
                for (int c = 0; c < Q; ++c) {
                    double v = 0.0;
                    for (int k = 0; k < Q; ++k) v += DM[r][k] * MiD[k][c];
                    res = fmax(res, fabs(v - (r == c ? 1.0 : 0.0)));
                }
            if (!(cond <= 1e8) || !(res <= 1e-14 * cond))
                rc = fail(h, DBM_ERR_SINGULAR,
                          "species %d: moment matrix ill-conditioned (cond_inf=%g, residual=%g); "
                          "choose eta > 0 and distinct ring speeds",
                          s, cond, res);
            memcpy(h->cinv[s], Mi, sizeof(Mi));
            if (rc != DBM_OK) break;
            // symmetry blocks used by the step kernel; they must reproduce M^-1
            double iA[16], iB[4], iH[4], iX[16], Mb[Q][Q];
            if (symmetry_blocks(h->p.sp[s], iA, iB, iH, iX) != 0) {
                rc = fail(h, DBM_ERR_SINGULAR, "species %d: a symmetry block of M is singular", s);
                break;
            }
            blocks_to_matrix(iA, iB, iH, iX, Mb);
            double dmax = 0.0, mmax = 0.0;
            for (int r = 0; r < Q; ++r)
                for (int c = 0; c < Q; ++c) {
                    dmax = fmax(dmax, fabs(Mb[r][c] - Mi[r][c]));
                    mmax = fmax(mmax, fabs(Mi[r][c]));
                }
            if (!(dmax <= 1e-13 * mmax)) {
                rc = fail(h, DBM_ERR_SINGULAR, "species %d: symmetry blocks disagree with M^-1 (%g)", s,
                          dmax / mmax);
                break;
            }
            memcpy(h->eqA[s], iA, sizeof(iA));
            memcpy(h->eqB[s], iB, sizeof(iB));
            memcpy(h->eqH[s], iH, sizeof(iH));
            memcpy(h->eqX[s], iX, sizeof(iX));
        }
    }
    if (rc != DBM_OK) {
        memcpy(g_init_error, h->err, sizeof(g_init_error));
        free(h);
        return rc;
    }
    g_init_error[0] = 0;
    compute_layout(h);
    *out = h;
    return DBM_OK;
}

int dbm_equilibrium_matrix(const dbm_handle *h, int species, double *out)
{
    if (!h || !out || species < 0 || species >= h->p.nspecies) return DBM_ERR_INVALID;
    memcpy(out, h->cinv[species], sizeof(h->cinv[species]));
    return DBM_OK;
}

int dbm_get_layout(const dbm_handle *h, dbm_layout *out)
{
    if (!h || !out) return DBM_ERR_INVALID;
    *out = h->lay;
    return DBM_OK;
}

int dbm_state_bytes(const dbm_handle *h, size_t *bytes)
{
    if (!h || !bytes) return DBM_ERR_INVALID;
    *bytes = h->lay.bytes;
    return DBM_OK;
}

int dbm_scratch_bytes(const dbm_handle *h, size_t *bytes)
{
    if (!h || !bytes) return DBM_ERR_INVALID;
    *bytes = SCRATCH_HEAD + (size_t)CONS_BLOCKS * (h->p.nspecies + 4) * sizeof(double);
    return DBM_OK;
}

int dbm_bind(dbm_handle *h, void *f_a, void *f_b, void *scratch)
{
    if (!h) return DBM_ERR_INVALID;
    if (!f_a || !f_b || !scratch || f_a == f_b)
        return fail(h, DBM_ERR_INVALID, "bind needs two distinct state buffers and a scratch buffer");
    if (((uintptr_t)f_a | (uintptr_t)f_b | (uintptr_t)scratch) & 255)
        return fail(h, DBM_ERR_INVALID, "buffers must be 256-byte aligned");
    h->f[0] = f_a;
    h->f[1] = f_b;
    h->scratch = scratch;
    h->cur = 0;
    h->bound = 1;
    make_tensor_maps(h);
    const int want = h->p.step_kernel;
    if ((want != DBM_KERNEL_AUTO && want != DBM_KERNEL_GENERIC) || uses_acc(h->p))
        if (!h->tma_ok)
            return fail(h, DBM_ERR_INVALID, "no TMA-staged step kernel for these parameters");
    return DBM_OK;
}

static int check_bound(dbm_handle *h)
{
    if (!h) return DBM_ERR_INVALID;
    if (!h->bound) return fail(h, DBM_ERR_UNBOUND, "no state buffers bound (call dbm_bind)");
    return DBM_OK;
}

// Where a field array lives: device memory (or host memory the device reads
// in place), page-locked host memory, or pageable host memory the device
// cannot reach (refused rather than passed to a kernel).
enum { MEM_DEVICE = 0, MEM_PINNED = 1, MEM_UNREACHABLE = 2 };

static int mem_kind(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return MEM_UNREACHABLE;
    }
    if (a.type == cudaMemoryTypeHost) return MEM_PINNED;
    if (a.type == cudaMemoryTypeUnregistered) {
        int dev = 0, pageable = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, dev);
        return pageable ? MEM_DEVICE : MEM_UNREACHABLE;
    }
    return MEM_DEVICE;
}

// Staging area for transfers between page-locked host memory and a call:
// the state buffer the next step will overwrite (free between steps), when
// it holds `bytes`; NULL otherwise.
static char *staging(dbm_handle *h, size_t bytes)
{
    return h->lay.bytes >= bytes ? (char *)h->f[h->cur ^ 1] : nullptr;
}

int dbm_set_state(dbm_handle *h, const double *rho_s, const double *ux, const double *uy,
                  const double *T, void *stream)
{
    int rc = check_bound(h);
    if (rc) return rc;
    if (!rho_s || !ux || !uy || !T) return fail(h, DBM_ERR_INVALID, "set_state: null field");
    cudaStream_t st = (cudaStream_t)stream;
    // fields in page-locked host memory are copied (copy engine, no SM time)
    // into the free state buffer and read from there, when they fit
    const size_t N = (size_t)h->p.nx * h->p.ny, S = h->p.nspecies;
    const double *src[4] = {rho_s, ux, uy, T};
    const size_t len[4] = {S * N, N, N, N};
    int kind[4];
    bool any_pinned = false;
    for (int k = 0; k < 4; ++k) {
        kind[k] = mem_kind(src[k]);
        if (kind[k] == MEM_UNREACHABLE)
            return fail(h, DBM_ERR_INVALID, "set_state: field %d is in pageable host memory the device cannot read", k);
        any_pinned |= kind[k] == MEM_PINNED;
    }
    char *stg = any_pinned ? staging(h, (S + 3) * N * sizeof(double)) : nullptr;
    if (stg) {
        size_t off = 0;
        for (int k = 0; k < 4; ++k) {
            if (kind[k] == MEM_PINNED) {
                rc = set_cuda_error(h, cudaMemcpyAsync(stg + off, src[k], len[k] * sizeof(double),
                                                       cudaMemcpyHostToDevice, st),
                                    "set_state: copy of a host field");
                if (rc) return rc;
                src[k] = (const double *)(stg + off);
            }
            off += len[k] * sizeof(double);
        }
    }
    rc = set_cuda_error(h, cudaMemsetAsync(h->scratch, 0, SCRATCH_HEAD, st), "clear health flag");
    if (rc) return rc;
    rc = launch_set_state(h, h->f[h->cur], src[0], src[1], src[2], src[3], st);
    if (rc == DBM_OK) h->steps = 0;
    return rc;
}

int dbm_set_f(dbm_handle *h, const double *f, void *stream)
{
    int rc = check_bound(h);
    if (rc) return rc;
    if (!f) return fail(h, DBM_ERR_INVALID, "set_f: null f");
    cudaStream_t st = (cudaStream_t)stream;
    rc = set_cuda_error(h, cudaMemsetAsync(h->scratch, 0, SCRATCH_HEAD, st), "clear health flag");
    if (rc) return rc;
    rc = launch_set_f(h, h->f[h->cur], f, st);
    if (rc == DBM_OK) h->steps = 0;
    return rc;
}

int dbm_get_f(dbm_handle *h, double *f, void *stream)
{
    int rc = check_bound(h);
    if (rc) return rc;
    if (!f) return fail(h, DBM_ERR_INVALID, "get_f: null f");
    return launch_get_f(h, h->f[h->cur], f, (cudaStream_t)stream);
}

int dbm_step(dbm_handle *h, int nsteps, void *stream)
{
    int rc = check_bound(h);
    if (rc) return rc;
    if (nsteps < 0) return fail(h, DBM_ERR_INVALID, "nsteps=%d < 0", nsteps);
    cudaStream_t st = (cudaStream_t)stream;
    nvtxRangePushA("dbm_step");  // host-side range over the enqueueing of the launches
    for (int t = 0; t < nsteps && rc == DBM_OK; ++t) {
        rc = launch_step(h, h->cur, st);
        if (rc) break;
        h->cur ^= 1;
        h->steps += 1;
    }
    nvtxRangePop();
    return rc;
}

int dbm_moments(dbm_handle *h, double *out, void *stream)
{
    int rc = check_bound(h);
    if (rc) return rc;
    if (!out) return fail(h, DBM_ERR_INVALID, "moments: null out");
    const int kind = mem_kind(out);
    if (kind == MEM_UNREACHABLE)
        return fail(h, DBM_ERR_INVALID, "moments: out is in pageable host memory the device cannot write");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)(4 * h->p.nspecies + 5) * h->p.nx * h->p.ny * sizeof(double);
    char *stg = kind == MEM_PINNED ? staging(h, bytes) : nullptr;
    if (!stg) return launch_moments(h, h->f[h->cur], out, st);
    // page-locked host output: the fields go to the free state buffer, then
    // one copy (copy engine, no SM time) to the host
    rc = launch_moments(h, h->f[h->cur], (double *)stg, st);
    if (rc) return rc;
    return set_cuda_error(h, cudaMemcpyAsync(out, stg, bytes, cudaMemcpyDeviceToHost, st), "moments: copy to host");
}

int dbm_nonequilibrium(dbm_handle *h, double *out, void *stream)
{
    int rc = check_bound(h);
    if (rc) return rc;
    if (!out) return fail(h, DBM_ERR_INVALID, "nonequilibrium: null out");
    return launch_noneq(h, h->f[h->cur], out, (cudaStream_t)stream);
}

int dbm_conservation(dbm_handle *h, double *out, void *stream)
{
    int rc = check_bound(h);
    if (rc) return rc;
    if (!out) return fail(h, DBM_ERR_INVALID, "conservation: null out");
    return launch_conservation(h, h->f[h->cur], out, (cudaStream_t)stream);
}

int dbm_conservation_noalloc(dbm_handle *h, const void *state, double *out, void *stream)
{
    if (!h) return DBM_ERR_INVALID;
    if (!out) return fail(h, DBM_ERR_INVALID, "conservation_noalloc: null out");
    if (!state) {
        if (!h->bound) return fail(h, DBM_ERR_UNBOUND, "conservation_noalloc: no state given and none bound");
        state = h->f[h->cur];
    }
    const size_t need = (size_t)CONS_BLOCKS * (h->p.nspecies + 4);
    if (need > DBM_NOALLOC_SCRATCH_DOUBLES)
        return fail(h, DBM_ERR_INVALID,
                    "conservation_noalloc: its static scratch holds %d doubles, %d species need %zu "
                    "(use dbm_conservation with a scratch buffer)",
                    DBM_NOALLOC_SCRATCH_DOUBLES, h->p.nspecies, need);
    return launch_conservation_noalloc(h, state, out, (cudaStream_t)stream);
}

int dbm_status(dbm_handle *h, void *stream, unsigned *bits)
{
    int rc = check_bound(h);
    if (rc) return rc;
    unsigned v = 0;
    cudaStream_t st = (cudaStream_t)stream;
    rc = set_cuda_error(h, cudaMemcpyAsync(&v, h->scratch, sizeof(v), cudaMemcpyDeviceToHost, st),
                        "read health flag");
    if (rc) return rc;
    rc = set_cuda_error(h, cudaStreamSynchronize(st), "synchronise for health flag");
    if (rc) return rc;
    if (bits) *bits = v;
    if (v & DBM_HEALTH_BOUNDS) return fail(h, DBM_ERR_BOUNDS, "an index fell outside its buffer (flag %u)", v);
    if (v & DBM_HEALTH_TIMEOUT) return fail(h, DBM_ERR_TIMEOUT, "a tile copy timed out (flag %u)", v);
    if (v & DBM_HEALTH_NONFINITE) return fail(h, DBM_ERR_NONFINITE, "non-finite moment (flag %u)", v);
    if (v) return fail(h, DBM_ERR_NEGATIVE, "non-positive density/temperature or negative n* (flag %u)", v);
    return DBM_OK;
}

long long dbm_steps_taken(const dbm_handle *h) { return h ? h->steps : -1; }

int dbm_step_tile(const dbm_handle *h, int *tile_x, int *tile_y, int *cells_per_thread)
{
    if (!h) return DBM_ERR_INVALID;
    if (!h->bound) return DBM_ERR_UNBOUND;
    const bool tiled = h->tma_ok && h->p.step_kernel != DBM_KERNEL_GENERIC;
    if (tile_x) *tile_x = tiled ? h->tma_tx : 0;
    if (tile_y) *tile_y = tiled ? h->tma_ty : 0;
    if (cells_per_thread) *cells_per_thread = tiled ? h->tma_cw : 0;
    return DBM_OK;
}

const char *dbm_last_error(const dbm_handle *h) { return h ? h->err : "null handle"; }

void dbm_destroy(dbm_handle *h) { free(h); }

}  // extern "C"
