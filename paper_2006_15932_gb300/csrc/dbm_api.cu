// dbm_api.cu -- host side of the C ABI declared in include/dbm.h:
// parameter validation, the FP64 host inversion of the D2V16 moment matrix
// M (section "Discrete Boltzmann model": f^eq = M^-1 f-hat), buffer
// geometry, binding, and the enqueueing of the device kernels.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

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

// LU factorisation with partial pivoting (Doolittle, in place), then
// M^-1 column by column from forward and back substitution.
// Returns 0, or -1 when a pivot vanishes.
static int lu_inverse(const double A[Q][Q], double Ainv[Q][Q])
{
    double LU[Q][Q];
    int perm[Q];
    memcpy(LU, A, sizeof(LU));
    for (int i = 0; i < Q; ++i) perm[i] = i;
    for (int k = 0; k < Q; ++k) {
        int piv = k;
        double best = fabs(LU[k][k]);
        for (int r = k + 1; r < Q; ++r)
            if (fabs(LU[r][k]) > best) {
                best = fabs(LU[r][k]);
                piv = r;
            }
        if (best == 0.0) return -1;
        if (piv != k) {
            for (int c = 0; c < Q; ++c) {
                const double t = LU[k][c];
                LU[k][c] = LU[piv][c];
                LU[piv][c] = t;
            }
            const int t = perm[k];
            perm[k] = perm[piv];
            perm[piv] = t;
        }
        for (int r = k + 1; r < Q; ++r) {
            LU[r][k] /= LU[k][k];
            const double l = LU[r][k];
            for (int c = k + 1; c < Q; ++c) LU[r][c] -= l * LU[k][c];
        }
    }
    for (int col = 0; col < Q; ++col) {
        double z[Q];
        for (int r = 0; r < Q; ++r) {  // L z = P e_col
            double s = (perm[r] == col) ? 1.0 : 0.0;
            for (int c = 0; c < r; ++c) s -= LU[r][c] * z[c];
            z[r] = s;
        }
        for (int r = Q - 1; r >= 0; --r) {  // U x = z
            double s = z[r];
            for (int c = r + 1; c < Q; ++c) s -= LU[r][c] * Ainv[c][col];
            Ainv[r][col] = s / LU[r][r];
        }
    }
    return 0;
}

// Compensated dot product c - sum_k a[k] b[k*stride] (Ogita-Rump-Oishi
// "Dot2": error-free products via fma and error-free sums), as accurate as
// if accumulated in twice the working precision.
static double residual_dot2(double c, const double *a, const double *b, int stride)
{
    double s = c, err = 0.0;
    for (int k = 0; k < Q; ++k) {
        const double p = -a[k] * b[k * stride];
        const double pe = fma(-a[k], b[k * stride], -p);
        const double t = s + p;
        const double z = t - s;
        err += ((s - (t - z)) + (p - z)) + pe;
        s = t;
    }
    return s + err;
}

// Newton-Schulz style refinement X <- X + X (I - A X) with the residual
// from residual_dot2: the error of X squares at each pass, so X becomes the
// inverse of A rounded correctly to double (ties aside).  Exact conservation
// by f^eq = M^-1 f-hat needs this: a few ulps of error in M^-1 bias the
// mass, momentum and energy of every collision the same way, and that bias
// accumulates step after step.
static void refine_inverse(const double A[Q][Q], double X[Q][Q], int passes)
{
    for (int it = 0; it < passes; ++it) {
        double R[Q][Q], Xn[Q][Q];
        for (int r = 0; r < Q; ++r)
            for (int c = 0; c < Q; ++c) R[r][c] = residual_dot2(r == c ? 1.0 : 0.0, A[r], &X[0][c], Q);
        for (int r = 0; r < Q; ++r)
            for (int c = 0; c < Q; ++c) {
                double d = 0.0;
                for (int k = 0; k < Q; ++k) d += X[r][k] * R[k][c];
                Xn[r][c] = X[r][c] + d;
            }
        memcpy(X, Xn, sizeof(Xn));
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
    L.pitch = ((GX + p.nx + 2) + 31) / 32 * 32;
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
            if (lu_inverse(M, Mi) != 0) {
                rc = fail(h, DBM_ERR_SINGULAR, "species %d: moment matrix M is singular", s);
                break;
            }
            refine_inverse(M, Mi, 3);
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
    return DBM_OK;
}

static int check_bound(dbm_handle *h)
{
    if (!h) return DBM_ERR_INVALID;
    if (!h->bound) return fail(h, DBM_ERR_UNBOUND, "no state buffers bound (call dbm_bind)");
    return DBM_OK;
}

int dbm_set_state(dbm_handle *h, const double *rho_s, const double *ux, const double *uy,
                  const double *T, void *stream)
{
    int rc = check_bound(h);
    if (rc) return rc;
    if (!rho_s || !ux || !uy || !T) return fail(h, DBM_ERR_INVALID, "set_state: null field");
    cudaStream_t st = (cudaStream_t)stream;
    rc = set_cuda_error(h, cudaMemsetAsync(h->scratch, 0, SCRATCH_HEAD, st), "clear health flag");
    if (rc) return rc;
    if (h->p.precision == DBM_BF16DEV) return fail(h, DBM_ERR_INVALID, "BF16DEV not built yet");
    rc = launch_set_state(h, h->f[h->cur], rho_s, ux, uy, T, st);
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
    for (int t = 0; t < nsteps; ++t) {
        rc = launch_step(h, h->f[h->cur], h->f[h->cur ^ 1], st);
        if (rc) return rc;
        h->cur ^= 1;
        h->steps += 1;
    }
    return DBM_OK;
}

int dbm_moments(dbm_handle *h, double *out, void *stream)
{
    int rc = check_bound(h);
    if (rc) return rc;
    if (!out) return fail(h, DBM_ERR_INVALID, "moments: null out");
    return launch_moments(h, h->f[h->cur], out, (cudaStream_t)stream);
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
    if (v & DBM_HEALTH_NONFINITE) return fail(h, DBM_ERR_NONFINITE, "non-finite moment (flag %u)", v);
    if (v) return fail(h, DBM_ERR_NEGATIVE, "non-positive density/temperature or negative n* (flag %u)", v);
    return DBM_OK;
}

long long dbm_steps_taken(const dbm_handle *h) { return h ? h->steps : -1; }

const char *dbm_last_error(const dbm_handle *h) { return h ? h->err : "null handle"; }

void dbm_destroy(dbm_handle *h) { free(h); }

}  // extern "C"
