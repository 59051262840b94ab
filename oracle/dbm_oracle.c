/*
 * dbm_oracle.c -- plain FP64 CPU oracle of the multi-component discrete
 * Boltzmann model (DBM) on the D2V16 velocity set of Lin, Luo, Fei & Succi,
 * "A multi-component discrete Boltzmann model for nonequilibrium reactive
 * flows" (arXiv 2006.15932).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library and
 * never calls it.
 *
 * Every routine follows the paper in its own order and notation:
 *   - the D2V16 velocities and the moment matrix M (section "Discrete
 *     Boltzmann model", the D2V16 definition and the list of M_ki);
 *   - the equilibrium moments f-hat (same section, the list f-hat_1..16,
 *     which restates Eqs. relation1..relation7);
 *   - f^eq = M^-1 f-hat (same section);
 *   - the BGK collision, reaction and force terms (Eqs. CollisionTerm,
 *     ReactionTerm, ForceTerm) and the one-step Arrhenius rate (Eq.
 *     ReactionFunction and the omega_ov formula below it);
 *   - forward-Euler time stepping with the NND finite-difference scheme for
 *     v.grad f (section "Numerical simulation");
 *   - the nonequilibrium moments Delta_2, Delta_3,1, Delta_3, Delta_4,2
 *     (Eqs. Delta2, Delta31, Delta3, Delta42) and the energy / energy-flux
 *     diagnostics defined after them.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   R1  mixture u and T are the values for which the collision term conserves
 *       total momentum and energy exactly for any tau^sigma:
 *         u = sum(rho^s u^s / tau^s) / sum(rho^s / tau^s)
 *         T = sum((m^s E^s - rho^s u.u) / tau^s) / sum(n^s (D+I^s) / tau^s)
 *       with E^s = sum_i f_i^s (v_i.v_i + eta_i^2).
 *   R2  reaction state after a time tau^s at the current rate:
 *         n^s* = n^s + tau^s a^s omega_ov,  T*^s = T + tau^s T',
 *         T' = [Q omega_ov - (T/2) sum_s (D+I^s) a^s omega_ov]
 *              / [(1/2) sum_s n^s (D+I^s)].
 *   R3  force: u^dag,s = u^s + a tau^s, T^dag,s = T^s.
 *   R4  NND flux (Zhang's published form), see nnd_dflux().
 *   R5  boundaries: two ghost layers, periodic wrap or zero-gradient copy.
 *   R6  diagnostics use the same mixture equilibrium f^eq(n^s, u, T) as the
 *       collision term.
 *   M_9i is printed as a duplicate of M_8i; it is read as
 *   (v^2 + eta^2) v_iy, the row that matches f-hat_9.
 *   The third-order relation uses the mixture T like f-hat_10..13.
 *
 * Layout of a distribution field: f[s][i][y][x], x fastest, no ghosts,
 * nx*ny cells, species-major.  All arithmetic is IEEE double; build with
 * -ffp-contract=off so that no multiply-add is fused.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_Q 16
#define ORC_DIM 2.0 /* D, the number of space dimensions */
#define ORC_MAXS 8

enum { ORC_PERIODIC = 0, ORC_OUTFLOW = 1 };

/* status bits returned by the stepping routines */
enum {
    ORC_OK = 0,
    ORC_BAD_DENSITY = 1,      /* n^s < -1e-6 sum|n|, no matter, or not finite */
    ORC_BAD_TEMPERATURE = 2,  /* T <= 0 or not finite */
    ORC_NEGATIVE_NSTAR = 4,   /* n^s* < 0 after the reaction */
    ORC_NONFINITE = 8         /* a non-finite f was produced */
};

typedef struct orc_species {
    double m;       /* molar mass m^s */
    double I;       /* extra degrees of freedom I^s */
    double tau;     /* relaxation time tau^s */
    double v[4];    /* ring speeds v_a..v_d */
    double eta[4];  /* ring internal speeds eta_a..eta_d */
    double a;       /* stoichiometric coefficient a^s */
} orc_species;

typedef struct orc_params {
    int nx, ny, ns;
    double dx, dy, dt;
    int bc_x, bc_y;
    int fuel, oxid;
    double k_ov, Ea_over_R, Q;
    double ax, ay;
    orc_species sp[ORC_MAXS];
} orc_params;

/* ------------------------------------------------------------------ */
/* Velocity space                                                      */
/* ------------------------------------------------------------------ */

/* D2V16 (section "Discrete Boltzmann model"): rings a and c hold the four
 * cyclic permutations of v(+-1, 0); rings b and d hold v(+-1, +-1).
 * Within a ring the order is +x, +y, -x, -y (axis rings) or
 * (+,+), (-,+), (-,-), (+,-) (diagonal rings). */
void orc_velocities(const orc_species *sp, double vx[ORC_Q], double vy[ORC_Q],
                    double eta[ORC_Q])
{
    static const double axis[4][2] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
    static const double diag[4][2] = {{1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    for (int r = 0; r < 4; ++r) {
        for (int k = 0; k < 4; ++k) {
            const int i = 4 * r + k;
            const double *d = (r % 2 == 0) ? axis[k] : diag[k];
            vx[i] = sp->v[r] * d[0];
            vy[i] = sp->v[r] * d[1];
            eta[i] = sp->eta[r];
        }
    }
}

/* The 16x16 matrix M with f-hat = M f (rows k = 1..16 of the M_ki list;
 * row 9 read as (v^2+eta^2) v_y).  Row-major: M[k*16 + i]. */
void orc_moment_matrix(const double vx[ORC_Q], const double vy[ORC_Q],
                       const double eta[ORC_Q], double M[ORC_Q * ORC_Q])
{
    for (int i = 0; i < ORC_Q; ++i) {
        const double x = vx[i], y = vy[i];
        const double q = x * x + y * y + eta[i] * eta[i];
        M[0 * ORC_Q + i] = 1.0;
        M[1 * ORC_Q + i] = x;
        M[2 * ORC_Q + i] = y;
        M[3 * ORC_Q + i] = q;
        M[4 * ORC_Q + i] = x * x;
        M[5 * ORC_Q + i] = x * y;
        M[6 * ORC_Q + i] = y * y;
        M[7 * ORC_Q + i] = q * x;
        M[8 * ORC_Q + i] = q * y;
        M[9 * ORC_Q + i] = x * x * x;
        M[10 * ORC_Q + i] = x * x * y;
        M[11 * ORC_Q + i] = x * y * y;
        M[12 * ORC_Q + i] = y * y * y;
        M[13 * ORC_Q + i] = q * x * x;
        M[14 * ORC_Q + i] = q * x * y;
        M[15 * ORC_Q + i] = q * y * y;
    }
}

/* Textbook Gauss-Jordan elimination with partial pivoting on [A | I].
 * Returns 0, or -1 when a pivot is exactly zero (A singular). */
int orc_invert(const double *A, double *Ainv, int n)
{
    double *w = (double *)malloc(sizeof(double) * (size_t)n * 2 * n);
    if (!w) return -2;
    for (int r = 0; r < n; ++r) {
        for (int c = 0; c < n; ++c) w[r * 2 * n + c] = A[r * n + c];
        for (int c = 0; c < n; ++c) w[r * 2 * n + n + c] = (r == c) ? 1.0 : 0.0;
    }
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(w[r * 2 * n + col]) > fabs(w[piv * 2 * n + col])) piv = r;
        if (w[piv * 2 * n + col] == 0.0) {
            free(w);
            return -1;
        }
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = w[col * 2 * n + c];
                w[col * 2 * n + c] = w[piv * 2 * n + c];
                w[piv * 2 * n + c] = t;
            }
        const double p = w[col * 2 * n + col];
        for (int c = 0; c < 2 * n; ++c) w[col * 2 * n + c] /= p;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            const double fac = w[r * 2 * n + col];
            if (fac == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) w[r * 2 * n + c] -= fac * w[col * 2 * n + c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = w[r * 2 * n + n + c];
    free(w);
    return 0;
}

/* Error-free transformations: s + e == a + b and p + e == a * b exactly. */
static void two_sum(double a, double b, double *s, double *e)
{
    const double t = a + b, z = t - a;
    *s = t;
    *e = (a - (t - z)) + (b - z);
}
static void two_prod(double a, double b, double *p, double *e)
{
    *p = a * b;
    *e = fma(a, b, -*p);
}

/* Iterative refinement X <- X + X (I - A X) of an approximate inverse.  The
 * residual I - A X is accumulated in double-double (error-free products and
 * sums), so each pass squares the relative error and X ends as the
 * correctly rounded inverse of the double matrix A (up to exact ties). */
void orc_refine_inverse(const double *A, double *X, int n, int passes)
{
    double *R = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *D = (double *)malloc(sizeof(double) * (size_t)n * n);
    if (!R || !D) {
        free(R);
        free(D);
        return;
    }
    for (int it = 0; it < passes; ++it) {
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c) {
                double hi = (r == c) ? 1.0 : 0.0, lo = 0.0;
                for (int k = 0; k < n; ++k) {
                    double p, pe, s, se;
                    two_prod(-A[r * n + k], X[k * n + c], &p, &pe);
                    two_sum(hi, p, &s, &se);
                    hi = s;
                    lo += se + pe;
                }
                R[r * n + c] = hi + lo;
            }
        for (int r = 0; r < n; ++r)
            for (int c = 0; c < n; ++c) {
                double s = 0.0;
                for (int k = 0; k < n; ++k) s += X[r * n + k] * R[k * n + c];
                D[r * n + c] = s;
            }
        for (int k = 0; k < n * n; ++k) X[k] += D[k];
    }
    free(R);
    free(D);
}

/* M^-1 for one species (the "C^-1" of the equilibrium inversion): the
 * inverse of the double matrix M, rounded correctly to double (Gauss-Jordan
 * followed by refinement).  An accurate M^-1 matters: an error of a few
 * units in the last place of M^-1 breaks the exact conservation of mass,
 * momentum and energy by f^eq by as much, and that bias accumulates over
 * thousands of steps. */
int orc_species_minv(const orc_species *sp, double Minv[ORC_Q * ORC_Q])
{
    double vx[ORC_Q], vy[ORC_Q], eta[ORC_Q], M[ORC_Q * ORC_Q];
    orc_velocities(sp, vx, vy, eta);
    orc_moment_matrix(vx, vy, eta, M);
    if (orc_invert(M, Minv, ORC_Q) != 0) return -1;
    orc_refine_inverse(M, Minv, ORC_Q, 3);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Equilibrium                                                         */
/* ------------------------------------------------------------------ */

/* The 16 equilibrium moments f-hat_1..16 of species with mass m and extra
 * degrees of freedom I at (n, u, T); theta = T/m, D = 2. */
void orc_fhat(double n, double ux, double uy, double T, double m, double I,
              double fh[ORC_Q])
{
    const double D = ORC_DIM;
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

/* y = A x for a 16x16 row-major A. */
void orc_matvec(const double A[ORC_Q * ORC_Q], const double x[ORC_Q], double y[ORC_Q])
{
    for (int r = 0; r < ORC_Q; ++r) {
        double s = 0.0;
        for (int c = 0; c < ORC_Q; ++c) s += A[r * ORC_Q + c] * x[c];
        y[r] = s;
    }
}

/* f^eq = M^-1 f-hat(n, u, T). */
void orc_feq(const double Minv[ORC_Q * ORC_Q], double n, double ux, double uy, double T,
             double m, double I, double feq[ORC_Q])
{
    double fh[ORC_Q];
    orc_fhat(n, ux, uy, T, m, I, fh);
    orc_matvec(Minv, fh, feq);
}

/* ------------------------------------------------------------------ */
/* Macroscopic quantities                                              */
/* ------------------------------------------------------------------ */

/* Species moments from f (Eqs. relation1..relation3 applied to f):
 * n = sum f, n u = sum f v, E = sum f (v.v + eta^2),
 * T^s = m (E/n - u.u) / (D + I). */
void orc_species_moments(const double f[ORC_Q], const double vx[ORC_Q], const double vy[ORC_Q],
                         const double eta[ORC_Q], double m, double I, double *n,
                         double *ux, double *uy, double *Ts, double *E)
{
    double sn = 0.0, jx = 0.0, jy = 0.0, se = 0.0;
    for (int i = 0; i < ORC_Q; ++i) {
        sn += f[i];
        jx += f[i] * vx[i];
        jy += f[i] * vy[i];
        se += f[i] * (vx[i] * vx[i] + vy[i] * vy[i] + eta[i] * eta[i]);
    }
    *n = sn;
    *E = se;
    if (sn == 0.0) {
        /* an absent species: report zero velocity and temperature */
        *ux = 0.0;
        *uy = 0.0;
        *Ts = 0.0;
        return;
    }
    *ux = jx / sn;
    *uy = jy / sn;
    *Ts = m * (se / sn - ((*ux) * (*ux) + (*uy) * (*uy))) / (ORC_DIM + I);
}

/* Mixture velocity and temperature, reading R1. */
void orc_mixture(int ns, const orc_species *sp, const double *n, const double *ux,
                 const double *uy, const double *E, double *Ux, double *Uy, double *T)
{
    double w = 0.0, wx = 0.0, wy = 0.0;
    for (int s = 0; s < ns; ++s) {
        const double rho = sp[s].m * n[s];
        w += rho / sp[s].tau;
        wx += rho * ux[s] / sp[s].tau;
        wy += rho * uy[s] / sp[s].tau;
    }
    *Ux = wx / w;
    *Uy = wy / w;
    const double u2 = (*Ux) * (*Ux) + (*Uy) * (*Uy);
    double num = 0.0, den = 0.0;
    for (int s = 0; s < ns; ++s) {
        const double rho = sp[s].m * n[s];
        num += (sp[s].m * E[s] - rho * u2) / sp[s].tau;
        den += n[s] * (ORC_DIM + sp[s].I) / sp[s].tau;
    }
    *T = num / den;
}

/* One-step overall rate omega_ov = k_ov n^fuel n^ox exp(-E_a / (R T)). */
double orc_omega(const orc_params *p, const double *n, double T)
{
    if (p->k_ov == 0.0) return 0.0;
    return p->k_ov * n[p->fuel] * n[p->oxid] * exp(-p->Ea_over_R / T);
}

/* Reading R2: T' from the heat release Q per mole of reaction. */
double orc_dTdt(const orc_params *p, const double *n, double T, double omega)
{
    double src = 0.0, cap = 0.0;
    for (int s = 0; s < p->ns; ++s) {
        src += (ORC_DIM + p->sp[s].I) * p->sp[s].a * omega;
        cap += n[s] * (ORC_DIM + p->sp[s].I);
    }
    return (p->Q * omega - 0.5 * T * src) / (0.5 * cap);
}

/* Collision + reaction + force at one cell: rhs[s][i] = Omega + R + G for
 * the S x 16 distributions fc[s][i] of that cell.  Minv holds S blocks of
 * 16x16.  Returns status bits. */
int orc_cell_rhs(const orc_params *p, const double *Minv, const double *fc, double *rhs)
{
    const int ns = p->ns;
    double n[ORC_MAXS], ux[ORC_MAXS], uy[ORC_MAXS], Ts[ORC_MAXS], E[ORC_MAXS];
    int st = ORC_OK;
    for (int s = 0; s < ns; ++s) {
        double vx[ORC_Q], vy[ORC_Q], eta[ORC_Q];
        orc_velocities(&p->sp[s], vx, vy, eta);
        orc_species_moments(fc + s * ORC_Q, vx, vy, eta, p->sp[s].m, p->sp[s].I, &n[s], &ux[s],
                            &uy[s], &Ts[s], &E[s]);
    }
    /* a species may be absent (n = 0) or slightly negative from numerical
     * diffusion; flag densities below -1e-6 of the mixture, or a mixture
     * without matter */
    double ntot = 0.0;
    for (int s = 0; s < ns; ++s) ntot += fabs(n[s]);
    for (int s = 0; s < ns; ++s)
        if (!(n[s] >= -1e-6 * ntot) || !isfinite(n[s])) st |= ORC_BAD_DENSITY;
    if (!(ntot > 0.0)) st |= ORC_BAD_DENSITY;
    double Ux, Uy, T;
    orc_mixture(ns, p->sp, n, ux, uy, E, &Ux, &Uy, &T);
    if (!(T > 0.0) || !isfinite(T)) st |= ORC_BAD_TEMPERATURE;
    const double omega = orc_omega(p, n, T);
    const double dTdt = orc_dTdt(p, n, T, omega);
    for (int s = 0; s < ns; ++s) {
        const orc_species *sp = &p->sp[s];
        const double *Mi = Minv + s * ORC_Q * ORC_Q;
        const double tau = sp->tau;
        /* Eq. CollisionTerm: f^eq(n^s, u, T) */
        double feq[ORC_Q];
        orc_feq(Mi, n[s], Ux, Uy, T, sp->m, sp->I, feq);
        /* Eq. ReactionTerm: f^eq(n^s*, u, T*) with reading R2 */
        const double nstar = n[s] + tau * sp->a * omega;
        const double Tstar = T + tau * dTdt;
        if (p->k_ov != 0.0 && nstar < -1e-6 * ntot) st |= ORC_NEGATIVE_NSTAR;
        double feq_r[ORC_Q];
        orc_feq(Mi, nstar, Ux, Uy, Tstar, sp->m, sp->I, feq_r);
        /* Eq. ForceTerm with reading R3: u^dag = u^s + a tau, T^dag = T^s */
        double feq_f1[ORC_Q], feq_f0[ORC_Q];
        orc_feq(Mi, n[s], ux[s] + p->ax * tau, uy[s] + p->ay * tau, Ts[s], sp->m, sp->I, feq_f1);
        orc_feq(Mi, n[s], ux[s], uy[s], Ts[s], sp->m, sp->I, feq_f0);
        for (int i = 0; i < ORC_Q; ++i) {
            const double f = fc[s * ORC_Q + i];
            const double Omega = -(f - feq[i]) / tau;
            const double R = (feq_r[i] - feq[i]) / tau;
            const double G = (feq_f1[i] - feq_f0[i]) / tau;
            rhs[s * ORC_Q + i] = Omega + R + G;
        }
    }
    return st;
}

/* ------------------------------------------------------------------ */
/* NND advection (section "Numerical simulation", reading R4)          */
/* ------------------------------------------------------------------ */

static double sgn(double a) { return (a > 0.0) ? 1.0 : ((a < 0.0) ? -1.0 : 0.0); }

/* minmod(a, b) = (sgn a + sgn b)/2 * min(|a|, |b|) */
double orc_minmod(double a, double b)
{
    const double fa = fabs(a), fb = fabs(b);
    return 0.5 * (sgn(a) + sgn(b)) * (fa < fb ? fa : fb);
}

/* d(c f)/dx at node j from w[0..4] = f_{j-2..j+2} and spacing h, by the NND
 * scheme: F = c f is split into F+ = (c+|c|)/2 f and F- = (c-|c|)/2 f and
 *   H_{j+1/2} = F+_j + mm(dF+_{j-1/2}, dF+_{j+1/2})/2
 *             + F-_{j+1} - mm(dF-_{j+1/2}, dF-_{j+3/2})/2,
 * dF_{k+1/2} = F_{k+1} - F_k, and d(cf)/dx = (H_{j+1/2} - H_{j-1/2}) / h. */
double orc_nnd_dflux(double c, const double w[5], double h)
{
    const double cp = 0.5 * (c + fabs(c)), cm = 0.5 * (c - fabs(c));
    double Fp[5], Fm[5];
    for (int k = 0; k < 5; ++k) {
        Fp[k] = cp * w[k];
        Fm[k] = cm * w[k];
    }
    /* node j is index 2 */
    const double Hr = Fp[2] + 0.5 * orc_minmod(Fp[2] - Fp[1], Fp[3] - Fp[2]) + Fm[3] -
                      0.5 * orc_minmod(Fm[3] - Fm[2], Fm[4] - Fm[3]);
    const double Hl = Fp[1] + 0.5 * orc_minmod(Fp[1] - Fp[0], Fp[2] - Fp[1]) + Fm[2] -
                      0.5 * orc_minmod(Fm[2] - Fm[1], Fm[3] - Fm[2]);
    return (Hr - Hl) / h;
}

/* ------------------------------------------------------------------ */
/* Grid                                                                */
/* ------------------------------------------------------------------ */

/* Reading R5: index of the cell whose value a (possibly ghost) index k
 * takes; periodic wrap or zero-gradient (copy of the edge cell). */
static int bc_index(int k, int n, int bc)
{
    if (bc == ORC_PERIODIC) return ((k % n) + n) % n;
    return k < 0 ? 0 : (k >= n ? n - 1 : k);
}

static size_t fidx(const orc_params *p, int s, int i, int x, int y)
{
    return (((size_t)s * ORC_Q + i) * p->ny + y) * p->nx + x;
}

/* All species M^-1 blocks (S x 256).  Returns -1 if any M is singular. */
int orc_prepare(const orc_params *p, double *Minv)
{
    for (int s = 0; s < p->ns; ++s)
        if (orc_species_minv(&p->sp[s], Minv + s * ORC_Q * ORC_Q) != 0) return -1;
    return 0;
}

/* New f of the cells (x, y) with x0 <= x < x1 and y0 <= y < y1 after one
 * forward-Euler step: f^{n+1} = f^n + dt [Omega + R + G - d(v_x f)/dx -
 * d(v_y f)/dy], everything on the right taken at time n.  fin is the whole
 * field; fout holds only the region, [s][i][y - y0][x - x0].  Returns
 * status bits. */
/* Threads of the OpenMP loops over rows (for timing the oracle on one core
 * and on all of them; no effect on any result).  n > 0 sets the number;
 * returns the number the next parallel loop uses (1 without OpenMP). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_step_region(const orc_params *p, const double *Minv, const double *fin, double *fout,
                    int x0, int x1, int y0, int y1)
{
    const int rw = x1 - x0, rh = y1 - y0;
    const int ns = p->ns;
    int status = ORC_OK;
#pragma omp parallel for schedule(static) reduction(| : status)
    for (int y = y0; y < y1; ++y) {
        double vx[ORC_MAXS][ORC_Q], vy[ORC_MAXS][ORC_Q], eta[ORC_MAXS][ORC_Q];
        for (int s = 0; s < ns; ++s) orc_velocities(&p->sp[s], vx[s], vy[s], eta[s]);
        double fc[ORC_MAXS * ORC_Q], rhs[ORC_MAXS * ORC_Q];
        for (int x = x0; x < x1; ++x) {
            for (int s = 0; s < ns; ++s)
                for (int i = 0; i < ORC_Q; ++i) fc[s * ORC_Q + i] = fin[fidx(p, s, i, x, y)];
            status |= orc_cell_rhs(p, Minv, fc, rhs);
            for (int s = 0; s < ns; ++s) {
                for (int i = 0; i < ORC_Q; ++i) {
                    double adv = 0.0;
                    if (vx[s][i] != 0.0) {
                        double w[5];
                        for (int k = -2; k <= 2; ++k)
                            w[k + 2] = fin[fidx(p, s, i, bc_index(x + k, p->nx, p->bc_x), y)];
                        adv += orc_nnd_dflux(vx[s][i], w, p->dx);
                    }
                    if (vy[s][i] != 0.0) {
                        double w[5];
                        for (int k = -2; k <= 2; ++k)
                            w[k + 2] = fin[fidx(p, s, i, x, bc_index(y + k, p->ny, p->bc_y))];
                        adv += orc_nnd_dflux(vy[s][i], w, p->dy);
                    }
                    const double fnew = fc[s * ORC_Q + i] + p->dt * (rhs[s * ORC_Q + i] - adv);
                    if (!isfinite(fnew)) status |= ORC_NONFINITE;
                    fout[(((size_t)s * ORC_Q + i) * rh + (y - y0)) * rw + (x - x0)] = fnew;
                }
            }
        }
    }
    return status;
}

/* nsteps steps of the whole grid, in place in f (work is a second buffer
 * of the same size).  Stops at the first step that raises a status bit. */
int orc_run(const orc_params *p, double *f, double *work, int nsteps)
{
    double *Minv = (double *)malloc(sizeof(double) * ORC_Q * ORC_Q * p->ns);
    if (!Minv) return -2;
    if (orc_prepare(p, Minv) != 0) {
        free(Minv);
        return -1;
    }
    const size_t total = (size_t)p->ns * ORC_Q * p->nx * p->ny;
    double *a = f, *b = work;
    int status = ORC_OK;
    for (int t = 0; t < nsteps && status == ORC_OK; ++t) {
        status = orc_step_region(p, Minv, a, b, 0, p->nx, 0, p->ny);
        double *tmp = a;
        a = b;
        b = tmp;
    }
    if (a != f) memcpy(f, a, sizeof(double) * total);
    free(Minv);
    return status;
}

/* f = f^eq(n^s = rho^s/m^s, u, T) from macroscopic fields
 * rho_s[s][y][x], ux, uy, T[y][x]. */
int orc_init_feq(const orc_params *p, const double *rho_s, const double *ux, const double *uy,
                 const double *T, double *f)
{
    double *Minv = (double *)malloc(sizeof(double) * ORC_Q * ORC_Q * p->ns);
    if (!Minv) return -2;
    if (orc_prepare(p, Minv) != 0) {
        free(Minv);
        return -1;
    }
    const size_t N = (size_t)p->nx * p->ny;
    for (int s = 0; s < p->ns; ++s) {
        for (size_t c = 0; c < N; ++c) {
            double feq[ORC_Q];
            orc_feq(Minv + s * ORC_Q * ORC_Q, rho_s[s * N + c] / p->sp[s].m, ux[c], uy[c], T[c],
                    p->sp[s].m, p->sp[s].I, feq);
            for (int i = 0; i < ORC_Q; ++i) f[((size_t)s * ORC_Q + i) * N + c] = feq[i];
        }
    }
    free(Minv);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Outputs                                                             */
/* ------------------------------------------------------------------ */

/* Per-cell macroscopic fields, field-major out[k][y][x], k =
 *   4s+0: n^s, 4s+1: u^s_x, 4s+2: u^s_y, 4s+3: T^s   (s = 0..S-1)
 *   4S+0: rho, 4S+1: u_x, 4S+2: u_y, 4S+3: T, 4S+4: p = n T
 * with rho = sum m^s n^s, n = sum n^s and (u, T) from reading R1. */
void orc_moments(const orc_params *p, const double *f, double *out)
{
    const int ns = p->ns;
    const size_t N = (size_t)p->nx * p->ny;
    for (size_t c = 0; c < N; ++c) {
        double n[ORC_MAXS], ux[ORC_MAXS], uy[ORC_MAXS], Ts[ORC_MAXS], E[ORC_MAXS];
        double rho = 0.0, ntot = 0.0;
        for (int s = 0; s < ns; ++s) {
            double vx[ORC_Q], vy[ORC_Q], eta[ORC_Q], fc[ORC_Q];
            orc_velocities(&p->sp[s], vx, vy, eta);
            for (int i = 0; i < ORC_Q; ++i) fc[i] = f[((size_t)s * ORC_Q + i) * N + c];
            orc_species_moments(fc, vx, vy, eta, p->sp[s].m, p->sp[s].I, &n[s], &ux[s], &uy[s],
                                &Ts[s], &E[s]);
            out[(size_t)(4 * s + 0) * N + c] = n[s];
            out[(size_t)(4 * s + 1) * N + c] = ux[s];
            out[(size_t)(4 * s + 2) * N + c] = uy[s];
            out[(size_t)(4 * s + 3) * N + c] = Ts[s];
            rho += p->sp[s].m * n[s];
            ntot += n[s];
        }
        double Ux, Uy, T;
        orc_mixture(ns, p->sp, n, ux, uy, E, &Ux, &Uy, &T);
        out[(size_t)(4 * ns + 0) * N + c] = rho;
        out[(size_t)(4 * ns + 1) * N + c] = Ux;
        out[(size_t)(4 * ns + 2) * N + c] = Uy;
        out[(size_t)(4 * ns + 3) * N + c] = T;
        out[(size_t)(4 * ns + 4) * N + c] = ntot * T;
    }
}

/* Nonequilibrium moments (Eqs. Delta2, Delta31, Delta3, Delta42) and the
 * energy diagnostics that follow them, 20 fields per species,
 * out[20 s + k][y][x]:
 *   k = 0..2   Delta_2 xx, xy, yy
 *   k = 3..4   Delta_3,1 x, y
 *   k = 5..8   Delta_3 xxx, xxy, xyy, yyy
 *   k = 9..11  Delta_4,2 xx, xy, yy
 *   k = 12..13 (1/2) M_2xx(f), (1/2) M_2yy(f)        translational energy
 *   k = 14..15 (1/2) M_2xx(f^eq), (1/2) M_2yy(f^eq)
 *   k = 16..17 (1/2) M_3,1x(f), (1/2) M_3,1y(f)      energy flux
 *   k = 18..19 (1/2) M_3,1x(f^eq), (1/2) M_3,1y(f^eq)
 * Every sum carries the factor m^s; f^eq = f^eq(n^s, u, T) (reading R6). */
void orc_nonequilibrium(const orc_params *p, const double *f, double *out)
{
    const int ns = p->ns;
    const size_t N = (size_t)p->nx * p->ny;
    double *Minv = (double *)malloc(sizeof(double) * ORC_Q * ORC_Q * ns);
    if (!Minv) return;
    orc_prepare(p, Minv);
    for (size_t c = 0; c < N; ++c) {
        double n[ORC_MAXS], ux[ORC_MAXS], uy[ORC_MAXS], Ts[ORC_MAXS], E[ORC_MAXS];
        double vx[ORC_MAXS][ORC_Q], vy[ORC_MAXS][ORC_Q], eta[ORC_MAXS][ORC_Q];
        double fc[ORC_MAXS][ORC_Q];
        for (int s = 0; s < ns; ++s) {
            orc_velocities(&p->sp[s], vx[s], vy[s], eta[s]);
            for (int i = 0; i < ORC_Q; ++i) fc[s][i] = f[((size_t)s * ORC_Q + i) * N + c];
            orc_species_moments(fc[s], vx[s], vy[s], eta[s], p->sp[s].m, p->sp[s].I, &n[s],
                                &ux[s], &uy[s], &Ts[s], &E[s]);
        }
        double Ux, Uy, T;
        orc_mixture(ns, p->sp, n, ux, uy, E, &Ux, &Uy, &T);
        for (int s = 0; s < ns; ++s) {
            const double m = p->sp[s].m;
            double feq[ORC_Q];
            orc_feq(Minv + s * ORC_Q * ORC_Q, n[s], Ux, Uy, T, m, p->sp[s].I, feq);
            double acc[20];
            for (int k = 0; k < 20; ++k) acc[k] = 0.0;
            for (int i = 0; i < ORC_Q; ++i) {
                const double x = vx[s][i], y = vy[s][i];
                const double q = x * x + y * y + eta[s][i] * eta[s][i];
                const double d = m * (fc[s][i] - feq[i]);
                const double mf = m * fc[s][i], me = m * feq[i];
                acc[0] += d * x * x;
                acc[1] += d * x * y;
                acc[2] += d * y * y;
                acc[3] += d * q * x;
                acc[4] += d * q * y;
                acc[5] += d * x * x * x;
                acc[6] += d * x * x * y;
                acc[7] += d * x * y * y;
                acc[8] += d * y * y * y;
                acc[9] += d * q * x * x;
                acc[10] += d * q * x * y;
                acc[11] += d * q * y * y;
                acc[12] += 0.5 * mf * x * x;
                acc[13] += 0.5 * mf * y * y;
                acc[14] += 0.5 * me * x * x;
                acc[15] += 0.5 * me * y * y;
                acc[16] += 0.5 * mf * q * x;
                acc[17] += 0.5 * mf * q * y;
                acc[18] += 0.5 * me * q * x;
                acc[19] += 0.5 * me * q * y;
            }
            for (int k = 0; k < 20; ++k) out[(size_t)(20 * s + k) * N + c] = acc[k];
        }
    }
    free(Minv);
}

/* Conserved totals summed over all cells, out[0..S+3]:
 *   out[s]   = sum rho^s                      (s = 0..S-1)
 *   out[S]   = sum rho u_x,  out[S+1] = sum rho u_y
 *   out[S+2] = sum_s (m^s/2) sum_i f (v.v + eta^2)      total energy
 *   out[S+3] = sum Q n^fuel / |a^fuel|    heat still bound in the fuel
 *              (0 without a reaction). */
void orc_conservation(const orc_params *p, const double *f, double *out)
{
    const int ns = p->ns;
    const size_t N = (size_t)p->nx * p->ny;
    for (int k = 0; k < ns + 4; ++k) out[k] = 0.0;
    for (int s = 0; s < ns; ++s) {
        double vx[ORC_Q], vy[ORC_Q], eta[ORC_Q];
        orc_velocities(&p->sp[s], vx, vy, eta);
        const double m = p->sp[s].m;
        for (size_t c = 0; c < N; ++c) {
            for (int i = 0; i < ORC_Q; ++i) {
                const double fv = f[((size_t)s * ORC_Q + i) * N + c];
                out[s] += m * fv;
                out[ns] += m * fv * vx[i];
                out[ns + 1] += m * fv * vy[i];
                out[ns + 2] += 0.5 * m * fv * (vx[i] * vx[i] + vy[i] * vy[i] + eta[i] * eta[i]);
                if (p->k_ov != 0.0 && s == p->fuel)
                    out[ns + 3] += p->Q * fv / fabs(p->sp[s].a);
            }
        }
    }
}
