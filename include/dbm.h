/*
 * dbm.h -- C ABI of the GB300 (sm_103a) solver for the multi-component
 * discrete Boltzmann model (DBM) of Lin, Luo, Fei & Succi, "A multi-component
 * discrete Boltzmann model for nonequilibrium reactive flows"
 * (arXiv 2006.15932), on its two-dimensional sixteen-velocity (D2V16) set.
 *
 * One call of dbm_step advances the species distributions f^s_i of every
 * cell by forward-Euler steps of the discrete Boltzmann equation (Eq.
 * DiscreteBoltzmannEquation):
 *     f^{n+1} = f^n + dt [ Omega + R + G - v_i . grad f^n ],
 * Omega = BGK collision (Eq. CollisionTerm), R = reaction (Eq. ReactionTerm),
 * G = force (Eq. ForceTerm), with the equilibria f^eq = M^-1 f-hat built from
 * the moment relations relation1..relation7, and the advection discretised by
 * the NND scheme (section "Numerical simulation").
 *
 * Conventions
 *  - Every call returns int: DBM_OK (0) or a negative dbm_status_code.
 *    Nothing is thrown across the ABI.  dbm_last_error() gives a message.
 *  - The library owns only the handle (host memory) and the per-species
 *    constants it derives (carried in kernel parameters).  The caller owns
 *    every device buffer and every stream; no call allocates device memory.
 *  - "stream" arguments are cudaStream_t values passed as void* (NULL is the
 *    legacy default stream).  Calls marked async only enqueue work.
 *  - Field arrays exchanged with the caller are dense FP64, x fastest:
 *    a scalar field is [ny][nx], a species field [S][ny][nx], a distribution
 *    [S][16][ny][nx].  They may live in device memory or in page-locked host
 *    memory that the device can address (cudaHostAlloc / cudaHostRegister);
 *    pageable host memory is accepted only where the device can read it in
 *    place (cudaDevAttrPageableMemoryAccess), else refused with
 *    DBM_ERR_INVALID.  dbm_set_state and dbm_moments move page-locked host
 *    fields through the handle's second state buffer (free between steps;
 *    the next step overwrites it) with one stream-ordered copy each, so the
 *    copy engine carries them and no SM waits on the host link; where that
 *    buffer is too small (one species, or BF16DEV moments) the kernels read
 *    or write the host memory directly.  Either way the results are the
 *    same bits as with device arrays.
 *  - Velocity index i = 0..15 runs over the rings a, b, c, d (4 each) in the
 *    order of the D2V16 definition: axis rings (v,0), (0,v), (-v,0), (0,-v);
 *    diagonal rings (v,v), (-v,v), (-v,-v), (v,-v).
 */
#ifndef DBM_H
#define DBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DBM_Q 16
#define DBM_MAX_SPECIES 8

enum dbm_bc { DBM_BC_PERIODIC = 0, DBM_BC_OUTFLOW = 1 };

/* Arithmetic and storage of the stepped state.  Every output array is
 * FP64.  dbm_nonequilibrium and dbm_conservation are computed in double in
 * every mode; dbm_moments in double for DBM_FP64 and, for the float states,
 * in float (their own precision) with the temperature subtraction in
 * float-float.
 *  DBM_FP64    f stored and stepped in double.
 *  DBM_FP32    f stored and stepped in float.  By default (DBM_THERMO_FLOATFLOAT)
 *              the species and mixture moment sums are float; the one
 *              cancelling subtraction of the mixture temperature, energy
 *              minus kinetic part, is carried in float-float (an error-free
 *              FMA product and Knuth's two-sum, on the FP32 pipes), and the
 *              Arrhenius rate uses float expf.  DBM_THERMO_FP64 computes the
 *              species moments, the mixture u and T (the temperature
 *              recovery from the energy moment, section "Discrete Boltzmann
 *              model") and the Arrhenius rate in double from the stored
 *              floats instead; the equilibrium, collision and advection stay
 *              float.  dbm_params.rounding selects round-to-nearest or
 *              stochastic rounding of the stored f.
 *  DBM_BF16DEV f stored as a bfloat16 deviation from the equilibrium of
 *              stored float moments (n^s, u, T), stepped in float. */
enum dbm_precision { DBM_FP64 = 0, DBM_FP32 = 1, DBM_BF16DEV = 2 };

/* Arithmetic options of the DBM_FP32 step (dbm_params.thermo and
 * dbm_params.rounding); both need S <= 4, a TMA-staged step kernel, and
 * cannot be batched.  The defaults run the fastest kernel. */
enum dbm_thermo {
    DBM_THERMO_FLOATFLOAT = 0, /* float moment sums, float-float temperature subtraction */
    DBM_THERMO_FP64 = 1        /* species moments, mixture u, T and the Arrhenius
                                  rate in double                                   */
};
enum dbm_rounding {
    DBM_ROUND_NEAREST = 0,     /* f^{n+1} = f^n + increment, rounded to nearest */
    DBM_ROUND_STOCHASTIC = 1   /* the exact sum f^n + increment (two-sum) and the
                                  reacted density n* rounded up or down at random
                                  with the probabilities that make the rounding
                                  unbiased, so rounding errors do not accumulate
                                  into a drift of the conserved totals; random
                                  numbers from a counter-based hash of (step,
                                  cell, value): deterministic for a given step
                                  count                                         */
};

enum dbm_status_code {
    DBM_OK = 0,
    DBM_ERR_INVALID = -1,     /* a parameter or argument is out of range      */
    DBM_ERR_SINGULAR = -2,    /* a moment matrix M is singular/ill-conditioned */
    DBM_ERR_UNBOUND = -3,     /* state buffers not bound yet                   */
    DBM_ERR_CUDA = -4,        /* a CUDA runtime call or launch failed           */
    DBM_ERR_NONFINITE = -5,   /* device health flag: a non-finite moment        */
    DBM_ERR_NEGATIVE = -6,    /* device health flag: negative density, T <= 0 or n* < 0 */
    DBM_ERR_STABILITY = -7,   /* CFL or dt/tau stability limit exceeded         */
    DBM_ERR_TIMEOUT = -8,     /* device health flag: a bounded wait gave up     */
    DBM_ERR_BOUNDS = -9       /* device health flag (checked builds): an index out of range */
};

/* Health-flag bits as kept on the device (dbm_status_bits). */
enum dbm_health_bits {
    DBM_HEALTH_DENSITY = 1,      /* n^s < -1e-6 sum|n^s|, no matter at all, or not finite */
    DBM_HEALTH_TEMPERATURE = 2,  /* mixture T <= 0 or not finite */
    DBM_HEALTH_NSTAR = 4,        /* n^s* < 0 after the reaction  */
    DBM_HEALTH_NONFINITE = 8,    /* a non-finite moment           */
    DBM_HEALTH_TIMEOUT = 16,     /* a tile copy did not complete within its wait limit */
    DBM_HEALTH_BOUNDS = 32       /* checked builds only (-DDBM_CHECKED): an index fell
                                    outside the buffer it addresses; the access was
                                    skipped */
};

/* Step kernel selection (dbm_params.step_kernel).  Every choice runs the
 * same explicitly rounded arithmetic and gives bitwise identical results;
 * they differ in speed only. */
enum dbm_step_kernel {
    DBM_KERNEL_AUTO = 0,      /* TMA-staged where built (FP32), else generic; tile as
                                 DBM_KERNEL_TMA                                      */
    DBM_KERNEL_GENERIC = 1,   /* stencil read from global memory                      */
    DBM_KERNEL_TMA = 2,       /* tile + halo staged in shared memory by TMA copies:
                                 S = 1: one cell per thread; S = 2: all planes in one
                                 copy, two cells per thread on grids of at least 4096
                                 tiles of 64 x 8 cells, else one cell per thread;
                                 S = 3, 4: one cell per thread; S >= 5: as
                                 DBM_KERNEL_TMA_STAGED                               */
    DBM_KERNEL_TMA_CELL = 3,  /* TMA-staged, all planes in one copy, one cell per
                                 thread (S <= 4)                                     */
    DBM_KERNEL_TMA_PAIR = 4,  /* TMA-staged, two adjacent cells per thread: S = 2 all
                                 planes in one copy, S >= 3 species-staged           */
    DBM_KERNEL_TMA_STAGED = 5 /* TMA-staged one species at a time through two shared-
                                 memory buffers (each species copied for its moment
                                 sums and again for its update), two adjacent cells
                                 per thread on 64 x 8 tiles; 2 <= S <= 8, without the
                                 thermo and rounding options                         */
};

/* Constants of one species sigma. */
typedef struct dbm_species {
    double m;        /* molar mass m^s (> 0)                                    */
    double I;        /* extra degrees of freedom I^s (>= 0); gamma = (D+I+2)/(D+I) */
    double tau;      /* relaxation time tau^s (> 0)                              */
    double v[4];     /* ring speeds v_a, v_b, v_c, v_d (> 0)                     */
    double eta[4];   /* internal speeds eta_a .. eta_d (>= 0, not all 0)         */
    double a_stoich; /* stoichiometric coefficient a^s of the one-step reaction  */
} dbm_species;

/* Problem description (section "Discrete Boltzmann model" for the physics,
 * section "Numerical simulation" for the discretisation). */
typedef struct dbm_params {
    int nx, ny;             /* interior cells (>= 1 each)                          */
    int nspecies;           /* S, 1 .. DBM_MAX_SPECIES                              */
    double dx, dy, dt;      /* grid spacing and time step (> 0)                     */
    int bc_x, bc_y;         /* dbm_bc per axis: periodic, or outflow (zero-gradient) */
    int fuel, oxidizer;     /* species indices of the Arrhenius rate               */
    double k_ov;            /* reaction coefficient; 0 switches the reaction off   */
    double Ea_over_R;       /* activation temperature E_a / R                       */
    double Q;               /* heat released per mole of reaction                   */
    double accel[2];        /* external acceleration a of the force term; 0 = off   */
    int precision;          /* dbm_precision                                         */
    int step_kernel;        /* dbm_step_kernel; all give bitwise identical results   */
    int wait_polls;         /* polls of a TMA-staged step's first wait for its tile
                               copy: 0 = library default (2^22), > 0 = that many,
                               < 0 = none (the wait gives up at once, the step
                               raises DBM_HEALTH_TIMEOUT and writes nothing: a
                               safe way to exercise the timeout path; the copy
                               still lands before the CTA exits)               */
    int thermo;             /* dbm_thermo (DBM_FP32 only)                          */
    int rounding;           /* dbm_rounding (DBM_FP32 only)                        */
    dbm_species sp[DBM_MAX_SPECIES];
} dbm_params;

/* Device storage geometry of one state buffer: plane p = s*16 + i holds
 * `rows` rows of `pitch` elements; interior cell (x, y) sits at element
 * p*plane + (y + gy)*pitch + (x + gx).  The margins hold ghost cells:
 * dbm_set_state / dbm_set_f fill them, and so do the FP64 step and the
 * generic FP32 step, which read their boundary stencils from them; the
 * TMA-staged FP32 step and the BF16DEV step read a boundary cell's stencil
 * from its periodic or outflow source cell instead and leave the margins
 * untouched.  Only interior cells carry the state.
 * For DBM_BF16DEV the buffer holds 16*S bfloat16 deviation planes followed
 * (at byte offset moments_offset) by S+3 float moment planes
 * (n^0..n^{S-1}, u_x, u_y, T) of the same geometry. */
typedef struct dbm_layout {
    int pitch, rows, gx, gy;
    long long plane;          /* elements per plane                       */
    int elem_bytes;           /* bytes per stored f element (8, 4 or 2)   */
    size_t moments_offset;    /* BF16DEV only: byte offset of the moments */
    size_t bytes;             /* bytes of one state buffer                */
} dbm_layout;

typedef struct dbm_handle dbm_handle;

/* Validate params, build M^s for every species (rows of the M_ki list, row 9
 * read as (v^2+eta^2) v_y) and invert it on the host in FP64 (LU with
 * partial pivoting).  Rejects: S outside 1..8, non-positive sizes, m, tau,
 * dx, dy, dt or ring speeds; a singular M, or an infinity-norm condition
 * number of the row-equilibrated M above 1e8 (DBM_ERR_SINGULAR); with the reaction on, bad fuel/oxidizer indices or
 * |sum_s a^s m^s| > 1e-12 sum_s |a^s m^s| (DBM_ERR_INVALID); a CFL number
 * max|v_ia| dt / d_a > 0.5 or dt >= 2 tau^s (DBM_ERR_STABILITY).
 * On success *out owns a new handle (free with dbm_destroy). */
int dbm_init(const dbm_params *params, dbm_handle **out);

/* Message of the last failed dbm_init on the calling thread ("" after a
 * successful one). */
const char *dbm_init_error(void);

/* The equilibrium matrix M^-1 of one species as used by the kernels,
 * out[16*16] row-major (row i = velocity, column k = moment f-hat_k), so
 * that f^eq_i = sum_k out[16 i + k] f-hat_k (section "Discrete Boltzmann
 * model").  It is the inverse of the double matrix M rounded correctly to
 * double (LU, then refinement with compensated residuals).  Host only. */
int dbm_equilibrium_matrix(const dbm_handle *h, int species, double *out);

/* Storage geometry and size of one state buffer for this handle. */
int dbm_get_layout(const dbm_handle *h, dbm_layout *out);

/* Bytes of one state buffer (the caller allocates two) and of the scratch
 * buffer (health flag and reduction partials). */
int dbm_state_bytes(const dbm_handle *h, size_t *bytes);
int dbm_scratch_bytes(const dbm_handle *h, size_t *bytes);

/* Bind caller-owned device buffers: f_a and f_b of dbm_state_bytes each
 * (256-byte aligned), scratch of dbm_scratch_bytes.  f_a becomes the current
 * state.  The buffers must outlive every call that uses them.  Builds the
 * TMA descriptors of the two buffers and fixes the step's tile
 * (dbm_step_tile); DBM_ERR_INVALID when dbm_params.step_kernel asks for a
 * TMA-staged kernel that cannot run (not FP32; one cell per thread or an
 * arithmetic option with S > 4; no descriptor). */
int dbm_bind(dbm_handle *h, void *f_a, void *f_b, void *scratch);

/* f = f^eq(n^s = rho^s / m^s, u, T) in every cell from the macroscopic
 * fields rho_s [S][ny][nx], ux, uy, T [ny][nx] (FP64); ghosts filled; health
 * flag cleared.  Async on stream. */
int dbm_set_state(dbm_handle *h, const double *rho_s, const double *ux, const double *uy,
                  const double *T, void *stream);

/* Load / read the raw distributions, dense FP64 [S][16][ny][nx] (checkpoint
 * and restore).  dbm_set_f fills the ghosts and clears the health flag;
 * in DBM_BF16DEV mode it stores the moments of f and the bfloat16 deviation
 * from their equilibrium, and dbm_get_f reconstructs f.  Async on stream. */
int dbm_set_f(dbm_handle *h, const double *f, void *stream);
int dbm_get_f(dbm_handle *h, double *f, void *stream);

/* Advance nsteps >= 0 forward-Euler steps (Eqs. DiscreteBoltzmannEquation,
 * CollisionTerm, ReactionTerm, ForceTerm; NND advection).  One fused kernel
 * launch per step (boundary conditions inside the same kernel).
 * Async on stream; never synchronises and never allocates. */
int dbm_step(dbm_handle *h, int nsteps, void *stream);

/* Macroscopic fields of the current state, FP64 out[(4S+5)][ny][nx]:
 *   rows 4s..4s+3: n^s, u^s_x, u^s_y, T^s = m^s (E^s/n^s - u^s.u^s)/(D+I^s)
 *   (u^s = T^s = 0 for an absent species, n^s = 0);
 *   rows 4S..4S+4: rho = sum m^s n^s, u_x, u_y, T (mixture, from conservation
 *   of the collision term), p = n T with n = sum n^s.
 * Evaluated in double for a DBM_FP64 state; for DBM_FP32 and DBM_BF16DEV
 * states in float (ring sums as in the step, the mixture temperature's
 * subtraction in float-float), a few float ulps from the exact moments of
 * the stored floats.  Async on stream. */
int dbm_moments(dbm_handle *h, double *out, void *stream);

/* Nonequilibrium moments, FP64 out[20 S][ny][nx], 20 rows per species s
 * (Eqs. Delta2, Delta31, Delta3, Delta42 and the energy diagnostics defined
 * after them; f^eq = f^eq(n^s, u, T) with the mixture u, T):
 *   0..2 Delta_2 xx, xy, yy       3..4 Delta_3,1 x, y
 *   5..8 Delta_3 xxx, xxy, xyy, yyy   9..11 Delta_4,2 xx, xy, yy
 *   12..13 M_2xx(f)/2, M_2yy(f)/2     14..15 M_2xx(f^eq)/2, M_2yy(f^eq)/2
 *   16..17 M_3,1x(f)/2, M_3,1y(f)/2   18..19 M_3,1x(f^eq)/2, M_3,1y(f^eq)/2
 * All sums carry the factor m^s.  Async on stream. */
int dbm_nonequilibrium(dbm_handle *h, double *out, void *stream);

/* Conserved totals over the interior cells, FP64 out[S+4] (device or
 * addressable host memory): out[s] = sum rho^s; out[S], out[S+1] = sum rho u;
 * out[S+2] = total energy sum_s (m^s/2) sum_i f (v.v + eta^2);
 * out[S+3] = sum Q n^fuel / |a^fuel| (heat still bound in the fuel; 0
 * without reaction).  Summed in FP64 in a fixed order (deterministic).
 * Uses the bound scratch buffer.  Async on stream. */
int dbm_conservation(dbm_handle *h, double *out, void *stream);

/* ------------------------------------------------------------------------
 * Batches: many independent problems stepped together.
 *
 * A batch groups bound FP32 handles with the same species count S <= 4
 * (grids, boundaries, species constants, reaction and time step may all
 * differ).  Each dbm_batch_step advances every instance: one kernel launch
 * per time step covers the tiles of all instances (each CTA a contiguous
 * range of tiles, or one tile per CTA), each tile staged by TMA through its
 * instance's own descriptor; pairs of steps are
 * replayed from captured CUDA graphs when `stream` is a created stream.
 * The caller owns the device table (dbm_batch_table_bytes, 128-byte
 * aligned).  While a batch exists, step its handles through it; a handle
 * reset with dbm_set_state / dbm_set_f is picked up on the next batch step.
 * ------------------------------------------------------------------------ */
typedef struct dbm_batch dbm_batch;

/* Bytes of the device table for these n handles. */
int dbm_batch_table_bytes(dbm_handle *const *handles, int n, size_t *bytes);

/* Build a batch over n handles; writes the table (async on stream, then
 * synchronises it).  DBM_ERR_INVALID if a handle is unbound, not FP32, has
 * S > 4 or a different S than the others, asks for a non-default thermo or
 * rounding option, or the table is too small. */
int dbm_batch_create(dbm_handle *const *handles, int n, void *table, size_t table_bytes, void *stream,
                     dbm_batch **out);

/* Choose the tile shape (32x10, 32x8, 32x16, 32x7 or 64x4 cells at one cell
 * per thread, or 64x8 or 32x16 cells at two adjacent cells per thread), the launch form (as
 * many CTAs as are resident at once, each walking a contiguous range of
 * tiles, or one CTA per tile) and whether the tile copies promote L2 fills
 * to 256 bytes, whichever step this batch fastest: each choice is timed on
 * `reps` trial launches that read the current states and write only the
 * buffers the next step overwrites, so no state advances.  Synchronises the
 * stream. */
int dbm_batch_tune(dbm_batch *b, void *stream, int reps);

/* Advance every instance of the batch by nsteps >= 0 (async on stream). */
int dbm_batch_step(dbm_batch *b, int nsteps, void *stream);

/* Current tile shape, number of tiles per step and CTAs per launch. */
int dbm_batch_info(const dbm_batch *b, int *tile_x, int *tile_y, int *tiles, int *ctas);

/* The batch's kernel configuration: tile shape and cells per thread (1,
 * or 2 adjacent cells of a row in packed FP32x2 arithmetic), launch form
 * (1: at most the CTAs resident at once, each over a contiguous range of
 * tiles; 0: one CTA per tile) and L2 promotion of the tile copies (1: 256 B;
 * 0: none).  Null outputs are skipped. */
int dbm_batch_get_config(const dbm_batch *b, int *tile_x, int *tile_y, int *cells_per_thread, int *persistent,
                         int *promote);

/* Set the configuration (a compiled shape: 32x10, 32x8, 32x16, 32x7 or
 * 64x4 at one cell per thread, 64x8 or 32x16 at two), rewriting the batch's
 * tables; synchronises the stream.  Every shape runs the same explicitly
 * rounded arithmetic as dbm_step, so an instance's result is bitwise the
 * same whatever the shape and whatever else the batch holds.
 * DBM_ERR_INVALID for a shape that is not compiled. */
int dbm_batch_set_config(dbm_batch *b, int tile_x, int tile_y, int cells_per_thread, int persistent, int promote,
                         void *stream);

const char *dbm_batch_last_error(const dbm_batch *b);
void dbm_batch_destroy(dbm_batch *b);

/* Capacity, in doubles, of the library's own device array that holds the
 * reduction partials of dbm_conservation_noalloc (32 KB on every GPU that
 * loads the library, kept until the process exits). */
#define DBM_NOALLOC_SCRATCH_DOUBLES 4096

/* The totals of dbm_conservation without any caller-provided scratch
 * buffer.  The paper has no counterpart to this entry point: it is for
 * callers that cannot allocate device memory when they need the totals --
 * for example a plug-in running inside a host application that owns all of
 * the GPU's memory and allows no further allocation -- and so cannot hand
 * the library a scratch buffer.
 *   state  a state buffer in this handle's layout (device memory), or NULL
 *          for the handle's current bound state;
 *   out    S+4 doubles, laid out as for dbm_conservation (device or
 *          addressable host memory).
 * The result equals dbm_conservation's (same reduction blocks and order).
 * The block partials go to a static device array of
 * DBM_NOALLOC_SCRATCH_DOUBLES doubles inside the library instead of the
 * scratch buffer; a problem whose partials do not fit (more than 4 species)
 * is rejected with DBM_ERR_INVALID.  The call makes no cudaMalloc, cudaFree
 * or other allocation.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current: make that
 * first call before any stream capture, and call with the device that holds
 * `state` current.  All calls on a device share the one array, and each
 * call overwrites every partial it reads (nothing needs clearing), so calls
 * that may overlap on the GPU race with each other: order them on one
 * stream or synchronise between them.  Async on stream. */
int dbm_conservation_noalloc(dbm_handle *h, const void *state, double *out, void *stream);

/* Synchronise the stream, read the sticky device health flag and map it to
 * DBM_OK, DBM_ERR_NEGATIVE or DBM_ERR_NONFINITE.  *bits (may be NULL)
 * receives the raw dbm_health_bits. */
int dbm_status(dbm_handle *h, void *stream, unsigned *bits);

/* Steps taken since the last dbm_set_state / dbm_set_f. */
long long dbm_steps_taken(const dbm_handle *h);

/* The shared-memory tile the step of a bound handle uses (chosen at
 * dbm_bind from dbm_params.step_kernel and the grid): tile_x x tile_y
 * cells, cells_per_thread 1 or 2 (adjacent cells of a row, packed FP32x2
 * arithmetic); all three 0 when the step runs a kernel without a tile
 * (generic global-memory stencil, FP64, BF16DEV).  Null outputs are
 * skipped.  DBM_ERR_UNBOUND before dbm_bind. */
int dbm_step_tile(const dbm_handle *h, int *tile_x, int *tile_y, int *cells_per_thread);

/* Message of the last failed call on this handle ("" if none).  The string
 * is owned by the handle. */
const char *dbm_last_error(const dbm_handle *h);

/* Release the handle (not the caller's buffers).  NULL is allowed. */
void dbm_destroy(dbm_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* DBM_H */
