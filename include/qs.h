/*
 * qs.h -- C ABI of the B300 (sm_103a) linearised quasistatic beam-plasma
 * sweep library (libqs.so).
 *
 * Model (arXiv 2607.24234, normalised to omega_p, k_p = omega_p/c, n_p,
 * m_e, e).  Per transverse Fourier mode k_perp the library advances the
 * beam-density perturbation n_bs and Theta_s = d_xi v_x - i k.v_perp of
 * each beam species s in slow time tau.  Every slow-time step is one fused
 * causal sweep along xi = t - x of
 *   - the plasma response (d_xi^2 + 1) n_p = rho_b = sum_s q_s n_bs
 *     (Sec. II, Eq. 5), integrated exactly across each xi cell with the
 *     beam charge constant on the cell;
 *   - the pseudo-potential Psi = n_p / (1 + k^2) (Eq. 14) and its
 *     derivatives d_xi Psi, d_xi^2 Psi = (rho - n_p) / (1 + k^2);
 *   - the beam push of Eqs. (8)-(9):
 *       d_tau Theta_s = (q_s/m_s)[(k^2/g) Psi - g^-3 d_xi^2 Psi],
 *       d_tau n_bs    = n_bs0(xi) Theta_s,
 *     as a kick-drift leapfrog (first step kicks by dt/2).
 * Dropping the g^-3 term (QS_MODEL_REDUCED) gives Eq. (18) for one
 * species; keeping it gives Eq. (15) per mode.
 *
 * Conventions for every entry point:
 *   - Device work is enqueued asynchronously on the CUDA stream given to
 *     qs_init (NULL = legacy default stream).  Only qs_sync and the
 *     host-pointer forms of qs_diag / qs_seed block.
 *   - Return value: QS_OK or an error code; no exception crosses the ABI.
 *     qs_last_error(ctx) returns a message for the last failure on ctx
 *     (ctx == NULL: the last failure of qs_init on this thread).
 *   - Argument errors are detected on the host before any launch.  Device
 *     errors (non-finite values, exhausted bounded waits) set a sticky
 *     device word that qs_sync / host qs_diag report; after one, the
 *     context returns QS_ERR_STATE until the next qs_seed.
 *   - The library owns all state buffers (allocated through the caller's
 *     allocator when one is given, else cudaMalloc) and frees them in
 *     qs_free.  The caller owns every buffer it passes in.
 */
#ifndef QS_H
#define QS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QS_OK = 0,
    QS_ERR_ARG = 1,          /* invalid argument or size                  */
    QS_ERR_OOM = 2,          /* allocation failed                         */
    QS_ERR_CUDA = 3,         /* a CUDA runtime/driver call failed         */
    QS_ERR_TIMEOUT = 4,      /* a bounded device wait ran out             */
    QS_ERR_NONFINITE = 5,    /* NaN/Inf appeared in the state             */
    QS_ERR_STATE = 6,        /* context poisoned by an earlier error      */
    QS_ERR_UNSUPPORTED = 7,  /* valid request this build does not serve   */
    QS_ERR_BOUNDS = 8        /* bounds-checked build: a device index left
                              * its buffer (the access was skipped)       */
} qs_status;

enum { QS_GEOM_KLIST = 0,    /* explicit list of k (2D slab, k along y)   */
       QS_GEOM_KGRID2 = 1 }; /* cell-centred (kx, ky) grid, optional disc */

enum { QS_FP64 = 0,          /* state and arithmetic in FP64              */
       QS_FP32_RENORM = 1 }; /* FP32 mantissas + power-of-two exponent    *
                              * per (mode, 32-cell group)                 */

enum { QS_MODEL_FULL = 0, QS_MODEL_REDUCED = 1 };

enum { QS_FRONT_QUIESCENT = 0,   /* plasma at rest ahead: P(0) = (0, 0)       */
       QS_FRONT_EQUILIBRIUM = 1, /* P(0) = (rho at cell 0, 0)                 */
       QS_FRONT_HELD = 2 };      /* P(0) fixed per mode by the caller
                                  * (Sec. III.C holds the front value)        */

enum { QS_PROF_FLATTOP = 0,      /* 1 for xi <= length, 0 behind              */
       QS_PROF_GAUSSIAN = 1,     /* exp(-(xi-center)^2 / (2 sigma^2))         */
       QS_PROF_RAMP_FLATTOP = 2, /* xi/ramp for xi < ramp, 1 up to length     */
       QS_PROF_USER = 3 };       /* user_profile[n_xi] at cell centres        */

typedef struct {
    double q;             /* charge in units of e (electron: -1)           */
    double m;             /* mass in units of m_e                           */
    double density_ratio; /* peak n_bs0 / n_p                              */
} qs_species;

/* Problem statement (Sec. II: species (q_s, m_s, n_bs0), gamma_b, the
 * longitudinal profile, the transverse wavenumbers and the xi / tau
 * grids).  Cell j covers [j dxi, (j+1) dxi); beam quantities live at the
 * cell centre (j + 1/2) dxi. */
typedef struct {
    int geom;                 /* QS_GEOM_*                                 */
    int prec;                 /* QS_FP64 | QS_FP32_RENORM                  */
    int model;                /* QS_MODEL_*                                */
    int front;                /* QS_FRONT_*                                */
    int n_species;            /* 1 or 2                                    */
    qs_species species[2];
    double gamma_b;           /* > 1                                       */
    int profile;              /* QS_PROF_*                                 */
    double length, sigma_xi, center_xi, ramp_len;
    const double *user_profile; /* host, n_xi doubles (QS_PROF_USER)       */
    int n_xi;                 /* >= 1                                      */
    double dxi;               /* > 0                                       */
    double dt;                /* > 0                                       */
    int n_k;                  /* QS_GEOM_KLIST: number of k                */
    const double *k_list;     /* host, n_k doubles                         */
    int nkx, nky;             /* QS_GEOM_KGRID2: k_i = (i-(n-1)/2) 2kmax/n */
    double kmax;
    int disc_mask;            /* 1: keep |k| <= kmax only                  */
    const double *held_front; /* QS_FRONT_HELD: host, 4 doubles per active
                               * mode (re n_p, im n_p, re n_p', im n_p')   */
} qs_params;

/* Caller-supplied device allocator (e.g. a framework's caching allocator).
 * alloc returns NULL on failure (the library then returns QS_ERR_OOM). */
typedef struct {
    void *(*alloc)(size_t bytes, void *user);
    void (*free)(void *ptr, void *user);
    void *user;
} qs_allocator;

typedef struct qs_ctx qs_ctx;

/* Create a context for n_inst >= 1 instances.  per_inst == NULL: all
 * instances use *p; else per_inst[i] describes instance i and must agree
 * with *p on geom, prec, model, front, n_species and the k set (instances
 * may differ in species densities, gamma_b, profile, n_xi and dxi).
 * alloc == NULL: cudaMalloc/cudaFree.  stream: a cudaStream_t or NULL.
 * On success *out owns the state, zero-initialised; call qs_seed next. */
qs_status qs_init(const qs_params *p, int n_inst, const qs_params *per_inst,
                  const qs_allocator *alloc, void *stream, qs_ctx **out);

enum { QS_SEED_NOISE = 0,   /* complex Gaussian white noise on n_b          */
       QS_SEED_IMPULSE = 1, /* d_tau rho(0) = amplitude * delta(xi) in cell 0 */
       QS_SEED_USER = 2,    /* n_b from `user`, Theta = 0                   */
       QS_SEED_STATE = 3 }; /* restore a QS_DIAG_STATE checkpoint            */

/* (Re)initialise the perturbation and reset the step counter to 0
 * (QS_SEED_STATE restores the checkpoint's counter instead).
 *  NOISE:   n_bs(xi_j) = amplitude * shape(xi_j) * (g1 + i g2)/sqrt 2 with
 *           g1, g2 standard normals from Philox4x32-10 keyed by `seed`, with
 *           counter (j, canonical mode id, instance, species); the mode
 *           paired with -k receives the complex conjugate.
 *  IMPULSE: Theta_0(cell 0) = amplitude / (q_0 n_b00(xi_0) dxi), n_b = 0:
 *           the impulse response (Green's function) source of Eq. (23).
 *  USER:    `user` = complex128 n_b as [inst][mode][species][xi]
 *           (interleaved re, im), instances concatenated.
 *  STATE:   `user` = bytes written by qs_diag(QS_DIAG_STATE).
 * user_on_host selects whether `user` is a host or a device pointer. */
qs_status qs_seed(qs_ctx *ctx, uint64_t seed, double amplitude, int kind,
                  const void *user, size_t user_bytes, int user_on_host);

/* Advance every instance by n_steps >= 1 slow-time steps (async). */
qs_status qs_step(qs_ctx *ctx, int n_steps);

/* Diagnostic record kinds (bit mask for qs_record, value for qs_diag). */
enum {
    QS_REC_MAG = 1,     /* 5 doubles per cell: ln|dn_b|, ln|dE|, ln|dB|,
                         * ln|F_perp|, ln|E_x| at the cell centre.  |dn_b|
                         * = (sum_s |n_bs|^2)^(1/2); fields (a reading, the
                         * paper derives only F_perp ~ grad_perp Psi):
                         * E_x = -d_xi Psi, E_perp = i k kappa (n_p - rho),
                         * |B_perp| = |k| kappa |rho|, F_perp = i k Psi.    */
    QS_REC_NP = 2,      /* complex n_p at the cell centre (2 doubles)      */
    QS_REC_MODEMAX = 4  /* per mode: max over xi of ln|dn_b|, ln|dE|, ln|dB| */
};

/* Attach a device buffer that subsequent qs_step calls fill with the
 * fields at tau = g dt for every global step g = g0 + i*stride (g0 = the
 * step counter now), as computed inside the sweep of step g (before its
 * update).  Layout per snapshot, for each kind present in `kinds` (in bit
 * order): MAG [5][cells][mode], NP [cells][mode][2], MODEMAX
 * [3][inst][mode], where `cells` runs over the instances' xi cells
 * concatenated and `mode` over the padded mode count (qs_query).
 * qs_step fails with QS_ERR_ARG rather than write past out_bytes.
 * kinds == 0 or out == NULL detaches. */
qs_status qs_record(qs_ctx *ctx, int kinds, int stride, void *dev_out,
                    size_t out_bytes);

enum { QS_DIAG_MAG = 1, QS_DIAG_NP = 2, QS_DIAG_MODEMAX = 4,
       QS_DIAG_XIMAX = 8,  /* per xi cell: max over modes of ln|dn_b|, ln|dE|,
                            * ln|dB| as [3][cells] (read-only pass only)     */
       QS_DIAG_STATE = 16, /* opaque checkpoint (state + exponents + step) */
       QS_DIAG_WAKE0 = 32  /* zeroth-order n_p response to the unperturbed
                            * beam charge: 2 doubles per cell per instance
                            * (cell exit, cell centre), Eq. (5)          */ };

/* Read-only diagnostic pass at the current state (tau = step * dt), one
 * snapshot in the qs_record layout (or the checkpoint / wake layout).
 * out_on_host = 1 copies to host memory and synchronises the stream. */
qs_status qs_diag(qs_ctx *ctx, int kind, void *out, size_t out_bytes,
                  int out_on_host);

enum { QS_Q_N_MODES = 0,      /* active modes                              */
       QS_Q_MODES_PADDED = 1, /* row length of every [cells][mode] array   */
       QS_Q_N_INST = 2,
       QS_Q_TOTAL_CELLS = 3,  /* sum over instances of n_xi                */
       QS_Q_STEP = 4,         /* global slow-time step counter             */
       QS_Q_STATE_BYTES = 5,  /* size of a QS_DIAG_STATE checkpoint        */
       QS_Q_SNAPSHOT_BYTES = 6, /* bytes of one snapshot for kinds = arg  */
       QS_Q_CELL_OFFSET = 7,  /* first cell of instance arg                */
       QS_Q_LAUNCH = 8,       /* packed launch shape in use (see qs_launch) */
       QS_Q_RES_EVERY = 9 };  /* resident variant's renormalisation interval
                               * (steps; 0: the variant is refused, see
                               * qs_growth_bound)                          */

/* Query a size or counter; `arg` is used by QS_Q_SNAPSHOT_BYTES (kinds)
 * and QS_Q_CELL_OFFSET (instance). */
qs_status qs_query(const qs_ctx *ctx, int what, int64_t arg, int64_t *value);

/* Copy the active modes' (kx, ky) to host arrays of QS_Q_N_MODES doubles
 * (KLIST: kx = k, ky = 0). */
qs_status qs_modes(const qs_ctx *ctx, double *kx, double *ky);

/* Launch shape of the sweep kernel. */
enum { QS_VARIANT_REGISTERS = 0,  /* thread per line, register prefetch       */
       QS_VARIANT_TMA = 1,        /* thread per line, warp-wide TMA tiles of
                                   * (cells x 32 modes) through shared memory */
       QS_VARIANT_SCAN = 2,       /* FP64 only, for few lines: the lanes of a
                                   * warp split xi into sub-chunks joined by a
                                   * shuffle scan of the cell propagators      */
       QS_VARIANT_RESIDENT = 3 }; /* FP32 only: whole warps hold a line in
                                   * registers for every step of a call (HBM
                                   * is read once and written once per call);
                                   * xi is joined by a block scan of the cell
                                   * propagators.  Steps that record, and field
                                   * passes, run the register kernel.  Range:
                                   * a line keeps 2^190 (e^131) below its
                                   * largest value, smaller cells flush to 0
                                   * (the streaming variants keep every 32-cell
                                   * group at full FP32 precision); a front
                                   * that grows far slower than the back of a
                                   * long beam over thousands of steps can fall
                                   * that far behind                          */
typedef struct {
    int warps_per_cta;   /* REGISTERS: 1, 2, 4 or 8 (TMA: always 1);
                          * RESIDENT: 1, 2, 4, 8 or 16 (CTA size; a line
                          * takes ceil(ceil(n_xi / cells) / 32) warps and
                          * must fit in one CTA)                            */
    int prefetch;        /* REGISTERS: cells per register batch (FP32 4|8,
                          * FP64 2|4); TMA: cells per tile (FP32 8|16,
                          * FP64 4|8); RESIDENT: cells per thread, 8|16 with
                          * any CTA size, 32 (one species) with 2|4|8 warps,
                          * 16 (two species) with 4|8|16 warps               */
    int persistent;      /* 1: LPT-ordered work list pulled by atomic ticket */
    int ctas_per_sm;     /* persistent grid size = ctas_per_sm * SM count    */
    int variant;         /* QS_VARIANT_*                                    */
    int scan_cells;      /* SCAN: cells per lane per sub-chunk (1..64); the
                          * lanes per mode along xi are `prefetch` (2..32).
                          * RESIDENT: QS_RES_THETA_REGS keeps Theta in
                          * registers at 32 cells of one species or 16 of
                          * two (1|2|4|8 warps); any other value keeps it in
                          * shared memory there                             */
} qs_launch;
enum { QS_RES_THETA_REGS = 1 };

qs_status qs_set_launch(qs_ctx *ctx, const qs_launch *l);
qs_status qs_get_launch(const qs_ctx *ctx, qs_launch *l);

/* Autotuner: time every candidate launch shape for `reps` steps on a copy
 * of the state (the context's state is unchanged), keep the fastest, and
 * read/write the choice in the JSON cache file `cache_path` (NULL: no
 * cache) keyed by precision, species count, xi-length bucket and SM count.
 * Synchronises the stream. */
qs_status qs_tune(qs_ctx *ctx, int reps, const char *cache_path);

/* Capture n_steps of qs_step in a CUDA graph (cached per n_steps) and
 * launch it.  Semantics as qs_step.  The record target must be detached. */
qs_status qs_step_graph(qs_ctx *ctx, int n_steps);

/* Green's-function path: advance the state by n_steps slow-time steps as a
 * causal convolution in xi (Sec. III.A's Green's-function picture, for the
 * discrete scheme).  For a uniform profile (the same dt n_bs0 in every cell
 * of an instance) and a quiescent front each step is linear, causal and
 * shift-invariant in xi with real coefficients, so n steps map every mode by
 * x_n(j) = sum_{l<=j} G_n(l) x_0(j - l), G_n the response to a unit impulse at
 * cell 0, which depends on the mode only through k^2.  The library sweeps
 * one impulse line per (k^2 class, input component) through the resident
 * FP32 kernel (Theta impulses only when Theta is not identically zero, i.e.
 * after any step or an impulse / checkpoint seed) and convolves every mode
 * with its class's responses.  Results agree with qs_step to FP32 accuracy
 * (not bitwise).  FP32 contexts only; QS_ERR_UNSUPPORTED for FP64, a
 * non-uniform profile, a front other than QS_FRONT_QUIESCENT, lines too long
 * for the resident kernel (> 8192 cells) or a convolution that does not fit
 * shared memory; QS_ERR_ARG with a record target attached.  Allocates
 * impulse-line buffers and a second state buffer on the first call (kept
 * until qs_free). */
qs_status qs_step_green(qs_ctx *ctx, int n_steps);

/* Wait for the stream and report device-side errors. */
qs_status qs_sync(qs_ctx *ctx);

/* Test hook for the bounded waits of the TMA variant (failure detection
 * without a GPU fault).  Every mbarrier wait of that kernel gives up after
 * spin_limit polls (default 2^24); with unsatisfiable = 1 each tile's
 * barrier expects 16 bytes more than its tensor copy delivers, so the first
 * wait runs out: the kernel records QS_ERR_TIMEOUT in the device error word,
 * drains its copies (again bounded) and returns, and qs_sync reports
 * QS_ERR_TIMEOUT.  The context is usable again after qs_debug_waits(ctx,
 * limit, 0) and a reseed.  Other kernels have no device-side waits. */
qs_status qs_debug_waits(qs_ctx *ctx, int64_t spin_limit, int unsatisfiable);

/* Upper bound of the scheme's growth per slow-time step for a problem
 * statement (host only, no CUDA call).  One step maps (n_b, Theta) by the
 * kick of Eqs. (8)-(9) and the drift, with |n_p| <= L max|rho| over a line
 * of length L (Eq. 5) and kappa k^2, kappa <= 1 (Eq. 14); with
 *   a = dt max|q/m| (1/gamma + 1/gamma^3) sum_s |q_s| (2 + L),
 *   b = dt max_s n_bs0 (peak of the profile),
 * the step is bounded, in suitably weighted max norms, by a symmetric 2 x 2
 * matrix whose spectral radius 1 + ab/2 + sqrt(ab + (ab)^2/4) gives
 * *efolds_per_step (its log).  *res_every: the renormalisation interval the
 * resident FP32 sweep uses for this problem, the largest power of two up to
 * 16 steps over which the bound (plus the one-time weight factor) stays
 * below e^28, or 0 when none does; a context refuses the resident variant
 * and the Green's-function path (QS_ERR_UNSUPPORTED) when any instance has
 * 0.  The bound is loose (the instabilities of Sec. III grow far slower),
 * it only guards the FP32 range.  Either pointer may be NULL. */
qs_status qs_growth_bound(const qs_params *p, double *efolds_per_step, int *res_every);

/* Build variants.  The library built with -DQS_CHECK_BOUNDS (libqs_checked.so)
 * tests every global-memory index of the sweep kernels against the extent of
 * its buffer; an index outside it sets a device error bit, the first bad index
 * is kept, the access is skipped (no trap, no fault), and the next qs_sync
 * returns QS_ERR_BOUNDS.  qs_build_flags() reports the variant. */
enum { QS_BUILD_CHECK_BOUNDS = 1 };
int qs_build_flags(void);

/* Test hook for the bounds checks (failure detection without a bad access):
 * the checked build is told that the last rows_cut rows of the state
 * (cells x species) are missing, so the sweep reports QS_ERR_BOUNDS at the
 * first access to them and skips it; the memory is there, nothing strays.
 * rows_cut = 0 restores the true extent.  No effect in the ordinary build. */
qs_status qs_debug_bounds(qs_ctx *ctx, int64_t rows_cut);

/* Guards: every context buffer is allocated 256 bytes longer, the tail is
 * filled with a fixed byte, and qs_sync (and host-pointer qs_diag) check the
 * tails; an overwritten one is reported as QS_ERR_BOUNDS ("the guard after
 * buffer i was overwritten").  Test hook: qs_debug_canary overwrites one
 * byte of buffer `buffer`'s guard (inside the allocation) so that the
 * detection can be tested without a stray write. */
qs_status qs_debug_canary(qs_ctx *ctx, int buffer);

/* Number of sweep-kernel launches enqueued by this context so far. */
int64_t qs_launch_count(const qs_ctx *ctx);

const char *qs_last_error(const qs_ctx *ctx);
void qs_free(qs_ctx *ctx);

/* ---------------------------------------------------------------------
 * Finite-width beam on a periodic transverse grid (Sec. IV.B: narrow
 * beams, self-modulation and hosing).  One species with a Gaussian (or
 * uniform) transverse profile n_b0(y, z), flat top in xi.  Per step: the
 * plasma response (Eq. 5) per transverse point, then per xi slice the
 * screened Poisson solve of Eq. (14) by 2-D FFT with spectral gradients,
 * and the push d_tau G = -(q/(m gamma)) [n_b0 (Psi - n_p) + grad n_b0 .
 * grad Psi], d_tau n_b = G (Eqs. 8-9 with the transverse divergence in
 * conservative form; the gamma^-3 term is dropped).  FP32 state
 * [xi][y][z], z fastest; cell centres y_i = (i + 1/2) L/N - L/2.
 * ------------------------------------------------------------------- */
typedef struct {
    qs_species species;   /* q, m, peak n_b0/n_p                           */
    double gamma_b;
    int n_xi;
    double dxi, dt;
    int n_perp;           /* N = 32, 64, 128 or 256 points per transverse axis */
    double L_perp;        /* periodic box size (both axes)                  */
    double sigma_r;       /* rms of the Gaussian profile                    */
    int uniform;          /* 1: n_b0 = peak everywhere                       */
} qs_r2_params;
typedef struct qs_r2 qs_r2;

qs_status qs_r2_init(const qs_r2_params *p, const qs_allocator *alloc, void *stream, qs_r2 **out);
/* n_b = amplitude (n_b0/peak) g + [n_b0(y - offset, z) - n_b0(y, z)], G = 0,
 * step counter reset; g standard normals from Philox4x32-10 keyed by seed
 * (counter (cell, point)), or the float32 field `user` [n_xi][N][N] (host
 * or device) when not NULL.  Synchronises the stream. */
qs_status qs_r2_seed(qs_r2 *c, uint64_t seed, double amplitude, double centroid_offset, const float *user,
                     size_t user_bytes, int user_on_host);
qs_status qs_r2_step(qs_r2 *c, int n_steps);
/* what: 0 n_b, 1 G, 2 n_p (cell centres, last step) -> float32 [n_xi][N][N]. */
qs_status qs_r2_read(qs_r2 *c, int what, float *out, size_t out_bytes, int on_host);
qs_status qs_r2_sync(qs_r2 *c);   /* QS_ERR_NONFINITE if a value overflowed */
int64_t qs_r2_launch_count(const qs_r2 *c);
void qs_r2_free(qs_r2 *c);

/* ---------------------------------------------------------------------
 * Learned surrogate (the paper has no learned component; this serves
 * parameter screening, with the solver as the fallback and as the reference
 * for the surrogate's error).
 * A small MLP n_in -> width (depth hidden layers, GELU erf form) -> 2
 * (regression output: log growth envelope; logit: CFI (0) / OTSI (1)),
 * BF16 weights and activations, FP32 accumulation on the tensor cores,
 * FP32 master weights, Adam; an ensemble of independent members (different
 * initial weights).  Loss per sample: (p0 - y0')^2 + BCE-with-logits(p1, y1)
 * with y0' the standardised target.  All pointers to samples are device
 * pointers: X [n][n_in] fp32, Y [n][2] fp32.
 * ------------------------------------------------------------------- */
typedef struct qs_mlp qs_mlp;

/* n_in <= 32, width multiple of 16, 1 <= depth <= 8, n_out = 2,
 * 1 <= ensemble <= 16, max_batch rows per training step / inference chunk. */
qs_status qs_mlp_create(int n_in, int width, int depth, int n_out, int ensemble, int max_batch,
                        uint64_t seed, const qs_allocator *alloc, void *stream, qs_mlp **out);
/* Input standardisation statistics (and regression-target statistics if Y
 * is not NULL) computed on the device from n training rows. */
qs_status qs_mlp_set_norm(qs_mlp *m, const float *X, int64_t n, const float *Y);
/* Copy member `member`'s fp32 master parameters to (set = 0) or from
 * (set = 1) a host array of qs_mlp_layout's nparam floats; setting also
 * refreshes the BF16 copy. */
qs_status qs_mlp_params(qs_mlp *m, int member, float *host, int64_t n, int set);
/* nparam per member; offsets[2l], offsets[2l+1] = start of W_l [out][in]
 * and b_l (layer 0's `in` is n_in rounded up to 16, extra columns zero);
 * norm[64]: input mean[0..31], inverse std[32..63] with norm[62], norm[63]
 * = regression target mean and std. */
qs_status qs_mlp_layout(const qs_mlp *m, int64_t *nparam, int64_t *offsets, float *norm);
/* One step on n <= max_batch rows: forward, loss, backward for every member;
 * Adam update if do_update.  loss_host (optional) receives the mean loss
 * over members (synchronises the stream). */
qs_status qs_mlp_train_step(qs_mlp *m, const float *X, const float *Y, int64_t n, float lr, int do_update,
                            float *loss_host);
/* Gradients of member `member` from the last train step (host copy). */
qs_status qs_mlp_grads(qs_mlp *m, int member, float *host_grad, int64_t n);
/* Ensemble inference: mean/var [n][2] on the device (output 0 in target
 * units); mask[i] = 1 marks rows whose output-0 variance exceeds
 * var_threshold, to be answered by the solver instead. */
qs_status qs_mlp_infer(qs_mlp *m, const float *X, int64_t n, float *mean, float *var, uint8_t *mask,
                       float var_threshold);
const char *qs_mlp_last_error(const qs_mlp *m);
void qs_mlp_free(qs_mlp *m);

/* Whole-model surrogate: train the ensemble on n device rows X [n][7],
 * Y [n][2] (fp32, as written by qs_sur_points) with the options of a flat
 * JSON object (numbers; defaults in brackets): "epochs" [8], "batch"
 * [16384], "lr" [0.002, cosine-decayed over the epochs], "ensemble" [4],
 * "width" [256], "depth" [3], "seed" [3] (initial weights and the per-epoch
 * shuffles), "var_threshold" [inf] (the fallback threshold of
 * qs_sur_infer).  json_cfg may be NULL.  ctx (may be NULL) lends its stream
 * and allocator.  Synchronises the stream every epoch (the shuffle is drawn
 * on the host).  On success *out owns the model; free it with qs_sur_free. */
typedef struct qs_sur qs_sur;
qs_status qs_sur_train(qs_ctx *ctx, const void *X, const void *Y, int64_t n, const char *json_cfg, qs_sur **out);
/* Ensemble inference on n device rows X [n][7]: y_mean, y_var [n][2] fp32
 * device (output 0 in target units); fallback_mask (device, may be NULL):
 * 1 where the output-0 variance exceeds the model's threshold, i.e. the
 * rows to answer with the solver. */
qs_status qs_sur_infer(qs_sur *s, const void *X, int64_t n, void *y_mean, void *y_var, uint8_t *fallback_mask);
/* Mean loss of each epoch's first batch (host; *n_out = epochs). */
qs_status qs_sur_losses(const qs_sur *s, float *host, int max_n, int *n_out);
qs_status qs_sur_set_threshold(qs_sur *s, float var_threshold);
void qs_sur_free(qs_sur *s);

/* Parameter screening, the solver answering the flagged queries.  X [n][7]
 * fp32 device: queries as written by qs_sur_points (columns 0..2 name a
 * parameter set, 3..6 the point (xi, t, |k|, angle)).  The ensemble answers
 * every query (y, y_var [n][2] fp32 device, as qs_sur_infer); queries whose
 * output-0 variance exceeds the model's threshold are answered by the solver
 * instead: each is matched to the entry of sets[0..n_sets) (host; same k set,
 * precision, model, front and species count) whose (ln n_b0/n_p, ln gamma_b,
 * length) equal its columns 0..2 to fp32 rounding; the sets that have such
 * queries run in solver contexts (instance counter of the noise = the set's
 * index, so set i draws the noise it would draw as instance i of one context
 * holding every set; seeded with noise_seed and amplitude), are stepped to
 * each queried t (a whole number of steps), and the targets of
 * qs_sur_points are evaluated at the queried cell and mode.  Those rows get
 * y0 = the solver's log envelope, y1 = +-30 (the class as a saturated
 * logit), zero variance, and mask = 1; the other rows keep the ensemble's
 * answer and mask = 0.  *n_solved (may be NULL) receives the number of
 * solver-answered rows.  The solver contexts use lend's stream and allocator
 * (lend may be NULL: default stream, cudaMalloc), hold at most ~16 GiB each
 * (sets are split across contexts beyond that), and are freed before the
 * call returns.  Synchronises the device.  QS_ERR_ARG if a flagged query
 * matches no set, lies outside its line, or names an inactive mode. */
qs_status qs_sur_screen(qs_sur *s, qs_ctx *lend, const qs_params *sets, int n_sets, uint64_t noise_seed,
                        double amplitude, const void *X, int64_t n, void *y, void *y_var, uint8_t *mask,
                        int64_t *n_solved);

/* Training samples for the surrogate from one snapshot of ctx (the
 * device buffer `snap` written by qs_diag(QS_DIAG_MAG) at the current step;
 * snap_bytes its size).  n samples, cells drawn uniformly over all
 * instances' cells and modes uniformly (Philox4x32-10 keyed by seed).
 * X [n][7] fp32 device: ln(n_b0/n_p), ln gamma_b, L, xi, t, |k|, atan2(ky,kx).
 * Y [n][2] fp32 device: ln(RMS of |dn_b| over xi +- 1) - ln(amplitude), and
 * 1 (OTSI) / 0 (CFI): whether the mode oscillates in xi over one plasma
 * wavelength, Re sum conj(Psi) d_xi^2 Psi < 0 (the d_xi^2 ~ -1 regime of
 * Sec. III.A), evaluated from the recorded F_perp, E_perp and B_perp.
 * Synchronises the stream. */
qs_status qs_sur_points(qs_ctx *ctx, const double *snap, size_t snap_bytes, double amplitude,
                        int64_t n, uint64_t seed, float *X, float *Y);

/* Arithmetic-rate probe (measurement aid; the paper has no counterpart).
 * The resident and Green's-function FP32 sweeps and the FP64 sweep are
 * bound by arithmetic rather than HBM, so their roofline fractions divide
 * by the rate the GPU actually sustains.  This enqueues on `stream` one
 * launch of `blocks` x `threads` (32..256, a multiple of 32) threads, each
 * running 8 independent chains of `iters` dependent fused multiply-adds:
 *   QS_PROBE_FFMA2  packed f32x2 FMA (__ffma2_rn, two lane-ops each),
 *   QS_PROBE_FFMA   scalar FP32 FMA (16 chains),
 *   QS_PROBE_DFMA   FP64 FMA; QS_PROBE_DADD, QS_PROBE_DMUL FP64 add, multiply.
 * *lane_ops (may be NULL) receives the number of FMA lane-operations the
 * launch performs; time it with CUDA events on `stream`.  dev_sink is a
 * device buffer of at least 8 bytes that the kernel never writes in practice
 * (it keeps the arithmetic from being optimised away).  QS_ERR_ARG for a bad
 * shape; QS_ERR_CUDA if the launch fails. */
enum { QS_PROBE_FFMA2 = 0, QS_PROBE_FFMA = 1, QS_PROBE_DFMA = 2,
       QS_PROBE_DADD = 3,   /* FP64 add (one lane-op each)                 */
       QS_PROBE_DMUL = 4 }; /* FP64 multiply (one lane-op each)            */
qs_status qs_probe_alu(int kind, int blocks, int threads, int64_t iters, void *dev_sink, void *stream,
                       double *lane_ops);

/* Allocation-free sweep (the paper has no counterpart; this is a service to
 * callers that must not allocate device memory when they step the solver,
 * e.g. a host framework whose memory pool forbids driver allocations in its
 * steady-state loop, or code where an allocation could synchronise the
 * device or fail mid-run).  No context is created and nothing is allocated:
 * no cudaMalloc, cudaFree or allocating library routine is called.
 *
 * The caller owns the state, in the library's internal layout with
 * Mp = active modes rounded up to a multiple of 32:
 *   QS_FP32_RENORM: state = float4 [n_xi][n_species][Mp]
 *                   (Re n_b, Im n_b, Re Theta, Im Theta) and exponents =
 *                   int32 [ceil(n_xi/32)][Mp] (value = mantissa * 2^(e >> 8));
 *                   theta = NULL.
 *   QS_FP64:        state = double2 n_b [n_xi][n_species][Mp],
 *                   theta = double2 Theta [n_xi][n_species][Mp];
 *                   exponents = NULL.
 * (the same bytes qs_diag(QS_DIAG_STATE) writes after its 64-byte header).
 * The call advances them in place by n_steps slow-time steps starting at
 * global step step0 (step 0 kicks by dt/2), asynchronously on `stream`.
 * If dev_status is not NULL, the device error bits of this call (1:
 * non-finite value) are copied to that device int at the end.
 *
 * Everything else the sweep needs -- mode tables, profile weights, work
 * list, scheduler ticket, error word -- lives in one fixed 4 MiB device
 * array of this library, held by every GPU that loads it until the process
 * exits.  Limits: it must hold 3*Mp doubles + ceil(M/64) work items +
 * n_xi*n_species profile weights (about 4 MiB in total, e.g. Mp up to
 * ~150,000 with n_xi = 8,192); larger problems are rejected with QS_ERR_ARG
 * before anything is enqueued.  QS_FRONT_HELD is not supported here
 * (QS_ERR_UNSUPPORTED); one instance per call.
 *
 * The first call on a device looks up the array's address once
 * (cudaGetSymbolAddress, with that device current): make that first call
 * before any stream capture.  Every call reuses the same array and leaves
 * its contents behind (the ticket and error word are cleared at the start
 * of each call), so calls whose work overlaps on the GPU, e.g. on two
 * streams, race on it.
 *
 * The tables are computed on the host and copied from ordinary (pageable)
 * host memory, so the call may wait for `stream` before it returns; a call
 * on a stream that is being captured returns QS_ERR_UNSUPPORTED with nothing
 * enqueued.  The problem statement is checked as in qs_init (QS_ERR_ARG for
 * non-finite or out-of-range values, QS_ERR_UNSUPPORTED for geometries this
 * build does not serve). */
qs_status qs_sweep_noalloc(const qs_params *p, void *state, void *theta, int *exponents,
                           int64_t step0, int n_steps, int *dev_status, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* QS_H */
