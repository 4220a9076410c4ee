/*
 * fkp.h - C ABI of the GB300 library for the FFT-based power-spectrum and
 * bispectrum multipole estimators of Scoccimarro (2015), "Fast Estimators
 * for Redshift-Space Clustering", arXiv:1506.02729.
 *
 * The library computes, for a galaxy catalog and its random catalog:
 *   P_0, P_2, P_4 (Sec. III.A, eqs. P0_impl, P2_impl, P4_impl) and the
 *   reduced-FFT hexadecapole P_4b (eqs. P4fast, P4_implb), and
 *   B_0, B_2, B_4 for closed triangles (Sec. III.B, eqs. BispMono, BispQuad)
 *   with the thin-shell shot noise of eq. SNbisp2thin and exact triangle
 *   counts N_T (eq. NT).
 *
 * Conventions (the readings the library fixes where the paper is silent):
 *   - Fourier sign e^{-ik.x}; the DFT phase origin is the box corner.
 *   - alpha = W_g / W_r (weighted) by default, N_g/N_r on request.
 *   - x^ (the line of sight) is taken at grid nodes about the observer.
 *   - CIC (assign = 2), TSC (3) or PCS (4) with nodes at origin + i*L/N,
 *     optionally interlaced (a second grid half a cell further).
 *   - Modes with any |n_a| = N/2 are excluded from every bin and shell.
 *   - P bins are half-open [kmin + i dk, kmin + (i+1) dk), decided in FP64.
 *   - P_4b = [35/2 <|F_2|^2> - 5 <Re F_2 F_0*> - 7/2 <|F_0|^2>] / I_22.
 *   - I_33 = alpha sum_r nbar^2 w^3.
 *   - Bispectrum shells: centre (first + s*step) k_f, width width*k_f.
 *
 * Errors: every int-returning call returns 0 on success or a negative
 * FKP_E* code; fkp_last_error() then returns a thread-local message.
 * Ownership: the caller owns every input array and every output array it
 * passes; the library owns its device workspaces (allocated when a plan is
 * created, freed by fkp_plan_destroy).  Input pointers are read only during
 * the call.  A plan is used by one thread and one stream at a time.
 */
#ifndef FKP_H
#define FKP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  FKP_OK = 0,
  FKP_EINVAL = -1,   /* bad sizes, bins, flags or NULL pointers            */
  FKP_EGEOM = -2,    /* object too close to the box edge, or shells alias  */
  FKP_ENOMEM = -3,   /* device allocation failed / over the HBM budget     */
  FKP_ETIMEOUT = -4, /* a bounded device-side wait gave up                 */
  FKP_ECUDA = -5,    /* a CUDA runtime call failed                         */
  FKP_ESTATE = -6    /* call not valid in the plan's state                 */
};

/* What to compute (bit flags).  FKP_P6B, FKP_P8B: the l = 6 and 8 power
 * multipoles by the line-of-sight split of Sec. II.B (the remark after eq.
 * P4fast: the 22 fields of l <= 4 give l = 6 and 8 too).  FKP_B4B: the split
 * hexadecapole bispectrum of eq. Bhexa2 (delta_2 on the two larger sides;
 * a true multipole on zero-area triangles).
 *
 * FKP_XHAT_OBJECT (a modifier, not an output): the moment fields of eqs. Qij,
 * Qijkl take each object's own line of sight x^ (eq. Qab with x^ of the
 * object) instead of the grid node's: every moment field is gridded from the
 * catalogs, sum w x^_a x^_b (...) W, before its FFT, so the estimator is the
 * gridded form of the direct sum over objects of w L_l(k^.x^) e^{-ik.x}.
 * Power multipoles of one grid only: fkp_plan_create rejects it with any
 * FKP_B* flag or an interlaced geometry (FKP_EINVAL), and such plans do not
 * take fkp_plan_cache_randoms, fkp_power_batch or fkp_power_from_grid
 * (FKP_ESTATE).  The plan holds one int64 grid per moment field (16 with
 * FKP_P4, 6 with FKP_P2 alone, 8 N^3 bytes each) and grids the catalogs once
 * per field. */
enum {
  FKP_P0 = 1, FKP_P2 = 2, FKP_P4 = 4, FKP_P4B = 8,
  FKP_B0 = 16, FKP_B2 = 32, FKP_B4 = 64,
  FKP_P6B = 128, FKP_P8B = 256, FKP_B4B = 512,
  FKP_XHAT_OBJECT = 1024
};

/* One catalog {x_j, w_j, nbar_j} (Sec. III.A, around eq. F0), structure of
 * arrays of n float32 values.  w may be NULL: then w_j = 1/(1 + nbar_j P_fkp)
 * (FKP weights).  on_device = 1: device pointers; 0: host pointers (pinned or
 * pageable), copied in by the call. */
typedef struct {
  const float *x, *y, *z, *w, *nbar;
  int64_t n;
  int on_device;
} fkp_catalog_t;

/* Box, grid and observer.  The grid has N^3 nodes at origin + i*L/N.
 * observer_at_infinity = 1 uses the constant unit vector los as x^.
 * assign: 2 = CIC, 3 = TSC, 4 = PCS (the cubic B-spline: the paper's
 * fourth-order interpolation, Sec. III.A after eq. mapFFT).
 * periodic = 0 rejects objects closer than assign/2 + 1 cells to a box face
 * (FKP_EGEOM); periodic = 1 wraps node indices mod N.
 * compensate = 1 divides every mode by prod_a sinc(pi n_a/N)^assign.
 * alpha_mode: 0 = W_g/W_r, 1 = N_g/N_r.
 * interlace = 1 grids every field twice, the second time on nodes at
 * origin + (i + 1/2) L/N, and averages F_l = [F_l^(1) + e^{-i pi (n_x + n_y +
 * n_z)/N} F_l^(2)] / 2 (the paper's interlaced grids: the odd alias images
 * cancel); it doubles the gridding and the x- and y-passes.  Not with
 * fkp_power_from_grid, fkp_power_from_grid_noalloc or fkp_power_batch. */
typedef struct {
  double L;
  double origin[3];
  double observer[3];
  int observer_at_infinity;
  double los[3];
  int N;
  int assign;
  int compensate;
  int periodic;
  double P_fkp;
  int alpha_mode;
  int interlace;
} fkp_geometry_t;

/* P bins: edges kmin + i*dk, i = 0..nbins (h/Mpc), half-open. */
typedef struct {
  double kmin, dk;
  int nbins;
} fkp_pbins_t;

/* Bispectrum shells in integer k_f units: shell s holds modes with
 * c_s - width/2 <= |n| < c_s + width/2, c_s = first + s*step. */
typedef struct {
  int first, step, width, nshells;
} fkp_bshells_t;

/* Power-spectrum results.  Array pointers are caller-allocated host arrays
 * of nbins entries (any may be NULL to skip).  Scalars are always filled.
 * P_l follow eqs. P0_impl, P2_impl, P4_impl, P4_implb; mono_raw is
 * <|F_0|^2>/I_22 before shot-noise subtraction. */
typedef struct {
  double *k_eff, *P0, *P2, *P4, *P4b, *mono_raw;
  int64_t *nmodes;
  double alpha, I22, I33, N0, N0_fkp, S3, W_g, W_r;
  double Lab[6];        /* eq. Lab at k = 0, order xx yy zz xy yz zx */
  int64_t n_gal, n_ran;
  float timing_ms[8];   /* scalars, assign, xpass, ypass, zpass, bisp ifft (the F^w passes and the shell
                         * IFFTs), contraction, total */
  int graph;            /* 1 when the call replayed the plan's CUDA graph (see fkp_plan_set_graphs) */
  /* split multipoles (FKP_P6B, FKP_P8B; nbins entries, may be NULL):
   *   P_6b = 13 s60 / I_22,  s60 = 11/5 [<Re F_4 F_2*> - 2/7 <Re F_2 F_0*> - 20/77 <Re F_4 F_0*>]
   *   P_8b = 17 s80 / I_22,  s80 = 1287/490 [<|F_4|^2> - 1/9 <|F_0|^2> - 100/693 <Re F_2 F_0*>
   *                                          - 162/1001 <Re F_4 F_0*> - 20/99 s60]
   * (L_2 L_4 and L_4^2 in Legendre polynomials, each product's factors about
   * two lines of sight; no shot-noise subtraction is needed). */
  double *P6b, *P8b;
} fkp_power_out;

/* Bispectrum results, ntri entries each (caller-allocated host arrays, any
 * may be NULL).  Triangles are shell triples a >= b >= c (largest side
 * first) with N_T > 0, in lexicographic (a, b, c) order. */
typedef struct {
  int16_t *tri;         /* [ntri][3] */
  int64_t *NT;          /* exact closed-triangle counts (eq. NT)              */
  uint8_t *centre_closed; /* 1 when c_b + c_c >= c_a                          */
  double *B0, *B2, *B4; /* eqs. BispMono, BispQuad (shot noise subtracted)  */
  double *N0, *N2, *N4; /* thin-shell shot noise of eq. SNbisp2thin          */
  double *T0, *T2, *T4; /* raw sums sum_x F_a^(l) F_b^(0) F_c^(0) (eq. Factorize) */
  double I33, S3;
  /* split hexadecapole (FKP_B4B; ntri entries, may be NULL): T22 = sum_x
   * F_a^(2) F_b^(2) F_c^(0) and B4b = [35/2 T22 - 5 T2 - 7/2 T0] / (N^3 N_T
   * I_33), eq. Bhexa2 from the raw sums (the self terms cancel on zero-area
   * triangles as for P_4b; no thin-shell noise is subtracted). */
  double *B4b, *T22;
} fkp_bisp_out;

/* Contraction of the triangle sums (eq. Factorize):
 *   FP32   CUDA cores, FP32 products, compensated FP32 sums, FP64 across slices;
 *   BF16X3 tcgen05 tensor cores, operands split v = hi + lo in BF16, products
 *          hi*hi + hi*lo + lo*hi, FP32 accumulation in tensor memory;
 *   BF16X6 tcgen05 tensor cores, 3-way split hi + mid + lo, the six products of
 *          order <= 2^-16: per-term error near FP32 rounding.
 * The tensor-core modes need (number of multipoles) x (shells) <= 128. */
enum { FKP_CONTRACT_FP32 = 0, FKP_CONTRACT_BF16X3 = 1, FKP_CONTRACT_BF16X6 = 2 };

/* Context: binds a CUDA device.  hbm_budget_bytes = 0 means no limit.
 * Returns FKP_EINVAL for a bad device index, FKP_ECUDA on runtime errors. */
int fkp_context_create(int device, size_t hbm_budget_bytes, void **ctx);
void fkp_context_destroy(void *ctx);

/* Plan: validates geometry and bins, builds the FP64 bin look-up table
 * (n^2 -> bin, eq. shell), the twiddle tables and, when B is wanted, the
 * shell tables; allocates the device workspace.  bshells may be NULL when
 * no FKP_B* flag is set.  FKP_EGEOM when B is wanted and 3*n_max >= N (the
 * triangle sum of eq. Factorize would alias). */
int fkp_plan_create(void *ctx, const fkp_geometry_t *geom, const fkp_pbins_t *pbins,
                    const fkp_bshells_t *bshells, uint32_t want, void **plan);
void fkp_plan_destroy(void *plan);

/* Sizes the caller needs for its outputs and the plan's device footprint
 * (workspace plus the catalog buffers it keeps between calls and, once
 * fkp_power_batch has run, its batch workspace). */
int fkp_plan_sizes(const void *plan, int *nbins, int *ntriangles, size_t *workspace_bytes);

/* Launch schedule of the three FFT passes of a plan: x_mult (x-pass blocks
 * per SM = resident blocks x x_mult: 1, 2, 4 or 8), and the threads per block
 * of the y- and z-passes (256 or 512).  The first plan of a given grid and
 * multipole order in a context times the x- and y-pass candidates on its own
 * workspace (about 12 launches of each pass) and keeps the fastest; later
 * plans of that kind reuse the choice.  The z-pass shape is fixed per grid
 * (256 threads up to N = 256, 512 above): it sets how the bin sums are
 * split into FP32 runs, so with it fixed every result is the same bit for bit
 * whatever the tuning picks (every reduction of the path has a fixed order or
 * is integer).  tuned_ms (3 floats, may be NULL) receives the passes' times.
 * fkp_plan_set_schedule overrides the choice for one plan (FKP_EINVAL
 * outside those values); another z_threads changes the bins' FP32 run
 * rounding (~1e-7). */
int fkp_plan_schedule(const void *plan, int *x_mult, int *y_threads, int *z_threads, float *tuned_ms);
int fkp_plan_set_schedule(void *plan, int x_mult, int y_threads, int z_threads);

/* CUDA graphs of the power path (default on).  With device catalogs, the
 * second fkp_power call on a plan with the same catalog pointers and sizes
 * captures the gridding, FFT passes and binning into a graph; later calls
 * with those catalogs replay it (one launch instead of about twenty).  A
 * different catalog runs the plain launches; host catalogs never use the
 * graph.  enable = 0 frees the graph and keeps plain launches.  Results
 * are the same either way. */
int fkp_plan_set_graphs(void *plan, int enable);

/* Random catalog shared by many mocks (Sec. III.C, Performance: gridding
 * the randoms is most of the time, 210 s of the paper's 232 s, and mocks for
 * a covariance estimate usually share one random catalog).  Grids `ran` once
 * onto the plan without alpha -- R(x) = sum_r w W(x - x_r), and for
 * bispectrum plans R^w(x) = sum_r w^2 W(x - x_r) -- and keeps its scalar sums
 * (W_r, sum w^2, sum w^3, sum nbar w^2, sum nbar^2 w^3, L^ab) and its size.
 * Later fkp_power, fkp_bispectrum and fkp_power_batch calls with ran (rans)
 * == NULL grid only the galaxies and use F = G - alpha R and F^w = G^w +
 * alpha^2 R^w with alpha from the galaxies' W_g and the cached W_r; results
 * equal those of passing the same random catalog (up to the rounding of
 * each random term to the grid's 2^-40 fixed point).  A new call replaces the
 * cache; ran->n = 0 drops it.  The cached grids take 8 N^3 bytes each.
 * FKP_EGEOM if a random lies too close to a box face (non-periodic plans). */
int fkp_plan_cache_randoms(void *plan, const fkp_catalog_t *ran, void *cuda_stream);

/* P_l of one survey (Sec. III.A).  Enqueues every step on cuda_stream (a
 * cudaStream_t, NULL = legacy default stream), then synchronizes it and
 * fills out.  ran == NULL uses the plan's cached random catalog
 * (fkp_plan_cache_randoms; FKP_ESTATE without one).  FKP_EGEOM if an object
 * lies too close to a box face (non-periodic plans). */
int fkp_power(void *plan, const fkp_catalog_t *gal, const fkp_catalog_t *ran,
              void *cuda_stream, fkp_power_out *out);

/* The gridded fields of one survey (eq. mapFFT and the F^w of eq. SNbisp2):
 * F(x) = sum_g w W(x - x_g) - alpha sum_r w W(x - x_r) and, for bispectrum
 * plans, F^w(x) = sum_g w^2 W(x - x_g) + alpha^2 sum_r w^2 W(x - x_r), with
 * the plan's assignment W and alpha = W_g / W_r, exactly as fkp_power and
 * fkp_bispectrum grid them.  Every tap's value is rounded to a multiple of
 * 2^-40 and the rounded values are summed as integers, so the grid is the
 * same whatever the order of the objects.  F and Fw (host or device, N^3
 * int64 each, [z][y][x] with x fastest, owned by the caller) receive the
 * fields in units of 2^-40; Fw may be NULL and must be NULL for plans
 * without bispectrum outputs (FKP_EINVAL).  which = 1 selects the second
 * grid of an interlaced plan (origin shifted by half a cell along each axis;
 * FKP_EINVAL otherwise).  ran == NULL uses the cached random catalog as
 * fkp_power does.  Synchronizes cuda_stream before it returns.  FKP_EGEOM if
 * an object lies too close to a box face (non-periodic plans). */
int fkp_grid(void *plan, const fkp_catalog_t *gal, const fkp_catalog_t *ran, int which,
             long long *F, long long *Fw, void *cuda_stream);

/* P_l of nmock independent surveys (mocks) on one plan's grid, for the
 * ensembles that covariance estimates need (abstract; Sec. III.C, Performance): gals[k] and
 * rans[k] (host or device, any sizes, randoms non-empty) give mock k, whose
 * results go to outs[k] (NULL: none).  Each mock is gridded with launches
 * shaped by its own catalogs; then the three FFT passes and the bin
 * reduction run once for all mocks (one launch each, the mock index in the
 * grid).  Every mock's results are those of fkp_power on the same catalogs:
 * the same grid, scalars and bins, bit for bit.  The plan keeps a batch workspace (grid, pass buffers and bins
 * per mock: about 15 GB per mock at 512^3, 1.9 GB at 256^3) sized for the
 * largest nmock seen; FKP_ENOMEM when that exceeds the context's HBM budget
 * or the device.  Stage times in outs[k].timing_ms are those of the whole
 * batch: [1] gridding of all mocks, [2..4] the fused x, y, z passes (z with
 * the bin reduction), [7] the whole batch.  nmock: 1 .. 65535.  rans == NULL:
 * every mock uses the plan's cached random catalog. */
int fkp_power_batch(void *plan, int nmock, const fkp_catalog_t *gals, const fkp_catalog_t *rans,
                    void *cuda_stream, fkp_power_out *outs);

/* The same estimator applied to a given real field F(x) (device pointer to
 * N^3 float32, layout [z][y][x]), with caller-supplied I_22 and N_0.  Test
 * hook for periodic-box checks. */
int fkp_power_from_grid(void *plan, const float *F_device, double I22, double N0,
                        void *cuda_stream, fkp_power_out *out);

/* P_l and B_l of one survey (Sec. III.B).  contraction is one of
 * FKP_CONTRACT_FP32, _BF16X3, _BF16X6.  ran == NULL uses the plan's cached
 * random catalog. */
int fkp_bispectrum(void *plan, const fkp_catalog_t *gal, const fkp_catalog_t *ran,
                   int contraction, void *cuda_stream, fkp_power_out *pout, fkp_bisp_out *bout);

/* The estimator of fkp_power_from_grid for small grids without allocating
 * any device memory: every device buffer it uses lives in one file-scope
 * device array of about 42 MB, held by each GPU that has mapped the library's
 * device code until the process exits.  The paper has no counterpart; this is
 * for callers that cannot call cudaMalloc while running (a process that
 * reserved all device memory for its own pool, a real-time loop that forbids
 * allocation after start-up, a plugin host that gives the library no
 * allocator).
 * With CUDA's lazy module loading (the default since CUDA 12.2) the array and
 * the kernels are mapped onto a device by the first call there, not when the
 * library is loaded: make one warm-up call per device (or run with
 * CUDA_MODULE_LOADING=EAGER) before reserving the rest of the device's memory,
 * or that first call can fail with FKP_ECUDA.
 * Arguments: geometry and P bins as for fkp_plan_create (no plan is made),
 * F_device the real field [z][y][x] (N^3 float32, device pointer), I22 and
 * N0 as for fkp_power_from_grid, results in out (caller-allocated arrays of
 * nbins entries, any may be NULL).
 * Limits: even N <= 64 and nbins <= 64; larger requests return FKP_EINVAL
 * with a message.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  Every call on a device shares the array and reinitialises what
 * must start at zero, so calls whose GPU work overlaps (two streams, or two
 * threads) race and must be serialised by the caller.  The call
 * synchronizes its stream before returning. */
int fkp_power_from_grid_noalloc(const fkp_geometry_t *geom, const fkp_pbins_t *pbins, const float *F_device,
                                double I22, double N0, void *cuda_stream, fkp_power_out *out);

/* ---------------------------------------------------------------------------
 * Request server (continuous batching).  The paper's use of the estimators is
 * covariance estimation from many realisations of a survey (Sec. III.C, the
 * ~10^4 mocks of its performance section); the server runs such requests as
 * they arrive.  It keeps nslots worker threads, each with its own CUDA
 * stream, and a pool of plans shared by the slots (a request reuses an idle
 * plan of its geometry, so workspaces stay on the device between requests).
 * A request is admitted when its estimated device footprint fits next to the
 * pooled plans and running requests within hbm_budget_bytes (0 = 90 % of the
 * free device memory at creation), evicting idle plans of other geometries
 * (least recently used first) when that makes room; the queue is first-in
 * first-out with skip-ahead.  Requests on different slots
 * run concurrently on the device.  Every result equals the one the same
 * request gives alone, bit for bit (integer gridding, fixed-order or integer
 * reductions, the z-pass shape fixed per grid).
 * ------------------------------------------------------------------------- */

/* One request: the arguments of fkp_plan_create plus catalogs and outputs.
 * The catalog arrays and the output arrays must stay valid until the ticket
 * has completed (fkp_server_wait returned). */
typedef struct {
  fkp_geometry_t geom;
  fkp_pbins_t pbins;
  fkp_bshells_t bshells;   /* read when want has an FKP_B* flag */
  uint32_t want;
  int contraction;         /* FKP_CONTRACT_* for bispectrum requests */
  fkp_catalog_t gal, ran;
  fkp_power_out *pout;     /* may be NULL */
  fkp_bisp_out *bout;      /* may be NULL */
} fkp_request_t;

typedef struct {
  int64_t submitted, completed, failed, rejected, queued;
  int running, peak_running;
  size_t bytes_in_use, peak_bytes, budget_bytes;
} fkp_server_stats_t;

/* Creates the server on a device.  FKP_EINVAL unless 1 <= nslots <= 64. */
int fkp_server_create(int device, int nslots, size_t hbm_budget_bytes, void **server);
/* Queues a request; *ticket identifies it.  FKP_ENOMEM when the request alone
 * exceeds the budget (it is not queued), FKP_EINVAL for malformed requests. */
int fkp_server_submit(void *server, const fkp_request_t *req, uint64_t *ticket);
/* *done = 1 when the request has finished (successfully or not). */
int fkp_server_poll(void *server, uint64_t ticket, int *done);
/* Waits up to timeout_ms (< 0: no limit) for the ticket; FKP_ETIMEOUT if it is
 * still running (the ticket stays valid).  On completion *status is the
 * request's own return code and *latency_ms the time from submission to
 * completion, and the ticket is retired.  When the request failed, its
 * worker's error message becomes this thread's fkp_last_error(). */
int fkp_server_wait(void *server, uint64_t ticket, int timeout_ms, int *status, double *latency_ms);
int fkp_server_stats(void *server, fkp_server_stats_t *stats);
/* Lets queued and running requests finish, then frees everything. */
void fkp_server_destroy(void *server);

/* Diagnostic of the bounded device-side waits (the FFT passes wait on an
 * mbarrier for each bulk tile copy, giving up after a fixed number of polls
 * and reporting FKP_ETIMEOUT instead of hanging).  Launches one block on
 * `device` that initialises an mbarrier, issues no copy, never arrives, and
 * waits on it with the same bounded wait for `polls` polls (1 .. 4194304).
 * The expected return is FKP_ETIMEOUT, with the device context left usable;
 * FKP_ESTATE means the wait completed (it must not), FKP_EINVAL bad
 * arguments, FKP_ECUDA a runtime failure.  Allocates and frees 4 bytes. */
int fkp_selftest_bounded_wait(int device, unsigned polls);

/* Host-only consistency check of the tables that map the moment fields to
 * the k_z-power groups (for lmax = 0, 2, 4): the field order matches the
 * kernels', and the coefficients reproduce S_2 = (k.x^)^2 and S_4 = (k.x^)^4
 * for unit vectors x^ (the multiplicities of eqs. delta2b, delta4b and the
 * trace identities of x^).  Needs no GPU.  Returns FKP_OK or FKP_ESTATE. */
int fkp_check_tables(void);

/* Thread-local message for the last error on this thread. */
const char *fkp_last_error(void);

/* Library version string. */
const char *fkp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FKP_H */
