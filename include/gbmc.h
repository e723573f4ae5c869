/*
 * gbmc -- GB300-native event-based continuous-energy Monte Carlo transport
 * hot path.  C ABI (C99, extern "C"): plain pointers and sizes only.
 *
 * The operations follow the method studied in Tramm et al., "Performance
 * Portable Monte Carlo Particle Transport on Intel, NVIDIA, and AMD GPUs":
 *   - event-based parallelism, one narrow kernel per event type over every
 *     queued particle (Sec. 2, "Event-Based Parallelism");
 *   - particles sorted by material and energy before the cross-section
 *     lookup, the dominant kernel (Sec. 2, "Sorting");
 *   - tallies scored during active batches (Sec. 2, "Tallying");
 *   - a cap on particles in flight, refilled from the batch's remaining
 *     source particles (Sec. 2, "In-Flight Particles");
 *   - surface (ray) tracking, delta tracking disabled (Sec. 3);
 *   - results reproducible between a serial history-based CPU run and the
 *     event-based GPU run up to floating-point summation order (Sec. 4.3).
 *
 * Conventions for every entry point:
 *   - return value: GBMC_OK (0) or a negative GBMC_ERR_* code; no exception
 *     or exit crosses the ABI; gbmc_last_error() returns a context-owned
 *     message describing the last failure;
 *   - host pointers are read (or written) during the call only and never
 *     retained; device memory is allocated and owned by the context unless
 *     an entry point says it takes device pointers from the caller;
 *   - units: energies in eV, lengths in cm, microscopic cross sections in
 *     barns, densities in atoms/(barn cm);
 *   - one context drives one device; calls on one context must not overlap.
 */
#ifndef GBMC_H
#define GBMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define GBMC_OK 0
#define GBMC_ERR_INVALID_ARG (-1)     /* argument failed validation */
#define GBMC_ERR_NOT_INITIALIZED (-2) /* tables / materials / tally not loaded */
#define GBMC_ERR_OOM (-3)             /* device allocation failed */
#define GBMC_ERR_CUDA (-4)            /* a CUDA runtime call failed */
#define GBMC_ERR_TIMEOUT (-5)         /* the device event loop hit its iteration bound */
#define GBMC_ERR_DEVICE_FLAG (-6)     /* a kernel flagged an inconsistency */
#define GBMC_ERR_UNSUPPORTED (-7)     /* feature not available on this device */

/* ---- table precision --------------------------------------------------- */
#define GBMC_FP64 0 /* binary64 tables, interpolation and sums */
#define GBMC_FP32 1 /* binary32 tables, interpolation and sums; binary64
                       positions, directions, distances and tallies */

/* ---- geometry kinds, boundary conditions, sources ---------------------- */
#define GBMC_GEOM_INFINITE 0 /* one homogeneous material, no surfaces */
#define GBMC_GEOM_LATTICE 1  /* n x n pin cells of pitch p: a cylinder of radius
                                r on each cell axis, height H along z */
#define GBMC_GEOM_SLAB 2     /* n_layers layers of thickness dx along x */
#define GBMC_BC_VACUUM 0
#define GBMC_BC_REFLECT 1
#define GBMC_SRC_ORIGIN 0    /* point at the origin, isotropic */
#define GBMC_SRC_BOX 1       /* uniform in the lattice box, isotropic */
#define GBMC_SRC_SLAB_FACE 2 /* point on x = 0, isotropic over the inward hemisphere */
#define GBMC_SRC_BANK 3      /* the fission bank set by gbmc_set_source_bank, isotropic
                              * (lattice or infinite medium; k-eigenvalue mode) */

/* ---- per-particle outcome status -------------------------------------- */
#define GBMC_STATUS_ABSORBED 1
#define GBMC_STATUS_LEAKED 2
#define GBMC_STATUS_CUTOFF 3     /* energy fell below E_cut */
#define GBMC_STATUS_LIMIT 4      /* GBMC_MAX_FLIGHTS flights reached */
#define GBMC_STATUS_LEAKED_FAR 5 /* slab: left through x = n_layers dx */
#define GBMC_STATUS_ROULETTE 6   /* killed by weight-window roulette */
#define GBMC_MAX_FLIGHTS 100000

/* ---- scalar tally slots (counts are int64, weights binary64) ----------- */
#define GBMC_S_COLLISION 0
#define GBMC_S_ABSORPTION 1
#define GBMC_S_LEAK 2
#define GBMC_S_CUTOFF 3
#define GBMC_S_LIMIT 4
#define GBMC_S_LEAK_FAR 5
#define GBMC_S_FLIGHT 6
#define GBMC_S_HISTORY 7
#define GBMC_S_SPLIT 8      /* copies made by weight-window splits (weight they carry) */
#define GBMC_S_ROULETTE 9   /* histories ended by roulette (weight before) */
#define GBMC_NSCAL 10

typedef struct gbmc_ctx gbmc_ctx;

/* Launch and scheduling options.  Any field left 0 takes its default. */
typedef struct {
    int32_t precision;       /* GBMC_FP64 or GBMC_FP32 (tables must be loaded in it) */
    int64_t max_in_flight;   /* cap on particles in flight (Sec. 2, "In-Flight
                                Particles"); 0: min(particles of the run, 8M) */
    int32_t sort;            /* 1 (default): sort the lookup queue by material
                                and energy (Sec. 2, "Sorting"); -1: do not sort */
    int32_t block_lookup;    /* threads per block of the lookup kernel (default 256) */
    int32_t block_event;     /* threads per block of the other event kernels (256) */
    int32_t blocks_per_sm;   /* event-kernel grid = SMs x blocks_per_sm (default 8) */
    int32_t max_iterations;  /* bound on event-loop iterations of one run
                                (default 4 * GBMC_MAX_FLIGHTS); reaching it
                                returns GBMC_ERR_TIMEOUT from the next read */
    int32_t sort_min;        /* sort only iterations with at least this many
                                lookups (default 4096) */
    int32_t warp_lookup_max; /* iterations with fewer lookups run one warp per
                                particle instead of one thread (default 4096;
                                -1: never) */
    int32_t tail_max;        /* once the source is exhausted and at most this many
                                particles are in flight, the loop stops and a
                                tail kernel finishes them, one warp per particle
                                (default 4096; -1: never) */
    int32_t sparse_windows;  /* binary32 lookup searches a finer coarse index (about
                                two buckets a grid point) whose buckets each hold a
                                32-byte window of four (E, sigma) pairs, read as one
                                256-bit load (1), instead of the 64-byte windows of
                                seven pairs (0, default).  One sector and one L1
                                wavefront per lane and nuclide where the lanes of a
                                warp read distinct windows (tables far beyond L2,
                                particles sparser in energy than the grid points).
                                Same results either way. */
    int32_t group_lookup_max; /* binary64 tables: iterations with fewer lookups (and
                                at least warp_lookup_max) run 4 lanes per particle,
                                each with a quarter of the nuclides (default 160000;
                                -1: never): shorter chains of dependent loads per
                                warp where the queue is too short to hide them */
    int32_t search;          /* bracket search of the energy grids: 1 (default) a
                                coarse index over each grid's bit patterns (binary64:
                                about one point a bucket, then at most about one
                                bisection step; binary32: a bucket window of the
                                bracket's pairs), the "double indexing" of the codes
                                the paper compares against (Sec. 3); -1 a plain
                                binary search of each whole grid.  Same results
                                either way (the bracket is unique). */
    int32_t reserved[2];
} gbmc_options;

/* One geometry (and its source).  Fields of other kinds are ignored. */
typedef struct {
    int32_t kind;     /* GBMC_GEOM_* */
    int32_t source;   /* GBMC_SRC_* */
    double E0;        /* source energy (eV) */
    double E_cut;     /* energy cutoff (eV): a scatter below it ends the history */
    int32_t mat;      /* INFINITE: material index */
    int32_t n;        /* LATTICE: cells per side */
    double pitch;     /* LATTICE: cell pitch p */
    double radius;    /* LATTICE: pin radius r, 0 < r < p/2 */
    double height;    /* LATTICE: height H (z in [0, H]) */
    int32_t mat_pin;  /* LATTICE: material inside the pins */
    int32_t mat_mod;  /* LATTICE: material outside the pins */
    int32_t bc_side;  /* LATTICE: x/y outer faces, GBMC_BC_* */
    int32_t bc_z;     /* LATTICE: z = 0 and z = H faces, GBMC_BC_* */
    int32_t n_layers; /* SLAB: number of layers (x in [0, n_layers dx]); both faces vacuum */
    double layer_dx;  /* SLAB: layer thickness */
    int32_t n_first;  /* SLAB: layers [0, n_first) hold mat_a, the rest mat_b */
    int32_t mat_a, mat_b;
} gbmc_geometry;

/* One independent fixed-source problem of a run. */
typedef struct {
    gbmc_geometry geom;
    uint64_t seed;           /* Philox key word 0 */
    uint32_t problem_index;  /* Philox key word 1 = problem_index << 32 | batch */
    uint32_t batch;
    int64_t first_id;        /* histories first_id .. first_id + n_particles - 1 */
    int64_t n_particles;
} gbmc_problem;

/* Counters of the last run (for throughput figures). */
typedef struct {
    int64_t iterations;       /* event-loop iterations */
    int64_t lookups;          /* macroscopic lookups (lookup-event particles) */
    int64_t micro_lookups;    /* nuclide lookups in the lookup event */
    int64_t flights;          /* advance events */
    int64_t crossings;        /* surface events */
    int64_t collisions;       /* collision events */
    int64_t histories;        /* particles born */
    int32_t device_error;     /* 0, or the first GBMC_ERR_* a kernel flagged */
    int32_t reserved;
    int64_t handoffs;         /* particles a ray-trace warp handed to the next
                                 iteration once its queue was exhausted and at
                                 most a quarter of its lanes were busy (each after
                                 at least one flight) */
} gbmc_stats;

/* Per-kernel device time of one profiled run (gbmc_profile_problems). */
#define GBMC_NKERNELS 8
typedef struct {
    /* kernels: 0 plan, 1 source, 2 sort scan (bucket offsets from the
       counts the queue appends keep), 3 sort scatter, 4 lookup, 5 ray trace
       (advance and surface events), 6 collision, 7 tail (finishes the last
       particles in flight) */
    double ms[GBMC_NKERNELS];        /* summed device time (CUDA events) */
    int64_t launches[GBMC_NKERNELS]; /* launches of each kernel */
} gbmc_kernel_times;

/* Fill *opt with the defaults. */
int gbmc_default_options(gbmc_options *opt);

/* Create a context on CUDA device `device` (opt may be NULL: defaults).
 * On success *out owns its device memory until gbmc_destroy. */
int gbmc_create(gbmc_ctx **out, int device, const gbmc_options *opt);

/* Release every device allocation of the context.  NULL is accepted. */
int gbmc_destroy(gbmc_ctx *ctx);

/* Message of the last failure on ctx ("" if none).  Owned by the context;
 * valid until the next call on it.  With ctx == NULL: the last gbmc_create
 * failure of this thread. */
const char *gbmc_last_error(const gbmc_ctx *ctx);

/* Replace the options.  Takes effect at the next run. */
int gbmc_set_options(gbmc_ctx *ctx, const gbmc_options *opt);

/* Load the pointwise nuclide tables (Sec. 2, "Sorting": the lookup reads
 * each nuclide's energy grid and cross sections).
 *   n_nuc     number of nuclides (>= 1)
 *   grid_off  [n_nuc+1] int64, grid_off[0] = 0, at least 2 points per nuclide
 *   energy    [grid_off[n_nuc]] eV, strictly increasing within each nuclide, > 0
 *   sigma_t   [grid_off[n_nuc]] barns, > 0, finite
 *   f_abs     [n_nuc] absorption fraction sigma_a / sigma_t in [0, 1]
 *   awr       [n_nuc] atomic-weight ratio A >= 1 (elastic kinematics)
 *   precision GBMC_FP64 or GBMC_FP32: which device copy to build; the
 *             binary32 copy is the round-to-nearest cast of each value and is
 *             rejected (GBMC_ERR_INVALID_ARG) if a grid stops being strictly
 *             increasing after the cast.  Loading one precision keeps the
 *             other's copy if it was loaded from the same tables before.
 * Host arrays are copied.  Replaces earlier tables of that precision. */
int gbmc_load_xs_tables(gbmc_ctx *ctx, int32_t n_nuc, const int64_t *grid_off,
                        const double *energy, const double *sigma_t,
                        const double *f_abs, const double *awr, int32_t precision);

/* Define the materials: material m holds nuclides nuc_id[mat_off[m] ..
 * mat_off[m+1]-1] with densities density[...] (atoms/(b cm), > 0).  The
 * listed order is the summation order of the macroscopic cross section.
 *   mat_off [n_mat+1] int32, nuc_id and density [mat_off[n_mat]].
 * Requires the tables (nuclide ids are range-checked).  Host arrays copied. */
int gbmc_init_materials(gbmc_ctx *ctx, int32_t n_mat, const int32_t *mat_off,
                        const int32_t *nuc_id, const double *density);

/* Energy bins of the track-length flux tally: edges [n_bins+1], strictly
 * increasing.  The bin of energy E is the largest b <= n_bins-1 with
 * edges[b] <= E (b = 0 below edges[0]).  Zeroes all tallies. */
int gbmc_set_tally(gbmc_ctx *ctx, int32_t n_bins, const double *edges);

/* Zero the tallies of every problem slot (stream-ordered on `stream`). */
int gbmc_reset_tallies(gbmc_ctx *ctx, void *stream);

/* Run one batch of one problem: histories prob->first_id .. + n_particles-1
 * of batch prob->batch, event by event on the GPU (Sec. 2).  Asynchronous on
 * `stream` (a cudaStream_t; NULL = legacy default stream).  Tallies
 * accumulate into problem slot 0 (reset when the slot layout changes);
 * per-particle outcomes of this run replace the previous ones.
 * Equivalent to gbmc_run_problems(ctx, 1, prob, stream). */
int gbmc_run_batch(gbmc_ctx *ctx, const gbmc_problem *prob, void *stream);

/* Run n_prob independent problems (each with its own geometry, source,
 * Philox key and particle count) in one device-driven event loop: their
 * particles share the in-flight bank, queues and kernels; tallies go to
 * problem slots 0 .. n_prob-1.  Asynchronous on `stream`. */
int gbmc_run_problems(gbmc_ctx *ctx, int32_t n_prob, const gbmc_problem *probs,
                      void *stream);

/* Concurrent event loops (Sec. 2, "GPU Streams": several independent event
 * loops share one GPU, so that the short final iterations of one, bound by
 * latency rather than work, overlap the full iterations of another).
 * Results are those of gbmc_run_problems(ctx, n_prob, probs, stream):
 * problem p's histories, outcomes (problem slot p), flux and scalar tallies
 * (slot p) are the same, and the tallies follow the same slot layout.  Only
 * the execution differs: the problems are taken in runs of per_run
 * consecutive problems, run r goes to event loop r % n_loops, each loop runs
 * its runs one after another, and the loops run concurrently.  A loop is a
 * particle bank, queues, control block, graph and CUDA stream of its own,
 * created on first use and kept by the context; all loops read the
 * context's tables and add into its tallies and outcome buffers.  The loops
 * start after the work already queued on `stream`, and `stream` waits for
 * all of them: the call is asynchronous on `stream`.
 *   n_loops  1..16 (device memory: one bank, queues and running-sum cache
 *            per loop, sized for its largest run);
 *   per_run  problems per run, >= 1 (1: one batch at a time per loop).
 * Afterwards gbmc_read_stats sums the counters of every run of the call and
 * gbmc_last_run_ms times the whole call.  Weight windows, k-eigenvalue
 * banking, bank sources and importance recording give GBMC_ERR_UNSUPPORTED
 * (they run in one event loop).  Other errors as gbmc_run_problems. */
int gbmc_run_concurrent(gbmc_ctx *ctx, int32_t n_prob, const gbmc_problem *probs,
                        int32_t n_loops, int32_t per_run, void *stream);

/* Host destination of one problem's results for
 * gbmc_run_concurrent_to_host: HOST arrays (pinned -- cudaHostAlloc or
 * cudaHostRegister -- for the copies to run asynchronously; a pageable one
 * makes its copy block the calling thread until the run has ended).  Any
 * pointer may be NULL (that part is not copied).  flux [n_cells * n_bins]
 * (cell-major), counts and weights [GBMC_NSCAL] (as gbmc_read_tallies gives
 * them), and the problem's per-particle outcomes [n_particles] each (as
 * gbmc_read_outcomes gives them for first 0). */
typedef struct {
    double *flux;
    int64_t *counts;
    double *weights;
    int32_t *n_coll;
    int8_t *status;
    int32_t *n_flights;
    uint32_t *n_draws;
    double *E, *x, *y, *z;
} gbmc_host_results;

/* gbmc_run_concurrent, and each run's results copied to the host as soon as
 * that run has ended: a loop's copies go on a copy stream of the loop's own,
 * so they overlap its next run and the other loops' work (the overlap of
 * transfers with compute the paper's streams give).  dst[p] (HOST array of
 * n_prob) receives problem p's tallies (slot p) and outcomes.  Asynchronous
 * on `stream`: the host arrays hold the results once `stream` has passed the
 * call (e.g. cudaStreamSynchronize).  Where the destinations of consecutive
 * problems of one run are adjacent in host memory (problem p + 1's array of a
 * field starting where problem p's ends), that field of those problems goes
 * in one copy; overlapping destinations are not allowed.  Errors a run flags on the device are
 * reported by the next gbmc_read_stats / gbmc_read_tallies.  dst NULL:
 * INVALID_ARG; other errors as gbmc_run_concurrent. */
int gbmc_run_concurrent_to_host(gbmc_ctx *ctx, int32_t n_prob, const gbmc_problem *probs,
                                int32_t n_loops, int32_t per_run, const gbmc_host_results *dst,
                                void *stream);

/* Page-locked host memory for result destinations (the paper has no
 * counterpart; the overlap of copies with compute that its streams give
 * needs such memory).  gbmc_host_alloc stores in *ptr a HOST pointer to
 * `bytes` bytes (bytes >= 1) of page-locked memory from cudaHostAlloc with
 * default flags, aligned for any element type, usable as any destination
 * of gbmc_host_results and by plain host code; the caller owns it and
 * releases it with gbmc_host_free.  Errors: ptr NULL or bytes 0 -> INVALID_ARG; the
 * allocation failing -> OOM (*ptr is then NULL).  gbmc_host_free(NULL) is
 * a no-op; freeing another pointer is undefined. */
int gbmc_host_alloc(size_t bytes, void **ptr);
int gbmc_host_free(void *ptr);

/* Synchronize the last run's stream and copy the tallies of problem slot
 * `slot`: flux [n_cells * n_bins] (cell-major; n_flux must equal it; NULL
 * skips), counts [GBMC_NSCAL] and weights [GBMC_NSCAL] (NULL skips).
 * Returns GBMC_ERR_TIMEOUT / GBMC_ERR_DEVICE_FLAG if the run reported one. */
int gbmc_read_tallies(gbmc_ctx *ctx, int32_t slot, double *flux, int64_t n_flux,
                      int64_t *counts, double *weights);

/* k-eigenvalue mode (power iteration; the paper's production setting runs
 * inactive then active generations, Sec. 2 "Tallying").  Fission data per
 * nuclide: nu = mean neutrons per fission (>= 0) and f_fis = sigma_f /
 * sigma_t (0 <= f_fis <= f_abs: fission is part of absorption).  HOST
 * arrays of n_nuc (the loaded tables' count), copied.  Errors: INVALID_ARG,
 * NOT_INITIALIZED before the tables. */
int gbmc_load_fission(gbmc_ctx *ctx, int32_t n_nuc, const double *nu, const double *f_fis);

/* Fission banking for the following runs (k_norm > 0; k_norm <= 0 turns it
 * off): at every collision in nuclide i a history banks floor(w nu_i
 * f_fis_i / k_norm + xi) sites at the collision point, xi being one more
 * draw taken right after the nuclide choice; at most max_sites (1..255)
 * per history (DEVICE_FLAG beyond).  After a run the sites form the bank in
 * history order (run index, then banking order), whatever the order of the
 * events.  Runs then take one problem and no weight windows (UNSUPPORTED).
 * k_norm is normally the previous generation's k estimate, so the bank
 * stays near the generation size; generation g's estimate is then
 * k_g = (bank size / N) k_norm. */
int gbmc_set_eigen(gbmc_ctx *ctx, double k_norm, int32_t max_sites);

/* The last k-eigenvalue run's bank: *n_out = its size; if xyz != NULL the
 * sites into HOST xyz[n_cap][3] (n_cap >= size, else INVALID_ARG).
 * Synchronizes.  NOT_INITIALIZED before a k-eigenvalue run. */
int gbmc_read_bank(gbmc_ctx *ctx, double *xyz, int64_t n_cap, int64_t *n_out);

/* Source bank of the runs whose geometry has source GBMC_SRC_BANK: HOST
 * xyz[n][3] (copied), or xyz == NULL for the last run's own bank (kept on the
 * device; n is then ignored).  n_total = the generation's size N: history id
 * i (0 <= i < N; the problem's ids must lie in [0, N)) starts at site
 * floor(i n / N) -- systematic sampling, so replicas that split the ids and
 * share one bank start exactly the histories of one run.  Synchronizes. */
int gbmc_set_source_bank(gbmc_ctx *ctx, const double *xyz, int64_t n, int64_t n_total);

/* Self-checks of the library's binary64 division on the integer units
 * (the binary64 units are this GPU's scarce resource), each result compared
 * bit for bit with the hardware binary64 operation, on n samples from a
 * seeded counter-based stream:
 *   kind 0: div_rn(a, b) against a / b -- random significands and signs,
 *           exponents across and beyond the normal range, the significand
 *           patterns where rounding is decided, zeros, infinities, NaNs;
 *   kind 1: the lookup's interpolation factor (E - e0) / de from an
 *           interval record (de = e1 - e0 and its fixed-point reciprocal,
 *           as the binary64 tables store them) against the same expression
 *           in binary64 -- 65536 grid-like intervals (widths 2^-52 e0 to
 *           2^14 e0, some of zero width), E at, next to, inside, below and
 *           far above the interval.
 * *n_bad = the number that differ (0 expected); first_bad (HOST, 2 doubles,
 * may be NULL) = the first differing operands (a, b), or (E, e0).  Errors:
 * INVALID_ARG for kind not 0/1 or n < 0.  Synchronous. */
int gbmc_check_division(gbmc_ctx *ctx, int32_t kind, int64_t n, uint64_t seed, int64_t *n_bad,
                        double *first_bad);

/* Track-length absorption-rate tally (reaction-rate tally; the next step
 * after the lookup and tally of Sec. 2 "Tallying", which says tallies are
 * scored in active batches): for every flight segment of length d,
 * w d Sigma_a(E) is added to the segment's (cell, energy bin), Sigma_a being
 * the macroscopic absorption cross section the lookup formed for the
 * segment's energy and material.  Laid out as the flux tally.  Off by
 * default; gbmc_set_reaction_tally(ctx, 1) turns it on for the following
 * runs, starting it at zero (gbmc_reset_tallies zeroes it with the others),
 * 0 turns it off and frees it.  Errors: INVALID_ARG for on not 0/1. */
int gbmc_set_reaction_tally(gbmc_ctx *ctx, int32_t on);

/* Copy problem slot `slot`'s absorption-rate tally [n_cells x n_bins]
 * (row = cell) to HOST absrate[n]; n must equal the slot's cells x bins.
 * Synchronizes with the last run.  Errors: NOT_INITIALIZED while the tally
 * is off or before a run, INVALID_ARG for a bad slot or size. */
int gbmc_read_reaction_tally(gbmc_ctx *ctx, int32_t slot, double *absrate, int64_t n);

/* Synchronize and copy per-particle outcomes of the last run for particles
 * first .. first+n-1 of problem slot `slot` (index within that problem's
 * batch).  Any output pointer may be NULL.  Final E and position are the
 * state at death. */
int gbmc_read_outcomes(gbmc_ctx *ctx, int32_t slot, int64_t first, int64_t n,
                       int32_t *n_coll, int8_t *status, int32_t *n_flights,
                       uint32_t *n_draws, double *E, double *x, double *y, double *z);

/* Synchronize and return the counters of the last run. */
int gbmc_read_stats(gbmc_ctx *ctx, gbmc_stats *out);

/* Macroscopic lookup only (the lookup event of Sec. 2 "Sorting", outside
 * the transport loop), on DEVICE pointers owned by the caller:
 *   d_E [n] binary64 energies within the tables' grids (outside them the
 *   first or last interval is extrapolated), d_mat [n] int32 material ids,
 *   outputs d_sigma_t and d_sigma_a [n] binary64.  A query whose material id
 *   is not in [0, n_mat) gets NaN in both outputs and reads no table.  The
 *   four arrays must each hold n elements of these types; the library cannot
 *   check device buffers, so shorter ones are read or written out of bounds.
 * precision selects the loaded table copy; binary32 lookups search the
 * window form the context's sparse_windows option selects (same results).
 * sort = 1 sorts the queries by (material, energy) into context-owned
 * scratch first (results are written back in query order).  Asynchronous
 * on `stream`. */
int gbmc_lookup_macro(gbmc_ctx *ctx, int32_t precision, const double *d_E,
                      const int32_t *d_mat, int64_t n, double *d_sigma_t,
                      double *d_sigma_a, int32_t sort, void *stream);

/* Run like gbmc_run_problems, but launch each iteration's kernels eagerly
 * (no graph) with a CUDA event around every kernel on `stream`, and add the
 * per-kernel device times to *out (zero it first).  Synchronizes once per
 * iteration, so the run is slower end to end; outcomes and tallies are the
 * same as gbmc_run_problems'.
 * Optional per-iteration trace (trace_cap = 0 or NULL pointers skip it):
 *   trace_ms     [trace_cap * GBMC_NKERNELS] device ms of each kernel,
 *   trace_queues [trace_cap * 4] lookups, ray-traced particles, and
 *                collision events of each iteration, and particles in flight,
 *   *trace_len   iterations recorded (at most trace_cap). */
int gbmc_profile_problems(gbmc_ctx *ctx, int32_t n_prob, const gbmc_problem *probs,
                          void *stream, gbmc_kernel_times *out, int32_t trace_cap,
                          double *trace_ms, int32_t *trace_queues, int32_t *trace_len);

/* Weight windows for problem slot 0 of the following runs (the variance
 * reduction the learned importance map drives; the paper has no counterpart
 * beyond its Monte Carlo method).  lower [n_cells * n_bins], cell-major like
 * the flux tally, gives the window's lower weight bound per (cell, energy
 * bin); 0 means no window there.  Upper bound = ratio * lower, survival
 * weight = survival * lower (need survival >= 1, ratio >= 2 * survival).
 * Checked after every scatter and, in a slab, after every layer crossing:
 * above the window a particle splits into min(floor(w / w_s), max_split)
 * copies of equal weight; below it, Russian roulette keeps it with weight
 * w_s with probability w / w_s (else status GBMC_STATUS_ROULETTE).  Copies
 * are new histories with their own streams (ids from the parent's stream
 * position); they are tallied but have no outcome record.  While windows
 * are set, half of the bank is kept free for copies and the tail kernel is
 * not used.  Host array copied. */
int gbmc_set_weight_windows(gbmc_ctx *ctx, int32_t n_cells, int32_t n_bins, const double *lower,
                            double ratio, double survival, int32_t max_split);

/* Copy the current window lower bounds (n = cells * bins) to the host. */
int gbmc_get_weight_windows(gbmc_ctx *ctx, double *lower, int64_t n);

/* Back to analog transport. */
int gbmc_clear_weight_windows(gbmc_ctx *ctx);

/* ---- learned importance map (weight windows) ---------------------------
 * A 4 -> 64 -> 64 -> 1 multilayer perceptron (ReLU after each hidden
 * layer) maps features of (x, y, z, ln E) to a log-importance; weight
 * windows are set inversely proportional to the importance.  Weights are
 * BF16; the 64 x 64 layer runs on the tensor cores (FP32 accumulation) in
 * inference and training.  The paper has no counterpart (it is the
 * variance-reduction extension the weight windows serve).
 * Parameter layout: W1[64][4], b1[64], W2[64][64] (row = output unit),
 * b2[64], W3[64], b3 -- GBMC_MLP_NPARAM BF16 values.
 * Features: f_i = (raw_i - offset_i) * scale_i, raw = (x, y, z, ln E). */
#define GBMC_MLP_HIDDEN 64
#define GBMC_MLP_NPARAM 4545

/* Set the network (BF16 bit patterns) and its feature map; resets the
 * optimizer.  Host arrays copied. */
int gbmc_set_importance_net(gbmc_ctx *ctx, const uint16_t *bf16_params, int32_t n_params,
                            const double *feat_offset, const double *feat_scale);

/* Copy the current (trained) BF16 parameters to the host; synchronizes. */
int gbmc_get_importance_net(gbmc_ctx *ctx, uint16_t *bf16_params, int32_t n_params);

/* Network outputs for n feature rows: DEVICE pointers d_feat [n][4]
 * (float), d_out [n] (float).  The 64 x 64 layer runs on the tensor cores
 * (tcgen05, TMEM accumulator).  Synchronizes with `stream`; TIMEOUT if a
 * bounded wait for the tensor cores gave up (d_out then incomplete). */
int gbmc_mlp_forward(gbmc_ctx *ctx, const float *d_feat, int64_t n, float *d_out, void *stream);

/* Loss L = sum_s w_s (out_s - y_s)^2 / sum_s w_s over n rows (DEVICE
 * pointers d_feat [n][4], d_target [n], d_weight [n]) and its gradient with
 * respect to the parameters (host grad [GBMC_MLP_NPARAM], fp32; host loss).
 * Synchronizes. */
int gbmc_mlp_gradient(gbmc_ctx *ctx, const float *d_feat, const float *d_target,
                      const float *d_weight, int64_t n, float *grad, float *loss, void *stream);

/* `steps` full-batch Adam steps (beta 0.9 / 0.999, learning rate lr) on the
 * same loss, entirely on the device (FP32 master weights, BF16 copies for
 * the tensor cores).  *loss receives the last step's loss.  Synchronizes. */
int gbmc_mlp_train(gbmc_ctx *ctx, const float *d_feat, const float *d_target,
                   const float *d_weight, int64_t n, int32_t steps, float lr, float *loss,
                   void *stream);

/* Features of the mesh (cells of geometry g x tally energy bins: cell
 * centre, logarithmic bin centre) into DEVICE d_feat [n][4] with the
 * network's feature map (the network must be set); *n_out = number of rows
 * (d_feat NULL: count only). */
int gbmc_mesh_features(gbmc_ctx *ctx, const gbmc_geometry *g, float *d_feat, int64_t n_cap,
                       int64_t *n_out, void *stream);

/* Weight windows of problem slot 0 from the network: on the mesh of g,
 * lower = C / exp(out) with C such that the source cell and energy bin has
 * survival weight 1.  Then as gbmc_set_weight_windows.  Synchronizes. */
int gbmc_weight_windows_from_net(gbmc_ctx *ctx, const gbmc_geometry *g, double ratio,
                                 double survival, int32_t max_split, void *stream);

/* Importance estimates from analog runs.  With g != NULL and capacity > 0,
 * following runs record, for every collision of a problem-slot-0 history,
 * its mesh cell (cell of g x energy bin before the collision) -- at most
 * `capacity` per run (NULL / 0: recording off).
 * gbmc_importance_accumulate, after each such run, scores those samples by
 * whether their history left through the slab's far face, into per-mesh
 * counts n and scores s (kept across runs).
 * gbmc_importance_training_set writes the mesh features (the network's
 * feature map: set the network first), targets and
 * weights to DEVICE arrays of n_cap rows: a cell's importance pools its
 * energy bins, I_c = (S_c + 5 p0) / (N_c + 5) with p0 the overall score
 * fraction; every bin of the cell gets target ln I_c and weight
 * N_c / (N_c + 5) (0 in cells no history reached). */
int gbmc_importance_record(gbmc_ctx *ctx, const gbmc_geometry *g, int64_t capacity);
int gbmc_importance_accumulate(gbmc_ctx *ctx, void *stream);
int gbmc_importance_training_set(gbmc_ctx *ctx, const gbmc_geometry *g, float *d_feat,
                                 float *d_target, float *d_weight, int64_t n_cap,
                                 int64_t *n_out, void *stream);

/* Result of gbmc_autotune. */
typedef struct {
    int32_t trials;            /* probe runs timed */
    int32_t reserved;
    double default_ms;         /* probe device time with the options on entry */
    double best_ms;            /* probe device time with the chosen options */
    double in_flight_fraction; /* chosen cap / particles of the run (1 = no refill) */
} gbmc_autotune_report;

/* Autotuner for the launch and queue settings of a run (the batched
 * multi-problem launch in particular): times probe runs of these problems,
 * with each particle count scaled by `fraction` (0 < fraction <= 1), over
 * candidate settings by coordinate descent -- event-kernel grid
 * (blocks_per_sm), in-flight cap (as a fraction of the run's particles,
 * Sec. 2 "In-Flight Particles"), the warp-per-particle lookup threshold and
 * the sort threshold -- and keeps the fastest.  Outcomes do not depend on
 * these settings, only speed does.  On return the context uses the chosen
 * options (also copied to *best_out if not NULL; its max_in_flight is the
 * chosen fraction of the full problems' particles), tallies are zeroed and
 * the last run's outcomes are the last probe's.  Synchronous. */
int gbmc_autotune(gbmc_ctx *ctx, int32_t n_prob, const gbmc_problem *probs, double fraction,
                  void *stream, gbmc_options *best_out, gbmc_autotune_report *report);

/* Sorted macroscopic lookup that allocates nothing (the paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory while they call the library -- code running while a stream
 * is being captured into a CUDA graph, where cudaMalloc is not allowed;
 * processes whose device memory is a fixed pool handed out elsewhere; loops
 * that must not take allocator locks or fail with out-of-memory midway).
 * Same arguments, results and order of results as gbmc_lookup_macro with
 * sort = 1, but its sort scratch is a fixed area compiled into the library:
 *   - at most 1048576 (2^20) queries per call; more returns
 *     GBMC_ERR_INVALID_ARG before anything is launched;
 *   - every GPU that loads the library holds that area (about 8.5 MB) until
 *     the process exits;
 *   - every call looks up the area's device address in the current context
 *     (cudaGetSymbolAddress; the first lookup in a context may load the
 *     library's device code), so it stays valid across cudaDeviceReset;
 *   - all calls share the one area: calls whose work overlaps on the GPU
 *     (other streams, other threads, other contexts on the same device)
 *     race and corrupt each other's results; order them on one stream;
 *   - it calls no cudaMalloc / cudaFree and no allocating library routine.
 * Inputs and outputs are DEVICE pointers owned by the caller, as in
 * gbmc_lookup_macro.  Asynchronous on `stream`. */
int gbmc_lookup_macro_noalloc(gbmc_ctx *ctx, int32_t precision, const double *d_E,
                              const int32_t *d_mat, int64_t n, double *d_sigma_t,
                              double *d_sigma_a, void *stream);

/* Measured binary64 throughput of this device (the denominator of the
 * binary64 kernels' rooflines; the paper names no such figure): independent
 * fused multiply-add chains, 8 per thread, 2^14 steps each, over SMs x 8
 * blocks of 256 threads, timed with CUDA events on the legacy default
 * stream (best of three after a warm-up).  *ops_per_s = binary64
 * instructions per second, counted per thread.  Synchronous; allocates
 * and frees a small device buffer. */
int gbmc_measure_fp64_rate(gbmc_ctx *ctx, double *ops_per_s);

/* Device timing of the last run's event loop (ms, CUDA events on the run's
 * stream around the graph launch); synchronizes. */
int gbmc_last_run_ms(gbmc_ctx *ctx, double *ms);

#ifdef __cplusplus
}
#endif
#endif /* GBMC_H */
