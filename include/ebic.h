/*
 * ebic.h -- C ABI of the GB300 (sm_103a) EBIC population-evaluation library.
 *
 * EBIC (evolutionary biclustering, as re-implemented by EBIC.jl, arXiv 2105.01196) searches for
 * biclusters whose rows follow a common order of columns.  An individual is an ordered series of
 * column indices (Sec. 2.3, "EBIC" paragraph); its fitness comes from the number of rows whose
 * values follow that order (Sec. 2.4, steps 2-3 and 7).  This library evaluates whole populations
 * on the GPU and runs the generation loop of Sec. 2.4 (steps 1-9) on the device.
 *
 * Conventions shared by every entry point
 *   - Status: 0 (EBIC_OK) on success, a negative EBIC_E* code otherwise.  No C++ exception and no
 *     abort crosses this boundary; the message of the last failure is ebic_last_error().
 *   - Pointers: every array argument may be host memory or device memory of the context's GPU; the
 *     library tells them apart with cudaPointerGetAttributes.  Host arrays are copied through
 *     library-owned device buffers.  The caller owns every pointer it passes; the library keeps
 *     no reference to one after the call returns.
 *   - Streams: all GPU work of a context runs on the stream given to ebic_create (or on a stream
 *     the context creates).  Every call returns only after that work has finished, so the caller
 *     may read outputs at once.  Contexts are independent: calls on different contexts may run
 *     concurrently from different host threads.  Calls on one context must not overlap.
 *   - Integers are little-endian two's complement; rows are int64, columns int32.
 *   - Comparisons: float32 values are compared strictly; ties (including -0 against +0) break both
 *     the increasing and the decreasing trend.  NaN and +-Inf are rejected when the matrix is
 *     loaded.
 */
#ifndef EBIC_GB300_H
#define EBIC_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define EBIC_API __attribute__((visibility("default")))
#else
#define EBIC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------------------- status codes */
#define EBIC_OK 0
#define EBIC_EINVAL (-1)   /* bad argument: shape, parameter, chromosome, pointer            */
#define EBIC_ENAN (-2)     /* the matrix holds NaN or +-Inf                                    */
#define EBIC_ENOMEM (-3)   /* a device or host allocation failed                               */
#define EBIC_ECUDA (-4)    /* a CUDA runtime call failed (the message names it)                */
#define EBIC_ETIMEOUT (-5) /* a bounded device-side wait gave up                               */
#define EBIC_ESTATE (-6)   /* call out of order (e.g. no matrix loaded, no run initialised)    */

/* ----------------------------------------------------------------------------- enumerations */
#define EBIC_MODE_AUTO 0   /* the autotuner chooses the evaluation kernel                      */
#define EBIC_MODE_DIRECT 1 /* direct comparison: per-row rank codes up to 1,024 columns, the
                              order keys above                                                 */
#define EBIC_MODE_BITMAP 2 /* column-pair comparison bitmap (built on first use); not with
                              last_kept (EBIC_EINVAL)                                          */
#define EBIC_MODE_PLAIN 3  /* one kernel launch per individual (reference GPU form)            */
#define EBIC_MODE_STAGED 4 /* direct comparison over TMA-staged row tiles in shared memory;
                              the direct form is used where the tile does not fit (> 1536 columns)
                              or a pair-test variant (non_strict, last_kept) is set            */

#define EBIC_LAYOUT_ROW_MAJOR 0 /* x[r * cols + c] */
#define EBIC_LAYOUT_COL_MAJOR 1 /* x[c * rows + r] */

#define EBIC_MAX_LEN 64          /* longest chromosome                                        */
#define EBIC_MAX_BICLUSTERS 256  /* largest top rank list                                     */

typedef struct ebic_ctx ebic_ctx;

/*
 * Parameters of the method (Sec. 2.4, last paragraph: negative trends on/off, approximate-trend
 * threshold, allowed overlap between trends, number of iterations and of biclusters; Table 1
 * gives the iteration cap -n 20000).  The paper fixes no other value; ebic_default_params fills
 * the defaults this library uses.
 *   neg_trends       1: a row also counts when it follows the reversed order (Sec. 2.4).
 *   ratio_num/den    approximate-trend ratio; a row passes when at least
 *                    t(L) = ceil(ratio * (L-1)) of its L-1 consecutive pairs follow the trend.
 *                    1/1 is the exact trend.  Requires 0 < ratio_num <= ratio_den.
 *   min_rows         fitness is 0 below this many accepted rows.
 *   col_cap          fitness = rows * 2^min(L, col_cap); 0 <= col_cap <= 16.
 *   overlap_num/den  a top-list entry may share at most this fraction of its columns with any
 *                    better entry (Sec. 2.4, "level of overlap allowed between the trends").
 *   n_biclusters     size K of the top rank list, 1..256 (Sec. 2.4, steps 3, 4, 9).
 *   init_min_len, init_max_len  initial chromosome lengths (Sec. 2.4, step 1).
 *   max_len          longest chromosome the operators build, <= min(64, cols).
 *   pop_size         population size P, 2..2^20.
 *   elite            top-list entries copied into each new population (step 4), <= K.
 *   tournament       tournament size (step 5), 1..16.
 *   max_attempts     children tried per slot before the slot is dead (tabu list), 1..16.
 *   tabu_hit_limit   tabu hits within one generation that stop the run (step 6); <= 0: never.
 *   seed             key of the Philox4x32-10 stream all random draws come from.
 *   mode             EBIC_MODE_*: evaluation kernel.
 *   use_graph        ebic_run_generations: 1 replays one captured CUDA graph per generation,
 *                    0 launches every kernel eagerly and synchronises after each generation.
 */
typedef struct ebic_params {
  int32_t neg_trends;
  int32_t ratio_num, ratio_den;
  int32_t min_rows;
  int32_t col_cap;
  int32_t overlap_num, overlap_den;
  int32_t n_biclusters;
  int32_t init_min_len, init_max_len;
  int32_t max_len;
  int32_t pop_size;
  int32_t elite;
  int32_t tournament;
  int32_t max_attempts;
  int32_t tabu_hit_limit;
  uint64_t seed;
  int32_t mode;
  int32_t use_graph;
  int32_t non_strict;  /* 1: ties hold for both directions (pair test >= / <=); default 0      */
  int32_t last_kept;   /* 1: each value is compared with the last value that kept the
                          direction instead of with its predecessor; no bitmap form (mode
                          EBIC_MODE_BITMAP is rejected, AUTO takes the direct form); default 0 */
  int32_t ipw;         /* individuals per work item of the staged bitmap form (bitmaps larger
                          than L2, ratio below 1): 0 (default) = the autotuner's choice, 1 when
                          untuned; 1-4 forces it.  Results never depend on it               */
  int32_t fuse_pairs;  /* generation loop with the bitmap form: a child of at most this many
                          column pairs whose pair test is exact (the ratio lets no pair fail,
                          ceil(ratio * pairs) = pairs) is evaluated by the warp that built it,
                          inside the evolve kernel; the other slots go to the evaluation
                          launch.  0 (default) = the library's choice, -1 = never, 1-63 = this
                          limit.  Results never depend on it                                */
} ebic_params;

/* Progress of a run (Sec. 2.4, steps 6 and 8). */
typedef struct ebic_run_report {
  int32_t gens_done;   /* last scored generation; 0 = only the initial population            */
  int32_t stopped;     /* 1 when step 6 (tabu-hit limit) ended the run                       */
  int32_t last_hits;   /* tabu hits of the last generation built                             */
  int32_t n_top;       /* entries in the top rank list                                       */
  int64_t n_evaluated; /* individuals scored since the run was initialised                   */
  int32_t eval_mode;   /* evaluation form used: EBIC_MODE_DIRECT, _STAGED or _BITMAP         */
  int32_t fuse_pairs;  /* pair limit of the evaluation inside the evolve kernel in this call
                          (0: none; see ebic_params.fuse_pairs)                              */
  int64_t n_fused;     /* of n_evaluated, the individuals evaluated inside the evolve kernel */
  int64_t n_table;     /* of n_fused, the one-pair individuals scored from the pair counts the
                          bitmap build records (popcounts of the pair rows; C <= 1,024)     */
} ebic_run_report;

/* Fills *p with the library defaults.  Never fails. */
EBIC_API void ebic_default_params(ebic_params *p);

/* Library version string (static storage). */
EBIC_API const char *ebic_version(void);

/*
 * Creates a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t of that device the
 * context will use (borrowed, not destroyed by the context), or NULL to make the context create
 * and own a non-blocking stream.  *out receives the context.
 * Errors: EBIC_EINVAL (out NULL, bad device), EBIC_ECUDA, EBIC_ENOMEM.
 */
EBIC_API int ebic_create(ebic_ctx **out, int32_t device, void *cuda_stream);

/* Frees every device and host resource of the context.  NULL is accepted. */
EBIC_API int ebic_destroy(ebic_ctx *ctx);

/* Message of the last failed call on this context ("" when none); static per context. */
EBIC_API const char *ebic_last_error(const ebic_ctx *ctx);

/*
 * Loads the expression matrix (Sec. 2.1: rows x columns of numeric values; Sec. 2.4 step 2
 * sends the data to the GPU).  x holds rows*cols float32 in `layout` (EBIC_LAYOUT_*), host or
 * device memory.  The library converts it into its own device copy: column-major uint32 order
 * keys with rows padded to a multiple of 128.  Loading a new matrix drops the bitmap cache and
 * any run state.
 * Errors: EBIC_EINVAL (rows < 1, cols < 2, cols > 65535, bad layout, NULL x), EBIC_ENAN (NaN or
 * Inf anywhere in x; the previous matrix is gone), EBIC_ENOMEM, EBIC_ECUDA.
 */
EBIC_API int ebic_load_matrix(ebic_ctx *ctx, const float *x, int64_t rows, int32_t cols, int32_t layout);

/*
 * Builds the column-pair comparison bitmap of the loaded matrix: for every ordered pair of
 * columns (a, b), word w bit j is [x(32w+j, b) > x(32w+j, a)].  Its size is
 * ebic_bitmap_bytes(rows, cols).  EBIC_MODE_BITMAP builds it on first use; this call builds it
 * ahead of time, queued on the context's stream (every later call of the context is ordered
 * after it).  Errors: EBIC_ESTATE (no matrix), EBIC_ENOMEM, EBIC_ECUDA.
 */
EBIC_API int ebic_build_bitmap(ebic_ctx *ctx);

/* Bytes of the pair bitmap for a rows x cols matrix (cols^2 * ceil128(rows) / 8). */
EBIC_API int64_t ebic_bitmap_bytes(int64_t rows, int32_t cols);

/*
 * Copies the pair bitmap into `out` (host or device, n_words uint32).  Layout: word
 * ((a * cols + b) * w_stride + w), w_stride = ceil128(rows) / 32; bit j of word w is row 32w+j.
 * Errors: EBIC_ESTATE (no bitmap built), EBIC_EINVAL (n_words too small), EBIC_ECUDA.
 */
EBIC_API int ebic_copy_bitmap(ebic_ctx *ctx, uint32_t *out, int64_t n_words);

/*
 * Copies the pair counts the bitmap build records (cols <= 1,024: the build from the rank codes'
 * bit planes) into `out` (host or device, n >= cols * cols uint64): for a < b, out[a * cols + b]
 * = rows of G[a][b] (key(b) > key(a), the popcount of that pair row) in the low 32 bits and
 * rows of G[b][a] in the high 32 bits; the other entries are 0.  A one-pair chromosome's trend
 * counts follow from them (the generation loop scores one-pair children this way).
 * Errors: EBIC_ESTATE (no bitmap built, or built without counts: cols > 1,024), EBIC_EINVAL (n
 * too small), EBIC_ECUDA.
 */
EBIC_API int ebic_copy_pair_counts(ebic_ctx *ctx, uint64_t *out, int64_t n);

/*
 * Evaluates a population (Sec. 2.4, steps 2-3: score every individual by the number of its
 * trend-preserving rows).  The population is CSR: individual i is
 * col_idx[offsets[i] .. offsets[i+1]-1], 2 <= length <= 64, distinct columns in [0, cols).
 * For each individual i:
 *   rows_pos[i]  rows with at least t(L) increasing consecutive pairs,
 *   rows_neg[i]  rows with at least t(L) decreasing pairs (0 unless p->neg_trends),
 *   rows_any[i]  rows passing either direction (counted once),
 *   fitness[i]   0 if rows_any < p->min_rows, else rows_any * 2^min(L, p->col_cap).
 * Any of the four outputs may be NULL.  Only neg_trends, ratio_*, non_strict, last_kept,
 * min_rows, col_cap and mode of *p are read.  n_ind = 0 is valid and does nothing.
 * Errors: EBIC_ESTATE (no matrix), EBIC_EINVAL (bad parameter or chromosome; nothing written),
 * EBIC_ENOMEM, EBIC_ECUDA.
 */
EBIC_API int ebic_eval_population(ebic_ctx *ctx, const int32_t *col_idx, const int32_t *offsets,
                         int32_t n_ind, const ebic_params *p, int32_t *rows_pos,
                         int32_t *rows_neg, int32_t *rows_any, uint64_t *fitness);

/*
 * Runs the EBIC generation loop on the device (Sec. 2.4 steps 1-8; strategies of Sec. 2.3):
 * the first call on a loaded matrix initialises and scores a random population (steps 1-3),
 * then up to n_gen generations follow: elitism (step 4), penalised tournament, crossover and one
 * of insertion/deletion/substitution/swap with tabu-list rejection (step 5), the tabu-hit stop
 * test (step 6), scoring and top-list update (step 7).  Later calls continue the same run
 * (resuming is exact: all randomness is counter-based).  Changing any parameter but mode,
 * use_graph, ipw or fuse_pairs, or loading a matrix, starts a new run.  With the bitmap form,
 * short children whose pair test is exact are evaluated inside the evolve kernel (fuse_pairs);
 * the results are the same either way.  *rep (may be NULL) receives the progress.
 * Errors: EBIC_ESTATE (no matrix), EBIC_EINVAL (bad parameter), EBIC_ENOMEM, EBIC_ECUDA,
 * EBIC_ETIMEOUT.
 */
EBIC_API int ebic_run_generations(ebic_ctx *ctx, const ebic_params *p, int32_t n_gen,
                         ebic_run_report *rep);

/*
 * Copies the top rank list (Sec. 2.4, steps 3, 7 and 9), best first, sorted by fitness then by
 * tabu key.  cols: n_top * 64 int32 (entry e's columns at cols[e*64 .. e*64+len-1]); lens,
 * fitness, keys (the tabu key: FNV-1a 64 of the column sequence), rows (3 int32 per entry:
 * pos, neg, any).  Arrays hold at least `capacity` entries; any may be NULL.  *n_top receives the
 * number of entries.  Errors: EBIC_ESTATE (no run), EBIC_EINVAL, EBIC_ECUDA.
 */
EBIC_API int ebic_get_toplist(ebic_ctx *ctx, int32_t capacity, int32_t *n_top, int32_t *cols,
                     int32_t *lens, uint64_t *fitness, uint64_t *keys, int32_t *rows);

/*
 * Copies the current population: cols (P * 64 int32, slot s at cols[s*64..]), lens, dead (1 =
 * the slot was rejected by the tabu list and not scored), fitness.  Any may be NULL.
 * Errors: EBIC_ESTATE, EBIC_EINVAL (capacity < P), EBIC_ECUDA.
 */
EBIC_API int ebic_get_population(ebic_ctx *ctx, int32_t capacity, int32_t *cols, int32_t *lens,
                        uint8_t *dead, uint64_t *fitness);

/*
 * Bicluster extraction (Sec. 2.4, step 9): for each top-list entry e, the rows it accepts as a
 * bitmask, rowmask[e * w_stride + w] bit j = row 32w + j, w_stride = ceil128(rows) / 32.
 * rowmask holds capacity * w_stride words.  *n_out receives the number of entries written.
 * Errors: EBIC_ESTATE (no run), EBIC_EINVAL (capacity too small), EBIC_ENOMEM, EBIC_ECUDA.
 */
EBIC_API int ebic_extract_biclusters(ebic_ctx *ctx, int32_t capacity, uint32_t *rowmask, int32_t *n_out);

/*
 * Checkpoint of the run state (generation index, population, fitness, penalties, top list and
 * tabu list).  ebic_state_bytes returns the size of the blob; ebic_save_state writes it into the
 * host buffer `blob` of `size` bytes; ebic_load_state restores it (same matrix, same parameters)
 * so that later generations equal those of an uninterrupted run.
 * Errors: EBIC_ESTATE (no run / no matrix), EBIC_EINVAL (size, corrupt blob), EBIC_ENOMEM,
 * EBIC_ECUDA.
 */
EBIC_API int64_t ebic_state_bytes(ebic_ctx *ctx);
EBIC_API int ebic_save_state(ebic_ctx *ctx, void *blob, int64_t size);
EBIC_API int ebic_load_state(ebic_ctx *ctx, const ebic_params *p, const void *blob, int64_t size);

/*
 * Kernel statistics for roofline accounting (no counterpart in the paper).  While enabled, the
 * context records CUDA events on its stream around every launch of the evaluation kernel, the
 * bitmap build and the generation-loop kernels (inside replayed CUDA graphs too, through event
 * nodes re-pointed at fresh events before each replay), and it counts every kernel it launches.
 *   kernel  EBIC_KERNEL_EVAL (direct or bitmap evaluation, single sweeps and generations),
 *           EBIC_KERNEL_BITMAP_BUILD, EBIC_KERNEL_EVOLVE (children of one generation),
 *           EBIC_KERNEL_FINISH (scoring, tabu list and top-list update of one generation),
 *           EBIC_KERNEL_RANK_CODES (per-row rank codes, built by ebic_load_matrix when cols
 *           <= 1,024), or EBIC_KERNEL_ALL (launch count only).
 *   ms         summed event time of the timed launches;
 *   alg_bytes  algorithmic bytes of those launches: the bitmap form reads sum_i (L_i - 1) pair
 *              words per 32 rows and direction, the direct form gathers sum_i L_i codes (1 or 2
 *              bytes; keys, 4 bytes, when cols > 1,024 and in the staged form) per row, the
 *              build writes cols^2 words per 32 rows, the rank-code kernel reads the keys and
 *              writes the codes;
 *   alg_ops    algorithmic comparisons: sum_i (L_i - 1) * rows per direction;
 *   units      (individual, row) evaluations.
 * ebic_profile_enable(ctx, 1) resets the counters; 0 stops recording.
 */
#define EBIC_KERNEL_EVAL 0
#define EBIC_KERNEL_BITMAP_BUILD 1
#define EBIC_KERNEL_ALL 2
#define EBIC_KERNEL_EVOLVE 3
#define EBIC_KERNEL_FINISH 4
#define EBIC_KERNEL_RANK_CODES 5
#define EBIC_KERNEL_COUNT 6

typedef struct ebic_kernel_stats {
  int64_t launches;
  int64_t timed_launches;
  double ms;
  double alg_bytes;
  double alg_ops;
  double units;
} ebic_kernel_stats;

EBIC_API int ebic_profile_enable(ebic_ctx *ctx, int32_t on);
EBIC_API int ebic_profile_read(ebic_ctx *ctx, int32_t kernel, ebic_kernel_stats *out);

/*
 * Autotuner (no counterpart in the paper; the paper's kernel has a single form).  Measures, with
 * CUDA events, one evaluation sweep of the population (CSR as in ebic_eval_population, host or
 * device) in the direct form (several work-item sizes), the staged direct form (when its tiles
 * fit) and, when the pair bitmap fits in half of the free device memory, the bitmap form
 * (building it; several work-item sizes, and 1, 2 or 4 individuals per work item when the
 * bitmap is larger than L2 and the ratio below 1).  It then records for the loaded matrix the
 * form and sizes minimising build + expected_sweeps * sweep time.  With expected_sweeps > 2 and
 * p valid for ebic_run_generations (the staged direct form excepted), it also times 16
 * generations of a scratch run per work-item size (and group size) of the chosen form
 * (graph-replayed, after a warm-up run) and records the fastest for the generation loop; the
 * run state is reset afterwards, so the caller's next run starts from its initial population.
 * EBIC_MODE_AUTO follows the decisions in ebic_eval_population and ebic_run_generations until
 * a matrix of another shape is loaded (the measured times depend on the shape, not on the
 * values, so a reload of the same shape keeps them); p->ipw > 0 overrides the group size and
 * p->fuse_pairs != 0 the loop's fusion limit (with the bitmap form, the loop measurement first
 * picks that limit, then the work-item and group sizes).
 * Results never depend on the choice.  *rep (may be NULL) receives the measurements.
 * Errors: EBIC_ESTATE (no matrix), EBIC_EINVAL (bad population or parameter, n_ind < 1,
 * expected_sweeps < 1), EBIC_ENOMEM, EBIC_ECUDA.
 */
typedef struct ebic_tune_report {
  int32_t mode;       /* chosen form: EBIC_MODE_DIRECT, EBIC_MODE_STAGED or EBIC_MODE_BITMAP */
  int32_t seg_direct; /* chosen work-item size of the direct form, passes of 128 rows (0 = default split) */
  int32_t seg_bitmap; /* the same for the bitmap form, passes of 128 words                  */
  int32_t seg_loop;   /* the same for the generation loop's evaluations in the chosen form   */
  double direct_ms;   /* best measured sweep of the direct form                               */
  double bitmap_ms;   /* best measured sweep of the bitmap form (-1 when not measured)        */
  double build_ms;    /* measured bitmap build (0 when the bitmap already existed)            */
  double staged_ms;   /* best measured sweep of the staged direct form (-1 when not measured) */
  int32_t ipw_bitmap; /* chosen individuals per work item of the staged bitmap form (1-4)     */
  int32_t ipw_loop;   /* the same for the generation loop                                     */
  int32_t fuse_loop;  /* chosen pair limit of the evaluation inside the evolve kernel (bitmap
                         form; -1: none, 0: not measured); see ebic_params.fuse_pairs          */
  int32_t reserved;
} ebic_tune_report;

EBIC_API int ebic_autotune(ebic_ctx *ctx, const int32_t *col_idx, const int32_t *offsets,
                           int32_t n_ind, const ebic_params *p, int32_t expected_sweeps,
                           ebic_tune_report *rep);

/*
 * Job server: continuous batching of independent EBIC runs on one GPU (no counterpart in the
 * paper, which runs one job at a time).  Jobs are admitted in arrival order, a later job that
 * fits going ahead of a head job that does not, while the admitted jobs' device-memory
 * footprints (ebic_job_footprint) stay within hbm_budget_bytes and at most max_running (1..64)
 * jobs run.  Every admitted job runs on its own worker thread, context and stream; kernels of
 * different jobs overlap on the device, and each job's results are the same as when it runs alone.
 *   ebic_server_submit copies the matrix (host or device memory; layout EBIC_LAYOUT_*) and queues
 *     the job (initialisation + n_gen generations, as ebic_run_generations); *job_id receives its
 *     id.  EBIC_ENOMEM: its footprint exceeds the whole budget.  EBIC_ESTATE: server stopping.
 *   ebic_server_wait waits up to timeout_ms (< 0: no limit; EBIC_ETIMEOUT when it expires) for the
 *     job, fills *res and, when capacity >= n_top, the top list (layout of ebic_get_toplist), and
 *     forgets the job.  res->status is the job's own status code.
 *   ebic_server_destroy lets running and admitted jobs finish and drops the queued ones.
 * ebic_job_footprint: device bytes one job holds at most (matrix keys, staging, rank codes and
 * their bit planes up to 1,024 columns, the pair bitmap when the cost model picks it, population,
 * tabu list, tables), or -1 for bad arguments.
 */
typedef struct ebic_server ebic_server;

typedef struct ebic_job_result {
  int64_t job_id;
  int32_t status;      /* EBIC_OK or the job's error code                                    */
  int32_t gens_done;   /* as ebic_run_report                                                 */
  int32_t stopped;
  int32_t n_top;
  int64_t n_evaluated;
  int32_t eval_mode;   /* the evaluation form the job used                                   */
  int32_t reserved;
  int64_t footprint_bytes;
  double queued_ms;    /* submission to admission                                            */
  double run_ms;       /* admission to completion                                            */
} ebic_job_result;

EBIC_API int64_t ebic_job_footprint(int64_t rows, int32_t cols, const ebic_params *p,
                                    int32_t n_gen);
EBIC_API int ebic_server_create(ebic_server **out, int32_t device, int64_t hbm_budget_bytes,
                                int32_t max_running);
EBIC_API int ebic_server_destroy(ebic_server *srv);
EBIC_API int ebic_server_submit(ebic_server *srv, const float *x, int64_t rows, int32_t cols,
                                int32_t layout, const ebic_params *p, int32_t n_gen,
                                int64_t *job_id);
EBIC_API int ebic_server_wait(ebic_server *srv, int64_t job_id, int32_t timeout_ms,
                              ebic_job_result *res, int32_t capacity, int32_t *top_cols,
                              int32_t *top_lens, uint64_t *top_fit, uint64_t *top_keys,
                              int32_t *top_rows);
/* Queue length, running jobs and reserved device bytes at this moment. */
EBIC_API int ebic_server_stats(ebic_server *srv, int32_t *queued, int32_t *running,
                               int64_t *reserved);

/*
 * Population evaluation that allocates no memory.  The paper has no counterpart: this entry
 * point exists for callers that cannot let a library allocate GPU memory.  One case is a
 * serving process whose framework has already reserved the device memory in its own pool, so
 * that a cudaMalloc fails or fragments the pool.  Another is a latency-critical caller that
 * cannot afford cudaMalloc's unbounded latency or cudaFree's device-wide synchronisation.  It
 * calls no cudaMalloc, cudaFree or other allocating routine and needs no context.
 *
 * Computes the same rows_pos / rows_neg / rows_any / fitness as ebic_eval_population (strict
 * float32 comparisons, ties break both trends, t(L) = ceil(ratio * (L-1))), with the direct
 * comparison form, from caller memory only:
 *   x         rows * cols float32, COLUMN-major (x[c * rows + r]), device memory of `device`;
 *   col_idx, offsets  CSR population as in ebic_eval_population, device memory;
 *   outputs   device memory of `device`; any may be NULL;
 *   p         neg_trends, ratio_num/den, min_rows, col_cap, non_strict and last_kept are read
 *             (mode, ipw and the generation-loop fields are ignored);
 *   cuda_stream  a cudaStream_t of `device` (NULL = the legacy default stream);
 *   msg       optional buffer of msg_len bytes for the message of a failure.
 * Scratch: the per-individual accumulators, a work counter and an error word live in one
 * file-scope static device array of 3 * EBIC_NOALLOC_MAX_IND + 2 int32 (768 KB), which every
 * GPU that loads the library holds until the process exits.  CUDA loads modules lazily, so the
 * first call on each device does a one-time set-up with that device current: it looks up the
 * array's device address and loads this entry point's kernels, which places the array and their
 * code in device memory.  Make that first call before any stream capture, and before a framework
 * reserves the device's memory for its own pool (the set-up needs about 1 MB); later calls on
 * that device load nothing.  Every call shares the array and clears the part it uses; calls
 * whose work overlaps on the GPU (on different streams or from different threads) race on it
 * and must be serialised by the caller.  The call reads the validation result back and
 * synchronises `cuda_stream` before it launches the evaluation, and returns after the work has
 * finished on `cuda_stream`.
 * Errors: EBIC_EINVAL (n_ind > EBIC_NOALLOC_MAX_IND, a host pointer, bad shape, parameter or
 * chromosome), EBIC_ENAN (NaN or Inf in x), EBIC_ECUDA.
 */
#define EBIC_NOALLOC_MAX_IND 65536
EBIC_API int ebic_eval_population_noalloc(const float *x, int64_t rows, int32_t cols,
                                          const int32_t *col_idx, const int32_t *offsets,
                                          int32_t n_ind, const ebic_params *p,
                                          int32_t *rows_pos, int32_t *rows_neg,
                                          int32_t *rows_any, uint64_t *fitness, int32_t device,
                                          void *cuda_stream, char *msg, int32_t msg_len);

#ifdef __cplusplus
}
#endif

#endif /* EBIC_GB300_H */
