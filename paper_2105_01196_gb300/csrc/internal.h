// Internal declarations of the EBIC GB300 library: the context, device buffers, the population
// view shared by the evaluation kernels, and the host launchers each .cu file provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/ebic.h"

#define EBIC_CHECK_CUDA(ctx, call)                                                    \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) return ebic_fail_cuda((ctx), e_, #call, __FILE__, __LINE__); \
  } while (0)

#define EBIC_TRY(call)          \
  do {                          \
    int s_ = (call);            \
    if (s_ != EBIC_OK) return s_; \
  } while (0)

// The library's device-memory pool of the current device (created on first use; freed memory
// stays cached in it up to a threshold, for the next allocation of any context), or null when
// the device has no memory-pool support.
cudaMemPool_t library_pool();

// Growable device allocation owned by a context.  Memory comes from the library pool in stream
// order on the owning context's stream: freeing waits only for that stream's earlier work (no
// device-wide synchronisation, so one context ending does not stall the others), and a new
// allocation is followed by one synchronisation of that stream so that host-side copies may use
// it at once.  Without pool support, plain cudaMalloc / cudaFree.
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;  // the stream the memory was allocated on (pool memory)
  bool pooled = false;
  cudaError_t ensure(size_t n, cudaStream_t stream) {
    if (n <= bytes && p) return cudaSuccess;
    release();
    if (n == 0) n = 16;
    cudaMemPool_t pool = library_pool();
    cudaError_t e;
    if (pool) {
      e = cudaMallocFromPoolAsync(&p, n, pool, stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
      pooled = true;
      s = stream;
    } else {
      e = cudaMalloc(&p, n);
      pooled = false;
    }
    if (e != cudaSuccess) {
      if (p && pooled) cudaFreeAsync(p, stream);
      p = nullptr;
      cudaGetLastError();
      return e;
    }
    bytes = n;
    return cudaSuccess;
  }
  void release() {
    if (p) {
      if (pooled)
        cudaFreeAsync(p, s);
      else
        cudaFree(p);
    }
    p = nullptr;
    bytes = 0;
  }
  template <class T>
  T *as() const { return reinterpret_cast<T *>(p); }
};

// Population as the kernels see it: CSR (off != nullptr, len derived) or fixed-stride storage
// with explicit lengths (off == nullptr).  dead (optional) marks slots that are not scored.  In
// the generation loop, a slot whose key a lower slot also produced is not scored either (dkeys,
// the duplicate table), and a set *stop flag turns the whole launch into a no-op.  With a list
// (bitmap kernels only) the launch evaluates the slots list[0 .. *list_n - 1] of the n slots
// instead of all of them; the count is read on the device when the launch starts.
struct PopView {
  const int32_t *cols;
  const int32_t *off;
  const int32_t *len;
  const uint8_t *dead;
  int32_t stride;
  int32_t n;
  const int32_t *stop;
  const uint64_t *hash;
  uint64_t *dkeys;
  uint32_t *dslot;
  uint32_t dmask;
  const int32_t *list;
  const int32_t *list_n;
};

// Matrix geometry and the outputs of one evaluation sweep.
struct EvalArgs {
  const uint32_t *keys;    // [C][R_pad] order keys
  const uint32_t *bitmap;  // [C][C][Wst] pair words (bitmap path)
  int64_t R, R_pad, Wst;   // rows, padded rows, words per column pair (R_pad / 32)
  int32_t C;
  int32_t neg, rnum, rden, min_rows, col_cap;
  int32_t non_strict, last_kept;  // pair-test variants (trend.cuh)
  int32_t *rows_pos, *rows_neg, *rows_any;  // accumulated with atomics (zeroed first)
  uint64_t *fitness;
  int32_t *work;            // dynamic work counter (zeroed first)
  int32_t seg_passes;       // passes (of 128 words or 128 rows) per work item
  int32_t n_seg;            // segments per individual
  int32_t ipw;              // individuals per work item (the staged bitmap form; else 1)
  // Optional side task of the generation loop, done by the launch's warps beside the evaluation
  // items (the staged kernel: before them): the previous generation's live keys (mv_hash[s] of
  // its slots s < mv_n with !mv_dead[s] and mv_len[s] >= 2) join the hashed tabu list
  // mv_table, new keys counted in *mv_count; and that generation's duplicate table (clr_n
  // slots of clr_keys / clr_slots) is cleared for the next generation.  mv_n = 0: none.
  const uint64_t *mv_hash;
  const uint8_t *mv_dead;
  const int32_t *mv_len;
  uint32_t mv_n;
  uint64_t *mv_table;
  uint32_t mv_tmask;
  unsigned long long *mv_count;
  uint64_t *clr_keys;
  uint32_t *clr_slots;
  uint32_t clr_n;
  int32_t *err;                   // kernels OR error bits in (4: a bounded wait expired)
  const struct DirectTma *dtma;   // host-side: staged direct form, when prepared
  const uint8_t *codes;           // [C][S] per-row rank codes (codes.cu), or nullptr
  int32_t code_bytes;             // bytes per code: 1 or 2 (0: the direct form reads keys)
  int64_t S;                      // rows per code column (a multiple of one pass)
  int32_t stage_bitmap;           // the bitmap kernel stages pair words in shared memory (set
                                  // when the bitmap exceeds L2: its words stream from HBM)
};

// Per-row rank codes (codes.cu): code width for C columns (1 for C <= 128, 2 for C <= 1024,
// else 0 = none), rows per pass of the code kernel, padded rows per code column, the number of
// bit planes of the codes (bits of C - 1) and their stride (planes stored per column and word: nb
// rounded up to a multiple of 4), the rank kernel (zero-fills the padding; writes the bit planes
// [C][Wst][stride] too when `planes` is not null) and the direct evaluation over codes.
int code_bytes_for(int32_t C);
int64_t code_rows_per_pass(int code_bytes);
int64_t code_stride_for(int64_t R, int code_bytes);
int code_plane_bits(int32_t C);
int code_plane_stride(int nb);
cudaError_t launch_rank_codes(const uint32_t *keys, int64_t R_pad, int32_t C, void *codes,
                              int code_bytes, int64_t S, uint32_t *planes, int64_t Wst,
                              int num_sms, cudaStream_t s);
// The rows [r_begin, r_end) only (multiples of 16), codes not cleared beforehand.
cudaError_t launch_rank_codes_rows(const uint32_t *keys, int64_t R_pad, int32_t C, void *codes,
                                   int code_bytes, int64_t S, uint32_t *planes, int64_t Wst,
                                   int num_sms, int64_t r_begin, int64_t r_end, cudaStream_t s);
cudaError_t launch_eval_codes(const EvalArgs &a, const PopView &pv, int num_sms, cudaStream_t s,
                              bool pdl);

// Tensor map and tile geometry of the TMA-staged direct form (direct_tma.cu).
struct DirectTma {
  alignas(64) unsigned char map[128];  // CUtensorMap of the keys [C][R_pad]
  int TR = 0, CB = 0, nbox = 0, stages = 0;
  int64_t stage_words = 0;
  bool ok = false;
};
void direct_tma_prepare(DirectTma *d, const uint32_t *keys, int64_t R_pad, int32_t C);
cudaError_t launch_eval_direct_tma(const DirectTma &d, const EvalArgs &a, const PopView &pv,
                                   int num_sms, cudaStream_t s, bool pdl);

// Kernel statistics (ebic_profile_*): launches counted always, event pairs while enabled.
struct KStats {
  int64_t launches = 0, timed = 0;
  double ms = 0, bytes = 0, ops = 0, units = 0;
};

struct PendingTiming {
  cudaEvent_t a, b;
  int kernel;
  double bytes, ops, units;
  bool own_a, own_b;  // the pair returns these events to the pool (shared ends are owned once)
};

struct ebic_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // a host matrix's segments are copied on copy_stream, each followed by an event that the
  // context stream waits for before it processes that segment (created on first use)
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> seg_ev;
  int num_sms = 0;
  int64_t l2_bytes = 0;  // the device's L2 size
  std::string err;

  // matrix
  int64_t R = 0, R_pad = 0, Wst = 0;
  int32_t C = 0;
  bool have_matrix = false;
  DevBuf keys, bitmap, stage_x;
  bool bitmap_ok = false;
  // rows of the pair rows of the bitmap, [C][C] 64-bit words: for a < b, popcount(G[a][b]) in
  // the low and popcount(G[b][a]) in the high 32 bits; built with the bitmap from the rank
  // codes' bit planes (C <= 1,024), else absent
  DevBuf pair_cnt;
  bool pair_cnt_ok = false;

  // scratch for single evaluations
  DevBuf d_err, d_work, ev_cols, ev_off, ev_out, ev_fit;

  // staged direct form of the loaded matrix, and the kernels' error word
  DirectTma dtma;
  DevBuf d_kerr;

  // per-row rank codes of the loaded matrix (code_bytes 0: none) and their bit planes
  // [C][Wst][code_plane_stride(plane_bits)] (the pair-bitmap build's operand), built together
  // on first use
  DevBuf codes, planes;
  int code_bytes = 0;
  int64_t code_stride = 0;
  int plane_bits = 0;
  bool codes_ready = false;

  // autotuner decisions for the loaded matrix (tune.cu)
  bool tuned = false;
  int tuned_mode = EBIC_MODE_DIRECT;
  int seg_direct = 0, seg_bitmap = 0;  // work-item sizes in passes; 0 = the built-in split
  int seg_loop = 0;                    // the same for the generation loop's evaluations
  int ipw_bitmap = 1, ipw_loop = 1;    // individuals per work item (staged bitmap form)
  int fuse_loop = 0;  // pair limit of the evaluation inside the evolve kernel (-1: none, 0: untuned)

  // generation loop state (evolve.cu)
  struct GenState *gen = nullptr;

  // profiling
  bool prof = false;
  KStats kst[EBIC_KERNEL_COUNT];
  std::vector<PendingTiming> pending;
  std::vector<cudaEvent_t> ev_pool;
};

// An event from the context's pool (nullptr when not profiling), and queuing a recorded pair.
cudaEvent_t prof_event(ebic_ctx *ctx);
void prof_push(ebic_ctx *ctx, cudaEvent_t a, cudaEvent_t b, int kernel, double bytes, double ops,
               double units, bool own_a = true, bool own_b = true);
// Records an event on the context stream before a timed launch (nullptr when not profiling).
cudaEvent_t prof_begin(ebic_ctx *ctx);
// Records the closing event and queues the pair with its algorithmic work.
void prof_end(ebic_ctx *ctx, cudaEvent_t a, int kernel, double bytes, double ops, double units);
// Counts launches of `kernel` (and of EBIC_KERNEL_ALL).
void prof_count(ebic_ctx *ctx, int kernel, int64_t n);
// After a stream synchronisation: turns queued event pairs into times.
void prof_collect(ebic_ctx *ctx);

int ebic_fail(ebic_ctx *ctx, int code, const std::string &msg);

// Builds the rank codes of the loaded matrix if it has some and they are not built yet.
int ensure_codes(ebic_ctx *ctx);
// Whether evaluation form `mode` runs the direct kernel (the staged form falls back to it).
int direct_form_used(const ebic_ctx *ctx, int mode, const ebic_params *p);
// Evaluation arguments with the loaded matrix's fields set (keys, bitmap, codes, sizes, error
// word, staged form); the caller sets the trend parameters, outputs and work counter.
EvalArgs eval_args_for(const ebic_ctx *ctx);
// Passes of 128 rows (keys), of one code load (codes) or of 128 bitmap words per individual.
int64_t eval_passes(const ebic_ctx *ctx, int mode);
// Algorithmic bytes of one evaluation sweep in `mode` (sum of lengths total_len).
double eval_bytes(const ebic_ctx *ctx, int mode, int64_t total_len, int64_t n_ind, int neg);
int ebic_fail_cuda(ebic_ctx *ctx, cudaError_t e, const char *what, const char *file, int line);

bool ebic_is_device_ptr(const void *p);

// A validated population on the device (abi.cu).
struct StagedPop {
  const int32_t *d_cols = nullptr, *d_off = nullptr;
  std::vector<int32_t> h_off;  // host copy of the offsets when requested
  int64_t total = 0;           // sum of lengths
  double mean_len = 0.0;
};
int stage_population(ebic_ctx *ctx, const int32_t *col_idx, const int32_t *offsets, int32_t n_ind,
                     bool want_host_offsets, StagedPop *out);

// params helpers (abi.cu)
int ebic_check_eval_params(ebic_ctx *ctx, const ebic_params *p);
int ebic_check_run_params(ebic_ctx *ctx, const ebic_params *p);

// matrix.cu
cudaError_t launch_upload(const float *x, int64_t R, int32_t C, int64_t R_pad, int32_t layout,
                          uint32_t *keys, int32_t *err, cudaStream_t s);
// Rows [r_begin, r_end) of a row-major upload (multiples of 32; x is the whole matrix).
cudaError_t launch_upload_rows(const float *x, int64_t R, int32_t C, int64_t R_pad,
                               uint32_t *keys, int32_t *err, int64_t r_begin, int64_t r_end,
                               cudaStream_t s);
cudaError_t launch_build_bitmap(const uint32_t *keys, int64_t R_pad, int32_t C, int64_t Wst,
                                uint32_t *bitmap, cudaStream_t s);
// The same bitmap from the bit planes of the rank codes (nb planes per column, nb <= 10); with
// cnt (C * C, zeroed beforehand) also the pair rows' popcounts: for a < b, cnt[a * C + b] =
// popcount(G[a][b]) | popcount(G[b][a]) << 32.
// chunk0 / chunk1: only the 32-word row chunks [chunk0, chunk1) (chunk1 < 0: to the end).
cudaError_t launch_build_bitmap_planes(const uint32_t *planes, int nb, int32_t C, int64_t Wst,
                                       uint32_t *bitmap, unsigned long long *cnt,
                                       cudaStream_t s, int64_t chunk0 = 0,
                                       int64_t chunk1 = -1);

// eval.cu
cudaError_t launch_validate_csr(const int32_t *cols, const int32_t *off, int32_t n, int32_t C,
                                int32_t *err, cudaStream_t s);
// Zeroes the outputs and the work counter, evaluates, writes fitness.  When ev0/ev1 are not
// null they are recorded on `s` immediately before and after the evaluation kernel.
cudaError_t launch_eval(int mode, const EvalArgs &a, const PopView &pv, int num_sms,
                        cudaStream_t s, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr);
// One launch evaluating individual i (columns d_cols[0..L-1] on the device); outputs must be
// zeroed beforehand.
cudaError_t launch_eval_plain(const EvalArgs &a, const int32_t *d_cols, int32_t L, int32_t i,
                              cudaStream_t s);
// The evaluation kernel alone (outputs and a.work must be zero): work split, grid, launch.
// With pdl, the launch may overlap the tail of the previous kernel in the stream (programmatic
// dependent launch); the kernel waits for that kernel's results before reading them.
cudaError_t launch_eval_kernel(int mode, const EvalArgs &a, const PopView &pv, int num_sms,
                               cudaStream_t s, bool pdl = false);
cudaError_t launch_fitness(const EvalArgs &a, const PopView &pv, cudaStream_t s);
// Raises the bitmap kernels' dynamic shared-memory limit on the current device (once per device;
// done before any graph capture, with the bitmap's build).
cudaError_t prepare_bitmap_eval();
int choose_mode(const ebic_ctx *ctx, int requested, int64_t n_ind, double mean_len,
                int expected_sweeps, int last_kept);
// The cost model behind AUTO without tuning (and the job server's footprint): whether building
// the pair bitmap and running `sweeps` bitmap sweeps is expected to beat `sweeps` direct sweeps.
// Costs are in units of about 1.3 ns on GB300, measured per unit on the tie-heavy workload
// (60,000 x 1,000, P 8,192): a bitmap word built (the bit-plane build), a pair word per
// individual and pair in a sweep (both directions), and 16 bytes of codes (or keys) gathered by
// the direct form.
inline bool cost_model_prefers_bitmap(double R_pad, double C, int code_bytes, double n_ind,
                                      double mean_len, double sweeps) {
  const double Wst = R_pad / 32.0;
  const double build = C * C * Wst;
  const double eval_bm = n_ind * (mean_len - 1.0) * Wst;
  const double direct = n_ind * mean_len * R_pad * (code_bytes ? code_bytes : 4) / 16.0;
  return build + sweeps * eval_bm < sweeps * direct;
}

// Capacities of the generation loop's hash tables (tables.cuh): powers of two at load factor
// <= 1 / kTableSpread.  The tabu list is sized for `keys` keys, the duplicate table for P.
constexpr int64_t kTableSpread = 8;
inline uint64_t pow2_at_least(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}
inline uint64_t tabu_capacity(int64_t keys) {
  const int64_t want = kTableSpread * keys;
  return pow2_at_least((uint64_t)(want > 1024 ? want : 1024));
}
inline uint64_t dedup_capacity(int64_t P) { return pow2_at_least((uint64_t)(kTableSpread * P)); }

// Returns a context's matrix- and run-sized buffers (keys, staging, codes, planes, bitmap, pair
// counts, evaluation scratch, the generation loop's state) to the pool, stream-ordered, and
// forgets the matrix; the context itself (stream, events, settings) stays usable.
void ctx_release_buffers(ebic_ctx *ctx);

// evolve.cu
void gen_state_free(struct GenState *g);
// Ends the current run: the state is cleared before the next run, buffers and graphs stay.
void gen_mark_reset(struct GenState *g);
// Drops the captured generation graphs (they hold launch arguments that changed).
void gen_drop_graphs(struct GenState *g);
// The generation loop's parameter check (evolve.cu).
int ebic_check_loop_params(ebic_ctx *ctx, const ebic_params *p);
