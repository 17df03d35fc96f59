// Autotuner: measures the evaluation kernels on a representative population of the loaded matrix
// and records, for this matrix, the evaluation form (direct comparison from L2, direct comparison
// over TMA-staged tiles, or pair bitmap) and the
// work-item size (passes of 128 rows or 128 words per item) that minimise the expected time of
// `expected_sweeps` evaluations, the bitmap build included when the bitmap does not exist yet.
// EBIC_MODE_AUTO then follows the recorded choice, both in ebic_eval_population and in the
// generation loop, until a matrix of another shape is loaded.  When a run of generations is
// expected, the loop's own work-item size is measured in a scratch run of the loop (selection
// soon makes its population shorter than the one given here).
#include <float.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace {

const int kSegCandidates[] = {0, 1, 2, 4, 8, 16, 32};  // 0 = the built-in split
const int kReps = 3;

// Minimum over kReps of one evaluation sweep (kernel only, CUDA events on the context stream).
int time_eval(ebic_ctx *ctx, int mode, EvalArgs a, const PopView &pv, int seg, int ipw,
              double *ms_out) {
  cudaEvent_t e0, e1;
  EBIC_CHECK_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ebic_fail(ctx, EBIC_ECUDA, "cudaEventCreate failed");
  }
  a.seg_passes = seg;
  a.ipw = ipw;
  double best = DBL_MAX;
  int status = EBIC_OK;
  for (int r = 0; r < kReps && status == EBIC_OK; ++r) {
    cudaError_t e = launch_eval(mode, a, pv, ctx->num_sms, ctx->stream, e0, e1);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      status = ebic_fail_cuda(ctx, e, "autotune sweep", __FILE__, __LINE__);
      break;
    }
    prof_count(ctx, EBIC_KERNEL_EVAL, 1);
    prof_count(ctx, -1, 1);
    best = std::min(best, (double)ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms_out = best;
  return status;
}

const int kLoopSegCandidates[] = {0, 1, 2, 4, 8, 16};  // 0 = the built-in split
const int kLoopGens = 16;

// Pair limits of the evaluation inside the evolve kernel measured for the bitmap form (-1: none).
const int kLoopFuseCandidates[] = {-1, 1, 2, 4, 8, 63};

// The generation loop's sizes, each candidate measured in the loop itself: a warm-up run
// (initial population and `gens` generations, which also captures the graphs), then the same
// run again with its generations timed by CUDA events on the context stream.  First (bitmap
// form) the pair limit of the evaluation inside the evolve kernel, with the built-in work-item
// split; then the work-item size and group size with that limit.  The run state is reset
// afterwards: the caller's next run starts from its own initial population.
int tune_loop(ebic_ctx *ctx, const ebic_params *p, int gens, int ipw_max, int *best_seg_out,
              int *best_ipw_out, int *best_fuse_out) {
  cudaEvent_t e0, e1;
  EBIC_CHECK_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return ebic_fail(ctx, EBIC_ECUDA, "cudaEventCreate failed");
  }
  ebic_params q = *p;
  q.mode = EBIC_MODE_AUTO;  // (the form just chosen)
  q.use_graph = 1;
  q.ipw = 0;                // (the candidates below)
  q.fuse_pairs = -1;
  const int64_t passes = eval_passes(ctx, ctx->tuned_mode);
  int status = EBIC_OK;
  ebic_run_report rep;
  // the loop with the current candidate: *ms for its `gens` timed generations
  auto time_loop = [&](float *ms) {
    for (int pass = 0; pass < 2 && status == EBIC_OK; ++pass) {
      if (ctx->gen) {
        // (the captured launches hold the sizes: captured again in the first pass)
        if (pass == 0) gen_drop_graphs(ctx->gen);
        gen_mark_reset(ctx->gen);
      }
      status = ebic_run_generations(ctx, &q, 0, &rep);
      if (status != EBIC_OK) break;
      cudaError_t e = cudaEventRecord(e0, ctx->stream);
      if (e == cudaSuccess) status = ebic_run_generations(ctx, &q, gens, &rep);
      if (status != EBIC_OK) break;
      if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
      if (e != cudaSuccess) status = ebic_fail_cuda(ctx, e, "loop tuning", __FILE__, __LINE__);
    }
  };
  double best = DBL_MAX;
  int best_fuse = 0;  // (not measured: other forms)
  if (ctx->tuned_mode == EBIC_MODE_BITMAP && !p->last_kept) {
    best_fuse = -1;
    ctx->seg_loop = 0;
    ctx->ipw_loop = 1;
    for (int f : kLoopFuseCandidates) {
      q.fuse_pairs = f;
      float ms = 0.f;
      time_loop(&ms);
      if (status != EBIC_OK) break;
      if (ms < best) {
        best = ms;
        best_fuse = f;
      }
    }
    q.fuse_pairs = best_fuse;
  }
  best = DBL_MAX;
  int best_seg = 0, best_ipw = 1;
  for (int cand = 0; status == EBIC_OK; ++cand) {
    const int n_seg_cands = (int)(sizeof(kLoopSegCandidates) / sizeof(int));
    const int ipw = 1 << (cand / n_seg_cands), seg = kLoopSegCandidates[cand % n_seg_cands];
    if (ipw > ipw_max) break;
    if (seg > passes) continue;
    ctx->seg_loop = seg;
    ctx->ipw_loop = ipw;
    float ms = 0.f;
    time_loop(&ms);
    if (status != EBIC_OK) break;
    if (ms < best) {
      best = ms;
      best_seg = seg;
      best_ipw = ipw;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (ctx->gen) {
    gen_drop_graphs(ctx->gen);
    gen_mark_reset(ctx->gen);
  }
  *best_seg_out = best_seg;
  *best_ipw_out = best_ipw;
  *best_fuse_out = best_fuse;
  return status;
}

}  // namespace

extern "C" int ebic_autotune(ebic_ctx *ctx, const int32_t *col_idx, const int32_t *offsets,
                             int32_t n_ind, const ebic_params *p, int32_t expected_sweeps,
                             ebic_tune_report *rep) {
  if (!ctx) return EBIC_EINVAL;
  if (!ctx->have_matrix) return ebic_fail(ctx, EBIC_ESTATE, "no matrix loaded");
  EBIC_TRY(ebic_check_eval_params(ctx, p));
  if (n_ind < 1 || n_ind > (1 << 24) || expected_sweeps < 1)
    return ebic_fail(ctx, EBIC_EINVAL, "need 1 <= n_ind <= 2^24 and expected_sweeps >= 1");
  if (!col_idx || !offsets) return ebic_fail(ctx, EBIC_EINVAL, "col_idx/offsets NULL");
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev};
  StagedPop sp;
  EBIC_TRY(stage_population(ctx, col_idx, offsets, n_ind, false, &sp));
  EBIC_CHECK_CUDA(ctx, ctx->ev_out.ensure((size_t)n_ind * 3 * sizeof(int32_t), ctx->stream));
  EBIC_CHECK_CUDA(ctx, ctx->ev_fit.ensure((size_t)n_ind * sizeof(uint64_t), ctx->stream));
  EBIC_TRY(ensure_codes(ctx));  // the direct form is always measured
  EvalArgs a = eval_args_for(ctx);
  a.bitmap = nullptr;
  a.neg = p->neg_trends;
  a.non_strict = p->non_strict;
  a.last_kept = p->last_kept;
  a.rnum = p->ratio_num;
  a.rden = p->ratio_den;
  a.min_rows = p->min_rows;
  a.col_cap = p->col_cap;
  a.rows_pos = ctx->ev_out.as<int32_t>();
  a.rows_neg = a.rows_pos + n_ind;
  a.rows_any = a.rows_neg + n_ind;
  a.fitness = ctx->ev_fit.as<uint64_t>();
  a.work = ctx->d_work.as<int32_t>();
  PopView pv{};
  pv.cols = sp.d_cols;
  pv.off = sp.d_off;
  pv.n = n_ind;

  ebic_tune_report r{};
  const int64_t passes_direct = eval_passes(ctx, EBIC_MODE_DIRECT),
                passes_bitmap = eval_passes(ctx, EBIC_MODE_BITMAP);
  double best_direct = DBL_MAX, best_bitmap = DBL_MAX;
  int seg_direct = 0, seg_bitmap = 0, ipw_bitmap = 1;
  for (int seg : kSegCandidates) {
    if (seg > passes_direct) break;
    double ms = 0;
    EBIC_TRY(time_eval(ctx, EBIC_MODE_DIRECT, a, pv, seg, 1, &ms));
    if (ms < best_direct) {
      best_direct = ms;
      seg_direct = seg;
    }
  }
  // the bitmap form, when its C^2 * R / 8 bytes fit comfortably
  double build_ms = 0.0;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = 0;
  }
  const bool had_bitmap = ctx->bitmap_ok;
  // (the last-kept pair test has no bitmap form)
  if (!p->last_kept &&
      (had_bitmap || (double)ebic_bitmap_bytes(ctx->R, ctx->C) < 0.5 * (double)free_b)) {
    if (!had_bitmap) {
      cudaEvent_t e0, e1;
      EBIC_CHECK_CUDA(ctx, cudaEventCreate(&e0));
      EBIC_CHECK_CUDA(ctx, cudaEventCreate(&e1));
      EBIC_CHECK_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
      const int st = ebic_build_bitmap(ctx);
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (st != EBIC_OK) return st;
      build_ms = ms;
    }
    a.bitmap = ctx->bitmap.as<uint32_t>();
    a.stage_bitmap = eval_args_for(ctx).stage_bitmap;  // (the form later runs will use)
    // (individuals per item: the staged form only)
    const int ipw_max = a.stage_bitmap && p->ratio_num < p->ratio_den ? 4 : 1;
    for (int ipw = 1; ipw <= ipw_max; ipw *= 2)
      for (int seg : kSegCandidates) {
        if (seg > passes_bitmap) break;
        double ms = 0;
        EBIC_TRY(time_eval(ctx, EBIC_MODE_BITMAP, a, pv, seg, ipw, &ms));
        if (ms < best_bitmap) {
          best_bitmap = ms;
          seg_bitmap = seg;
          ipw_bitmap = ipw;
        }
      }
  }
  // the staged direct form, when its tiles fit in shared memory
  double best_staged = DBL_MAX;
  if (ctx->dtma.ok && !p->non_strict && !p->last_kept) {  // the staged kernel's pair test
    EBIC_TRY(time_eval(ctx, EBIC_MODE_STAGED, a, pv, 0, 1, &best_staged));
  }
  const int direct_mode = best_staged < best_direct ? EBIC_MODE_STAGED : EBIC_MODE_DIRECT;
  const double cost_direct = (double)expected_sweeps * (best_staged < best_direct ? best_staged
                                                                                    : best_direct);
  const double cost_bitmap = best_bitmap == DBL_MAX
                                 ? DBL_MAX
                                 : build_ms + (double)expected_sweeps * best_bitmap;
  ctx->tuned = true;
  ctx->tuned_mode = cost_bitmap < cost_direct ? EBIC_MODE_BITMAP : direct_mode;
  ctx->seg_direct = seg_direct;
  ctx->seg_bitmap = seg_bitmap;
  ctx->ipw_bitmap = ipw_bitmap;
  ctx->seg_loop = 0;
  ctx->ipw_loop = 1;
  ctx->fuse_loop = 0;
  // A run of generations expected: the loop's population soon differs from this one (selection
  // shortens it), so its work-item size is measured in the loop itself.
  if (expected_sweeps > 2 && ctx->tuned_mode != EBIC_MODE_STAGED &&
      ebic_check_loop_params(ctx, p) == EBIC_OK) {
    int best_seg = 0, best_ipw = 1, best_fuse = 0;
    const bool staged = ctx->tuned_mode == EBIC_MODE_BITMAP && eval_args_for(ctx).stage_bitmap &&
                        p->ratio_num < p->ratio_den;
    EBIC_TRY(tune_loop(ctx, p, std::min(expected_sweeps - 1, kLoopGens), staged ? 4 : 1,
                       &best_seg, &best_ipw, &best_fuse));
    ctx->seg_loop = best_seg;
    ctx->ipw_loop = best_ipw;
    ctx->fuse_loop = best_fuse;
  }
  if (rep) {
    r.mode = ctx->tuned_mode;
    r.seg_direct = seg_direct;
    r.seg_bitmap = seg_bitmap;
    r.seg_loop = ctx->seg_loop;
    r.ipw_bitmap = ctx->ipw_bitmap;
    r.ipw_loop = ctx->ipw_loop;
    r.fuse_loop = ctx->fuse_loop;
    r.direct_ms = best_direct;
    r.staged_ms = best_staged == DBL_MAX ? -1.0 : best_staged;
    r.bitmap_ms = best_bitmap == DBL_MAX ? -1.0 : best_bitmap;
    r.build_ms = build_ms;
    *rep = r;
  }
  return EBIC_OK;
}
