// C ABI of the EBIC GB300 library: contexts, matrix upload, the pair bitmap and population
// evaluation.  The generation-loop entry points live in evolve.cu.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>

#include "internal.h"

namespace {

// Restores the caller's current device when an entry point returns.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace

// Up to this many freed bytes stay cached in the library pool of a device (beyond it, memory
// goes back to the device at the next synchronisation).
constexpr uint64_t kPoolKeepBytes = 8ull << 30;
constexpr int kPoolDevices = 64;

cudaMemPool_t library_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[kPoolDevices] = {};
  static bool tried[kPoolDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kPoolDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (!tried[dev]) {
    tried[dev] = true;
    int supported = 0;
    if (cudaDeviceGetAttribute(&supported, cudaDevAttrMemoryPoolsSupported, dev) == cudaSuccess &&
        supported) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.handleTypes = cudaMemHandleTypeNone;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t pool = nullptr;
      if (cudaMemPoolCreate(&pool, &props) == cudaSuccess) {
        uint64_t keep = kPoolKeepBytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = pool;
      }
    }
    cudaGetLastError();
  }
  return pools[dev];
}

int ebic_fail(ebic_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int ebic_fail_cuda(ebic_ctx *ctx, cudaError_t e, const char *what, const char *file, int line) {
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  cudaGetLastError();
  if (ctx) ctx->err = buf;
  return e == cudaErrorMemoryAllocation ? EBIC_ENOMEM : EBIC_ECUDA;
}

bool ebic_is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

static int check_device_ptr(ebic_ctx *ctx, const void *p, const char *name) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return EBIC_OK;
  }
  if ((attr.type == cudaMemoryTypeDevice) && attr.device != ctx->device)
    return ebic_fail(ctx, EBIC_EINVAL, std::string(name) + " is memory of another device");
  return EBIC_OK;
}

int ebic_check_eval_params(ebic_ctx *ctx, const ebic_params *p) {
  if (!p) return ebic_fail(ctx, EBIC_EINVAL, "params is NULL");
  if (!(p->ratio_num > 0 && p->ratio_num <= p->ratio_den))
    return ebic_fail(ctx, EBIC_EINVAL, "need 0 < ratio_num <= ratio_den");
  if (p->ratio_den > (1 << 24))
    return ebic_fail(ctx, EBIC_EINVAL, "ratio_den must be <= 2^24");
  if (p->neg_trends != 0 && p->neg_trends != 1)
    return ebic_fail(ctx, EBIC_EINVAL, "neg_trends must be 0 or 1");
  if (p->col_cap < 0 || p->col_cap > 16 || p->min_rows < 0)
    return ebic_fail(ctx, EBIC_EINVAL, "need 0 <= col_cap <= 16 and min_rows >= 0");
  if (p->mode < EBIC_MODE_AUTO || p->mode > EBIC_MODE_STAGED)
    return ebic_fail(ctx, EBIC_EINVAL, "unknown mode");
  if ((p->non_strict != 0 && p->non_strict != 1) || (p->last_kept != 0 && p->last_kept != 1))
    return ebic_fail(ctx, EBIC_EINVAL, "non_strict and last_kept must be 0 or 1");
  if (p->last_kept && p->mode == EBIC_MODE_BITMAP)
    return ebic_fail(ctx, EBIC_EINVAL, "the last-kept pair test has no bitmap form");
  if (p->ipw < 0 || p->ipw > 4 || p->fuse_pairs < -1 || p->fuse_pairs >= EBIC_MAX_LEN)
    return ebic_fail(ctx, EBIC_EINVAL, "ipw must be in [0, 4] and fuse_pairs in [-1, 63]");
  return EBIC_OK;
}

cudaEvent_t prof_event(ebic_ctx *ctx) {
  if (!ctx->prof) return nullptr;
  cudaEvent_t e = nullptr;
  if (!ctx->ev_pool.empty()) {
    e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

void prof_push(ebic_ctx *ctx, cudaEvent_t a, cudaEvent_t b, int kernel, double bytes, double ops,
               double units, bool own_a, bool own_b) {
  if (a && b) {
    ctx->pending.push_back(PendingTiming{a, b, kernel, bytes, ops, units, own_a, own_b});
  } else {
    if (a) ctx->ev_pool.push_back(a);
    if (b) ctx->ev_pool.push_back(b);
  }
}

cudaEvent_t prof_begin(ebic_ctx *ctx) {
  if (!ctx->prof) return nullptr;
  cudaEvent_t e = nullptr;
  if (!ctx->ev_pool.empty()) {
    e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  cudaEventRecord(e, ctx->stream);
  return e;
}

void prof_end(ebic_ctx *ctx, cudaEvent_t a, int kernel, double bytes, double ops, double units) {
  if (!a) return;
  cudaEvent_t b = nullptr;
  if (!ctx->ev_pool.empty()) {
    b = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
  } else if (cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    ctx->ev_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, ctx->stream);
  ctx->pending.push_back(PendingTiming{a, b, kernel, bytes, ops, units, true, true});
}

void prof_count(ebic_ctx *ctx, int kernel, int64_t n) {
  if (kernel >= 0 && kernel < EBIC_KERNEL_COUNT && kernel != EBIC_KERNEL_ALL)
    ctx->kst[kernel].launches += n;
  ctx->kst[EBIC_KERNEL_ALL].launches += n;
}

void prof_collect(ebic_ctx *ctx) {
  for (const PendingTiming &t : ctx->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      KStats &k = ctx->kst[t.kernel];
      k.timed += 1;
      k.ms += ms;
      k.bytes += t.bytes;
      k.ops += t.ops;
      k.units += t.units;
    } else {
      cudaGetLastError();
    }
    if (t.own_a) ctx->ev_pool.push_back(t.a);
    if (t.own_b) ctx->ev_pool.push_back(t.b);
  }
  ctx->pending.clear();
}

// Validates a CSR population (on the host for host arrays, on the device for device arrays)
// and makes it available on the device.  Host arrays are copied into the context's buffers.
int stage_population(ebic_ctx *ctx, const int32_t *col_idx, const int32_t *offsets, int32_t n_ind,
                     bool want_host_offsets, StagedPop *out) {
  const bool dev_cols = ebic_is_device_ptr(col_idx), dev_off = ebic_is_device_ptr(offsets);
  if (dev_cols != dev_off)
    return ebic_fail(ctx, EBIC_EINVAL, "col_idx and offsets must both be host or both device");
  cudaStream_t s = ctx->stream;
  const int32_t *d_cols = col_idx, *d_off = offsets;
  std::vector<int32_t> &h_off = out->h_off;
  double mean_len = 0.0;
  int64_t total = 0;
  if (!dev_cols) {
    // Host CSR: the offsets are checked here (they size the copy), the columns on the device
    // after the copy, by the kernel that checks device populations (a host loop over every
    // column pair took milliseconds for 8,192 individuals of up to 64 columns).
    for (int32_t i = 0; i < n_ind; ++i) {
      const int64_t L = (int64_t)offsets[i + 1] - offsets[i];
      if (offsets[i] < 0 || L < 2 || L > EBIC_MAX_LEN)
        return ebic_fail(ctx, EBIC_EINVAL, "individual " + std::to_string(i) +
                                               ": length must be in [2, 64]");
    }
    total = (int64_t)offsets[n_ind] - offsets[0];
    mean_len = (double)total / n_ind;
    EBIC_CHECK_CUDA(ctx, ctx->ev_cols.ensure((size_t)(offsets[n_ind]) * 4 + 16, ctx->stream));
    EBIC_CHECK_CUDA(ctx, ctx->ev_off.ensure((size_t)(n_ind + 1) * 4, ctx->stream));
    EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(ctx->ev_cols.p, col_idx, (size_t)offsets[n_ind] * 4,
                                         cudaMemcpyHostToDevice, s));
    EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(ctx->ev_off.p, offsets, (size_t)(n_ind + 1) * 4,
                                         cudaMemcpyHostToDevice, s));
    d_cols = ctx->ev_cols.as<int32_t>();
    d_off = ctx->ev_off.as<int32_t>();
    EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(ctx->d_err.p, 0, sizeof(int32_t), s));
    EBIC_CHECK_CUDA(ctx, launch_validate_csr(d_cols, d_off, n_ind, ctx->C,
                                             ctx->d_err.as<int32_t>(), s));
    prof_count(ctx, -1, 1);
    int32_t herr = 0;
    EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(&herr, ctx->d_err.p, 4, cudaMemcpyDeviceToHost, s));
    EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(s));
    if (herr) return ebic_fail(ctx, EBIC_EINVAL, "invalid chromosome in the population");
    if (want_host_offsets) h_off.assign(offsets, offsets + n_ind + 1);
  } else {
    // Device CSR: validate on the device before any kernel indexes the matrix with it.
    EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(ctx->d_err.p, 0, sizeof(int32_t), s));
    EBIC_CHECK_CUDA(ctx, launch_validate_csr(col_idx, offsets, n_ind, ctx->C,
                                             ctx->d_err.as<int32_t>(), s));
    prof_count(ctx, -1, 1);
    int32_t herr = 0;
    int32_t ends[2] = {0, 0};
    EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(&herr, ctx->d_err.p, 4, cudaMemcpyDeviceToHost, s));
    EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(&ends[0], offsets, 4, cudaMemcpyDeviceToHost, s));
    EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(&ends[1], offsets + n_ind, 4, cudaMemcpyDeviceToHost, s));
    if (want_host_offsets) {
      h_off.resize(n_ind + 1);
      EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(h_off.data(), offsets, (size_t)(n_ind + 1) * 4,
                                           cudaMemcpyDeviceToHost, s));
    }
    EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(s));
    if (herr) return ebic_fail(ctx, EBIC_EINVAL, "invalid chromosome in the population");
    total = (int64_t)ends[1] - ends[0];
    mean_len = (double)total / n_ind;
  }

  out->d_cols = d_cols;
  out->d_off = d_off;
  out->total = total;
  out->mean_len = mean_len;
  return EBIC_OK;
}

extern "C" {

int ebic_profile_enable(ebic_ctx *ctx, int32_t on) {
  if (!ctx) return EBIC_EINVAL;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaGetLastError();
  prof_collect(ctx);
  if (on) {
    for (KStats &k : ctx->kst) k = KStats();
  }
  ctx->prof = on != 0;
  return EBIC_OK;
}

int ebic_profile_read(ebic_ctx *ctx, int32_t kernel, ebic_kernel_stats *out) {
  if (!ctx || !out || kernel < 0 || kernel >= EBIC_KERNEL_COUNT) return EBIC_EINVAL;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaGetLastError();
  prof_collect(ctx);
  const KStats &k = ctx->kst[kernel];
  out->launches = k.launches;
  out->timed_launches = k.timed;
  out->ms = k.ms;
  out->alg_bytes = k.bytes;
  out->alg_ops = k.ops;
  out->units = k.units;
  return EBIC_OK;
}

const char *ebic_version(void) { return "ebic-gb300 0.1 (sm_103a)"; }

void ebic_default_params(ebic_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->neg_trends = 1;
  p->ratio_num = 85;
  p->ratio_den = 100;
  p->min_rows = 2;
  p->col_cap = 10;
  p->overlap_num = 1;
  p->overlap_den = 2;
  p->n_biclusters = 10;
  p->init_min_len = 2;
  p->init_max_len = 8;
  p->max_len = 20;
  p->pop_size = 800;
  p->elite = 10;
  p->tournament = 4;
  p->max_attempts = 4;
  p->tabu_hit_limit = 800;
  p->seed = 20210710ull;
  p->mode = EBIC_MODE_AUTO;
  p->use_graph = 1;
}

int ebic_create(ebic_ctx **out, int32_t device, void *cuda_stream) {
  if (!out) return EBIC_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return EBIC_ECUDA;
  }
  if (device < 0 || device >= ndev) return EBIC_EINVAL;
  ebic_ctx *ctx = new (std::nothrow) ebic_ctx();
  if (!ctx) return EBIC_ENOMEM;
  ctx->device = device;
  DeviceGuard g(device);
  int l2 = 0;
  if (cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, device) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return EBIC_ECUDA;
  }
  ctx->l2_bytes = l2;
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return EBIC_ECUDA;
    }
    ctx->own_stream = true;
  }
  if (ctx->d_err.ensure(64, ctx->stream) != cudaSuccess ||
      ctx->d_work.ensure(64, ctx->stream) != cudaSuccess ||
      ctx->d_kerr.ensure(64, ctx->stream) != cudaSuccess ||
      cudaMemset(ctx->d_kerr.p, 0, 64) != cudaSuccess) {
    ebic_destroy(ctx);
    return EBIC_ENOMEM;
  }
  *out = ctx;
  return EBIC_OK;
}

int ebic_destroy(ebic_ctx *ctx) {
  if (!ctx) return EBIC_OK;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaGetLastError();
  gen_state_free(ctx->gen);
  ctx->gen = nullptr;
  DevBuf *bufs[] = {&ctx->keys, &ctx->bitmap, &ctx->stage_x, &ctx->d_err, &ctx->d_work,
                    &ctx->ev_cols, &ctx->ev_off, &ctx->ev_out, &ctx->ev_fit, &ctx->d_kerr,
                    &ctx->codes, &ctx->planes, &ctx->pair_cnt};
  for (DevBuf *b : bufs) b->release();
  prof_collect(ctx);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->seg_ev) cudaEventDestroy(e);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return EBIC_OK;
}

const char *ebic_last_error(const ebic_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

int64_t ebic_bitmap_bytes(int64_t rows, int32_t cols) {
  if (rows < 1 || cols < 1) return 0;
  return (int64_t)cols * cols * (round_up(rows, 128) / 32) * 4;
}

}  // extern "C"

void ctx_release_buffers(ebic_ctx *ctx) {
  gen_state_free(ctx->gen);
  ctx->gen = nullptr;
  DevBuf *bufs[] = {&ctx->keys, &ctx->bitmap, &ctx->stage_x, &ctx->ev_cols, &ctx->ev_off,
                    &ctx->ev_out, &ctx->ev_fit, &ctx->codes, &ctx->planes, &ctx->pair_cnt};
  for (DevBuf *b : bufs) b->release();
  ctx->have_matrix = false;
  ctx->bitmap_ok = false;
  ctx->pair_cnt_ok = false;
  ctx->codes_ready = false;
  ctx->tuned = false;
  ctx->R = ctx->R_pad = ctx->Wst = 0;
  ctx->C = 0;
}

namespace {

// The segmented load of a row-major host matrix (see ebic_load_matrix): kLoadSegments segments
// of a multiple of 8,192 rows (whole 1,024-row chunks of the bitmap, whole tiles of every
// kernel), the last one with the padded tail.
constexpr int64_t kLoadSegments = 4;

int load_matrix_segmented(ebic_ctx *ctx, const float *x, int64_t rows, int32_t cols,
                          int64_t R_pad) {
  const bool bitmap = ctx->tuned_mode == EBIC_MODE_BITMAP;
  const int64_t C = cols, Wst = R_pad / 32;
  const int cb = code_bytes_for(cols), nb = code_plane_bits(cols);
  const int64_t S = code_stride_for(rows, cb);
  cudaStream_t s = ctx->stream;
  EBIC_CHECK_CUDA(ctx, ctx->stage_x.ensure((size_t)rows * C * sizeof(float), s));
  EBIC_CHECK_CUDA(ctx, ctx->codes.ensure((size_t)C * S * cb, s));
  EBIC_CHECK_CUDA(ctx, ctx->planes.ensure((size_t)C * code_plane_stride(nb) * Wst * 4, s));
  EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(ctx->codes.p, 0, (size_t)C * S * cb, s));
  if (bitmap) {
    EBIC_CHECK_CUDA(ctx, ctx->bitmap.ensure((size_t)ebic_bitmap_bytes(rows, cols), s));
    EBIC_CHECK_CUDA(ctx, prepare_bitmap_eval());
    const size_t nc = (size_t)C * C * sizeof(unsigned long long);
    EBIC_CHECK_CUDA(ctx, ctx->pair_cnt.ensure(nc, s));
    EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(ctx->pair_cnt.p, 0, nc, s));
  }
  if (!ctx->copy_stream)
    EBIC_CHECK_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
  const int64_t seg =
      std::max<int64_t>(8192, round_up((R_pad + kLoadSegments - 1) / kLoadSegments, 8192));
  const int64_t n_seg = (R_pad + seg - 1) / seg;
  while ((int64_t)ctx->seg_ev.size() < n_seg + 1) {
    cudaEvent_t e = nullptr;
    EBIC_CHECK_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    ctx->seg_ev.push_back(e);
  }
  // the copy stream starts after the context stream's earlier work (which may still read the
  // staging buffer)
  EBIC_CHECK_CUDA(ctx, cudaEventRecord(ctx->seg_ev[n_seg], s));
  EBIC_CHECK_CUDA(ctx, cudaStreamWaitEvent(ctx->copy_stream, ctx->seg_ev[n_seg], 0));
  EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(ctx->d_err.p, 0, sizeof(int32_t), s));
  float *stage = ctx->stage_x.as<float>();
  for (int64_t i = 0; i < n_seg; ++i) {
    const int64_t r0 = i * seg, r1 = std::min(R_pad, r0 + seg);
    if (r0 < rows) {
      const int64_t n = std::min(r1, rows) - r0;
      EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(stage + r0 * C, x + r0 * C, (size_t)(n * C) * 4,
                                           cudaMemcpyHostToDevice, ctx->copy_stream));
      EBIC_CHECK_CUDA(ctx, cudaEventRecord(ctx->seg_ev[i], ctx->copy_stream));
      EBIC_CHECK_CUDA(ctx, cudaStreamWaitEvent(s, ctx->seg_ev[i], 0));
    }
    EBIC_CHECK_CUDA(ctx, launch_upload_rows(stage, rows, cols, R_pad, ctx->keys.as<uint32_t>(),
                                            ctx->d_err.as<int32_t>(), r0, r1, s));
    EBIC_CHECK_CUDA(ctx, launch_rank_codes_rows(ctx->keys.as<uint32_t>(), R_pad, cols,
                                                ctx->codes.p, cb, S, ctx->planes.as<uint32_t>(),
                                                Wst, ctx->num_sms, r0, r1, s));
    prof_count(ctx, -1, 1);
    prof_count(ctx, EBIC_KERNEL_RANK_CODES, 1);
  }
  if (bitmap) {
    EBIC_CHECK_CUDA(ctx, launch_build_bitmap_planes(ctx->planes.as<uint32_t>(), nb, cols, Wst,
                                                    ctx->bitmap.as<uint32_t>(),
                                                    ctx->pair_cnt.as<unsigned long long>(), s));
    prof_count(ctx, EBIC_KERNEL_BITMAP_BUILD, 1);
  }
  int32_t herr = 0;
  EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(&herr, ctx->d_err.p, sizeof(int32_t),
                                       cudaMemcpyDeviceToHost, s));
  EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(s));
  if (herr) return ebic_fail(ctx, EBIC_ENAN, "matrix holds NaN or Inf");
  ctx->R = rows;
  ctx->C = cols;
  ctx->R_pad = R_pad;
  ctx->Wst = Wst;
  direct_tma_prepare(&ctx->dtma, ctx->keys.as<uint32_t>(), R_pad, cols);
  ctx->code_bytes = cb;
  ctx->code_stride = S;
  ctx->plane_bits = nb;
  ctx->codes_ready = true;
  ctx->bitmap_ok = bitmap;
  ctx->pair_cnt_ok = bitmap;
  ctx->have_matrix = true;
  ctx->err.clear();
  return EBIC_OK;
}

}  // namespace

extern "C" {

int ebic_load_matrix(ebic_ctx *ctx, const float *x, int64_t rows, int32_t cols, int32_t layout) {
  if (!ctx) return EBIC_EINVAL;
  if (!x) return ebic_fail(ctx, EBIC_EINVAL, "x is NULL");
  if (rows < 1 || cols < 2 || cols > 65535)
    return ebic_fail(ctx, EBIC_EINVAL, "need rows >= 1 and 2 <= cols <= 65535");
  if (layout != EBIC_LAYOUT_ROW_MAJOR && layout != EBIC_LAYOUT_COL_MAJOR)
    return ebic_fail(ctx, EBIC_EINVAL, "unknown layout");
  if (rows > (int64_t(1) << 31) - 128)
    return ebic_fail(ctx, EBIC_EINVAL, "rows must be < 2^31 - 128");
  DeviceGuard g(ctx->device);
  EBIC_TRY(check_device_ptr(ctx, x, "x"));
  // (the autotuner's measurements depend on the matrix's shape only, not on its values: a
  // matrix of the same shape keeps its decisions)
  if (rows != ctx->R || cols != ctx->C) ctx->tuned = false;
  ctx->have_matrix = false;
  ctx->bitmap_ok = false;
  ctx->pair_cnt_ok = false;
  // A matrix of the same shape keeps the generation loop's buffers and captured graphs (their
  // device addresses and sizes stay valid); the run state is cleared before the next run.
  if (ctx->gen && rows == ctx->R && cols == ctx->C) {
    gen_mark_reset(ctx->gen);
  } else {
    gen_state_free(ctx->gen);
    ctx->gen = nullptr;
  }
  const int64_t R_pad = round_up(rows, 128);
  EBIC_CHECK_CUDA(ctx, ctx->keys.ensure((size_t)cols * R_pad * sizeof(uint32_t), ctx->stream));
  // A host matrix of a shape the autotuner measured, in a form that reads rank codes: the copy
  // goes in segments, and each segment's keys, rank codes and bit planes are built while the
  // next segment is copied; the pair words (bitmap form) follow in one launch over every row.
  if (!ebic_is_device_ptr(x) && layout == EBIC_LAYOUT_ROW_MAJOR && code_bytes_for(cols) &&
      ctx->tuned && ctx->tuned_mode != EBIC_MODE_STAGED && !ctx->prof)
    return load_matrix_segmented(ctx, x, rows, cols, R_pad);
  const float *src = x;
  if (!ebic_is_device_ptr(x)) {
    EBIC_CHECK_CUDA(ctx, ctx->stage_x.ensure((size_t)rows * cols * sizeof(float), ctx->stream));
    EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(ctx->stage_x.p, x, (size_t)rows * cols * sizeof(float),
                                         cudaMemcpyHostToDevice, ctx->stream));
    src = ctx->stage_x.as<float>();
  }
  EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(ctx->d_err.p, 0, sizeof(int32_t), ctx->stream));
  EBIC_CHECK_CUDA(ctx, launch_upload(src, rows, cols, R_pad, layout, ctx->keys.as<uint32_t>(),
                                     ctx->d_err.as<int32_t>(), ctx->stream));
  prof_count(ctx, -1, 1);
  int32_t herr = 0;
  EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(&herr, ctx->d_err.p, sizeof(int32_t),
                                       cudaMemcpyDeviceToHost, ctx->stream));
  EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (herr) return ebic_fail(ctx, EBIC_ENAN, "matrix holds NaN or Inf");
  ctx->R = rows;
  ctx->C = cols;
  ctx->R_pad = R_pad;
  ctx->Wst = R_pad / 32;
  direct_tma_prepare(&ctx->dtma, ctx->keys.as<uint32_t>(), R_pad, cols);
  // per-row rank codes for the direct form (C <= 1,024), built on the direct form's first use
  ctx->code_bytes = code_bytes_for(cols);
  ctx->code_stride = ctx->code_bytes ? code_stride_for(rows, ctx->code_bytes) : 0;
  ctx->codes_ready = false;
  ctx->have_matrix = true;
  ctx->err.clear();
  return EBIC_OK;
}

int ebic_build_bitmap(ebic_ctx *ctx) {
  if (!ctx) return EBIC_EINVAL;
  if (!ctx->have_matrix) return ebic_fail(ctx, EBIC_ESTATE, "no matrix loaded");
  if (ctx->bitmap_ok) return EBIC_OK;
  DeviceGuard g(ctx->device);
  const size_t bytes = (size_t)ebic_bitmap_bytes(ctx->R, ctx->C);
  EBIC_CHECK_CUDA(ctx, ctx->bitmap.ensure(bytes, ctx->stream));
  EBIC_CHECK_CUDA(ctx, prepare_bitmap_eval());
  // With rank codes (C <= 1,024) the words come from the codes' bit planes, else from the keys.
  if (ctx->code_bytes) EBIC_TRY(ensure_codes(ctx));
  // (and the pair counts, C * C words, accumulated by the same kernel)
  if (ctx->code_bytes) {
    const size_t nc = (size_t)ctx->C * ctx->C * sizeof(unsigned long long);
    EBIC_CHECK_CUDA(ctx, ctx->pair_cnt.ensure(nc, ctx->stream));
    EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(ctx->pair_cnt.p, 0, nc, ctx->stream));
  }
  cudaEvent_t ev = prof_begin(ctx);
  if (ctx->code_bytes)
    EBIC_CHECK_CUDA(ctx, launch_build_bitmap_planes(ctx->planes.as<uint32_t>(), ctx->plane_bits,
                                                    ctx->C, ctx->Wst, ctx->bitmap.as<uint32_t>(),
                                                    ctx->pair_cnt.as<unsigned long long>(),
                                                    ctx->stream));
  else
    EBIC_CHECK_CUDA(ctx, launch_build_bitmap(ctx->keys.as<uint32_t>(), ctx->R_pad, ctx->C,
                                             ctx->Wst, ctx->bitmap.as<uint32_t>(), ctx->stream));
  prof_end(ctx, ev, EBIC_KERNEL_BITMAP_BUILD, (double)bytes,
           (double)ctx->C * ctx->C * (double)ctx->R, 0.0);
  prof_count(ctx, EBIC_KERNEL_BITMAP_BUILD, 1);
  if (ctx->prof) {  // (later work on the stream is ordered after the build anyway)
    EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
  }
  ctx->bitmap_ok = true;
  ctx->pair_cnt_ok = ctx->code_bytes != 0;
  return EBIC_OK;
}

int ebic_copy_bitmap(ebic_ctx *ctx, uint32_t *out, int64_t n_words) {
  if (!ctx) return EBIC_EINVAL;
  if (!ctx->bitmap_ok) return ebic_fail(ctx, EBIC_ESTATE, "no bitmap built");
  const int64_t need = ebic_bitmap_bytes(ctx->R, ctx->C) / 4;
  if (!out || n_words < need) return ebic_fail(ctx, EBIC_EINVAL, "output too small");
  DeviceGuard g(ctx->device);
  EBIC_TRY(check_device_ptr(ctx, out, "out"));
  EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(out, ctx->bitmap.p, (size_t)need * 4, cudaMemcpyDefault,
                                       ctx->stream));
  EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return EBIC_OK;
}

int ebic_copy_pair_counts(ebic_ctx *ctx, uint64_t *out, int64_t n) {
  if (!ctx) return EBIC_EINVAL;
  if (!ctx->bitmap_ok || !ctx->pair_cnt_ok)
    return ebic_fail(ctx, EBIC_ESTATE, "no pair counts built (bitmap from rank codes)");
  const int64_t need = (int64_t)ctx->C * ctx->C;
  if (!out || n < need) return ebic_fail(ctx, EBIC_EINVAL, "output too small");
  DeviceGuard g(ctx->device);
  EBIC_TRY(check_device_ptr(ctx, out, "out"));
  EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(out, ctx->pair_cnt.p, (size_t)need * 8, cudaMemcpyDefault,
                                       ctx->stream));
  EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return EBIC_OK;
}

int ebic_eval_population(ebic_ctx *ctx, const int32_t *col_idx, const int32_t *offsets,
                         int32_t n_ind, const ebic_params *p, int32_t *rows_pos,
                         int32_t *rows_neg, int32_t *rows_any, uint64_t *fitness) {
  if (!ctx) return EBIC_EINVAL;
  if (!ctx->have_matrix) return ebic_fail(ctx, EBIC_ESTATE, "no matrix loaded");
  EBIC_TRY(ebic_check_eval_params(ctx, p));
  if (n_ind < 0 || n_ind > (1 << 24)) return ebic_fail(ctx, EBIC_EINVAL, "need 0 <= n_ind <= 2^24");
  if (n_ind == 0) return EBIC_OK;
  if (!col_idx || !offsets) return ebic_fail(ctx, EBIC_EINVAL, "col_idx/offsets NULL");
  DeviceGuard g(ctx->device);
  EBIC_TRY(check_device_ptr(ctx, col_idx, "col_idx"));
  EBIC_TRY(check_device_ptr(ctx, offsets, "offsets"));
  void *outs[4] = {rows_pos, rows_neg, rows_any, fitness};
  for (void *o : outs)
    if (o) EBIC_TRY(check_device_ptr(ctx, o, "output"));
  cudaStream_t s = ctx->stream;
  StagedPop sp;
  EBIC_TRY(stage_population(ctx, col_idx, offsets, n_ind, p->mode == EBIC_MODE_PLAIN, &sp));
  const int32_t *d_cols = sp.d_cols, *d_off = sp.d_off;
  const std::vector<int32_t> &h_off = sp.h_off;
  const double mean_len = sp.mean_len;
  const int64_t total = sp.total;

  int mode = choose_mode(ctx, p->mode, n_ind, mean_len, 1, p->last_kept);
  if (mode == EBIC_MODE_BITMAP && !ctx->bitmap_ok) EBIC_TRY(ebic_build_bitmap(ctx));
  if (direct_form_used(ctx, mode, p)) EBIC_TRY(ensure_codes(ctx));

  EBIC_CHECK_CUDA(ctx, ctx->ev_out.ensure((size_t)n_ind * 3 * sizeof(int32_t), ctx->stream));
  EBIC_CHECK_CUDA(ctx, ctx->ev_fit.ensure((size_t)n_ind * sizeof(uint64_t), ctx->stream));
  EvalArgs a = eval_args_for(ctx);
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
  a.seg_passes = ctx->tuned ? (mode == EBIC_MODE_BITMAP ? ctx->seg_bitmap
                                                      : (mode == EBIC_MODE_DIRECT ? ctx->seg_direct : 0))
                            : 0;
  a.ipw = p->ipw > 0 ? p->ipw : (ctx->tuned && mode == EBIC_MODE_BITMAP ? ctx->ipw_bitmap : 1);
  PopView pv{};
  pv.cols = d_cols;
  pv.off = d_off;
  pv.n = n_ind;

  const double pairs = (double)(total - n_ind), nd = a.neg ? 2.0 : 1.0;
  const double ev_bytes = eval_bytes(ctx, mode, total, n_ind, a.neg);
  const double ev_ops = pairs * (double)ctx->R * nd, ev_units = (double)n_ind * (double)ctx->R;
  if (mode == EBIC_MODE_PLAIN) {
    EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(a.rows_pos, 0, (size_t)n_ind * 3 * 4, s));
    cudaEvent_t ev = prof_begin(ctx);
    for (int32_t i = 0; i < n_ind; ++i)
      EBIC_CHECK_CUDA(ctx, launch_eval_plain(a, d_cols + h_off[i], h_off[i + 1] - h_off[i], i, s));
    prof_end(ctx, ev, EBIC_KERNEL_EVAL, (double)total * (double)ctx->R_pad * 4.0, ev_ops,
             ev_units);
    prof_count(ctx, EBIC_KERNEL_EVAL, n_ind);
    EBIC_CHECK_CUDA(ctx, launch_fitness(a, pv, s));
    prof_count(ctx, -1, 1);
  } else {
    cudaEvent_t e0 = prof_event(ctx), e1 = prof_event(ctx);
    EBIC_CHECK_CUDA(ctx, launch_eval(mode, a, pv, ctx->num_sms, s, e0, e1));
    prof_push(ctx, e0, e1, EBIC_KERNEL_EVAL, ev_bytes, ev_ops, ev_units);
    prof_count(ctx, EBIC_KERNEL_EVAL, 1);
    prof_count(ctx, -1, 1);
  }
  int32_t *dsts[3] = {rows_pos, rows_neg, rows_any};
  for (int k = 0; k < 3; ++k)
    if (dsts[k])
      EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(dsts[k], a.rows_pos + (size_t)k * n_ind,
                                           (size_t)n_ind * 4, cudaMemcpyDefault, s));
  if (fitness)
    EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(fitness, a.fitness, (size_t)n_ind * 8,
                                         cudaMemcpyDefault, s));
  int32_t kerr = 0;
  EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(&kerr, ctx->d_kerr.p, 4, cudaMemcpyDeviceToHost, s));
  EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(s));
  prof_collect(ctx);
  if (kerr) {
    cudaMemset(ctx->d_kerr.p, 0, 4);
    return ebic_fail(ctx, EBIC_ETIMEOUT, "a bounded device wait expired in the evaluation");
  }
  return EBIC_OK;
}

}  // extern "C"

int ensure_codes(ebic_ctx *ctx) {
  if (!ctx->code_bytes || ctx->codes_ready) return EBIC_OK;
  const int64_t S = ctx->code_stride, C = ctx->C;
  ctx->plane_bits = code_plane_bits(ctx->C);
  EBIC_CHECK_CUDA(ctx, ctx->codes.ensure((size_t)C * S * ctx->code_bytes, ctx->stream));
  EBIC_CHECK_CUDA(ctx, ctx->planes.ensure(
                           (size_t)C * code_plane_stride(ctx->plane_bits) * ctx->Wst * 4,
                           ctx->stream));
  cudaEvent_t ev = prof_begin(ctx);
  EBIC_CHECK_CUDA(ctx, launch_rank_codes(ctx->keys.as<uint32_t>(), ctx->R_pad, ctx->C,
                                         ctx->codes.p, ctx->code_bytes, S,
                                         ctx->planes.as<uint32_t>(), ctx->Wst, ctx->num_sms,
                                         ctx->stream));
  // algorithmic bytes: keys read, codes and planes written
  prof_end(ctx, ev, EBIC_KERNEL_RANK_CODES,
           (double)C * ctx->R_pad * 4.0 + (double)C * S * ctx->code_bytes +
               (double)C * ctx->plane_bits * ctx->Wst * 4.0,
           (double)C * ctx->R_pad, (double)ctx->R_pad);
  prof_count(ctx, EBIC_KERNEL_RANK_CODES, 1);
  if (ctx->prof) {  // (later work on the stream is ordered after the build anyway)
    EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    prof_collect(ctx);
  }
  ctx->codes_ready = true;
  return EBIC_OK;
}

int direct_form_used(const ebic_ctx *ctx, int mode, const ebic_params *p) {
  if (mode == EBIC_MODE_DIRECT) return 1;
  return mode == EBIC_MODE_STAGED && (!ctx->dtma.ok || p->non_strict || p->last_kept);
}


// Evaluation-kernel choice for EBIC_MODE_AUTO: a cost model in row-words, refined by the
// autotuner when it has measured this matrix.  The bitmap costs a one-off build of C^2 * Wst
// words and then (L-1) * Wst words per individual and direction; the direct form gathers
// L * R_pad keys per individual.
EvalArgs eval_args_for(const ebic_ctx *ctx) {
  EvalArgs a{};
  a.keys = ctx->keys.as<uint32_t>();
  a.bitmap = ctx->bitmap_ok ? ctx->bitmap.as<uint32_t>() : nullptr;
  a.R = ctx->R;
  a.R_pad = ctx->R_pad;
  a.Wst = ctx->Wst;
  a.C = ctx->C;
  a.err = ctx->d_kerr.as<int32_t>();
  a.dtma = ctx->dtma.ok ? &ctx->dtma : nullptr;
  a.codes = ctx->codes_ready ? ctx->codes.as<uint8_t>() : nullptr;
  a.code_bytes = ctx->codes_ready ? ctx->code_bytes : 0;
  a.S = ctx->codes_ready ? ctx->code_stride : 0;
  a.stage_bitmap = ctx->bitmap_ok && (double)ebic_bitmap_bytes(ctx->R, ctx->C) > (double)ctx->l2_bytes;
  a.ipw = 1;
  return a;
}

int64_t eval_passes(const ebic_ctx *ctx, int mode) {
  if (mode == EBIC_MODE_BITMAP) return (ctx->Wst + 127) / 128;
  if (ctx->codes_ready) return ctx->code_stride / code_rows_per_pass(ctx->code_bytes);
  return ctx->R_pad / 128;
}

double eval_bytes(const ebic_ctx *ctx, int mode, int64_t total_len, int64_t n_ind, int neg) {
  // algorithmic bytes of one sweep: the pair words (bitmap), else one code or key per row and
  // chromosome column (the staged form reads each tile of keys once per group of individuals;
  // its algorithmic gathers are counted like the key form's)
  if (mode == EBIC_MODE_BITMAP)
    return (double)(total_len - n_ind) * (double)ctx->Wst * 4.0 * (neg ? 2.0 : 1.0);
  if (mode == EBIC_MODE_DIRECT && ctx->codes_ready)
    return (double)total_len * (double)ctx->code_stride * ctx->code_bytes;
  return (double)total_len * (double)ctx->R_pad * 4.0;
}

int choose_mode(const ebic_ctx *ctx, int requested, int64_t n_ind, double mean_len,
                int expected_sweeps, int last_kept) {
  if (requested != EBIC_MODE_AUTO) return requested;
  if (last_kept) {  // no bitmap form
    return ctx->tuned && ctx->tuned_mode != EBIC_MODE_BITMAP ? ctx->tuned_mode : EBIC_MODE_DIRECT;
  }
  if (ctx->tuned) return ctx->tuned_mode;
  if (ctx->bitmap_ok) return EBIC_MODE_BITMAP;
  const double Wst = (double)ctx->Wst, C = (double)ctx->C;
  const double bitmap_bytes = C * C * Wst * 4.0;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    free_b = 0;
  }
  if (bitmap_bytes > 0.5 * (double)free_b) return EBIC_MODE_DIRECT;
  return cost_model_prefers_bitmap((double)ctx->R_pad, C, ctx->code_bytes, (double)n_ind,
                                   mean_len, (double)expected_sweeps)
             ? EBIC_MODE_BITMAP
             : EBIC_MODE_DIRECT;
}
