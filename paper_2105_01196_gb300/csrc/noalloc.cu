// Population evaluation without any memory allocation (ebic_eval_population_noalloc).
//
// Some callers cannot let a library call cudaMalloc or cudaFree.  Examples: a serving process
// whose framework has already reserved the GPU's memory in its own pool, where a further
// allocation fails or fragments the pool; and latency-critical callers, for whom cudaFree's
// device-wide synchronisation and the allocator's unbounded latency are not acceptable.  This
// entry point takes every input and output from the caller, and keeps its scratch (per-individual
// count accumulators, the work-queue counter and an error word) in one file-scope
// `static __device__` array of fixed size, which every GPU that loads the library holds until
// the process exits.
//
// Host code cannot name that array's device address directly: in host code its name stands for
// a host-side shadow.  The address is therefore fetched once per device with
// cudaGetSymbolAddress (with that device current) and handed to the kernels.
//
// CUDA loads modules lazily by default, so this file's module (the array and the kernels' code)
// is placed in device memory only when first used on a device.  The first call on each device
// therefore does that set-up explicitly: it resolves the array's address and queries every
// kernel's attributes, which loads all of them.  Later calls on that device load nothing.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "internal.h"
#include "trend.cuh"

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kNaWarps = 8;
constexpr int kNaThreads = kNaWarps * 32;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  int32_t counts[3 * EBIC_NOALLOC_MAX_IND];  // rows_pos | rows_neg | rows_any accumulators
  int32_t work;                              // work-queue counter
  int32_t err;                               // 1: non-finite matrix value, 2: bad chromosome
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_setup_mu;
NoAllocScratch *g_scratch_addr[kMaxDevices] = {};

__device__ __forceinline__ int threshold(int L, int num, int den) {
  return (num * (L - 1) + den - 1) / den;
}

// Checks the matrix for NaN/Inf and the population for invalid chromosomes.
__global__ void k_na_validate(const float *__restrict__ x, int64_t total,
                              const int32_t *__restrict__ cols, const int32_t *__restrict__ off,
                              int32_t n, int32_t C, NoAllocScratch *sc) {
  bool bad_x = false;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = tid; q < total; q += stride) {
    const uint32_t u = __float_as_uint(__ldg(x + q));
    bad_x |= (u & 0x7F800000u) == 0x7F800000u;
  }
  if (__any_sync(kFull, bad_x) && (threadIdx.x & 31) == 0) atomicOr(&sc->err, 1);
  for (int64_t i = tid; i < n; i += stride) {
    const int s = off[i], L = off[i + 1] - s;
    bool bad = s < 0 || L < 2 || L > EBIC_MAX_LEN;
    for (int k = 0; k < L && !bad; ++k) {
      const int c = cols[s + k];
      if (c < 0 || c >= C) bad = true;
      for (int j = 0; j < k && !bad; ++j)
        if (cols[s + j] == c) bad = true;
    }
    if (bad) atomicOr(&sc->err, 2);
  }
}

// Direct float32 comparisons (-0 equals +0; no FTZ in this file's compilation), one row per
// lane, warps pulling (individual, segment of 32-row passes) items from sc->work.  NS / LK are
// the pair-test variants of trend.cuh.
template <bool NEG, bool NS, bool LK>
__global__ void __launch_bounds__(kNaThreads) k_na_eval(const float *__restrict__ x, int64_t R,
                                                        const int32_t *__restrict__ cols,
                                                        const int32_t *__restrict__ off,
                                                        int32_t n, int32_t n_seg,
                                                        int32_t seg_passes, int32_t rnum,
                                                        int32_t rden, NoAllocScratch *sc) {
  __shared__ int64_t s_base[kNaWarps][EBIC_MAX_LEN];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t passes_total = (R + 31) / 32;
  const int32_t n_items = n * n_seg;
  for (;;) {
    int q = 0;
    if (lane == 0) q = atomicAdd(&sc->work, 1);
    q = __shfl_sync(kFull, q, 0);
    if (q >= n_items) break;
    const int i = q / n_seg, seg = q - i * n_seg;
    const int st = off[i], L = off[i + 1] - st;
    __syncwarp();
    for (int k = lane; k < L; k += 32) s_base[warp][k] = (int64_t)cols[st + k] * R;
    __syncwarp();
    const int t = threshold(L, rnum, rden);
    const int64_t p0 = (int64_t)seg * seg_passes;
    const int64_t p1 = min(p0 + seg_passes, passes_total);
    int cp = 0, cn = 0, ca = 0;
    for (int64_t pass = p0; pass < p1; ++pass) {
      const int64_t r = pass * 32 + lane;
      if (r < R) {
        RowTrend<float, NEG, NS, LK> tr;
        tr.start(__ldg(x + s_base[warp][0] + r));
        for (int k = 1; k < L; ++k) tr.step(__ldg(x + s_base[warp][k] + r));
        const bool po = tr.inc >= t, ne = NEG && tr.dec >= t;
        cp += po;
        cn += ne;
        ca += po || ne;
      }
    }
    cp = __reduce_add_sync(kFull, cp);
    cn = __reduce_add_sync(kFull, cn);
    ca = __reduce_add_sync(kFull, ca);
    if (lane == 0) {
      if (cp) atomicAdd(&sc->counts[i], cp);
      if (cn) atomicAdd(&sc->counts[n + i], cn);
      if (ca) atomicAdd(&sc->counts[2 * n + i], ca);
    }
  }
}

__global__ void k_na_finish(const int32_t *__restrict__ off, int32_t n, int32_t min_rows,
                            int32_t col_cap, const NoAllocScratch *sc, int32_t *rows_pos,
                            int32_t *rows_neg, int32_t *rows_any, uint64_t *fitness) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int rp = sc->counts[i], rn = sc->counts[n + i], ra = sc->counts[2 * n + i];
  if (rows_pos) rows_pos[i] = rp;
  if (rows_neg) rows_neg[i] = rn;
  if (rows_any) rows_any[i] = ra;
  if (fitness) {
    const int L = off[i + 1] - off[i];
    const int sh = L < col_cap ? L : col_cap;
    fitness[i] = ra < min_rows ? 0ull : ((uint64_t)ra << sh);
  }
}

using NaKernel = void (*)(const float *, int64_t, const int32_t *, const int32_t *, int32_t,
                          int32_t, int32_t, int32_t, int32_t, NoAllocScratch *);
// Indexed by neg_trends * 4 + non_strict * 2 + last_kept.
const NaKernel kNaEval[8] = {k_na_eval<false, false, false>, k_na_eval<false, false, true>,
                             k_na_eval<false, true, false>,  k_na_eval<false, true, true>,
                             k_na_eval<true, false, false>,  k_na_eval<true, false, true>,
                             k_na_eval<true, true, false>,   k_na_eval<true, true, true>};

// Set-up for `device`, done once: with the device current, fetch the device address of the
// scratch array and query every kernel of this file, so that the module (array and code) is in
// device memory before the call returns.  Returns the cached address on later calls.
cudaError_t scratch_for_device(int device, NoAllocScratch **out) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_addr[device]) {
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return e;
    void *ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    cudaFuncAttributes fa;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_validate);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_na_finish);
    for (int k = 0; k < 8 && e == cudaSuccess; ++k) e = cudaFuncGetAttributes(&fa, kNaEval[k]);
    if (prev >= 0 && prev != device) cudaSetDevice(prev);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<NoAllocScratch *>(ptr);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

int fail(char *msg, int32_t msg_len, int code, const char *text) {
  if (msg && msg_len > 0) snprintf(msg, (size_t)msg_len, "%s", text);
  return code;
}

bool on_device(const void *p, int device) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) &&
         (a.type == cudaMemoryTypeManaged || a.device == device);
}

}  // namespace

extern "C" int ebic_eval_population_noalloc(const float *x, int64_t rows, int32_t cols,
                                            const int32_t *col_idx, const int32_t *offsets,
                                            int32_t n_ind, const ebic_params *p,
                                            int32_t *rows_pos, int32_t *rows_neg,
                                            int32_t *rows_any, uint64_t *fitness,
                                            int32_t device, void *cuda_stream, char *msg,
                                            int32_t msg_len) {
  if (msg && msg_len > 0) msg[0] = '\0';
  if (!p) return fail(msg, msg_len, EBIC_EINVAL, "params is NULL");
  if (!(p->ratio_num > 0 && p->ratio_num <= p->ratio_den) || p->ratio_den > (1 << 24))
    return fail(msg, msg_len, EBIC_EINVAL, "need 0 < ratio_num <= ratio_den <= 2^24");
  if ((p->neg_trends != 0 && p->neg_trends != 1) || p->col_cap < 0 || p->col_cap > 16 ||
      p->min_rows < 0)
    return fail(msg, msg_len, EBIC_EINVAL, "bad neg_trends, col_cap or min_rows");
  if ((p->non_strict != 0 && p->non_strict != 1) || (p->last_kept != 0 && p->last_kept != 1))
    return fail(msg, msg_len, EBIC_EINVAL, "non_strict and last_kept must be 0 or 1");
  if (rows < 1 || rows > (int64_t(1) << 31) - 32 || cols < 2 || cols > 65535)
    return fail(msg, msg_len, EBIC_EINVAL, "need 1 <= rows < 2^31 - 32 and 2 <= cols <= 65535");
  if (n_ind < 0 || n_ind > EBIC_NOALLOC_MAX_IND)
    return fail(msg, msg_len, EBIC_EINVAL,
                "n_ind is beyond EBIC_NOALLOC_MAX_IND (65536), the size of the static scratch");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return fail(msg, msg_len, EBIC_ECUDA, "cudaGetDeviceCount failed");
  }
  if (device < 0 || device >= ndev || device >= kMaxDevices)
    return fail(msg, msg_len, EBIC_EINVAL, "bad device");
  if (n_ind == 0) return EBIC_OK;
  if (!on_device(x, device) || !on_device(col_idx, device) || !on_device(offsets, device))
    return fail(msg, msg_len, EBIC_EINVAL,
                "x, col_idx and offsets must be device memory of `device`");
  void *outs[4] = {rows_pos, rows_neg, rows_any, fitness};
  for (void *o : outs)
    if (o && !on_device(o, device))
      return fail(msg, msg_len, EBIC_EINVAL, "outputs must be device memory of `device`");

  NoAllocScratch *sc = nullptr;
  cudaError_t e = scratch_for_device(device, &sc);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(msg, msg_len, EBIC_ECUDA,
                "set-up failed: the scratch array's address or the kernels could not be loaded");
  }
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    prev = -1;
  }
  if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) {
    cudaGetLastError();
    return fail(msg, msg_len, EBIC_ECUDA, "cudaSetDevice failed");
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int status = EBIC_OK;
  do {
    // The array keeps the previous call's contents: clear the accumulators this call uses, the
    // work counter and the error word.
    if ((e = cudaMemsetAsync(sc->counts, 0, (size_t)3 * n_ind * sizeof(int32_t), s)) != cudaSuccess)
      break;
    if ((e = cudaMemsetAsync(&sc->work, 0, 2 * sizeof(int32_t), s)) != cudaSuccess) break;
    k_na_validate<<<1024, 256, 0, s>>>(x, rows * (int64_t)cols, col_idx, offsets, n_ind, cols,
                                       sc);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    int32_t herr = 0;
    if ((e = cudaMemcpyAsync(&herr, &sc->err, sizeof(herr), cudaMemcpyDeviceToHost, s)) !=
        cudaSuccess)
      break;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) break;
    if (herr & 1) {
      status = fail(msg, msg_len, EBIC_ENAN, "matrix holds NaN or Inf");
      break;
    }
    if (herr & 2) {
      status = fail(msg, msg_len, EBIC_EINVAL, "invalid chromosome in the population");
      break;
    }
    int num_sms = 0;
    if ((e = cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device)) !=
        cudaSuccess)
      break;
    const int64_t passes_total = (rows + 31) / 32;
    int64_t seg = ((int64_t)n_ind * passes_total) / ((int64_t)8 * num_sms * kNaWarps * 2);
    if (seg < 1) seg = 1;
    if (seg > passes_total) seg = passes_total;
    int64_t n_seg = (passes_total + seg - 1) / seg;
    while ((int64_t)n_ind * n_seg > (1LL << 30)) {
      seg *= 2;
      n_seg = (passes_total + seg - 1) / seg;
    }
    int64_t grid = ((int64_t)n_ind * n_seg + kNaWarps - 1) / kNaWarps;
    if (grid > (int64_t)num_sms * 2) grid = (int64_t)num_sms * 2;
    const NaKernel kern =
        kNaEval[(p->neg_trends ? 4 : 0) + (p->non_strict ? 2 : 0) + (p->last_kept ? 1 : 0)];
    kern<<<(unsigned)grid, kNaThreads, 0, s>>>(x, rows, col_idx, offsets, n_ind, (int32_t)n_seg,
                                               (int32_t)seg, p->ratio_num, p->ratio_den, sc);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    k_na_finish<<<(n_ind + 255) / 256, 256, 0, s>>>(offsets, n_ind, p->min_rows, p->col_cap, sc,
                                                    rows_pos, rows_neg, rows_any, fitness);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    e = cudaStreamSynchronize(s);
  } while (false);
  if (prev >= 0 && prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    char buf[256];
    snprintf(buf, sizeof(buf), "CUDA error: %s", cudaGetErrorString(e));
    return fail(msg, msg_len, EBIC_ECUDA, buf);
  }
  return status;
}
