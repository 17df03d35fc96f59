// Per-row rank codes and the direct-comparison evaluation over them (the trend counts of
// Sec. 2.3 / Sec. 2.4 steps 2-3, as in eval.cu).
//
// Every comparison the trend counts make is between two entries of the same row.  Replacing the
// entry of row r, column c by its rank within the row,
//   code(r, c) = #{k : key(r, k) < key(r, c)},
// preserves each such comparison exactly: key(r, a) > key(r, b) implies that every k counted
// for b is also counted for a, and so is b itself, hence code(r, a) > code(r, b); equal keys
// count the same set.  Codes lie in [0, C-1], so for C <= 128 they fit in 7 bits of a byte and
// for C <= 1,024 in 15 bits of a 16-bit half-word (column-major [C][S], rows padded to one pass
// of the kernel with code 0, which never forms a trend).
//
// The evaluation kernel then reads one byte (or two) per row and column instead of four, and
// compares 4 (or 2) rows per 32-bit word with SIMD-within-a-register arithmetic: with the top bit
// of each field free,
//   ((cur | H) - (prev + ONE)) & H  has the top bit of a field set exactly where cur > prev
// (no field borrows: every field difference stays in [0, 2^b - 1]).  Per-row counts (at most
// 63) accumulate in the fields, and a field's count is >= t exactly where
// (count + 2^(b-1) - t) has its top bit set.
#include <algorithm>
#include <mutex>

#include "internal.h"
#include "items.cuh"
#include "tables.cuh"

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kRankRows = 32;                        // rows per rank-code tile
constexpr size_t kRankSmemMax = 1024 * kRankRows * 4;  // C <= 1,024
constexpr int kMaxDevices = 64;
constexpr int kVec = 1;  // 16-byte loads per lane and column in one pass

__device__ __forceinline__ int threshold(int L, int num, int den) {
  return (num * (L - 1) + den - 1) / den;
}

__device__ __forceinline__ void wait_prior_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------------------------- rank codes

// A block ranks 32 rows at a time: the rows' keys of every column are staged in shared memory
// as [C][32] (lane = row, so a warp's loads are conflict-free), and each thread ranks four
// columns of its row per sweep over the C keys.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_rank_codes(const uint32_t *__restrict__ keys,
                                                         int64_t R_pad, int32_t C, int64_t S,
                                                         T *__restrict__ codes) {
  extern __shared__ uint32_t s_k[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n_tiles = R_pad / kRankRows;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t r0 = tile * kRankRows;
    __syncthreads();  // the previous tile's keys are no longer read
    for (int c = warp; c < C; c += kWarps) s_k[c * kRankRows + lane] = keys[(int64_t)c * R_pad + r0 + lane];
    __syncthreads();
    for (int c0 = warp; c0 < C; c0 += 4 * kWarps) {
      uint32_t x[4];
      int n[4] = {0, 0, 0, 0};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = c0 + j * kWarps;
        x[j] = c < C ? s_k[c * kRankRows + lane] : 0u;
      }
#pragma unroll 4
      for (int k = 0; k < C; ++k) {
        const uint32_t v = s_k[k * kRankRows + lane];
#pragma unroll
        for (int j = 0; j < 4; ++j) n[j] += v < x[j];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = c0 + j * kWarps;
        if (c < C) codes[(int64_t)c * S + r0 + lane] = (T)n[j];
      }
    }
  }
}

// ------------------------------------------------------------------------------- evaluation

// W = bytes per code.  A pass covers 32 lanes x kVec 16-byte loads (16 / W rows each) per column.
// NS / LK: the pair-test variants of trend.cuh.  Each direction keeps a reference word: its
// fields hold the predecessor (or, with LK, the last value the direction kept) plus OFF for the
// upward test and with the top bit set for the downward one, so that
//   up:   ((cur | H) - up_ref) & H      down: (down_ref - (cur + OFF)) & H
// set a field's top bit where the pair holds (OFF = 1 per field for the strict tests, 0 for
// greater-or-equal / smaller-or-equal).  With LK a field's reference is replaced only where its
// test held.  With ties counting, the pad rows past R (code 0) would pass and are masked out.
// (Four blocks per SM: up to 64 registers, no spills; measured faster than five blocks of 48.)
template <int W, bool NEG, bool NS, bool LK>
__global__ void __launch_bounds__(kThreads, 4) k_eval_codes(EvalArgs a, PopView pv) {
  constexpr uint32_t H = W == 1 ? 0x80808080u : 0x80008000u;    // top bit of every field
  constexpr uint32_t ONE = W == 1 ? 0x01010101u : 0x00010001u;  // 1 in every field
  constexpr uint32_t OFF = NS ? 0u : ONE;
  constexpr uint32_t FMAX = W == 1 ? 0xFFu : 0xFFFFu;           // a full field
  constexpr int SH = W == 1 ? 7 : 15;
  constexpr int FW = 4 / W;                                     // fields per word
  constexpr int kRowsPerPass = 32 * 16 * kVec / W;
  constexpr int NW = 4 * kVec;  // 32-bit words per lane
  __shared__ int64_t s_base[kWarps][EBIC_MAX_LEN];
  wait_prior_grid();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t passes_total = a.S / kRowsPerPass;
  const int32_t n_side = items::move_chunks(a), n_all = n_side + pv.n * a.n_seg;
  // Items are taken segment-major (all individuals of a row segment before the next segment),
  // so the codes of the segment stay in L2 while every individual reads them.  (Fetching the
  // next item's index ahead of the current item's work measured slower.)
  for (int q = items::first(); q < n_all; q = items::next(a.work, lane, q, n_all)) {
    if (q < n_side) {
      if (items::stopped(pv)) return;  // a stopped run changes nothing
      items::move_chunk(a, q, lane);
      continue;
    }
    const int seg = (q - n_side) / pv.n, i = (q - n_side) - seg * pv.n;  // segment-major
    const items::Meta m = items::load_meta(pv, i, lane);
    if (items::stopped(pv)) return;  // (read with the item's loads; before any store)
    const int L = m.dead ? 0 : m.L;
    if (L >= 2) {
      const items::Insert ins = items::insert_start(pv, seg, m.h, lane);
      __syncwarp();
      s_base[warp][lane] = (int64_t)m.c0 * a.S * W;
      s_base[warp][lane + 32] = (int64_t)m.c1 * a.S * W;
      __syncwarp();
      const int t = threshold(L, a.rnum, a.rden);
      const uint32_t tadd = (uint32_t)((1 << SH) - t) * ONE;
      const int64_t p0 = (int64_t)seg * a.seg_passes;
      const int64_t p1 = min(p0 + a.seg_passes, passes_total);
      int cp = 0, cn = 0, ca = 0;
      for (int64_t pass = p0; pass < p1; ++pass) {
        // lane's 16-byte chunks: lane + 32 v for v < kVec (each warp load is contiguous)
        const uint8_t *base = a.codes + pass * (kRowsPerPass * W) + lane * 16;
        uint32_t dn_ref[NW], up_ref[NW], inc[NW], dec[NW];
#pragma unroll
        for (int v = 0; v < kVec; ++v) {
          const uint4 v0 = __ldg(reinterpret_cast<const uint4 *>(base + v * 512 + s_base[warp][0]));
          const uint32_t w0[4] = {v0.x, v0.y, v0.z, v0.w};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            dn_ref[4 * v + j] = w0[j] | H;
            up_ref[4 * v + j] = w0[j] + OFF;
            inc[4 * v + j] = 0u;
            dec[4 * v + j] = 0u;
          }
        }
#pragma unroll 8
        for (int k = 1; k < L; ++k) {
          uint32_t cur[NW];
#pragma unroll
          for (int v = 0; v < kVec; ++v) {
            const uint4 x = __ldg(reinterpret_cast<const uint4 *>(base + v * 512 + s_base[warp][k]));
            cur[4 * v] = x.x;
            cur[4 * v + 1] = x.y;
            cur[4 * v + 2] = x.z;
            cur[4 * v + 3] = x.w;
          }
#pragma unroll
          for (int j = 0; j < NW; ++j) {
            const uint32_t cH = cur[j] | H, cO = cur[j] + OFF;
            // (m >> SH) as the high word of m * 2^(32-SH): with the accumulate, one multiply-add
            // on the FMA pipe instead of a shift and an add on the integer ALU pipe, which this
            // loop otherwise saturates
            const uint32_t u1 = __umulhi((cH - up_ref[j]) & H, 1u << (32 - SH));
            inc[j] += u1;
            uint32_t d1 = 0u;
            if (NEG) {
              d1 = __umulhi((dn_ref[j] - cO) & H, 1u << (32 - SH));
              dec[j] += d1;
            }
            if (LK) {  // replace the reference only in the fields whose pair held
              const uint32_t fu = u1 * FMAX;
              up_ref[j] = (cO & fu) | (up_ref[j] & ~fu);
              if (NEG) {
                const uint32_t fd = d1 * FMAX;
                dn_ref[j] = (cH & fd) | (dn_ref[j] & ~fd);
              }
            } else {
              up_ref[j] = cO;
              dn_ref[j] = cH;
            }
          }
        }
        const bool tail = NS && (pass + 1) * kRowsPerPass > a.R;  // pass holds pad rows
#pragma unroll
        for (int j = 0; j < NW; ++j) {
          uint32_t po = (inc[j] + tadd) & H;
          uint32_t ne = NEG ? ((dec[j] + tadd) & H) : 0u;
          if (tail) {
            const int64_t row0 = pass * kRowsPerPass + ((j >> 2) * 512 + lane * 16 + 4 * (j & 3)) / W;
            uint32_t vm = 0u;
#pragma unroll
            for (int f = 0; f < FW; ++f)
              if (row0 + f < a.R) vm |= 1u << (8 * W * (f + 1) - 1);
            po &= vm;
            ne &= vm;
          }
          cp += __popc(po);
          if (NEG) {
            cn += __popc(ne);
            ca += __popc(po | ne);
          }
        }
      }
      if (!NEG) ca = cp;
      items::insert_finish(pv, ins, m.h, i);
      cp = __reduce_add_sync(kFull, cp);
      cn = __reduce_add_sync(kFull, cn);
      ca = __reduce_add_sync(kFull, ca);
      if (lane == 0) {
        if (cp) atomicAdd(a.rows_pos + i, cp);
        if (cn) atomicAdd(a.rows_neg + i, cn);
        if (ca) atomicAdd(a.rows_any + i, ca);
      }
    }
  }
}

template <class K>
int blocks_per_sm(K kern, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  return nb < 1 ? 1 : nb;
}

template <class... Args>
cudaError_t launch_pdl_opt(void (*kern)(Args...), dim3 grid, dim3 block, cudaStream_t s,
                           bool pdl, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

}  // namespace

int code_bytes_for(int32_t C) { return C <= 128 ? 1 : (C <= 1024 ? 2 : 0); }

int64_t code_rows_per_pass(int code_bytes) { return 32 * 16 * kVec / code_bytes; }

int64_t code_stride_for(int64_t R, int code_bytes) {
  const int64_t q = code_rows_per_pass(code_bytes);
  return (R + q - 1) / q * q;
}

cudaError_t launch_rank_codes(const uint32_t *keys, int64_t R_pad, int32_t C, void *codes,
                              int code_bytes, int64_t S, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(codes, 0, (size_t)C * S * code_bytes, s);
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)C * kRankRows * 4;
  if (smem > kRankSmemMax) return cudaErrorInvalidValue;
  // one fixed limit for every context (no call lowers another's), set once per device
  int dev = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  static std::mutex mu;
  static bool attr_set[kMaxDevices] = {};
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
      if ((e = cudaFuncSetAttribute(k_rank_codes<uint8_t>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kRankSmemMax)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(k_rank_codes<uint16_t>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kRankSmemMax)) != cudaSuccess)
        return e;
      attr_set[dev] = true;
    }
  }
  const int64_t n_tiles = R_pad / kRankRows;
  if (code_bytes == 1) {
    const int64_t grid = std::min<int64_t>(n_tiles, (int64_t)num_sms * blocks_per_sm(k_rank_codes<uint8_t>, smem));
    k_rank_codes<uint8_t><<<(unsigned)grid, kThreads, smem, s>>>(keys, R_pad, C, S,
                                                                 static_cast<uint8_t *>(codes));
  } else {
    const int64_t grid = std::min<int64_t>(n_tiles, (int64_t)num_sms * blocks_per_sm(k_rank_codes<uint16_t>, smem));
    k_rank_codes<uint16_t><<<(unsigned)grid, kThreads, smem, s>>>(keys, R_pad, C, S,
                                                                  static_cast<uint16_t *>(codes));
  }
  return cudaGetLastError();
}

cudaError_t launch_eval_codes(const EvalArgs &a0, const PopView &pv, int num_sms, cudaStream_t s,
                              bool pdl) {
  if (pv.n <= 0) return cudaSuccess;
  EvalArgs a = a0;
  const int W = a.code_bytes;
  const int64_t passes_total = a.S / code_rows_per_pass(W);
  using Kernel = void (*)(EvalArgs, PopView);
  static const Kernel table[16] = {
      k_eval_codes<1, false, false, false>, k_eval_codes<1, false, false, true>,
      k_eval_codes<1, false, true, false>,  k_eval_codes<1, false, true, true>,
      k_eval_codes<1, true, false, false>,  k_eval_codes<1, true, false, true>,
      k_eval_codes<1, true, true, false>,   k_eval_codes<1, true, true, true>,
      k_eval_codes<2, false, false, false>, k_eval_codes<2, false, false, true>,
      k_eval_codes<2, false, true, false>,  k_eval_codes<2, false, true, true>,
      k_eval_codes<2, true, false, false>,  k_eval_codes<2, true, false, true>,
      k_eval_codes<2, true, true, false>,   k_eval_codes<2, true, true, true>};
  const Kernel kern = table[(W == 2 ? 8 : 0) + (a.neg ? 4 : 0) + (a.non_strict ? 2 : 0) +
                            (a.last_kept ? 1 : 0)];
  const int bps = blocks_per_sm(kern, 0);
  const int64_t warps = (int64_t)num_sms * bps * kWarps;
  // Segments: the autotuner's size when it set one, else enough work items for ~8 per
  // resident warp; at most 2^30 items in total.
  int64_t seg = a0.seg_passes > 0 ? a0.seg_passes : ((int64_t)pv.n * passes_total) / (8 * warps);
  if (seg < 1) seg = 1;
  if (seg > passes_total) seg = passes_total;
  int64_t n_seg = (passes_total + seg - 1) / seg;
  while ((int64_t)pv.n * n_seg > (1LL << 30)) {
    seg *= 2;
    n_seg = (passes_total + seg - 1) / seg;
  }
  a.seg_passes = (int32_t)seg;
  a.n_seg = (int32_t)n_seg;
  // (the side task's chunks count too: with a warp for every item they run beside the others)
  const int64_t items = (int64_t)pv.n * n_seg + (a.mv_table ? (a.mv_n + 31) / 32 : 0);
  int64_t grid = (int64_t)num_sms * bps;
  const int64_t need = (items + kWarps - 1) / kWarps;
  if (grid > need) grid = need;
  return launch_pdl_opt(kern, dim3((unsigned)grid), dim3(kThreads), s, pdl, a, pv);
}
