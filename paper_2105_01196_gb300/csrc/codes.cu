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
constexpr int kMaxDevices = 64;
constexpr int kVec = 1;  // 16-byte loads per lane and column in one pass

__device__ __forceinline__ int threshold(int L, int num, int den) {
  return (num * (L - 1) + den - 1) / den;
}

__device__ __forceinline__ void wait_prior_grid() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ------------------------------------------------------------------------------- rank codes

// One warp ranks one row at a time.  Its C keys (padded with 0xFFFFFFFF, above every key of a
// finite value, to N = 32 * EPL) are sorted ascending in registers, sorted position
// e = lane * EPL + j in register j of `lane`, by a bitonic network in the form whose every
// compare-exchange sends the minimum to the lower position: each merge phase of size k starts by
// comparing e with its mirror e ^ (k - 1) in the k-block, then halves the distance.  Exchanges
// at distance < EPL stay inside a lane; the others pair lanes through one shuffle.  The sorted
// row goes to shared memory and the rank of each key is the number of sorted keys below it,
// found by a branchless binary search (equal keys get equal codes, as the definition requires).
// A block owns 16 consecutive rows: their keys are staged column by column with coalesced loads
// in a shared [C][17] tile, each row's codes replace its keys in the tile, and the tile is
// written out column by column (codes [C][S]) together with the codes' bit planes: plane p of
// column c, word w has bit j = bit p of code(32 w + j, c), the operand of the pair-bitmap build
// (matrix.cu), stored [C][Wst][NBP] (a word's nb planes together, NBP = nb rounded up to a
// multiple of 4, so that they load as 16-byte vectors); a block fills one half of each word.
constexpr int kRankRows = 16;                 // rows per block tile
constexpr int kTileStride = kRankRows + 1;    // tile entries per column (bank spread)

template <int EPL>
__device__ __forceinline__ void bitonic_sort_row(uint32_t (&v)[EPL], int lane) {
  constexpr int LOG_EPL = EPL == 1 ? 0 : EPL == 2 ? 1 : EPL == 4 ? 2 : EPL == 8 ? 3 : EPL == 16 ? 4 : 5;
  constexpr int LOG_N = LOG_EPL + 5;
#pragma unroll
  for (int lk = 1; lk <= LOG_N; ++lk) {
    const int k = 1 << lk;  // size of the blocks merged in this phase
    if (k <= EPL) {         // mirror exchange inside the lane
#pragma unroll
      for (int j = 0; j < EPL; ++j) {
        const int jp = j ^ (k - 1);
        if ((j & (k >> 1)) == 0) {
          const uint32_t lo = min(v[j], v[jp]), hi = max(v[j], v[jp]);
          v[j] = lo;
          v[jp] = hi;
        }
      }
    } else {  // mirror exchange with lane ^ (k / EPL - 1), register EPL - 1 - j
      const int m = k / EPL - 1;
      const bool upper = (lane & (k / (2 * EPL))) != 0;
#pragma unroll
      for (int j = 0; j < EPL / 2 + (EPL == 1); ++j) {
        const int jm = EPL - 1 - j;
        const uint32_t oa = __shfl_xor_sync(kFull, v[jm], m);
        const uint32_t ob = __shfl_xor_sync(kFull, v[j], m);
        v[j] = upper ? max(v[j], oa) : min(v[j], oa);
        if (jm != j) v[jm] = upper ? max(v[jm], ob) : min(v[jm], ob);
      }
    }
#pragma unroll
    for (int ls = lk - 2; ls >= 0; --ls) {
      const int st = 1 << ls;  // half-cleaner distance
      if (st < EPL) {
#pragma unroll
        for (int j = 0; j < EPL; ++j) {
          if ((j & st) == 0) {
            const int jp = j ^ st;
            const uint32_t lo = min(v[j], v[jp]), hi = max(v[j], v[jp]);
            v[j] = lo;
            v[jp] = hi;
          }
        }
      } else {
        const int ld = st / EPL;
        const bool upper = (lane & ld) != 0;
#pragma unroll
        for (int j = 0; j < EPL; ++j) {
          const uint32_t o = __shfl_xor_sync(kFull, v[j], ld);
          v[j] = upper ? max(v[j], o) : min(v[j], o);
        }
      }
    }
  }
}

// Sorted position e sits at e + e / 32 in a warp's shared buffer (one pad word per 32: the
// stores of positions lane * EPL + j from every lane fall in distinct banks).
__device__ __forceinline__ int sorted_slot(int e) { return e + (e >> 5); }

// #{sorted keys < q} over N sorted keys (N a power of two), walking the padded positions: from a
// multiple of 32 a step s >= 32 tests element pos + s - 1 at padded offset s + s/32 - 2 and
// moves by s + s/32; smaller steps stay inside one 32-block.
template <int N>
__device__ __forceinline__ int count_below(const uint32_t *srt, uint32_t q) {
  const uint32_t *p = srt;
#pragma unroll
  for (int step = N / 2; step >= 1; step >>= 1) {
    const int d = step >= 32 ? step + step / 32 : step;
    const int t = step >= 32 ? d - 2 : d - 1;
    if (p[t] < q) p += d;
  }
  if (*p < q) ++p;
  const int pp = (int)(p - srt);
  return pp - pp / 33;
}

// T: code type (uint8_t for C <= 128, uint16_t for C <= 1,024); EPL: keys per lane
// (32 * EPL >= C).  planes may be null (no bit planes wanted); nb planes per column.
template <typename T, int EPL>
__global__ void __launch_bounds__(kThreads, 2)
    k_rank_codes(const uint32_t *__restrict__ keys, int64_t R_pad, int32_t C, int64_t S,
                 T *__restrict__ codes, uint32_t *__restrict__ planes, int64_t Wst, int nb,
                 int64_t t_begin, int64_t t_end) {
  constexpr int N = 32 * EPL;
  constexpr int kSorted = N + N / 32;  // words of one warp's sorted buffer
  extern __shared__ __align__(16) uint32_t s_rank[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *srt = s_rank + warp * kSorted;
  uint32_t *tile = s_rank + kWarps * kSorted;  // [C][kTileStride]: keys, then codes in place
  uint16_t *planes16 = reinterpret_cast<uint16_t *>(planes);
  const int nbp = (nb + 3) & ~3;  // planes per (column, word) in the layout
  // (tiles [t_begin, t_end) of the R_pad / kRankRows)
  for (int64_t t = t_begin + blockIdx.x; t < t_end; t += gridDim.x) {
    const int64_t r0 = t * kRankRows;
    for (int i = threadIdx.x; i < C * kRankRows; i += kThreads) {
      const int c = i / kRankRows, rho = i % kRankRows;
      tile[c * kTileStride + rho] = __ldg(keys + (int64_t)c * R_pad + r0 + rho);
    }
    __syncthreads();
    for (int rho = warp; rho < kRankRows; rho += kWarps) {
      uint32_t v[EPL];
#pragma unroll
      for (int j = 0; j < EPL; ++j) {
        const int c = j * 32 + lane;  // (any placement of the keys before sorting will do)
        v[j] = c < C ? tile[c * kTileStride + rho] : 0xFFFFFFFFu;
      }
      bitonic_sort_row<EPL>(v, lane);
      __syncwarp();  // the previous row's searches are done with the buffer
#pragma unroll
      for (int j = 0; j < EPL; ++j) srt[sorted_slot(lane * EPL + j)] = v[j];
      __syncwarp();
#pragma unroll
      for (int j = 0; j < EPL; ++j) {
        const int c = j * 32 + lane;  // (this row's slot of column c: only this warp's)
        if (c < C) tile[c * kTileStride + rho] = (uint32_t)count_below<N>(srt, tile[c * kTileStride + rho]);
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < C * kRankRows; i += kThreads) {
      const int c = i / kRankRows, rho = i % kRankRows;
      codes[(int64_t)c * S + r0 + rho] = (T)tile[c * kTileStride + rho];
    }
    if (planes) {
      // two columns per warp step: lanes 0-15 hold column c's 16 rows, lanes 16-31 column c + 1's
      const int64_t w = r0 / 32, half = (r0 / kRankRows) & 1;
      const int sub = lane >> 4;
      for (int c2 = 2 * warp; c2 < C; c2 += 2 * kWarps) {
        const int c = c2 + sub;
        const uint32_t code = c < C ? tile[c * kTileStride + (lane & 15)] : 0u;
        uint32_t mine = 0;
        for (int p = 0; p < nb; ++p) {
          const uint32_t bits = __ballot_sync(kFull, (code >> p) & 1u);
          if ((lane & 15) == p) mine = sub ? (bits >> 16) : (bits & 0xFFFFu);
        }
        const int p = lane & 15;
        if (p < nb && c < C)
          planes16[2 * (((int64_t)c * Wst + w) * nbp + p) + half] = (uint16_t)mine;
      }
    }
    __syncthreads();  // the tile is read before the next rows overwrite it
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

int code_plane_bits(int32_t C) {
  int nb = 1;
  while ((1 << nb) < C) ++nb;  // codes lie in [0, C - 1]
  return nb;
}

int code_plane_stride(int nb) { return (nb + 3) & ~3; }

namespace {

template <typename T, int EPL>
cudaError_t launch_rank_epl(const uint32_t *keys, int64_t R_pad, int32_t C, T *codes, int64_t S,
                            uint32_t *planes, int64_t Wst, int nb, int num_sms, cudaStream_t s,
                            int64_t r_begin, int64_t r_end) {
  constexpr int N = 32 * EPL;
  const size_t smem = (size_t)kWarps * (N + N / 32) * 4 + (size_t)C * kTileStride * 4;
  // one fixed limit for every context (no call lowers another's), set once per device
  constexpr size_t kLimit = (size_t)kWarps * (1024 + 32) * 4 + (size_t)1024 * kTileStride * 4;
  static_assert(kLimit <= 227 * 1024, "rank-code shared memory");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static bool attr_set[kMaxDevices] = {};
  {
    std::lock_guard<std::mutex> lock(mu);
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
      if ((e = cudaFuncSetAttribute(k_rank_codes<T, EPL>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kLimit)) !=
          cudaSuccess)
        return e;
      attr_set[dev] = true;
    }
  }
  const int64_t t_begin = r_begin / kRankRows, t_end = r_end / kRankRows;
  const int64_t grid = std::min<int64_t>(
      t_end - t_begin, (int64_t)num_sms * blocks_per_sm(k_rank_codes<T, EPL>, smem));
  k_rank_codes<T, EPL><<<(unsigned)grid, kThreads, smem, s>>>(keys, R_pad, C, S, codes, planes,
                                                                Wst, nb, t_begin, t_end);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_rank_codes_rows(const uint32_t *keys, int64_t R_pad, int32_t C, void *codes,
                                   int code_bytes, int64_t S, uint32_t *planes, int64_t Wst,
                                   int num_sms, int64_t r_begin, int64_t r_end, cudaStream_t s) {
  if (C > 1024 || code_bytes != (C <= 128 ? 1 : 2)) return cudaErrorInvalidValue;
  if (r_begin < 0 || r_begin % kRankRows || r_end > R_pad || r_end % kRankRows ||
      r_end <= r_begin)
    return cudaErrorInvalidValue;
  const int nb = code_plane_bits(C);
#define EBIC_RANK(T, EPL, cd) \
  launch_rank_epl<T, EPL>(keys, R_pad, C, cd, S, planes, Wst, nb, num_sms, s, r_begin, r_end)
  if (code_bytes == 1) {
    uint8_t *cd = static_cast<uint8_t *>(codes);
    return C <= 32 ? EBIC_RANK(uint8_t, 1, cd) : C <= 64 ? EBIC_RANK(uint8_t, 2, cd)
                                                         : EBIC_RANK(uint8_t, 4, cd);
  }
  uint16_t *cd = static_cast<uint16_t *>(codes);
  return C <= 256 ? EBIC_RANK(uint16_t, 8, cd) : C <= 512 ? EBIC_RANK(uint16_t, 16, cd)
                                                          : EBIC_RANK(uint16_t, 32, cd);
#undef EBIC_RANK
}

cudaError_t launch_rank_codes(const uint32_t *keys, int64_t R_pad, int32_t C, void *codes,
                              int code_bytes, int64_t S, uint32_t *planes, int64_t Wst,
                              int num_sms, cudaStream_t s) {
  // (the rows of the code columns past R_pad, up to S, stay zero)
  cudaError_t e = cudaMemsetAsync(codes, 0, (size_t)C * S * code_bytes, s);
  if (e != cudaSuccess) return e;
  return launch_rank_codes_rows(keys, R_pad, C, codes, code_bytes, S, planes, Wst, num_sms, 0,
                                R_pad, s);
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
