// Matrix upload (order keys, column-major) and the column-pair comparison bitmap.
//
// Order key: the float32 bit pattern u, with -0 mapped to +0, becomes
//   k(u) = u ^ 0xFFFFFFFF for negative values, u | 0x80000000 otherwise,
// an increasing map of the finite floats onto uint32, so `k(a) > k(b)` is exactly `a > b`
// (ties, including -0 against +0, compare equal) whatever the FTZ/DAZ mode of the arithmetic.
// The trend definition the keys serve is Sec. 2.3 ("EBIC" paragraph) of the EBIC.jl paper.
#include <algorithm>

#include "internal.h"

namespace {

constexpr uint32_t kSign = 0x80000000u;
constexpr uint32_t kExpMask = 0x7F800000u;

__device__ __forceinline__ uint32_t order_key(uint32_t u) {
  if (u == kSign) u = 0u;
  return (u & kSign) ? ~u : (u | kSign);
}

__device__ __forceinline__ bool not_finite(uint32_t u) { return (u & kExpMask) == kExpMask; }

// Row-major x[R][C] -> keys[C][R_pad] through a 32x32 shared-memory tile (coalesced on both
// sides).  Rows in [R, R_pad) get key 0, which never compares greater than anything.
// (rows [r_begin, r_end) of the R_pad: block x covers rows r_begin + 32 x ..)
__global__ void k_upload_rowmajor(const float *__restrict__ x, int64_t R, int32_t C,
                                  int64_t R_pad, uint32_t *__restrict__ keys,
                                  int32_t *__restrict__ err, int64_t r_begin, int64_t r_end) {
  __shared__ uint32_t tile[32][33];
  const int64_t r0 = r_begin + (int64_t)blockIdx.x * 32;
  const int32_t c0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;
  bool bad = false;
#pragma unroll
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + j;
    const int32_t c = c0 + tx;
    uint32_t k = 0u;
    if (r < R && c < C) {
      const uint32_t u = __float_as_uint(__ldg(x + r * C + c));
      bad |= not_finite(u);
      k = order_key(u);
    }
    tile[j][tx] = k;
  }
  if (__any_sync(0xFFFFFFFFu, bad) && (tx == 0)) atomicOr(err, 1);
  __syncthreads();
#pragma unroll
  for (int j = ty; j < 32; j += 8) {
    const int32_t c = c0 + j;
    const int64_t r = r0 + tx;
    if (c < C && r < r_end) keys[(int64_t)c * R_pad + r] = tile[tx][j];
  }
}

// Column-major x[C][R] -> keys[C][R_pad], one element per thread, grid-stride.
__global__ void k_upload_colmajor(const float *__restrict__ x, int64_t R, int32_t C,
                                  int64_t R_pad, uint32_t *__restrict__ keys,
                                  int32_t *__restrict__ err) {
  const int64_t total = (int64_t)C * R_pad;
  bool bad = false;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = q / R_pad, r = q - c * R_pad;
    uint32_t k = 0u;
    if (r < R) {
      const uint32_t u = __float_as_uint(__ldg(x + c * R + r));
      bad |= not_finite(u);
      k = order_key(u);
    }
    keys[q] = k;
  }
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, 1);
}

// Pair bitmap: G[(a*C + b)*Wst + w] bit j = [key(32w+j, b) > key(32w+j, a)].
// A block covers 32 words (1024 rows) of kBW columns a (one per warp, its 1024 keys held in
// registers).  Each unordered pair a < b is compared once: the ballot of kb > ka gives G[a][b]
// and the ballot of kb < ka gives G[b][a] (ties set neither).  The b-columns of the chunk stream
// through a double-buffered shared-memory stage filled with cp.async, so their loads overlap
// the ballots; lane 0 parks the 32 ballots of a pair in shared memory and the warp then writes
// them as two coalesced 128-byte rows.  With few (chunk, a-block) pairs (small matrices), the
// stages of b-columns are also split across blockIdx.z (stage st goes to z = st mod gridDim.z),
// so the launch still fills the GPU and the long first a-blocks share their work.
constexpr int kBW = 8;  // warps (a-columns) per block
constexpr int kBS = 4;  // b-columns per stage

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__global__ void __launch_bounds__(kBW * 32, 4) k_build_bitmap(const uint32_t *__restrict__ keys,
                                                              int64_t R_pad, int32_t C,
                                                              int64_t Wst,
                                                              uint32_t *__restrict__ G) {
  __shared__ __align__(16) uint32_t sb[2][kBS][1024];
  __shared__ uint32_t s_out[kBW][2][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t w0 = (int64_t)blockIdx.x * 32;
  const int nw = (int)((Wst - w0 < 32) ? (Wst - w0) : 32);  // words of this chunk
  const int a0 = blockIdx.y * kBW;
  const int a = a0 + warp;
  const bool a_ok = a < C;
  uint32_t ka[32];
#pragma unroll
  for (int j = 0; j < 32; ++j)
    ka[j] = (a_ok && j < nw) ? __ldg(keys + (int64_t)a * R_pad + (w0 + j) * 32 + lane) : 0u;
  if (a_ok && lane < nw && blockIdx.z == 0) G[((int64_t)a * C + a) * Wst + w0 + lane] = 0u;
  const int bstart = a0 + 1;
  const int nstages = bstart < C ? (C - bstart + kBS - 1) / kBS : 0;
  const int S = (int)gridDim.z, z = (int)blockIdx.z;
  const int my_stages = nstages > z ? (nstages - z + S - 1) / S : 0;  // stages z, z + S, ...
  const int pieces = nw * 8;  // 16-byte pieces of one column's chunk
  auto issue = [&](int st, int buf) {
    const int b0 = bstart + st * kBS;
    for (int i = threadIdx.x; i < kBS * pieces; i += blockDim.x) {
      const int bb = i / pieces, piece = i - bb * pieces;
      const int b = b0 + bb;
      if (b < C)
        cp_async16(&sb[buf][bb][piece * 4], keys + (int64_t)b * R_pad + w0 * 32 + piece * 4);
    }
    cp_commit();
  };
  if (my_stages > 0) issue(z, 0);
  for (int k = 0; k < my_stages; ++k) {
    const int st = z + k * S;
    if (k + 1 < my_stages) {
      issue(st + S, (k + 1) & 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    const int buf = k & 1, b0 = bstart + st * kBS;
    if (a_ok) {
      for (int bb = 0; bb < kBS; ++bb) {
        const int b = b0 + bb;
        if (b >= C) break;
        if (b <= a) continue;
        const uint32_t *col = sb[buf][bb];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const uint32_t kb = col[j * 32 + lane];
          const uint32_t gt = __ballot_sync(0xFFFFFFFFu, kb > ka[j]);
          const uint32_t lt = __ballot_sync(0xFFFFFFFFu, kb < ka[j]);
          if (lane == 0) {
            s_out[warp][0][j] = gt;
            s_out[warp][1][j] = lt;
          }
        }
        __syncwarp();
        if (lane < nw) {
          G[((int64_t)a * C + b) * Wst + w0 + lane] = s_out[warp][0][lane];
          G[((int64_t)b * C + a) * Wst + w0 + lane] = s_out[warp][1][lane];
        }
        __syncwarp();
      }
    }
    __syncthreads();  // this buffer is consumed before it is refilled
  }
}

// Pair bitmap from the bit planes of the per-row rank codes (codes.cu): comparing codes is
// comparing keys (the codes keep every within-row order), and a word of planes holds one bit of
// 32 rows' codes, so one lane compares 32 rows at once.  Going from the lowest plane to the
// highest, with A and B the planes of columns a and b,
//   gt = (B & ~A) | (~(A ^ B) & gt)      lt = (A & ~B) | (~(A ^ B) & lt)
// (each one three-input logic instruction, lop3 with truth tables 0x8E and 0xB2) leave
// gt = [code_b > code_a] = G[a][b] and lt = [code_a > code_b] = G[b][a] in every bit: a higher
// differing bit overrides the lower ones, equal bits keep them.  Ties and pad rows (code 0
// everywhere) set neither.
// A warp owns four a-columns (their planes in registers) and one 32-word chunk of rows (a word
// per lane, so every store is one coalesced 128-byte row piece), and walks b over a piece of at
// most kPiece columns after its own; the b planes of a block's eight warps come through L1.
// The b-range of an a-block is cut into pieces so that every block has about the same work
// (the first a-blocks pair with many more columns than the last ones).  The row chunk is the
// fastest block index, so the blocks resident together write adjacent 128-byte pieces of the
// same pair rows, which L2 then merges into whole sectors before they reach DRAM.  Piece p of
// a-block g starts at column 32 (g + 4 p); the pieces run in the order of that start (then of
// g), so the blocks in flight together read the same b planes, which stay in L2 between them.
constexpr int kPA = 4;       // a-columns per warp
constexpr int kPiece = 128;  // b-columns per block (at most)
constexpr int kMaxABlocks = 32;  // a-blocks of 32 columns: C <= 1,024
constexpr int kMaxPieces = kMaxABlocks * (1024 / kPiece);

struct PieceTable {
  uint16_t item[kMaxPieces];  // piece y of the launch: a-block << 8 | piece within the a-block
};

template <int LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}

template <int NB>
__device__ __forceinline__ void plane_compare(const uint32_t (&A)[NB], const uint32_t (&B)[NB],
                                              uint32_t &gt, uint32_t &lt) {
  gt = 0u;
  lt = 0u;
#pragma unroll
  for (int p = 0; p < NB; ++p) {
    gt = lop3<0x8E>(A[p], B[p], gt);  // (B & ~A) | (~(A ^ B) & gt)
    lt = lop3<0xB2>(A[p], B[p], lt);  // (A & ~B) | (~(A ^ B) & lt)
  }
}

constexpr int kBB = 16;  // b-columns per staged batch (48 KB of static shared memory at NB = 10)

__device__ __forceinline__ void cp_async16_bm(void *smem, const void *gmem) {
  const unsigned saddr = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit_bm() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_wait_bm() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The b planes of a block's piece are staged in shared memory, kBB columns at a time and
// double-buffered (cp.async by the whole block; the next batch is in flight while the current
// one is compared), so the eight warps share one copy and read it with constant offsets.  The
// planes are stored [C][Wst][NBP] (NBP = NB rounded up to 4): a column's chunk of 32 words is
// one contiguous span, copied as is, and each lane reads its word's planes as NBP / 4 16-byte
// vectors (lanes 48 or 16 bytes apart: no bank conflicts; 32 bytes apart at NBP = 8: two-way).
// The pair counts are accumulated too (cnt, zeroed beforehand): for a < b, cnt[a * C + b] holds
// the rows of G[a][b] (its popcount) in its low 32 bits and those of G[b][a] in its high 32
// bits.  Each warp adds its 32 words' counts of a pair by one warp sum (the two directions'
// counts packed in 16-bit halves, at most 1,024 each) and one 64-bit atomic.
// In the last row chunk, lanes past Wst hold zero planes for a (not loaded) and for b (their
// staged words are zeroed once and never copied): every such row compares equal, so their words
// are zero (and not stored) and add nothing to the sums.
template <int NB>
__global__ void __launch_bounds__(256, 2) k_build_bitmap_planes(const uint32_t *__restrict__ planes,
                                                             int32_t C, int64_t Wst,
                                                             PieceTable tab,
                                                             uint32_t *__restrict__ G,
                                                             unsigned long long *__restrict__ cnt,
                                                             int64_t chunk0) {
  constexpr int NBP = (NB + 3) & ~3;
  __shared__ __align__(16) uint32_t s_b[2][kBB][32][NBP];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // this block's a-block and piece (blockIdx.x is the row chunk: the blocks running together
  // write neighbouring pieces of the same pair rows)
  const int item = tab.item[blockIdx.y];
  const int ablk = item >> 8, piece = item & 0xFF;
  const int64_t w0 = (chunk0 + (int64_t)blockIdx.x) * 32, w = w0 + lane;
  const bool w_ok = w < Wst;
  const int a0 = (ablk * 8 + warp) * kPA;
  const int b_lo = ablk * 8 * kPA + piece * kPiece;  // the piece's b-range
  const int b_hi = min(C, b_lo + kPiece);
  const int b_first = max(b_lo, ablk * 8 * kPA + kPA);  // the first b any warp of the block needs
  uint32_t A[kPA][NB];
#pragma unroll
  for (int i = 0; i < kPA; ++i) {
    const bool on = a0 + i < C && w_ok;
    const uint4 *src = reinterpret_cast<const uint4 *>(planes + ((int64_t)(a0 + i) * Wst + w) * NBP);
#pragma unroll
    for (int q = 0; q < NBP / 4; ++q) {
      const uint4 v = on ? __ldg(src + q) : make_uint4(0u, 0u, 0u, 0u);
      const uint32_t e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (4 * q + k < NB) A[i][4 * q + k] = e[k];
    }
  }
  const int64_t row = (int64_t)C * Wst;  // words between G[a][.] and G[a + 1][.]
  // this warp's 32 words' counts of G[a][b] (gt) and G[b][a] (lt), packed, summed over the lanes
  auto warp_counts = [&](uint32_t gt, uint32_t lt) -> unsigned {
    return __reduce_add_sync(0xFFFFFFFFu, (unsigned)__popc(gt) + ((unsigned)__popc(lt) << 16));
  };
  auto add_counts = [&](int a, int b, unsigned n) {  // (a < b)
    if (n)
      atomicAdd(cnt + (int64_t)a * C + b,
                (unsigned long long)(n & 0xFFFFu) | ((unsigned long long)(n >> 16) << 32));
  };
  if (piece == 0 && a0 < C) {
    // the diagonal words, and the pairs among the warp's own columns
#pragma unroll
    for (int i = 0; i < kPA; ++i) {
      const int a = a0 + i;
      if (a >= C) break;
      if (w_ok) G[(int64_t)a * row + (int64_t)a * Wst + w] = 0u;
#pragma unroll
      for (int i2 = i + 1; i2 < kPA; ++i2) {
        const int b = a0 + i2;
        if (b < C) {
          uint32_t gt, lt;
          plane_compare<NB>(A[i], A[i2], gt, lt);
          if (w_ok) {
            __stcs(G + (int64_t)a * row + (int64_t)b * Wst + w, gt);
            __stcs(G + (int64_t)b * row + (int64_t)a * Wst + w, lt);
          }
          const unsigned n = warp_counts(gt, lt);
          if (lane == 0) add_counts(a, b, n);
        }
      }
    }
  }
  if (b_first >= b_hi) return;  // (the whole block: no b beyond its columns in this piece)
  // staging: batch t holds b = b_first + t kBB + bb; copy j of a batch is 16-byte part j % span
  // of column bb = j / span (span: the chunk's words x NBP / 4; Wst % 4 == 0)
  const int n_batches = (b_hi - b_first + kBB - 1) / kBB;
  const int valid = (int)(Wst - w0 >= 32 ? 32 : Wst - w0);  // words of this chunk
  const int span = valid * NBP / 4;
  if (valid < 32) {  // the tail lanes' staged words, in both buffers
    for (int j = threadIdx.x; j < 2 * kBB * (32 - valid) * NBP; j += blockDim.x) {
      const int k = j % NBP, l = valid + (j / NBP) % (32 - valid), bb = j / (NBP * (32 - valid));
      (&s_b[0][0][0][0])[((int64_t)bb * 32 + l) * NBP + k] = 0u;
    }
  }
  auto issue = [&](int t) {
    const int bs = b_first + t * kBB, nbb = min(kBB, b_hi - bs);
    for (int j = threadIdx.x; j < nbb * span; j += blockDim.x) {
      const int bb = j / span, part = j - bb * span;
      cp_async16_bm(&s_b[t & 1][bb][0][0] + part * 4,
                    planes + ((int64_t)(bs + bb) * Wst + w0) * NBP + part * 4);
    }
    cp_commit_bm();
  };
  // G[a][b] at a * row + b * Wst, G[b][a] at b * row + a * Wst; (a + i)'s words sit i rows (or
  // i * Wst words) past a's: 32-bit offsets from two pointers
  const uint32_t row32 = (uint32_t)row, wst32 = (uint32_t)Wst;  // (checked at launch)
  const bool active = a0 < C;  // (the whole warp; lanes past Wst store nothing)
  issue(0);
  for (int t = 0; t < n_batches; ++t) {
    if (t + 1 < n_batches) {
      issue(t + 1);
      cp_wait_bm<1>();
    } else {
      cp_wait_bm<0>();
    }
    __syncthreads();  // batch t is in shared memory for every warp
    const int bs = b_first + t * kBB, nbb = min(kBB, b_hi - bs);
    const int bb0 = max(0, a0 + kPA - bs);  // the first b after the warp's own columns
    if (active && bb0 < nbb) {
      uint32_t *g_ab = G + (int64_t)a0 * row + (int64_t)(bs + bb0) * Wst + w;
      uint32_t *g_ba = G + (int64_t)(bs + bb0) * row + (int64_t)a0 * Wst + w;
      // (b columns are independent: unrolled, their comparator chains interleave; the build at
      // 60,000 x 1,000 took 2.00 ms unrolled 4 times, 2.21-2.22 ms 1 or 2 times, 2.21 ms 8 times,
      // 2.17 ms 16 times; with a test of b against the warp's columns inside the loop, a select of
      // the tail lanes' counts and the counts optional, 2.33 ms rolled and 2.18 ms at best)
#pragma unroll 4
      for (int bb = bb0; bb < nbb; ++bb) {
        uint32_t B[NB];
#pragma unroll
        for (int q = 0; q < NBP / 4; ++q) {
          const uint4 v = *reinterpret_cast<const uint4 *>(&s_b[t & 1][bb][lane][4 * q]);
          const uint32_t e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int k = 0; k < 4; ++k)
            if (4 * q + k < NB) B[4 * q + k] = e[k];
        }
        unsigned n[kPA];
#pragma unroll
        for (int i = 0; i < kPA; ++i) {
          uint32_t gt, lt;
          plane_compare<NB>(A[i], B, gt, lt);
          if (w_ok) {
            __stcs(g_ab + (uint32_t)i * row32, gt);
            __stcs(g_ba + (uint32_t)i * wst32, lt);
          }
          n[i] = warp_counts(gt, lt);
        }
        if (lane < kPA) {  // lane i adds pair (a0 + i, b)'s counts
          unsigned mine = n[0];
#pragma unroll
          for (int i = 1; i < kPA; ++i) mine = lane == i ? n[i] : mine;
          add_counts(a0 + lane, bs + bb, mine);
        }
        g_ab += Wst;
        g_ba += row;
      }
    }
    __syncthreads();  // every warp is done with this buffer before batch t + 2 refills it
  }
}

}  // namespace

cudaError_t launch_upload_rows(const float *x, int64_t R, int32_t C, int64_t R_pad,
                               uint32_t *keys, int32_t *err, int64_t r_begin, int64_t r_end,
                               cudaStream_t s) {
  if (r_begin < 0 || r_begin % 32 || r_end > R_pad || r_end % 32 || r_end <= r_begin)
    return cudaErrorInvalidValue;
  dim3 grid((unsigned)((r_end - r_begin) / 32), (unsigned)((C + 31) / 32));
  k_upload_rowmajor<<<grid, dim3(32, 8), 0, s>>>(x, R, C, R_pad, keys, err, r_begin, r_end);
  return cudaGetLastError();
}

cudaError_t launch_upload(const float *x, int64_t R, int32_t C, int64_t R_pad, int32_t layout,
                          uint32_t *keys, int32_t *err, cudaStream_t s) {
  if (layout == EBIC_LAYOUT_ROW_MAJOR) {
    return launch_upload_rows(x, R, C, R_pad, keys, err, 0, R_pad, s);
  } else {
    const int64_t total = (int64_t)C * R_pad;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_upload_colmajor<<<(unsigned)blocks, 256, 0, s>>>(x, R, C, R_pad, keys, err);
  }
  return cudaGetLastError();
}

cudaError_t launch_build_bitmap(const uint32_t *keys, int64_t R_pad, int32_t C, int64_t Wst,
                                uint32_t *bitmap, cudaStream_t s) {
  const int64_t gx = (Wst + 31) / 32, gy = (C + kBW - 1) / kBW;
  // enough blocks for about four per SM, split over the b-stages of the first a-block at most
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 1;
  }
  const int64_t max_split = std::max<int64_t>(1, (C - 1 + kBS - 1) / kBS);
  const int64_t split =
      std::min<int64_t>(max_split, std::max<int64_t>(1, (4LL * sms + gx * gy - 1) / (gx * gy)));
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)std::min<int64_t>(split, 65535));
  k_build_bitmap<<<grid, kBW * 32, 0, s>>>(keys, R_pad, C, Wst, bitmap);
  return cudaGetLastError();
}

cudaError_t launch_build_bitmap_planes(const uint32_t *planes, int nb, int32_t C, int64_t Wst,
                                       uint32_t *bitmap, unsigned long long *cnt,
                                       cudaStream_t s, int64_t chunk0, int64_t chunk1) {
  const int64_t n_all = (Wst + 31) / 32;
  if (chunk1 < 0 || chunk1 > n_all) chunk1 = n_all;
  if (chunk0 < 0 || chunk0 >= chunk1) return chunk0 == chunk1 ? cudaSuccess : cudaErrorInvalidValue;
  const int64_t n_chunks = chunk1 - chunk0;
  const int n_ablk = (C + 8 * kPA - 1) / (8 * kPA);
  if (!cnt) return cudaErrorInvalidValue;  // (the pair counts are always accumulated)
  // (the kernel offsets rows of the bitmap by up to 3 * C * Wst words in 32 bits)
  if (n_ablk > kMaxABlocks || n_chunks > 0x7FFFFFFF || 4 * (int64_t)C * Wst > 0xFFFFFFFFll)
    return cudaErrorInvalidValue;
  // every (a-block g, piece p) with b in [32 g, C), in the order of the piece's first column
  // 32 (g + 4 p), then of g
  PieceTable tab{};
  int total = 0;
  const int k_max = (C + 8 * kPA - 1) / (8 * kPA);
  for (int k = 0; k < k_max; ++k)
    for (int g = k % 4; g <= k && g < n_ablk; g += 4) {
      const int piece = (k - g) / 4;  // (starts at column 32 k < C)
      tab.item[total++] = (uint16_t)(g << 8 | piece);
    }
  const dim3 grid((unsigned)n_chunks, (unsigned)total), block(256);  // (total <= 32 * 8 pieces)
  switch (nb) {
    case 1: k_build_bitmap_planes<1><<<grid, block, 0, s>>>(planes, C, Wst, tab, bitmap, cnt, chunk0);
      break;
    case 2: k_build_bitmap_planes<2><<<grid, block, 0, s>>>(planes, C, Wst, tab, bitmap, cnt, chunk0);
      break;
    case 3: k_build_bitmap_planes<3><<<grid, block, 0, s>>>(planes, C, Wst, tab, bitmap, cnt, chunk0);
      break;
    case 4: k_build_bitmap_planes<4><<<grid, block, 0, s>>>(planes, C, Wst, tab, bitmap, cnt, chunk0);
      break;
    case 5: k_build_bitmap_planes<5><<<grid, block, 0, s>>>(planes, C, Wst, tab, bitmap, cnt, chunk0);
      break;
    case 6: k_build_bitmap_planes<6><<<grid, block, 0, s>>>(planes, C, Wst, tab, bitmap, cnt, chunk0);
      break;
    case 7: k_build_bitmap_planes<7><<<grid, block, 0, s>>>(planes, C, Wst, tab, bitmap, cnt, chunk0);
      break;
    case 8: k_build_bitmap_planes<8><<<grid, block, 0, s>>>(planes, C, Wst, tab, bitmap, cnt, chunk0);
      break;
    case 9: k_build_bitmap_planes<9><<<grid, block, 0, s>>>(planes, C, Wst, tab, bitmap, cnt, chunk0);
      break;
    case 10: k_build_bitmap_planes<10><<<grid, block, 0, s>>>(planes, C, Wst, tab, bitmap, cnt, chunk0);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}
