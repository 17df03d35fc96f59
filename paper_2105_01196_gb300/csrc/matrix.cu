// Matrix upload (order keys, column-major) and the column-pair comparison bitmap.
//
// Order key: the float32 bit pattern u, with -0 mapped to +0, becomes
//   k(u) = u ^ 0xFFFFFFFF for negative values, u | 0x80000000 otherwise,
// an increasing map of the finite floats onto uint32, so `k(a) > k(b)` is exactly `a > b`
// (ties, including -0 against +0, compare equal) whatever the FTZ/DAZ mode of the arithmetic.
// The trend definition the keys serve is Sec. 2.3 ("EBIC" paragraph) of the EBIC.jl paper.
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
__global__ void k_upload_rowmajor(const float *__restrict__ x, int64_t R, int32_t C,
                                  int64_t R_pad, uint32_t *__restrict__ keys,
                                  int32_t *__restrict__ err) {
  __shared__ uint32_t tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
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
    if (c < C && r < R_pad) keys[(int64_t)c * R_pad + r] = tile[tx][j];
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
// Block = 8 warps, one column a per warp; a block covers 32 words (1024 rows) of rows.  The
// b-columns of the chunk are staged in shared memory in groups of kBStage columns and shared by
// the 8 warps; each warp keeps its a-column chunk in registers and forms one word per ballot.
constexpr int kBStage = 8;

__global__ void __launch_bounds__(256) k_build_bitmap(const uint32_t *__restrict__ keys,
                                                      int64_t R_pad, int32_t C, int64_t Wst,
                                                      uint32_t *__restrict__ G) {
  __shared__ uint32_t sb[kBStage][1024];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t w0 = (int64_t)blockIdx.x * 32;
  const int64_t nw = (Wst - w0 < 32) ? (Wst - w0) : 32;  // words of this chunk
  const int32_t a = blockIdx.y * 8 + warp;
  const bool a_ok = a < C;
  uint32_t ka[32];
#pragma unroll
  for (int j = 0; j < 32; ++j)
    ka[j] = (a_ok && j < nw) ? __ldg(keys + (int64_t)a * R_pad + (w0 + j) * 32 + lane) : 0u;

  for (int32_t b0 = 0; b0 < C; b0 += kBStage) {
    const int nb = (C - b0 < kBStage) ? (C - b0) : kBStage;
    __syncthreads();
    for (int q = threadIdx.x; q < nb * 1024; q += blockDim.x) {
      const int bb = q >> 10, rr = q & 1023;
      const int64_t row = w0 * 32 + rr;
      sb[bb][rr] = (row < R_pad) ? __ldg(keys + (int64_t)(b0 + bb) * R_pad + row) : 0u;
    }
    __syncthreads();
    if (!a_ok) continue;
    for (int bb = 0; bb < nb; ++bb) {
      uint32_t word = 0u;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, sb[bb][j * 32 + lane] > ka[j]);
        if (lane == j) word = m;
      }
      if (lane < nw) G[((int64_t)a * C + (b0 + bb)) * Wst + w0 + lane] = word;
    }
  }
}

}  // namespace

cudaError_t launch_upload(const float *x, int64_t R, int32_t C, int64_t R_pad, int32_t layout,
                          uint32_t *keys, int32_t *err, cudaStream_t s) {
  if (layout == EBIC_LAYOUT_ROW_MAJOR) {
    dim3 grid((unsigned)(R_pad / 32), (unsigned)((C + 31) / 32));
    k_upload_rowmajor<<<grid, dim3(32, 8), 0, s>>>(x, R, C, R_pad, keys, err);
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
  dim3 grid((unsigned)((Wst + 31) / 32), (unsigned)((C + 7) / 8));
  k_build_bitmap<<<grid, 256, 0, s>>>(keys, R_pad, C, Wst, bitmap);
  return cudaGetLastError();
}
