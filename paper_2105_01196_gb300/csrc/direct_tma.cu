// Direct-comparison evaluation with TMA-staged row tiles (the trend counts of Sec. 2.3 /
// Sec. 2.4 steps 2-3, as in eval.cu).
//
// A work item is (row tile, group of individuals).  A tile is TR rows of every column of the
// column-major order keys; the tensor memory accelerator copies it into shared memory as
// ceil(C / CB) boxes of TR x CB keys (cp.async.bulk.tensor, completion on an mbarrier), so every
// column's TR rows sit contiguously.  The tile then serves all individuals of the group: each warp
// takes an individual, its lanes hold four consecutive rows each (16-byte shared-memory loads),
// count the increasing and decreasing consecutive pairs, and the warp counts accepted rows with
// ballots.  Two stages let the copy of a CTA's next tile overlap the current one when both fit.
// Waits on the mbarrier are bounded: on expiry the kernel records an error word and stops.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "internal.h"
#include "items.cuh"
#include "tables.cuh"
#include "tma.cuh"

namespace {

using tma::mbar_expect_tx;
using tma::mbar_init;
using tma::mbar_wait;

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr size_t kStagedSmemMax = 192 * 1024;  // stage buffers; the static part comes on top

__device__ __forceinline__ int threshold(int L, int num, int den) {
  return (num * (L - 1) + den - 1) / den;
}

struct StagedArgs {
  int32_t TR, CB, nbox, stages;  // rows per tile, columns per box, boxes per tile, 1 or 2
  int32_t n_tiles, n_groups, group_size;
  int32_t stage_words;           // keys per stage buffer (nbox * CB * TR)
};

template <bool NEG>
__global__ void __launch_bounds__(kThreads, 1)
    k_eval_direct_tma(const __grid_constant__ CUtensorMap map, EvalArgs a, PopView pv,
                      StagedArgs sa) {
  extern __shared__ __align__(128) uint32_t s_tile[];
  __shared__ __align__(8) uint64_t s_bar[2];
  __shared__ int32_t s_base[kWarps][EBIC_MAX_LEN];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  if (pv.stop && *pv.stop) return;
  // the generation loop's side tasks: the previous generation's keys join the tabu list, and
  // this generation's live keys enter its duplicate table (tested after the launch)
  items::move_all(a);
  if (pv.dkeys)
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < pv.n; i += gridDim.x * blockDim.x)
      if (!(pv.dead && pv.dead[i])) dedup_insert(pv.dkeys, pv.dslot, pv.dmask, pv.hash[i], i);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_items = sa.n_tiles * sa.n_groups;
  const uint32_t stage_bytes = (uint32_t)sa.stage_words * 4u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < sa.stages; ++s) mbar_init(&s_bar[s], 1);
    tma::fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int item, int stage) {  // thread 0: copy the tile of `item` into `stage`
    const int tile = item / sa.n_groups;
    uint32_t *dst = s_tile + (size_t)stage * sa.stage_words;
    mbar_expect_tx(&s_bar[stage], stage_bytes);
    for (int b = 0; b < sa.nbox; ++b)
      tma::tensor_load_2d(dst + (size_t)b * sa.CB * sa.TR, &map, tile * sa.TR, b * sa.CB,
                          &s_bar[stage]);
  };
  int item = blockIdx.x;
  bool pending[2] = {false, false};  // a copy into the stage is in flight (tracked by thread 0)
  if (threadIdx.x == 0 && item < n_items) {
    issue(item, 0);
    pending[0] = true;
  }
  uint32_t phase[2] = {0u, 0u};
  bool failed = false;
  const bool vec = (sa.TR % 128) == 0;
  const int slots = vec ? sa.TR / 128 : sa.TR / 32;  // row slots per lane
  for (int k = 0; item < n_items; ++k, item += gridDim.x) {
    const int stage = sa.stages == 2 ? (k & 1) : 0;
    const int next = item + gridDim.x;
    if (sa.stages == 2 && threadIdx.x == 0 && next < n_items) {
      issue(next, stage ^ 1);
      pending[stage ^ 1] = true;
    }
    const bool ok = mbar_wait(&s_bar[stage], phase[stage]);
    if (__syncthreads_or(!ok)) {  // the same decision in every thread
      failed = true;
      break;
    }
    pending[stage] = false;
    phase[stage] ^= 1u;
    const uint32_t *tile = s_tile + (size_t)stage * sa.stage_words;
    const int t = item / sa.n_groups, grp = item - t * sa.n_groups;
    const int i0 = grp * sa.group_size, i1 = min(pv.n, i0 + sa.group_size);
    for (int i = i0 + warp; i < i1; i += kWarps) {
      if (pv.dead && pv.dead[i]) continue;
      const int st = pv.off ? pv.off[i] : i * pv.stride;
      const int L = pv.off ? pv.off[i + 1] - st : pv.len[i];
      if (L < 2) continue;
      __syncwarp();
      for (int c = lane; c < L; c += 32) s_base[warp][c] = pv.cols[st + c] * sa.TR;
      __syncwarp();
      const int thr = threshold(L, a.rnum, a.rden);
      int cp = 0, cn = 0, ca = 0;
      for (int q = 0; q < slots; ++q) {
        if (vec) {  // four consecutive rows per lane, 16-byte loads
          const int r = q * 128 + lane * 4;
          uint4 prev = *reinterpret_cast<const uint4 *>(tile + s_base[warp][0] + r);
          int n0 = 0, n1 = 0, n2 = 0, n3 = 0, m0 = 0, m1 = 0, m2 = 0, m3 = 0;
#pragma unroll 4
          for (int c = 1; c < L; ++c) {
            const uint4 cur = *reinterpret_cast<const uint4 *>(tile + s_base[warp][c] + r);
            n0 += cur.x > prev.x;
            n1 += cur.y > prev.y;
            n2 += cur.z > prev.z;
            n3 += cur.w > prev.w;
            if (NEG) {
              m0 += cur.x < prev.x;
              m1 += cur.y < prev.y;
              m2 += cur.z < prev.z;
              m3 += cur.w < prev.w;
            }
            prev = cur;
          }
          const int incs[4] = {n0, n1, n2, n3}, decs[4] = {m0, m1, m2, m3};
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const bool po = incs[j] >= thr, ne = NEG && decs[j] >= thr;
            cp += __popc(__ballot_sync(kFull, po));
            if (NEG) {
              cn += __popc(__ballot_sync(kFull, ne));
              ca += __popc(__ballot_sync(kFull, po || ne));
            }
          }
        } else {  // one row per lane
          const int r = q * 32 + lane;
          uint32_t prev = tile[s_base[warp][0] + r];
          int inc = 0, dec = 0;
#pragma unroll 4
          for (int c = 1; c < L; ++c) {
            const uint32_t cur = tile[s_base[warp][c] + r];
            inc += cur > prev;
            if (NEG) dec += cur < prev;
            prev = cur;
          }
          const bool po = inc >= thr, ne = NEG && dec >= thr;
          cp += __popc(__ballot_sync(kFull, po));
          if (NEG) {
            cn += __popc(__ballot_sync(kFull, ne));
            ca += __popc(__ballot_sync(kFull, po || ne));
          }
        }
      }
      if (!NEG) ca = cp;
      if (lane == 0) {
        if (cp) atomicAdd(a.rows_pos + i, cp);
        if (cn) atomicAdd(a.rows_neg + i, cn);
        if (ca) atomicAdd(a.rows_any + i, ca);
      }
    }
    __syncthreads();  // the stage is consumed before it is refilled
    if (sa.stages == 1 && threadIdx.x == 0 && next < n_items) {
      issue(next, 0);
      pending[0] = true;
    }
  }
  if (failed && threadIdx.x == 0) {
    if (a.err) atomicOr(a.err, 4);
    // wait (bounded) for this block's copies still in flight before its shared memory goes away
    for (int s = 0; s < sa.stages; ++s)
      if (pending[s]) mbar_wait(&s_bar[s], phase[s]);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

}  // namespace

// Tile geometry and tensor map for the keys of the loaded matrix.  Tiles are a multiple of 128
// rows (four rows per lane) when two stages of at least 128 rows fit, else a multiple of 32 rows
// in one stage.  ok = false when not even 32 rows of all columns fit in shared memory (more than
// 1,536 columns) or no encoder is available; the direct form then reads the keys from global
// memory instead.
void direct_tma_prepare(DirectTma *d, const uint32_t *keys, int64_t R_pad, int32_t C) {
  d->ok = false;
  const size_t budget = kStagedSmemMax;
  const int64_t per_row = 4 * (int64_t)((C + 255) / 256) * (C < 256 ? C : 256);
  int64_t TR = (int64_t)(budget / 2) / per_row / 128 * 128;  // two stages of 4 rows per lane
  int stages = 2;
  int64_t step = 128;
  if (TR < 128) {
    TR = (int64_t)budget / per_row / 32 * 32;  // one stage of 1 row per lane
    stages = 1;
    step = 32;
  }
  if (TR < 32) return;
  if (TR > 256) TR = 256;  // a tensor-map box spans at most 256 elements per dimension
  while (R_pad % TR) TR -= step;
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return;
  const int CB = C < 256 ? C : 256;
  const int nbox = (C + CB - 1) / CB;
  cuuint64_t dims[2] = {(cuuint64_t)R_pad, (cuuint64_t)C};
  cuuint64_t strides[1] = {(cuuint64_t)R_pad * 4};
  cuuint32_t box[2] = {(cuuint32_t)TR, (cuuint32_t)CB};
  cuuint32_t estr[2] = {1, 1};
  CUtensorMap *map = reinterpret_cast<CUtensorMap *>(d->map);
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<uint32_t *>(keys), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return;
  // one fixed limit for both instantiations (no context lowers another's)
  if (cudaFuncSetAttribute(k_eval_direct_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kStagedSmemMax) != cudaSuccess ||
      cudaFuncSetAttribute(k_eval_direct_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kStagedSmemMax) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  d->TR = (int)TR;
  d->CB = CB;
  d->nbox = nbox;
  d->stages = stages;
  d->stage_words = (int64_t)nbox * CB * TR;
  d->ok = true;
}

cudaError_t launch_eval_direct_tma(const DirectTma &d, const EvalArgs &a, const PopView &pv,
                                   int num_sms, cudaStream_t s, bool pdl) {
  StagedArgs sa;
  sa.TR = d.TR;
  sa.CB = d.CB;
  sa.nbox = d.nbox;
  sa.stages = d.stages;
  sa.stage_words = (int32_t)d.stage_words;
  sa.n_tiles = (int32_t)(a.R_pad / d.TR);
  // groups: about 4 items per CTA, each group at least 8 individuals
  int64_t groups = (4LL * num_sms + sa.n_tiles - 1) / sa.n_tiles;
  groups = std::max<int64_t>(1, std::min<int64_t>(groups, (pv.n + 7) / 8));
  sa.n_groups = (int32_t)groups;
  sa.group_size = (int32_t)((pv.n + groups - 1) / groups);
  const size_t smem = (size_t)sa.stages * sa.stage_words * 4;
  const CUtensorMap *map = reinterpret_cast<const CUtensorMap *>(d.map);
  const int64_t items = (int64_t)sa.n_tiles * sa.n_groups;
  const unsigned grid = (unsigned)std::min<int64_t>(items, num_sms);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  if (a.neg) return cudaLaunchKernelEx(&cfg, k_eval_direct_tma<true>, *map, a, pv, sa);
  return cudaLaunchKernelEx(&cfg, k_eval_direct_tma<false>, *map, a, pv, sa);
}
