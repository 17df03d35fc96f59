// Work items of the persistent evaluation kernels (eval.cu, codes.cu).
//
// Warps take items in one sequence (statically for small launches, else from one atomic counter):
// first - in the generation loop - the P / 32 chunks of its side task (the previous generation's
// keys join the tabu list, its duplicate table is cleared), then the (individual, row segment)
// evaluation items, segment-major.  The launch has a warp for every item when it can, so the
// chunks run beside the evaluations; when warps take several items, the chunks taken first keep
// them out of the launch's tail.
//
// The per-item bookkeeping is arranged so that its loads leave in as few dependent round trips as
// possible: length, start, dead flag, hash and (for the generation loop's fixed-stride rows) the
// 64 column words are loaded together, and the entry of the slot's key into the generation's
// duplicate table is started before the evaluation loads and finished after them.
#pragma once

#include "internal.h"
#include "tables.cuh"

namespace items {

constexpr unsigned kFull = 0xFFFFFFFFu;

// Number of side-task chunks (32 slots of the previous generation each).
__device__ __forceinline__ int move_chunks(const EvalArgs &a) {
  return a.mv_table ? (int)((a.mv_n + 31u) / 32u) : 0;
}

// Slot s of the previous generation: its key joins the tabu list when the slot was live (its
// tabu flag 1 marks a dead slot; 0 and 2 are live, 2 having been evaluated by the evolve kernel).
__device__ __forceinline__ unsigned move_slot(const EvalArgs &a, uint32_t s) {
  const uint8_t d = a.mv_dead[s];
  const int32_t L = a.mv_len[s];
  const uint64_t h = a.mv_hash[s];
  return (d != 1 && L >= 2 && tabu_insert(a.mv_table, a.mv_tmask, h)) ? 1u : 0u;
}

// One side-task chunk: slot 32 m + lane of the previous generation joins the tabu list, and the
// chunk clears its share of that generation's duplicate table (plain stores).
__device__ __forceinline__ void move_chunk(const EvalArgs &a, int m, int lane) {
  const uint32_t s = (uint32_t)m * 32u + (uint32_t)lane;
  unsigned added = s < a.mv_n ? move_slot(a, s) : 0u;
  const uint32_t n_ch = (a.mv_n + 31u) / 32u, per = (a.clr_n + n_ch - 1u) / n_ch;
  const uint32_t j1 = min(a.clr_n, ((uint32_t)m + 1u) * per);
  for (uint32_t j = (uint32_t)m * per + (uint32_t)lane; j < j1; j += 32u) {
    a.clr_keys[j] = 0ull;
    a.clr_slots[j] = 0u;
  }
  added = __reduce_add_sync(kFull, added);
  if (lane == 0 && added) atomicAdd(a.mv_count, (unsigned long long)added);
}

// The whole side task, spread over every thread of the calling grid (the staged kernel).
static __device__ __noinline__ void move_all(const EvalArgs &a) {
  if (!a.mv_table) return;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  unsigned long long added = 0ull;
  for (uint32_t s = tid; s < a.mv_n; s += stride) added += move_slot(a, s);
  for (uint32_t j = tid; j < a.clr_n; j += stride) {
    a.clr_keys[j] = 0ull;
    a.clr_slots[j] = 0u;
  }
  if (added) atomicAdd(a.mv_count, added);
}

// A warp's first item is its index w in the launch (no round trip to the counter).  With at
// most two items per warp of the launch (n_all <= 2 W, W warps) the second is w + W, again without
// the counter: every warp of such a launch would otherwise meet the others at the one counter
// address right after its first item, and those returning atomics serialise (measured: up to
// 5 us for the last warp of a 2,432-warp launch).  Larger launches take the later items from the
// counter, after the first items of all the launch's warps, to balance uneven items.
__device__ __forceinline__ int first() {
  return (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
}

__device__ __forceinline__ int next(int32_t *work, int lane, int q, int n_all) {
  const int W = (int)(gridDim.x * (blockDim.x >> 5));
  if (n_all <= 2 * W) return q + W;
  int x = 0;
  if (lane == 0) x = atomicAdd(work, 1);
  return __shfl_sync(kFull, x, 0) + W;
}

// Individuals of the launch: the view's n, or the count of its slot list (read on the device).
__device__ __forceinline__ int count(const PopView &pv) {
  return pv.list ? min(*pv.list_n, pv.n) : pv.n;
}

// Slot of the launch's individual i.
__device__ __forceinline__ int slot(const PopView &pv, int i) { return pv.list ? pv.list[i] : i; }

// Whether the run has stopped (the flag is read beside an item's first loads, and tested before
// the item's first store).
__device__ __forceinline__ bool stopped(const PopView &pv) { return pv.stop && *pv.stop; }

struct Meta {
  int st, L;     // start in cols, length
  bool dead;     // tabu-dead slot (never scored)
  uint64_t h;    // key (duplicate table), 0 when there is none
  int c0, c1;    // columns k = lane and k = lane + 32 (0 past the length)
};

// One individual's bookkeeping.  The generation loop's rows have a fixed stride of 64 columns,
// so their column words load in the same round trip as the length.
__device__ __forceinline__ Meta load_meta(const PopView &pv, int i, int lane) {
  Meta m;
  if (pv.off) {
    m.st = pv.off[i];
    m.L = pv.off[i + 1] - m.st;
  } else {
    m.st = i * pv.stride;
    m.L = pv.len[i];
  }
  m.dead = pv.dead && pv.dead[i];
  m.h = pv.dkeys ? pv.hash[i] : 0ull;
  if (!pv.off) {
    m.c0 = pv.cols[m.st + lane];
    m.c1 = pv.cols[m.st + 32 + lane];
    if (lane >= m.L) m.c0 = 0;
    if (lane + 32 >= m.L) m.c1 = 0;
  } else {
    m.c0 = lane < m.L ? pv.cols[m.st + lane] : 0;
    m.c1 = lane + 32 < m.L ? pv.cols[m.st + 32 + lane] : 0;
  }
  return m;
}

// The generation loop's duplicate table: each live slot's key enters it once, from the item of
// the slot's first row segment (the duplicate test itself runs after this launch, in k_finish).
// The compare-and-swap leaves before the evaluation loads and its result is used after them.
struct Insert {
  uint64_t prev;  // what the first probe position held
  uint32_t idx;   // first probe position
  bool on;        // lane 0 of the slot's first item, with a duplicate table
};

__device__ __forceinline__ Insert insert_start(const PopView &pv, int seg, uint64_t h, int lane) {
  Insert in{0ull, 0u, pv.dkeys != nullptr && seg == 0 && lane == 0};
  if (in.on) {
    in.idx = table_index(h, pv.dmask);
    in.prev = atomicCAS(reinterpret_cast<unsigned long long *>(pv.dkeys + in.idx), 0ull,
                        (unsigned long long)h);
  }
  return in;
}

// Completes the insertion: the slot word keeps the lowest slot (see dedup_insert).
__device__ __forceinline__ void insert_finish(const PopView &pv, const Insert &in, uint64_t h,
                                              int s) {
  if (!in.on) return;
  if (in.prev == 0ull || in.prev == h) {
    atomicMax(pv.dslot + in.idx, 0xFFFFFFFFu - (uint32_t)s);
    return;
  }
  // the first position holds another key: continue the linear probe from the next one
  uint32_t i = (in.idx + 1u) & pv.dmask;
  for (uint32_t n = 1; n <= pv.dmask; ++n) {
    const unsigned long long prev =
        atomicCAS(reinterpret_cast<unsigned long long *>(pv.dkeys + i), 0ull,
                  (unsigned long long)h);
    if (prev == 0ull || prev == h) {
      atomicMax(pv.dslot + i, 0xFFFFFFFFu - (uint32_t)s);
      return;
    }
    i = (i + 1u) & pv.dmask;
  }
}

}  // namespace items
