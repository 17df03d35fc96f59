// Device-side EBIC generation loop (EBIC.jl paper, Sec. 2.4 steps 1-9; strategies of Sec. 2.3:
// elitism, tournament selection with an exponential penalty on overused columns, tabu list of
// chromosome hashes, tabu-hit termination; parameters of Sec. 2.4's last paragraph).
//
// One generation is three kernels, captured as CUDA graphs (one per buffer parity, and one of
// sixteen consecutive generations per starting parity) and replayed:
//   k_evolve    one block per slot, one warp per tabu attempt: elites from the top list (step
//               4), otherwise penalised tournament, optional one-point crossover and one
//               mutation, tabu probe; the lowest attempt that misses the tabu list wins (step 5).
//               With the bitmap form, a live child whose pair test is exact and that has few
//               pairs is evaluated right there by the winning warp (step 7), which also enters
//               its key into the generation's duplicate table; the other live slots are listed
//               for the evaluation launch;
//   k_eval_*    the persistent evaluation kernel (eval.cu, codes.cu) over the new population,
//               or over the listed slots, skipping tabu-dead slots (step 7); it also enters the
//               live keys it evaluates into this generation's duplicate table, inserts the
//               previous generation's live keys into the hashed tabu list and clears that
//               generation's duplicate table;
//   k_finish    all blocks: final dead flags (tabu or duplicate), tabu hits, fitness, candidates
//               for the top list; then the last block to finish: tabu-hit stop test (step 6),
//               top rank list update (step 7), column usage, counters for the next generation.
// k_init builds the initial population (step 1), one warp per slot.
// Generation g reads population buffer (g-1)&1 and writes g&1, and uses duplicate table g&1.
// The tabu list a child is probed against is the hashed set of generations <= g-2 plus the
// duplicate table of generation g-1 (its live keys), which is the whole tabu list as it stood at
// the start of generation g.  Once the stop flag is set every kernel returns before its first
// store, so further replays are no-ops.  The random words come from Philox4x32-10 (Salmon et
// al., SC'11) with counter (generation, slot, attempt, block).
#include <string.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "tables.cuh"

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kS = EBIC_MAX_LEN;  // population slot stride (columns)
constexpr int kTopThreads = 1024;
constexpr int kSortSmemMax = 4096;  // most candidates sorted in shared memory
constexpr size_t kFinishSmemMax = 180 * 1024;  // dynamic shared memory limit set for k_finish

struct TopEntry {
  uint64_t f, h;
  int32_t len, rp, rn, ra;
  int32_t cols[kS];
};

struct GenCtl {
  int32_t gen;         // last scored generation, -1 before initialisation
  int32_t stopped;     // step 6 ended the run
  int32_t hits_cur;    // tabu hits of the generation being built
  int32_t hits_last;   // tabu hits of the last generation built
  int32_t n_top;       // entries in the top list
  int32_t live_cur;    // live slots of the generation being scored
  int32_t n_cand;      // top-list candidates collected by k_finish
  int32_t done;        // blocks of k_finish that have finished their slots
  int32_t n_todo;      // slots the evolve kernel left to the evaluation launch (its list)
  int32_t fused_cur;   // live slots of the generation being scored evaluated by the evolve kernel
  int32_t evo_next;    // slots k_evolve_seq's warps have taken beyond their first
  int32_t table_cur;   // of fused_cur, the one-pair slots scored from the pair-count table
  long long n_evaluated;
  long long tabu_count;
  long long sum_len;   // sum of the lengths of all scored live slots (evaluation work)
  long long len_cur;   // the same for the generation being scored
  long long n_fused;   // of n_evaluated, the slots the evolve kernel evaluated
  long long fused_len; // the sum of their lengths
  long long flen_cur;  // the same for the generation being scored
  long long n_table;   // of n_fused, the one-pair slots scored from the pair-count table
};

// One population buffer (P slots of stride kS).
struct Buf {
  int32_t *cols, *len, *att_hits, *rows;  // rows: [3][P] pos, neg, any
  uint8_t *att_dead, *dead;
  uint64_t *hash, *fit;
};

struct GenArgs {
  GenCtl *ctl;
  TopEntry *top;
  int32_t *usage;
  uint64_t *tabu;
  uint32_t tmask;
  uint64_t *dkeys[2];  // duplicate tables, one per generation parity
  uint32_t *dslot[2];
  uint32_t dmask;
  int32_t *rows_scr;  // [3][P] evaluation output (zeroed by k_finish)
  int32_t *work;
  uint64_t *cand_f, *cand_h;
  int32_t *cand_s;
  int32_t cand_cap;
  int32_t sort_cap;   // candidates sorted in shared memory up to this many (a power of two)
  uint64_t seed;
  int32_t P, C, K, E, T, A, max_len, init_min, init_max;
  int32_t min_rows, col_cap, ov_num, ov_den, tabu_limit;
  // Evaluation inside the evolve kernel (fuse_np > 0, bitmap form): the pair words, the test's
  // variant and ratio, and the list of the slots left to the evaluation launch (ctl->n_todo).
  const uint32_t *bitmap;  // [C][C][Wst]
  // [C][C], for a < b: rows of G[a][b] | rows of G[b][a] << 32 (or null)
  const unsigned long long *pair_cnt;
  int64_t Wst, R;
  int32_t neg, ns, rnum, rden, fuse_np;
  int32_t *todo;
};

// Waits for the preceding kernel of a programmatic launch (no-op otherwise).
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// ------------------------------------------------------------------ Philox4x32-10 word stream

constexpr uint32_t kMul0 = 0xD2511F53u, kMul1 = 0xCD9E8D57u;
constexpr uint32_t kWeyl0 = 0x9E3779B9u, kWeyl1 = 0xBB67AE85u;

// One Philox4x32-10 block: counter (c0, c1, c2, c3), key (k0, k1).
__device__ __forceinline__ void philox_block(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                                             uint32_t c2, uint32_t c3, uint32_t w[4]) {
  uint32_t x0 = c0, x1 = c1, x2 = c2, x3 = c3, a0 = k0, a1 = k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      a0 += kWeyl0;
      a1 += kWeyl1;
    }
    const uint32_t lo0 = kMul0 * x0, hi0 = __umulhi(kMul0, x0);
    const uint32_t lo1 = kMul1 * x2, hi1 = __umulhi(kMul1, x2);
    const uint32_t y0 = hi1 ^ x1 ^ a0, y2 = hi0 ^ x3 ^ a1;
    x0 = y0;
    x1 = lo1;
    x2 = y2;
    x3 = lo0;
  }
  w[0] = x0;
  w[1] = x1;
  w[2] = x2;
  w[3] = x3;
}

// The same as a call (for the rare refills of WarpStream, which would otherwise be inlined at
// every draw).
__device__ __noinline__ uint4 philox_block_call(uint32_t k0, uint32_t k1, uint32_t c0, uint32_t c1,
                                                uint32_t c2, uint32_t c3) {
  uint32_t w[4];
  philox_block(k0, k1, c0, c1, c2, c3, w);
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// The word stream of counter (g, s, a) - the words of Philox blocks 0, 1, 2, ... in order - for
// a whole warp: lane j holds block base + j, so one round of Philox in all lanes yields 128
// words, and word i comes from lane i / 4 - base by a shuffle (every lane calls next() together
// and gets the same word).
struct WarpStream {
  uint32_t k0, k1, c0, c1, c2;
  uint32_t w[4];
  uint32_t base, pos;  // first block held; next word index
  int lane;
  __device__ WarpStream(uint64_t seed, uint32_t g, uint32_t s, uint32_t a, int lane_)
      : k0((uint32_t)seed), k1((uint32_t)(seed >> 32)), c0(g), c1(s), c2(a), base(0), pos(0),
        lane(lane_) {
    philox_block(k0, k1, c0, c1, c2, base + (uint32_t)lane, w);
  }
  __device__ uint32_t next() {
    const uint32_t b = pos >> 2;
    if (b >= base + 32u) {  // (warp-uniform) the next 32 blocks
      base += 32u;
      const uint4 v = philox_block_call(k0, k1, c0, c1, c2, base + (uint32_t)lane);
      w[0] = v.x;
      w[1] = v.y;
      w[2] = v.z;
      w[3] = v.w;
    }
    const uint32_t k = pos & 3u;
    const uint32_t mine = k == 0 ? w[0] : (k == 1 ? w[1] : (k == 2 ? w[2] : w[3]));
    ++pos;
    return __shfl_sync(0xFFFFFFFFu, mine, (int)(b - base));
  }
  __device__ uint32_t below(uint32_t n) { return __umulhi(next(), n); }
};

// ------------------------------------------------------------------ FNV-1a 64 chromosome key

__device__ uint64_t chromosome_key(const int32_t *c, int L) {
  uint64_t h = 0xCBF29CE484222325ull;
  for (int k = 0; k < L; ++k) {
    const uint32_t v = (uint32_t)c[k];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      h ^= (v >> (8 * b)) & 0xFFu;
      h *= 0x100000001B3ull;
    }
  }
  return h ? h : 0x9E3779B97F4A7C15ull;
}

// ------------------------------------------------------------------ selection

// Sign of fa * 2^s - fb for s >= 0, exactly.
__device__ __forceinline__ int cmp_shifted(uint64_t fa, int s, uint64_t fb) {
  if (fa == 0ull) return fb == 0ull ? 0 : -1;
  if (s >= 64) return 1;
  const uint64_t q = fb >> s;  // fa * 2^s > fb  <=>  fa > floor(fb / 2^s)
  if (fa > q) return 1;
  if (fa < q) return -1;
  return (fb & ((s ? (1ull << s) : 1ull) - 1ull)) ? -1 : 0;
}

// Sign of fa * 2^-ua - fb * 2^-ub, exactly (ua, ub >= 0).
__device__ __forceinline__ int cmp_penalised(uint64_t fa, int ua, uint64_t fb, int ub) {
  return ub >= ua ? cmp_shifted(fa, ub - ua, fb) : -cmp_shifted(fb, ua - ub, fa);
}

// ------------------------------------------------------------------ variation

// ------------------------------------------------------------------ kernels


// ------------------------------------------------------------------ warp-cooperative children
// One warp builds one child.  The word stream and every decision are uniform across the warp (all
// lanes compute the same Philox words), and the lanes share the data-parallel work: parent
// copies, membership tests by ballot, shifts, the crossover's compaction and the tournament's
// penalty sums.  The child lives in shared memory (kS + 1 ints per warp).

__device__ __forceinline__ unsigned lanes_below(int lane) { return (1u << lane) - 1u; }

// Whether v occurs in c[0..L) (L <= 64).
__device__ __forceinline__ bool w_contains(const int32_t *c, int L, int v, int lane) {
  const bool hit = (lane < L && c[lane] == v) || (lane + 32 < L && c[lane + 32] == v);
  return __any_sync(kFull, hit);
}

__device__ int w_draw_free(WarpStream &st, int C, const int32_t *c, int L, int lane) {
  for (int t = 0; t < 64; ++t) {
    const int v = (int)st.below((uint32_t)C);
    if (!w_contains(c, L, v, lane)) return v;
  }
  return -1;
}

// Tournament of T candidates drawn in stream order, up to eight at a time.  Four lanes serve each
// candidate: one round of loads brings its fitness, length and all 64 column words (the tail past
// the length is zero), a second its column usage.  The columns go to the warp's scratch rows so
// that the winner's chromosome is copied to `win` without another trip to global memory.  Same
// winner as the sequential rule (exact penalised comparison, ties to the lower slot).
__device__ int w_tournament(WarpStream &st, const GenArgs &ga, const Buf &pb, int32_t *scratch,
                            int32_t *win, int *win_len, int lane, const int32_t *usage) {
  int best = -1, ub = 0, bl = 0;
  uint64_t fb = 0ull;
  const int mine = lane >> 2, sub = lane & 3;
  for (int t0 = 0; t0 < ga.T; t0 += 8) {
    int ids[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) ids[q] = (t0 + q < ga.T) ? (int)st.below((uint32_t)ga.P) : -1;
    int my = -1;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (q == mine) my = ids[q];
    uint64_t f = 0ull;
    int u = 0, L = 0;
    if (my >= 0) {
      // lane `sub` of the candidate holds the 16-byte chunks sub, sub + 4, sub + 8, sub + 12
      const int4 *cc4 = reinterpret_cast<const int4 *>(pb.cols + (size_t)my * kS);
      L = pb.len[my];
      f = pb.fit[my];
      int4 v[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) v[r] = cc4[sub + 4 * r];
      int4 *row4 = reinterpret_cast<int4 *>(scratch + mine * kS);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int k = 4 * (sub + 4 * r);
        const int u0 = k < L ? usage[v[r].x] : 0, u1 = k + 1 < L ? usage[v[r].y] : 0;
        const int u2 = k + 2 < L ? usage[v[r].z] : 0, u3 = k + 3 < L ? usage[v[r].w] : 0;
        u += u0 + u1 + u2 + u3;
        row4[sub + 4 * r] = v[r];
      }
    }
    u += __shfl_xor_sync(kFull, u, 1);
    u += __shfl_xor_sync(kFull, u, 2);
    __syncwarp();
    int take = -1;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const uint64_t fq = __shfl_sync(kFull, f, q * 4);
      const int uq = __shfl_sync(kFull, u, q * 4);
      const int lq = __shfl_sync(kFull, L, q * 4);
      const int iq = ids[q];
      if (iq < 0) continue;
      const int c = best < 0 ? 1 : cmp_penalised(fq, uq, fb, ub);
      if (c > 0 || (c == 0 && iq < best)) {
        best = iq;
        fb = fq;
        ub = uq;
        bl = lq;
        take = q;
      }
    }
    if (take >= 0) {  // the winner so far is in this group: keep its columns
      const int32_t *row = scratch + take * kS;
      win[lane] = row[lane];
      win[lane + 32] = row[lane + 32];
    }
    __syncwarp();
  }
  *win_len = bl;
  return best;
}

// Whether candidate (fa, ua, ia) beats (fb, ub, ib): exact penalised comparison, ties to the
// lower slot; a missing candidate (slot < 0) never wins.
__device__ __forceinline__ bool beats(uint64_t fa, int ua, int ia, uint64_t fb, int ub, int ib) {
  if (ia < 0) return false;
  if (ib < 0) return true;
  const int c = cmp_penalised(fa, ua, fb, ub);
  return c > 0 || (c == 0 && ia < ib);
}

// Both tournaments of a child when T <= 4: the first one's T candidates, the crossover word and
// the second one's T candidates are drawn in stream order (the second set from a copy of the
// stream, adopted only when the crossover happens).  The sets take candidate places 0..T-1 and
// 4..4+T-1, four lanes each, so all candidates' data arrive in one round of loads and each set's
// winner comes out of a two-step butterfly over its places.  The winner is the one w_tournament
// picks (the maximum of one total order: penalised score, then the lower slot).  Returns whether
// the crossover happens.
__device__ bool w_tournament_pair(WarpStream &st, const GenArgs &ga, const Buf &pb,
                                  int32_t *scratch, int32_t *A, int *LA, int32_t *B, int *LB,
                                  int lane, const int32_t *usage) {
  const int T = ga.T;
  int ids[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) ids[q] = -1;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q < T) ids[q] = (int)st.below((uint32_t)ga.P);
  const bool cross = st.next() < (1u << 30);  // one-point crossover, probability 1/4
  WarpStream st2 = st;
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (q < T) ids[4 + q] = (int)st2.below((uint32_t)ga.P);
  if (cross) st = st2;
  const int mine = lane >> 2, sub = lane & 3;
  int my = -1;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (q == mine) my = ids[q];
  if (!cross && mine >= 4) my = -1;  // the second set is not needed
  uint64_t f = 0ull;
  int u = 0, L = 0;
  if (my >= 0) {
    const int4 *cc4 = reinterpret_cast<const int4 *>(pb.cols + (size_t)my * kS);
    L = pb.len[my];
    f = pb.fit[my];
    int4 v[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r] = cc4[sub + 4 * r];
    int4 *row4 = reinterpret_cast<int4 *>(scratch + mine * kS);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int k = 4 * (sub + 4 * r);
      const int u0 = k < L ? usage[v[r].x] : 0, u1 = k + 1 < L ? usage[v[r].y] : 0;
      const int u2 = k + 2 < L ? usage[v[r].z] : 0, u3 = k + 3 < L ? usage[v[r].w] : 0;
      u += u0 + u1 + u2 + u3;
      row4[sub + 4 * r] = v[r];
    }
  }
  u += __shfl_xor_sync(kFull, u, 1);
  u += __shfl_xor_sync(kFull, u, 2);
  // butterfly over the places of each set (lanes 0-15: first set, 16-31: second set)
  int wi = my, wq = mine, wl = L, wu = u;
  uint64_t wf = f;
#pragma unroll
  for (int off = 4; off <= 8; off <<= 1) {
    const uint64_t of = __shfl_xor_sync(kFull, wf, off);
    const int ou = __shfl_xor_sync(kFull, wu, off), oi = __shfl_xor_sync(kFull, wi, off);
    const int ol = __shfl_xor_sync(kFull, wl, off), oq = __shfl_xor_sync(kFull, wq, off);
    if (beats(of, ou, oi, wf, wu, wi)) {
      wf = of;
      wu = ou;
      wi = oi;
      wl = ol;
      wq = oq;
    }
  }
  const int take0 = __shfl_sync(kFull, wq, 0), take1 = __shfl_sync(kFull, wq, 16);
  const int bl0 = __shfl_sync(kFull, wl, 0), bl1 = __shfl_sync(kFull, wl, 16);
  __syncwarp();  // the scratch rows are written
  const int32_t *ra = scratch + take0 * kS;
  A[lane] = ra[lane];
  A[lane + 32] = ra[lane + 32];
  *LA = bl0;
  if (cross) {
    const int32_t *rb = scratch + take1 * kS;
    B[lane] = rb[lane];
    B[lane + 32] = rb[lane + 32];
    *LB = bl1;
  }
  __syncwarp();
  return cross;
}

__device__ void w_copy(int32_t *c, const int32_t *src, int L, int lane) {
  if (lane < L) c[lane] = src[lane];
  if (lane + 32 < L) c[lane + 32] = src[lane + 32];
  __syncwarp();
}

__device__ void w_swap(WarpStream &st, int32_t *c, int L, int lane) {
  if (L < 2) return;  // never reached: every live chromosome has at least two columns
  const int p = (int)st.below((uint32_t)L);
  int q = (int)st.below((uint32_t)(L - 1));
  if (q >= p) ++q;
  if (lane == 0) {
    const int t = c[p];
    c[p] = c[q];
    c[q] = t;
  }
  __syncwarp();
}

__device__ void w_mutate(WarpStream &st, int32_t *c, int &L, int C, int max_len, int lane) {
  for (int tries = 0; tries < 8; ++tries) {
    const uint32_t op = st.next() >> 30;
    if (op == 0u) {  // insertion
      if (L >= max_len || L >= C) continue;
      const int pos = (int)st.below((uint32_t)(L + 1));
      const int v = w_draw_free(st, C, c, L, lane);
      if (v < 0) continue;
      const bool m0 = lane >= pos && lane < L, m1 = lane + 32 >= pos && lane + 32 < L;
      const int x0 = m0 ? c[lane] : 0, x1 = m1 ? c[lane + 32] : 0;
      __syncwarp();
      if (m0) c[lane + 1] = x0;
      if (m1) c[lane + 33] = x1;
      if (lane == 0) c[pos] = v;
      __syncwarp();
      ++L;
      return;
    }
    if (op == 1u) {  // deletion
      if (L <= 2) continue;
      const int pos = (int)st.below((uint32_t)L);
      const bool m0 = lane >= pos && lane < L - 1, m1 = lane + 32 >= pos && lane + 32 < L - 1;
      const int x0 = m0 ? c[lane + 1] : 0, x1 = m1 ? c[lane + 33] : 0;
      __syncwarp();
      if (m0) c[lane] = x0;
      if (m1) c[lane + 32] = x1;
      __syncwarp();
      --L;
      return;
    }
    if (op == 2u) {  // substitution
      if (L >= C) continue;
      const int pos = (int)st.below((uint32_t)L);
      const int v = w_draw_free(st, C, c, L, lane);
      if (v < 0) continue;
      if (lane == 0) c[pos] = v;
      __syncwarp();
      return;
    }
    w_swap(st, c, L, lane);
    return;
  }
  w_swap(st, c, L, lane);
}

__device__ void w_make_child(const GenArgs &ga, const Buf &pb, int g, int s, int a, int32_t *c,
                             int32_t *scratch, int32_t *A, int32_t *B, int &L, int lane,
                             const int32_t *usage) {
  WarpStream st(ga.seed, (uint32_t)g, (uint32_t)s, (uint32_t)a, lane);
  int LA = 0, LB = 0;
  bool cross;
  if (ga.T <= 4) {
    cross = w_tournament_pair(st, ga, pb, scratch, A, &LA, B, &LB, lane, usage);
  } else {
    w_tournament(st, ga, pb, scratch, A, &LA, lane, usage);
    cross = st.next() < (1u << 30);  // one-point crossover, probability 1/4
    if (cross) w_tournament(st, ga, pb, scratch, B, &LB, lane, usage);
  }
  if (cross) {
    // (the min() guards only matter for a chromosome shorter than 2, which is never built)
    const int cut1 = min(1 + (int)st.below((uint32_t)(LA - 1)), max(LA, 1));
    const int cut2 = min(1 + (int)st.below((uint32_t)(LB - 1)), LB);
    w_copy(c, A, cut1, lane);
    const int ns = LB - cut2;  // suffix length
    if (cut1 + ns <= 32) {
      // prefix in lanes [0, cut1), suffix in lanes [cut1, cut1 + ns): one match finds the
      // suffix columns present in the prefix (other lanes hold values no column has)
      const bool suf = lane >= cut1 && lane < cut1 + ns;
      const int v = lane < cut1 ? A[lane] : (suf ? B[cut2 + lane - cut1] : -1 - lane);
      const unsigned eq = __match_any_sync(kFull, v);
      const unsigned pre = cut1 >= 32 ? kFull : ((1u << cut1) - 1u);
      const bool keep = suf && !(eq & pre);
      const unsigned m = __ballot_sync(kFull, keep);
      const int pos = cut1 + __popc(m & lanes_below(lane));
      if (keep && pos < ga.max_len) c[pos] = v;
      __syncwarp();
      L = min(cut1 + __popc(m), ga.max_len);
    } else {
      const int k0 = cut2 + lane, k1 = cut2 + lane + 32;
      const int b0 = k0 < LB ? B[k0] : -1, b1 = k1 < LB ? B[k1] : -1;
      bool in0 = false, in1 = false;
      for (int q = 0; q < cut1; ++q) {
        const int hq = c[q];
        in0 |= b0 == hq;
        in1 |= b1 == hq;
      }
      const bool keep0 = b0 >= 0 && !in0, keep1 = b1 >= 0 && !in1;
      const unsigned m0 = __ballot_sync(kFull, keep0), m1 = __ballot_sync(kFull, keep1);
      const int pos0 = cut1 + __popc(m0 & lanes_below(lane));
      const int pos1 = cut1 + __popc(m0) + __popc(m1 & lanes_below(lane));
      if (keep0 && pos0 < ga.max_len) c[pos0] = b0;
      if (keep1 && pos1 < ga.max_len) c[pos1] = b1;
      __syncwarp();
      L = min(cut1 + __popc(m0) + __popc(m1), ga.max_len);
    }
    if (L < 2) {
      w_copy(c, A, LA, lane);
      L = LA;
    }
  } else {
    w_copy(c, A, LA, lane);
    L = LA;
  }
  w_mutate(st, c, L, ga.C, ga.max_len, lane);
}

// ------------------------------------------------------- evaluation inside the evolve kernel
//
// A child whose pair test is exact - the threshold ceil(ratio * pairs) equals its number of
// pairs, so a row must satisfy every pair (Sec. 2.2) - and that has at most fuse_np pairs is
// evaluated by the warp that built it, on the pair bitmap G (bit j of word w of row a * C + b:
// row 32 w + j has key(b) > key(a)).  A row follows the positive trend when every pair's word has
// its bit, the negative trend when every reversed pair's word has it (ties counting both ways:
// the complements of the opposite words, pad rows masked).  One unit is one pair row's 128 words
// of one pass (16 bytes per lane); units are copied asynchronously into the warp's shared region,
// two groups of kFuseGroup in flight (four with a region borrowed from a warp of the block that
// has no slot left), and each lane reads back only the bytes it copied.
constexpr int kFuseGroup = 4;               // units per copy group
constexpr int kFuseSlots = 2 * kFuseGroup;  // units staged per warp
constexpr int kFuseWords = 128;             // words of one unit

__device__ __forceinline__ void fuse_copy16(uint32_t *dst, const uint32_t *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"((uint64_t)__cvta_generic_to_global(src))
               : "memory");
}

__device__ __forceinline__ void fuse_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Waits until at most N of this thread's copy groups are pending (a hardware wait).
template <int N>
__device__ __forceinline__ void fuse_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ uint4 fuse_and(uint4 a, uint4 b) {
  return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}

__device__ __forceinline__ int fuse_popc(uint4 v) {
  return __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
}

// Rows of word w that exist (bit j: row 32 w + j < R).
__device__ __forceinline__ uint32_t fuse_valid(int64_t w, int64_t R) {
  const int64_t n = R - 32 * w;
  return n >= 32 ? kFull : (n <= 0 ? 0u : ((1u << n) - 1u));
}

// Whether the evolve kernel evaluates a live child of L columns itself.
__device__ __forceinline__ bool fuse_child(const GenArgs &ga, int L) {
  const int np = L - 1;
  return np <= ga.fuse_np && (ga.rnum * np + ga.rden - 1) / ga.rden == np;
}

// The counts of one pass (lane's 4 words w .. w + 3; act: they exist) from the ANDs of its pair
// rows in each direction.
__device__ __forceinline__ void fuse_pass_counts(const GenArgs &ga, bool neg, bool ns, bool act,
                                                 int64_t w, uint4 ap, uint4 an, int &cp, int &cn,
                                                 int &ca) {
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
  uint4 pos = act ? ap : zero4, ng = (neg && act) ? an : zero4;
  if (ns && act) {  // (pad rows hold complemented zeros)
    const uint4 vm = make_uint4(fuse_valid(w, ga.R), fuse_valid(w + 1, ga.R),
                                fuse_valid(w + 2, ga.R), fuse_valid(w + 3, ga.R));
    pos = fuse_and(pos, vm);
    ng = fuse_and(ng, vm);
  }
  cp += fuse_popc(pos);
  cn += fuse_popc(ng);
  ca += fuse_popc(make_uint4(pos.x | ng.x, pos.y | ng.y, pos.z | ng.z, pos.w | ng.w));
}

// The exact test when a pass's UPP pair rows (pairs x directions) fit in one copy group: a group
// holds kFuseGroup / UPP whole passes, and each lane keeps the UPP rows' addresses (src[u]: its
// words of pass 0; unit u of a pass is pair u / 2's positive (even u) or negative row with
// negative trends, else pair u's row).  NG groups are in flight: 2 in the warp's own region, 4
// with a second region (stage2) borrowed from a warp of the block that has no slot left.
template <int UPP, int NG>
__device__ void w_eval_exact_small(const GenArgs &ga, const uint32_t *const (&src)[4],
                                   uint32_t *stage, uint32_t *stage2, int lane, int &cp, int &cn,
                                   int &ca) {
  constexpr int PPG = kFuseGroup / UPP;  // passes per group
  const bool neg = ga.neg != 0, ns = ga.ns != 0;
  const int64_t Wst = ga.Wst;
  const int passes = (int)((Wst + kFuseWords - 1) / kFuseWords);
  const int n_groups = (passes + PPG - 1) / PPG;
  // group gi's units: half gi & 1 of the own region, or of the borrowed one when gi % NG >= 2
  auto unit = [&](int gi, int k) -> uint32_t * {
    uint32_t *base = (NG > 2 && (gi % NG) >= 2) ? stage2 : stage;
    return base + lane * 4 + ((gi & 1) * kFuseGroup + k) * kFuseWords;
  };
  auto issue = [&](int gi) {
#pragma unroll
    for (int pp = 0; pp < PPG; ++pp) {
      const int q = gi * PPG + pp;
      if (q < passes && (int64_t)q * kFuseWords + lane * 4 < Wst) {
#pragma unroll
        for (int u = 0; u < UPP; ++u)
          fuse_copy16(unit(gi, pp * UPP + u), src[u] + (int64_t)q * kFuseWords);
      }
    }
    fuse_commit();
  };
  const uint4 ones = make_uint4(kFull, kFull, kFull, kFull);
#pragma unroll
  for (int gi = 0; gi < NG; ++gi)
    if (gi < n_groups) issue(gi);
  for (int gi = 0; gi < n_groups; ++gi) {
    // (groups after gi still pending: at most NG - 1)
    const int later = min(NG - 1, n_groups - 1 - gi);
    if (NG > 2 && later >= 3)
      fuse_wait<3>();
    else if (NG > 2 && later == 2)
      fuse_wait<2>();
    else if (later >= 1)
      fuse_wait<1>();
    else
      fuse_wait<0>();
#pragma unroll
    for (int pp = 0; pp < PPG; ++pp) {
      const int q = gi * PPG + pp;
      const int64_t w = (int64_t)q * kFuseWords + lane * 4;
      const bool act = q < passes && w < Wst;
      uint4 ap = ones, an = ones;
      if (act) {
#pragma unroll
        for (int u = 0; u < UPP; ++u) {
          uint4 v = *reinterpret_cast<const uint4 *>(unit(gi, pp * UPP + u));
          if (ns) v = make_uint4(~v.x, ~v.y, ~v.z, ~v.w);
          if (neg && (u & 1))
            an = fuse_and(an, v);
          else
            ap = fuse_and(ap, v);
        }
      }
      if (q < passes) fuse_pass_counts(ga, neg, ns, act, w, ap, an, cp, cn, ca);
    }
    if (gi + NG < n_groups) issue(gi + NG);
  }
}

// Row counts (positive trend, negative trend, either) of the exact test of c[0 .. L-1] (L >= 2),
// in every lane.  stage: the warp's kFuseSlots * kFuseWords words of shared memory (16-byte
// aligned), free for this call; stage2: a second such region (borrowed), or null.  Only passes of
// at most kFuseGroup pair rows use the second region.
__device__ void w_eval_exact(const GenArgs &ga, const int32_t *c, int L, uint32_t *stage,
                             uint32_t *stage2, int lane, int &rp, int &rn, int &ra) {
  const int np = L - 1;
  const bool neg = ga.neg != 0, ns = ga.ns != 0;
  const int upp = neg ? 2 * np : np;  // units per pass: pair j's positive (then negative) row
  const int64_t Wst = ga.Wst;
  if (upp <= kFuseGroup) {
    // every lane: the addresses of the pass's rows (pairs 0 .. np-1 <= 3: columns c[0 .. 4])
    const uint32_t C = (uint32_t)ga.C;
    const uint32_t *src[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = neg ? (u >> 1) : u;
      const bool nd = neg && (u & 1);
      const int jj = j < np ? j : 0;  // (rows past upp are never read)
      const uint32_t a = (uint32_t)c[jj], b = (uint32_t)c[jj + 1];
      const uint32_t row = (ns != nd) ? b * C + a : a * C + b;
      src[u] = ga.bitmap + (int64_t)row * Wst + lane * 4;
    }
    int cp = 0, cn = 0, ca = 0;
    __syncwarp();  // every lane's earlier use of the region is done
    if (stage2) {
      switch (upp) {
        case 1: w_eval_exact_small<1, 4>(ga, src, stage, stage2, lane, cp, cn, ca); break;
        case 2: w_eval_exact_small<2, 4>(ga, src, stage, stage2, lane, cp, cn, ca); break;
        case 3: w_eval_exact_small<3, 4>(ga, src, stage, stage2, lane, cp, cn, ca); break;
        default: w_eval_exact_small<4, 4>(ga, src, stage, stage2, lane, cp, cn, ca); break;
      }
    } else {
      switch (upp) {
        case 1: w_eval_exact_small<1, 2>(ga, src, stage, stage, lane, cp, cn, ca); break;
        case 2: w_eval_exact_small<2, 2>(ga, src, stage, stage, lane, cp, cn, ca); break;
        case 3: w_eval_exact_small<3, 2>(ga, src, stage, stage, lane, cp, cn, ca); break;
        default: w_eval_exact_small<4, 2>(ga, src, stage, stage, lane, cp, cn, ca); break;
      }
    }
    rp = __reduce_add_sync(kFull, cp);
    rn = __reduce_add_sync(kFull, cn);
    ra = __reduce_add_sync(kFull, ca);
    return;
  }
  const int passes = (int)((Wst + kFuseWords - 1) / kFuseWords);
  const int n_groups = (passes * upp + kFuseGroup - 1) / kFuseGroup;
  // lane l: the word rows of pairs l and l + 32 (pair j = (c[j], c[j + 1])), positive and
  // negative direction
  uint32_t row_p[2] = {0u, 0u}, row_n[2] = {0u, 0u};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = lane + 32 * h;
    if (j < np) {
      const uint32_t a = (uint32_t)c[j], b = (uint32_t)c[j + 1], C = (uint32_t)ga.C;
      row_p[h] = ns ? b * C + a : a * C + b;
      row_n[h] = ns ? a * C + b : b * C + a;
    }
  }
  int iq = 0, ir = 0;  // next unit to copy: pass, unit within the pass
  auto issue_group = [&](int gi) {
#pragma unroll
    for (int k = 0; k < kFuseGroup; ++k) {
      if (iq < passes) {
        const int j = neg ? (ir >> 1) : ir, h = j >> 5;  // (the same in every lane)
        const bool nd = neg && (ir & 1);
        const uint32_t row =
            __shfl_sync(kFull, h ? (nd ? row_n[1] : row_p[1]) : (nd ? row_n[0] : row_p[0]),
                        j & 31);
        const int64_t w = (int64_t)iq * kFuseWords + lane * 4;
        if (w < Wst)  // (Wst is a multiple of 4: a lane's 4 words all exist or not)
          fuse_copy16(stage + ((gi & 1) * kFuseGroup + k) * kFuseWords + lane * 4,
                      ga.bitmap + (int64_t)row * Wst + w);
        if (++ir == upp) {
          ir = 0;
          ++iq;
        }
      }
    }
    fuse_commit();
  };
  const uint4 ones = make_uint4(kFull, kFull, kFull, kFull), zero4 = make_uint4(0u, 0u, 0u, 0u);
  uint4 ap = ones, an = ones;
  int cq = 0, cr = 0, cp = 0, cn = 0, ca = 0;
  __syncwarp();  // every lane's earlier use of the region is done
  issue_group(0);
  if (n_groups > 1) issue_group(1);
  for (int gi = 0; gi < n_groups; ++gi) {
    if (gi + 1 < n_groups)
      fuse_wait<1>();
    else
      fuse_wait<0>();
#pragma unroll
    for (int k = 0; k < kFuseGroup; ++k) {
      if (cq < passes) {
        const int64_t w = (int64_t)cq * kFuseWords + lane * 4;
        const bool act = w < Wst;
        if (act) {
          uint4 v = *reinterpret_cast<const uint4 *>(
              stage + ((gi & 1) * kFuseGroup + k) * kFuseWords + lane * 4);
          if (ns) v = make_uint4(~v.x, ~v.y, ~v.z, ~v.w);
          if (neg && (cr & 1))
            an = fuse_and(an, v);
          else
            ap = fuse_and(ap, v);
        }
        if (++cr == upp) {  // the pass is complete
          uint4 pos = act ? ap : zero4, ng = (neg && act) ? an : zero4;
          if (ns && act) {
            const uint4 vm = make_uint4(fuse_valid(w, ga.R), fuse_valid(w + 1, ga.R),
                                        fuse_valid(w + 2, ga.R), fuse_valid(w + 3, ga.R));
            pos = fuse_and(pos, vm);
            ng = fuse_and(ng, vm);
          }
          cp += fuse_popc(pos);
          cn += fuse_popc(ng);
          ca += fuse_popc(make_uint4(pos.x | ng.x, pos.y | ng.y, pos.z | ng.z, pos.w | ng.w));
          ap = ones;
          an = ones;
          cr = 0;
          ++cq;
        }
      }
    }
    if (gi + 2 < n_groups) issue_group(gi + 2);
  }
  rp = __reduce_add_sync(kFull, cp);
  rn = __reduce_add_sync(kFull, cn);
  ra = __reduce_add_sync(kFull, ca);
}

// Per-warp shared memory of k_evolve, in ints: the child (kS + 1 used), then 8 tournament scratch
// rows and the two parents; once the child is final, the region after it stages the pair words
// of its evaluation (kFuseSlots units).  Every part starts on a 16-byte boundary (the scratch
// rows are written with 16-byte stores, the staged units by 16-byte copies), and the total is a
// multiple of 16 bytes.
constexpr int kEvoChild = 0, kEvoScratch = kS + 4, kEvoA = kEvoScratch + 8 * kS,
              kEvoB = kEvoA + kS, kEvoStage = kEvoScratch;
constexpr int kEvolveWarpInts =
    kEvoScratch + (10 * kS > kFuseSlots * kFuseWords ? 10 * kS : kFuseSlots * kFuseWords);
static_assert(kEvoScratch % 4 == 0, "scratch rows and staged units start on 16-byte boundaries");

// The end of a live slot s's evolve step when fusion is on: the slot is evaluated here (its
// counts stored, its key entered in generation g's duplicate table, as the evaluation launch
// would) or listed for the evaluation launch.  Returns its tabu-flag value: 2 evaluated from the
// pair words, 3 (a one-pair chromosome) from the pair-count table, 0 listed.
// s_free (k_evolve_seq; null otherwise): bit w set while warp w of the block has no slot left,
// its region (of kEvolveWarpInts ints from `regions`) then free; a pair-word evaluation borrows
// one such region for two more copy groups in flight and gives it back at its end.
__device__ int fuse_or_list(const GenArgs &ga, const int32_t *c, int L, uint64_t h, int s,
                            int par, uint32_t *stage, int lane, int32_t *regions,
                            uint32_t *s_free) {
  if (fuse_child(ga, L)) {
    int rp = 0, rn = 0, ra = 0;
    const bool table = L == 2 && ga.pair_cnt != nullptr;
    if (table) {
      // one pair (a, b): G[a][b] holds the rows with key(b) > key(a) and G[b][a] the others
      // that differ (the two are disjoint); with ties counting both ways the rows of a
      // direction are the complement of the opposite direction's, and every row holds one
      if (lane == 0) {
        const int a = c[0], b = c[1];
        const bool lo = a < b;  // (the table holds a pair under its lower column)
        const unsigned long long v =
            ga.pair_cnt[(int64_t)(lo ? a : b) * ga.C + (lo ? b : a)];
        const int lo32 = (int)(uint32_t)v, hi32 = (int)(uint32_t)(v >> 32);
        const int ab = lo ? lo32 : hi32, ba = lo ? hi32 : lo32;
        const int R = (int)ga.R;
        if (!ga.ns) {
          rp = ab;
          rn = ga.neg ? ba : 0;
          ra = rp + rn;
        } else {
          rp = R - ba;
          rn = ga.neg ? R - ab : 0;
          ra = ga.neg ? R : rp;
        }
      }
    } else {
      int lent = -1;  // the warp whose region is borrowed
      if (s_free) {
        if (lane == 0) {
          const uint32_t m = *reinterpret_cast<volatile uint32_t *>(s_free);
          if (m) {
            const uint32_t bit = m & (0u - m);  // (the lowest free region)
            if (atomicAnd(s_free, ~bit) & bit) lent = __ffs(bit) - 1;
          }
        }
        lent = __shfl_sync(kFull, lent, 0);
      }
      uint32_t *stage2 =
          lent >= 0 ? reinterpret_cast<uint32_t *>(regions + lent * kEvolveWarpInts + kEvoStage)
                    : nullptr;
      w_eval_exact(ga, c, L, stage, stage2, lane, rp, rn, ra);
      if (lent >= 0) {
        __syncwarp();  // (every lane's copies into it have landed and been read)
        if (lane == 0) atomicOr(s_free, 1u << lent);
      }
    }
    if (lane == 0) {
      ga.rows_scr[s] = rp;
      ga.rows_scr[ga.P + s] = rn;
      ga.rows_scr[2 * ga.P + s] = ra;
      dedup_insert(ga.dkeys[par], ga.dslot[par], ga.dmask, h, s);
    }
    return table ? 3 : 2;
  }
  if (lane == 0) ga.todo[atomicAdd(&ga.ctl->n_todo, 1)] = s;
  return 0;
}

// Step 1: the initial population, one warp per slot (generation 0, attempt 0 of the word
// stream): length init_min + below(init_max - init_min + 1), then that many columns, each by at
// most 64 draws that avoid the columns already present (the chromosome ends early when all 64
// hit).
constexpr int kInitWarps = 8;
__global__ void __launch_bounds__(kInitWarps * 32) k_init(GenArgs ga, Buf nb) {
  __shared__ int32_t s_c[kInitWarps][kS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int s = blockIdx.x * kInitWarps + warp;
  if (s >= ga.P) return;  // (whole warps)
  int32_t *c = s_c[warp];
  WarpStream st(ga.seed, 0u, (uint32_t)s, 0u, lane);
  const int want = ga.init_min + (int)st.below((uint32_t)(ga.init_max - ga.init_min + 1));
  int L = 0;
  for (int j = 0; j < want; ++j) {
    const int v = w_draw_free(st, ga.C, c, L, lane);
    if (v < 0) break;
    if (lane == 0) c[L] = v;
    __syncwarp();
    ++L;
  }
  int32_t *out = nb.cols + (size_t)s * kS;
  out[lane] = lane < L ? c[lane] : 0;
  out[lane + 32] = lane + 32 < L ? c[lane + 32] : 0;
  if (lane == 0) {
    nb.len[s] = L;
    nb.att_dead[s] = L < 2;
    nb.att_hits[s] = 0;
    nb.hash[s] = chromosome_key(c, L);  // (the scoring launch enters live keys in the table)
  }
}

// One block per slot, one warp per attempt (G warps, G = the power of two >= max_attempts): the
// lowest attempt whose key misses the tabu list wins, which is exactly the sequential retry
// rule; when every attempt hits, the slot is dead and keeps the last attempt's child.
constexpr int kMaxAttemptWarps = 16;
// Matrices of up to this many columns have k_evolve's column-usage table in shared memory.
constexpr int kUsageSmemMax = 4096;
// Warps of k_evolve one SM holds at once (its registers allow 32).
constexpr int kEvolveResidentWarps = 32;

// Dynamic shared memory of a k_evolve launch with G warps.
size_t evolve_smem(int G, int C) {
  return (size_t)G * kEvolveWarpInts * 4 + (C <= kUsageSmemMax ? (size_t)(C + 3) / 4 * 16 : 0);
}
static_assert(kEvolveWarpInts % 4 == 0, "per-warp region must keep 16-byte alignment");

__global__ void __launch_bounds__(kMaxAttemptWarps * 32) k_evolve(GenArgs ga, Buf pb, Buf nb,
                                                                  int par) {
  extern __shared__ __align__(16) int32_t s_evo[];  // kEvolveWarpInts per warp, then usage
  __shared__ int s_ok[kMaxAttemptWarps];
  wait_prior_grid();
  const int stopped = ga.ctl->stopped, gen = ga.ctl->gen, n_top = ga.ctl->n_top;
  // the column-usage table goes to shared memory (its loads leave with the counters' loads)
  const int32_t *usage = ga.usage;
  if (ga.C <= kUsageSmemMax) {
    int32_t *s_usage = s_evo + (blockDim.x >> 5) * kEvolveWarpInts;
    for (int c = threadIdx.x; c < ga.C; c += blockDim.x) s_usage[c] = ga.usage[c];
    usage = s_usage;
  }
  if (stopped) return;
  __syncthreads();
  const int lane = threadIdx.x & 31, a = threadIdx.x >> 5;
  const int s = blockIdx.x;
  const int g = gen + 1;
  const int n_el = min(ga.E, n_top);
  int32_t *out = nb.cols + (size_t)s * kS;
  if (s < n_el) {  // elitism: copy top-list entry s (its key is already in the tabu list)
    if (a == 0) {
      const TopEntry &e = ga.top[s];
      out[lane] = lane < e.len ? e.cols[lane] : 0;
      out[lane + 32] = lane + 32 < e.len ? e.cols[lane + 32] : 0;
      if (lane == 0) {
        nb.len[s] = e.len;
        nb.hash[s] = e.h;
        nb.att_dead[s] = 0;
        nb.att_hits[s] = 0;
        if (ga.fuse_np > 0) ga.todo[atomicAdd(&ga.ctl->n_todo, 1)] = s;
      }
    }
    return;
  }
  int32_t *base = s_evo + a * kEvolveWarpInts;
  int32_t *scratch = base + kEvoScratch, *A = base + kEvoA, *B = base + kEvoB;
  int32_t *c = base + kEvoChild;
  int L = 0;
  uint64_t h = 0ull;
  int ok = 0;
  if (a < ga.A) {
    w_make_child(ga, pb, g, s, a, c, scratch, A, B, L, lane, usage);
    h = chromosome_key(c, L);
    // lane 0 probes the hashed tabu list, lane 1 generation g-1's live keys
    const bool hit = (lane == 0 && tabu_contains(ga.tabu, ga.tmask, h)) ||
                     (lane == 1 && tabu_contains(ga.dkeys[par ^ 1], ga.dmask, h));
    ok = !__any_sync(kFull, hit);
  }
  if (lane == 0) s_ok[a] = ok;
  __syncthreads();
  int win = -1;
  for (int q = 0; q < ga.A; ++q)
    if (s_ok[q]) {
      win = q;
      break;
    }
  const bool dead = win < 0;
  if (dead) win = ga.A - 1;
  if (a != win) return;
  out[lane] = lane < L ? c[lane] : 0;
  out[lane + 32] = lane + 32 < L ? c[lane + 32] : 0;
  const int fused = (!dead && ga.fuse_np > 0)
                        ? fuse_or_list(ga, c, L, h, s, par,
                                       reinterpret_cast<uint32_t *>(base + kEvoStage), lane,
                                       nullptr, nullptr)
                        : 0;
  if (lane == 0) {
    nb.len[s] = L;
    nb.hash[s] = h;
    // 1: dead; 2 or 3: live and evaluated here; 0: live, left to the evaluation launch (which
    // enters the live keys in D[par])
    nb.att_dead[s] = dead ? 1 : fused;
    nb.att_hits[s] = dead ? ga.A : win;
  }
}

// The same step for large populations, one warp per slot: a slot's attempts run one after the
// other in its warp, until one misses the tabu list, which is the retry rule itself (the lowest
// missing attempt wins; all A hit: the slot is dead with the last attempt's child).  Parallel
// attempt warps only shorten a slot's latency; when the launch has more slots than the GPU holds
// at once, the slots themselves fill it, and a warp per slot keeps four times as many of them in
// flight.  The launch is persistent: as many blocks of kSeqWarps warps as are resident at once,
// each warp taking its first slot by its index and later ones from a counter as it finishes, so
// warps building children (dependent loads, little traffic) and warps evaluating them (pair-word
// streams) overlap instead of alternating in waves of blocks.  The block's warps share one copy
// of the column-usage table.
constexpr int kSeqWarps = 8;

__global__ void __launch_bounds__(kSeqWarps * 32, 4) k_evolve_seq(GenArgs ga, Buf pb, Buf nb,
                                                               int par) {
  extern __shared__ __align__(16) int32_t s_evo[];  // kEvolveWarpInts per warp, then usage
  __shared__ uint32_t s_free;  // bit w: warp w has no slot left, its region free to borrow
  wait_prior_grid();
  const int stopped = ga.ctl->stopped, gen = ga.ctl->gen, n_top = ga.ctl->n_top;
  const int32_t *usage = ga.usage;
  if (ga.C <= kUsageSmemMax) {
    int32_t *s_usage = s_evo + kSeqWarps * kEvolveWarpInts;
    for (int c = threadIdx.x; c < ga.C; c += blockDim.x) s_usage[c] = ga.usage[c];
    usage = s_usage;
  }
  if (stopped) return;
  if (threadIdx.x == 0) s_free = 0u;
  __syncthreads();  // (no block-wide operation follows)
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int W = (int)gridDim.x * kSeqWarps;
  const int g = gen + 1;
  const int n_el = min(ga.E, n_top);
  int32_t *base = s_evo + w * kEvolveWarpInts;
  int32_t *scratch = base + kEvoScratch, *A = base + kEvoA, *B = base + kEvoB;
  int32_t *c = base + kEvoChild;
  for (int s = blockIdx.x * kSeqWarps + w; s < ga.P;) {
    int32_t *out = nb.cols + (size_t)s * kS;
    if (s < n_el) {  // elitism: copy top-list entry s (its key is already in the tabu list)
      const TopEntry &e = ga.top[s];
      out[lane] = lane < e.len ? e.cols[lane] : 0;
      out[lane + 32] = lane + 32 < e.len ? e.cols[lane + 32] : 0;
      if (lane == 0) {
        nb.len[s] = e.len;
        nb.hash[s] = e.h;
        nb.att_dead[s] = 0;
        nb.att_hits[s] = 0;
        if (ga.fuse_np > 0) ga.todo[atomicAdd(&ga.ctl->n_todo, 1)] = s;
      }
    } else {
      int L = 0, win = -1;
      uint64_t h = 0ull;
      for (int a = 0; a < ga.A; ++a) {
        w_make_child(ga, pb, g, s, a, c, scratch, A, B, L, lane, usage);
        h = chromosome_key(c, L);
        // lane 0 probes the hashed tabu list, lane 1 generation g-1's live keys
        const bool hit = (lane == 0 && tabu_contains(ga.tabu, ga.tmask, h)) ||
                         (lane == 1 && tabu_contains(ga.dkeys[par ^ 1], ga.dmask, h));
        if (!__any_sync(kFull, hit)) {
          win = a;
          break;
        }
      }
      const bool dead = win < 0;
      __syncwarp();
      out[lane] = lane < L ? c[lane] : 0;
      out[lane + 32] = lane + 32 < L ? c[lane + 32] : 0;
      const int fused = (!dead && ga.fuse_np > 0)
                            ? fuse_or_list(ga, c, L, h, s, par,
                                           reinterpret_cast<uint32_t *>(base + kEvoStage), lane,
                                           s_evo, &s_free)
                            : 0;
      if (lane == 0) {
        nb.len[s] = L;
        nb.hash[s] = h;
        nb.att_dead[s] = dead ? 1 : fused;  // (as in k_evolve)
        nb.att_hits[s] = dead ? ga.A : win;
      }
    }
    if (W >= ga.P) break;  // (every slot was some warp's first)
    int nx = 0;
    if (lane == 0) nx = atomicAdd(&ga.ctl->evo_next, 1);
    s = __shfl_sync(kFull, nx, 0) + W;
    __syncwarp();  // (the region's last reads are done before the next slot writes it)
  }
  // no slot left: the warp's region can stage a sibling's evaluation
  __syncwarp();
  if (lane == 0) atomicOr(&s_free, 1u << w);
}

__device__ __forceinline__ bool key_before(uint64_t fa, uint64_t ha, uint64_t fb, uint64_t hb) {
  return fa > fb || (fa == fb && ha < hb);
}

// Bitonic sort of n (f, h, s) candidates into "rank" order (f descending, key ascending) by the
// whole block; arrays hold N = next power of two >= n entries (padding written here).
__device__ void block_sort(uint64_t *f, uint64_t *h, int32_t *sl, int n) {
  int N = 1;
  while (N < n) N <<= 1;
  for (int i = n + threadIdx.x; i < N; i += blockDim.x) {
    f[i] = 0ull;
    h[i] = ~0ull;
    sl[i] = 0x7FFFFFFF;
  }
  __syncthreads();
  for (int k = 2; k <= N; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool asc = (i & k) == 0;
          const uint64_t fi = f[i], fl = f[l], hi = h[i], hl = h[l];
          const bool l_first = key_before(fl, hl, fi, hi);
          if (asc ? l_first : !l_first) {
            f[i] = fl;
            f[l] = fi;
            h[i] = hl;
            h[l] = hi;
            const int32_t t = sl[i];
            sl[i] = sl[l];
            sl[l] = t;
          }
        }
      }
      __syncthreads();
    }
  }
}

constexpr int kChunk = 32;  // candidates whose data is staged in shared memory at a time

struct TopSmem {
  TopEntry *pool;    // K + 1 entries
  uint32_t *colbits; // ceil(C / 32) words
  int32_t *idx;      // K + 1: pool index of list position
  int32_t *idx2;     // K + 1
  int32_t *ov;       // K + 1: columns each list entry shares with the candidate
  uint8_t *used;     // K + 1
  uint64_t *sf, *sh; // sort_cap
  int32_t *ss;
  int32_t *ccols;    // kChunk x kS: columns of the staged candidates
  int32_t *cmeta;    // kChunk x 4: length, rows_pos, rows_neg, rows_any
};

// Number of columns of pool entry e present in colbits (warp-wide).
__device__ __forceinline__ int overlap(const TopSmem &sm, const TopEntry &e, int lane) {
  int cnt = 0;
  for (int k = lane; k < e.len; k += 32) {
    const int v = e.cols[k];
    cnt += (sm.colbits[v >> 5] >> (v & 31)) & 1u;
  }
  return __reduce_add_sync(kFull, cnt);
}

// Top-list update over the staged, sorted candidates q0..q1-1 (their data is in sm.ccols /
// sm.cmeta at q - q0), one candidate after the other, by the whole block: warp 0 finds the
// candidate's rank and marks its columns; every warp then counts, for its share of the list's
// entries, the columns the entry shares with the candidate (sm.ov); warp 0 applies the
// admission and eviction rule with those counts.  Returns the new list length; *s_stop is set
// when a candidate ranks at position >= K (every later candidate ranks lower still).  Called by
// every thread of the block.
__device__ int process_chunk(const GenArgs &ga, const TopSmem &sm, int n, const uint64_t *cf,
                             const uint64_t *ch, int q0, int q1, int *s_stop) {
  __shared__ int s_pos, s_dup, s_n;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (threadIdx.x == 0) s_n = n;
  for (int q = q0; q < q1; ++q) {
    const uint64_t f = cf[q], h = ch[q];
    const int32_t *cc = sm.ccols + (q - q0) * kS;
    const int L = sm.cmeta[(q - q0) * 4];
    const int c0 = lane < L ? cc[lane] : 0, c1 = lane + 32 < L ? cc[lane + 32] : 0;
    if (warp == 0) {
      int pos = 0;
      bool dup = false;
      for (int e0 = 0; e0 < n; e0 += 32) {
        const int e = e0 + lane;
        bool isdup = false, before = false;
        if (e < n) {
          const TopEntry &E = sm.pool[sm.idx[e]];
          isdup = E.h == h;
          before = key_before(E.f, E.h, f, h);
        }
        dup |= __any_sync(kFull, isdup);
        pos += __popc(__ballot_sync(kFull, before));
      }
      if (!dup && pos < ga.K) {  // the candidate's columns, for the overlap counts
        if (lane < L) atomicOr(&sm.colbits[c0 >> 5], 1u << (c0 & 31));
        if (lane + 32 < L) atomicOr(&sm.colbits[c1 >> 5], 1u << (c1 & 31));
      }
      if (lane == 0) {
        s_pos = pos;
        s_dup = dup;
      }
    }
    __syncthreads();
    const int pos = s_pos;
    if (s_dup) {  // (uniform) every thread has read s_pos / s_dup before warp 0 rewrites them
      __syncthreads();
      continue;
    }
    if (pos >= ga.K) {    // the list is full and every later candidate ranks after it
      if (threadIdx.x == 0) *s_stop = 1;
      break;
    }
    for (int e = warp; e < n; e += nwarps) {
      const int inter = overlap(sm, sm.pool[sm.idx[e]], lane);
      if (lane == 0) sm.ov[e] = inter;
    }
    __syncthreads();
    if (warp == 0) {
      bool ok = true;
      for (int e = lane; e < pos; e += 32)
        ok &= (long long)sm.ov[e] * ga.ov_den <= (long long)ga.ov_num * L;
      ok = __all_sync(kFull, ok);
      if (ok) {
        // a free pool slot: the pool has K + 1 entries and the list at most K
        int fr = -1;
        for (int b0 = 0; b0 <= ga.K && fr < 0; b0 += 32) {
          const int b = b0 + lane;
          const unsigned m = __ballot_sync(kFull, b <= ga.K && !sm.used[b]);
          if (m) fr = b0 + __ffs(m) - 1;
        }
        TopEntry &ne = sm.pool[fr];
        ne.cols[lane] = lane < L ? c0 : 0;
        ne.cols[lane + 32] = lane + 32 < L ? c1 : 0;
        if (lane == 0) {
          ne.len = L;
          ne.f = f;
          ne.h = h;
          ne.rp = sm.cmeta[(q - q0) * 4 + 1];
          ne.rn = sm.cmeta[(q - q0) * 4 + 2];
          ne.ra = sm.cmeta[(q - q0) * 4 + 3];
          sm.used[fr] = 1;
        }
        // entries after the candidate stay when they share at most the allowed fraction of
        // their own columns with it (in order, the list cut to K)
        for (int e = lane; e < pos; e += 32) sm.idx2[e] = sm.idx[e];
        int m = pos + 1;
        for (int e0 = pos; e0 < n; e0 += 32) {
          const int e = e0 + lane;
          bool keep = false;
          int pe = 0;
          if (e < n) {
            pe = sm.idx[e];
            keep = (long long)sm.ov[e] * ga.ov_den <= (long long)ga.ov_num * sm.pool[pe].len;
          }
          const unsigned km = __ballot_sync(kFull, keep);
          const int dst = m + __popc(km & lanes_below(lane));
          if (e < n) {
            if (keep && dst < ga.K) sm.idx2[dst] = pe;
            else sm.used[pe] = 0;
          }
          m += __popc(km);
        }
        m = min(m, ga.K);
        __syncwarp();
        if (lane == 0) sm.idx2[pos] = fr;
        __syncwarp();
        for (int e = lane; e < m; e += 32) sm.idx[e] = sm.idx2[e];
        if (lane == 0) s_n = m;
      }
      __syncwarp();
      if (lane < L) atomicAnd(&sm.colbits[c0 >> 5], ~(1u << (c0 & 31)));
      if (lane + 32 < L) atomicAnd(&sm.colbits[c1 >> 5], ~(1u << (c1 & 31)));
    }
    __syncthreads();
    n = s_n;
  }
  __syncthreads();
  return s_n;
}

// Bitonic sort of up to 32 candidates across the lanes of one warp (lane i holds candidate i or
// a sentinel that sorts last); results land in sf/sh/ss[0..count).
__device__ void warp_sort(const uint64_t *gf, const uint64_t *gh, const int32_t *gs, int count,
                          uint64_t *sf, uint64_t *sh, int32_t *ss, int lane) {
  uint64_t f = lane < count ? gf[lane] : 0ull;
  uint64_t h = lane < count ? gh[lane] : ~0ull;
  int32_t sl = lane < count ? gs[lane] : 0x7FFFFFFF;
  __syncwarp();
  for (int k = 2; k <= 32; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      const uint64_t pf = __shfl_xor_sync(kFull, f, j), ph = __shfl_xor_sync(kFull, h, j);
      const int32_t ps = __shfl_xor_sync(kFull, sl, j);
      const bool up = (lane & k) == 0, lower = (lane & j) == 0;
      const bool partner_first = key_before(pf, ph, f, h);
      const bool partner_later = key_before(f, h, pf, ph);
      const bool take = (lower == up) ? partner_first : partner_later;
      if (take) {
        f = pf;
        h = ph;
        sl = ps;
      }
    }
  }
  if (lane < count) {
    sf[lane] = f;
    sh[lane] = h;
    ss[lane] = sl;
  }
}

// Sorts `count` candidates held in global arrays (within a warp, in shared memory, or in place
// in global memory, by size), then stages them kChunk at a time in shared memory and lets warp 0
// process each chunk.  Returns the new list length (valid in every thread).
__device__ int sort_and_process(const GenArgs &ga, const Buf &nb, const TopSmem &sm, int n,
                                int count, bool in_smem, int *s_n, int *s_stop) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int N = 1;
  while (N < count) N <<= 1;
  const uint64_t *cf;
  const uint64_t *ch;
  const int32_t *cs;
  if (in_smem) {  // already in sm.sf / sh / ss (count <= sort_cap)
    if (count <= 32) {
      if (warp == 0) warp_sort(sm.sf, sm.sh, sm.ss, count, sm.sf, sm.sh, sm.ss, lane);
    } else {
      block_sort(sm.sf, sm.sh, sm.ss, count);
    }
    __syncthreads();
    cf = sm.sf;
    ch = sm.sh;
    cs = sm.ss;
  } else if (count <= 32) {
    // written by other blocks: read from L2
    if (warp == 0) {
      const uint64_t *gf = ga.cand_f, *gh = ga.cand_h;
      const int32_t *gs = ga.cand_s;
      for (int i = lane; i < count; i += 32) {
        sm.sf[i] = __ldcg(gf + i);
        sm.sh[i] = __ldcg(gh + i);
        sm.ss[i] = __ldcg(gs + i);
      }
      __syncwarp();
      warp_sort(sm.sf, sm.sh, sm.ss, count, sm.sf, sm.sh, sm.ss, lane);
    }
    __syncthreads();
    cf = sm.sf;
    ch = sm.sh;
    cs = sm.ss;
  } else if (N <= ga.sort_cap) {
    for (int i = threadIdx.x; i < count; i += blockDim.x) {
      sm.sf[i] = __ldcg(ga.cand_f + i);
      sm.sh[i] = __ldcg(ga.cand_h + i);
      sm.ss[i] = __ldcg(ga.cand_s + i);
    }
    __syncthreads();
    block_sort(sm.sf, sm.sh, sm.ss, count);
    cf = sm.sf;
    ch = sm.sh;
    cs = sm.ss;
  } else {
    block_sort(ga.cand_f, ga.cand_h, ga.cand_s, count);
    cf = ga.cand_f;
    ch = ga.cand_h;
    cs = ga.cand_s;
  }
  if (threadIdx.x == 0) {
    *s_n = n;
    *s_stop = 0;
  }
  for (int q0 = 0; q0 < count; q0 += kChunk) {
    const int q1 = min(count, q0 + kChunk);
    for (int i = threadIdx.x; i < (q1 - q0) * kS; i += blockDim.x) {
      const int q = q0 + i / kS, k = i - (i / kS) * kS;
      sm.ccols[i] = __ldcg(nb.cols + (size_t)cs[q] * kS + k);
    }
    for (int i = threadIdx.x; i < q1 - q0; i += blockDim.x) {
      const int sl = cs[q0 + i];
      sm.cmeta[i * 4] = __ldcg(nb.len + sl);
      sm.cmeta[i * 4 + 1] = __ldcg(nb.rows + sl);
      sm.cmeta[i * 4 + 2] = __ldcg(nb.rows + ga.P + sl);
      sm.cmeta[i * 4 + 3] = __ldcg(nb.rows + 2 * ga.P + sl);
    }
    __syncthreads();
    const int m = process_chunk(ga, sm, *s_n, cf, ch, q0, q1, s_stop);
    if (threadIdx.x == 0) *s_n = m;
    __syncthreads();
    if (*s_stop) break;
  }
  return *s_n;
}

// A slot's inputs to scoring: every load first, then the duplicate lookup (probed whatever
// the dead flag says, so that its loads need not wait for it).
struct SlotIn {
  bool att_dead, fused, table, in_dup;
  uint64_t h;
  int L, ah, rp, rn, ra;
};

__device__ __forceinline__ SlotIn load_slot(const GenArgs &ga, const Buf &nb, int par, int s) {
  SlotIn in;
  const uint8_t ad = nb.att_dead[s];  // 1: dead; 2, 3: live, evaluated by the evolve kernel
  in.att_dead = ad == 1;
  in.fused = ad >= 2;
  in.table = ad == 3;
  in.h = nb.hash[s];
  in.L = nb.len[s];
  in.ah = nb.att_hits[s];
  in.rp = ga.rows_scr[s];
  in.rn = ga.rows_scr[ga.P + s];
  in.ra = ga.rows_scr[2 * ga.P + s];
  in.in_dup = dedup_is_dup(ga.dkeys[par], ga.dslot[par], ga.dmask, in.h, s);
  return in;
}

// Scoring, tabu bookkeeping and the top-list update of generation g (parity par).  Every block
// scores a share of the slots; the last block to finish then runs the single-block part.
__global__ void __launch_bounds__(kTopThreads, 1) k_finish(GenArgs ga, Buf nb, int par) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_hits, s_live, s_lsum, s_fused, s_flsum, s_table, s_last, s_n, s_cnt, s_stop,
      s_nc;
  GenCtl *ctl = ga.ctl;
  wait_prior_grid();
  // The counters, the list's last entry and this thread's first slot are loaded in one round,
  // ahead of the stop test (which must still come before any store).
  const int stopped = ctl->stopped, n0 = ctl->n_top, gen0 = ctl->gen;
  const uint64_t last_f = ga.top[ga.K - 1].f, last_h = ga.top[ga.K - 1].h;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  SlotIn first;
  if (tid < ga.P) first = load_slot(ga, nb, par, tid);
  if (stopped) return;
  // A single block keeps the candidates and counters in shared memory; several blocks use the
  // global arrays and counters and hand over to the last block to finish.
  const bool single = gridDim.x == 1 && ga.P <= ga.sort_cap;
  TopSmem sm;
  const int cw = (ga.C + 31) / 32;
  sm.pool = reinterpret_cast<TopEntry *>(smem);
  sm.sf = reinterpret_cast<uint64_t *>(sm.pool + ga.K + 1);
  sm.sh = sm.sf + ga.sort_cap;
  sm.colbits = reinterpret_cast<uint32_t *>(sm.sh + ga.sort_cap);
  sm.ss = reinterpret_cast<int32_t *>(sm.colbits + cw);
  sm.idx = sm.ss + ga.sort_cap;
  sm.idx2 = sm.idx + ga.K + 1;
  sm.ov = sm.idx2 + ga.K + 1;
  sm.ccols = sm.ov + ga.K + 1;
  sm.cmeta = sm.ccols + kChunk * kS;
  sm.used = reinterpret_cast<uint8_t *>(sm.cmeta + kChunk * 4);
  if (threadIdx.x == 0) {
    s_hits = 0;
    s_live = 0;
    s_lsum = 0;
    s_fused = 0;
    s_flsum = 0;
    s_table = 0;
    s_nc = 0;
  }
  __syncthreads();
  const bool had_threshold = n0 >= ga.K;
  const uint64_t tf = had_threshold ? last_f : 0ull;
  const uint64_t th = had_threshold ? last_h : 0ull;
  // Elites (copies of the first n_el entries) are no candidates: while their entry is in the
  // list they are skipped as duplicates, and an entry evicted by a better candidate fails the
  // same overlap test as its copy would, so leaving them out changes nothing.
  const int n_el = gen0 < 0 ? 0 : min(ga.E, n0);
  int hits = 0, live = 0, lsum = 0, fused = 0, flsum = 0, table = 0;
  for (int s = tid; s < ga.P; s += stride) {
    const SlotIn in = s == tid ? first : load_slot(ga, nb, par, s);
    const bool att_dead = in.att_dead;
    const uint64_t h = in.h;
    const int L = in.L, ah = in.ah, rp = in.rp, rn = in.rn, ra = in.ra;
    const bool dup = !att_dead && in.in_dup;
    const bool dead = att_dead || dup;
    const uint64_t f =
        (dead || ra < ga.min_rows) ? 0ull : ((uint64_t)ra << (L < ga.col_cap ? L : ga.col_cap));
    nb.dead[s] = dead;
    ga.rows_scr[s] = 0;
    ga.rows_scr[ga.P + s] = 0;
    ga.rows_scr[2 * ga.P + s] = 0;
    nb.rows[s] = dead ? 0 : rp;  // (a duplicate was evaluated, and is not scored)
    nb.rows[ga.P + s] = dead ? 0 : rn;
    nb.rows[2 * ga.P + s] = dead ? 0 : ra;
    nb.fit[s] = f;
    hits += ah + (dup ? 1 : 0);
    live += !dead;
    lsum += dead ? 0 : L;
    fused += (!dead && in.fused) ? 1 : 0;
    flsum += (!dead && in.fused) ? L : 0;
    table += (!dead && in.table) ? 1 : 0;
    if (s >= n_el && !dead && f > 0ull && (!had_threshold || key_before(f, h, tf, th))) {
      if (single) {  // at most P <= sort_cap candidates
        const int q = atomicAdd(&s_nc, 1);
        sm.sf[q] = f;
        sm.sh[q] = h;
        sm.ss[q] = s;
      } else {
        const int q = atomicAdd(&ctl->n_cand, 1);
        ga.cand_f[q] = f;
        ga.cand_h[q] = h;
        ga.cand_s[q] = s;
      }
    }
  }
  hits = __reduce_add_sync(kFull, hits);
  live = __reduce_add_sync(kFull, live);
  lsum = __reduce_add_sync(kFull, lsum);
  fused = __reduce_add_sync(kFull, fused);
  flsum = __reduce_add_sync(kFull, flsum);
  table = __reduce_add_sync(kFull, table);
  if ((threadIdx.x & 31) == 0) {
    if (hits) atomicAdd(&s_hits, hits);
    if (live) atomicAdd(&s_live, live);
    if (lsum) atomicAdd(&s_lsum, lsum);
    if (fused) atomicAdd(&s_fused, fused);
    if (flsum) atomicAdd(&s_flsum, flsum);
    if (table) atomicAdd(&s_table, table);
  }
  __syncthreads();
  int hits_g, live_g, nc, fused_g, table_g;
  long long len_g, flen_g;
  if (single) {
    hits_g = s_hits;
    live_g = s_live;
    len_g = s_lsum;
    fused_g = s_fused;
    flen_g = s_flsum;
    table_g = s_table;
    nc = s_nc;
  } else {
    if (threadIdx.x == 0) {
      if (s_hits) atomicAdd(&ctl->hits_cur, s_hits);
      if (s_live) atomicAdd(&ctl->live_cur, s_live);
      if (s_lsum)
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->len_cur),
                  (unsigned long long)s_lsum);
      if (s_fused) atomicAdd(&ctl->fused_cur, s_fused);
      if (s_table) atomicAdd(&ctl->table_cur, s_table);
      if (s_flsum)
        atomicAdd(reinterpret_cast<unsigned long long *>(&ctl->flen_cur),
                  (unsigned long long)s_flsum);
      __threadfence();
      s_last = atomicAdd(&ctl->done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    hits_g = __ldcg(&ctl->hits_cur);
    live_g = __ldcg(&ctl->live_cur);
    len_g = __ldcg(&ctl->len_cur);
    fused_g = __ldcg(&ctl->fused_cur);
    flen_g = __ldcg(&ctl->flen_cur);
    table_g = __ldcg(&ctl->table_cur);
    nc = __ldcg(&ctl->n_cand);
  }

  // ---- last block: step 6, then the top rank list (step 7)
  const bool init = ctl->gen < 0;
  if (!init && ga.tabu_limit > 0 && hits_g >= ga.tabu_limit) {
    if (threadIdx.x == 0) {
      ctl->hits_last = hits_g;
      ctl->stopped = 1;
      ctl->n_evaluated += live_g;          // the generation was evaluated, then discarded
      ctl->sum_len += len_g;
      ctl->n_fused += fused_g;
      ctl->fused_len += flen_g;
      ctl->n_table += table_g;
    }
    return;
  }
  if (nc == 0) {  // no candidate ranks before the list's last entry: the list stays as it is
    if (threadIdx.x == 0) {
      ctl->hits_last = hits_g;
      ctl->gen += 1;
      ctl->n_evaluated += live_g;
      ctl->sum_len += len_g;
      ctl->n_fused += fused_g;
      ctl->fused_len += flen_g;
      ctl->n_table += table_g;
      ctl->len_cur = 0;
      ctl->hits_cur = 0;
      ctl->live_cur = 0;
      ctl->fused_cur = 0;
      ctl->flen_cur = 0;
      ctl->table_cur = 0;
      ctl->n_todo = 0;
      ctl->evo_next = 0;
      ctl->n_cand = 0;
      ctl->done = 0;
      *ga.work = 0;
    }
    return;
  }
  for (int i = threadIdx.x; i < cw; i += blockDim.x) sm.colbits[i] = 0u;
  for (int e = threadIdx.x; e <= ga.K; e += blockDim.x) {
    sm.used[e] = e < n0;
    sm.idx[e] = e;
  }
  for (int q = threadIdx.x; q < n0 * (int)(sizeof(TopEntry) / 4); q += blockDim.x)
    reinterpret_cast<int32_t *>(sm.pool)[q] = reinterpret_cast<const int32_t *>(ga.top)[q];
  __syncthreads();
  int n = n0;
  if (nc > 0) n = sort_and_process(ga, nb, sm, n, nc, single, &s_n, &s_stop);
  if (had_threshold && n < ga.K) {
    // Evictions left room: the candidates ranking after the old threshold come next.
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < ga.P; s += blockDim.x) {
      const uint64_t f = __ldcg(nb.fit + s), h = __ldcg(nb.hash + s);
      if (!__ldcg(nb.dead + s) && f > 0ull && !key_before(f, h, tf, th)) {
        const int q = atomicAdd(&s_cnt, 1);
        ga.cand_f[q] = f;
        ga.cand_h[q] = h;
        ga.cand_s[q] = s;
      }
    }
    __syncthreads();
    const int cnt = s_cnt;
    __syncthreads();
    if (cnt > 0) n = sort_and_process(ga, nb, sm, n, cnt, false, &s_n, &s_stop);
  }
  const int words = (int)(sizeof(TopEntry) / 4);
  for (int q = threadIdx.x; q < n * words; q += blockDim.x) {
    const int e = q / words, w = q - e * words;
    reinterpret_cast<int32_t *>(ga.top + e)[w] =
        reinterpret_cast<const int32_t *>(sm.pool + sm.idx[e])[w];
  }
  for (int c = threadIdx.x; c < ga.C; c += blockDim.x) ga.usage[c] = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < n * kS; q += blockDim.x) {
    const int e = q / kS, k = q - e * kS;
    const TopEntry &E = sm.pool[sm.idx[e]];
    if (k < E.len) atomicAdd(&ga.usage[E.cols[k]], 1);
  }
  if (threadIdx.x == 0) {
    ctl->hits_last = hits_g;
    ctl->n_top = n;
    ctl->gen += 1;
    ctl->n_evaluated += live_g;
    ctl->sum_len += len_g;
    ctl->n_fused += fused_g;
    ctl->fused_len += flen_g;
    ctl->n_table += table_g;
    ctl->len_cur = 0;
    ctl->hits_cur = 0;
    ctl->live_cur = 0;
    ctl->fused_cur = 0;
    ctl->flen_cur = 0;
    ctl->table_cur = 0;
    ctl->n_todo = 0;
    ctl->evo_next = 0;
    ctl->n_cand = 0;
    ctl->done = 0;
    *ga.work = 0;
  }
}

// Step 9: row masks of the top-list entries, one warp per (entry, 32-row word), from the keys.
__global__ void __launch_bounds__(256) k_extract(const uint32_t *__restrict__ keys, int64_t R,
                                                 int64_t R_pad, int64_t Wst, const TopEntry *top,
                                                 const GenCtl *ctl, int neg, int rnum, int rden,
                                                 uint32_t *__restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n = ctl->n_top;
  if (gw >= (int64_t)n * Wst) return;
  const int e = (int)(gw / Wst);
  const int64_t w = gw - (int64_t)e * Wst;
  const TopEntry &E = top[e];
  const int64_t r = w * 32 + lane;
  bool acc = false;
  if (r < R) {
    const int t = (rnum * (E.len - 1) + rden - 1) / rden;
    uint32_t prev = keys[(int64_t)E.cols[0] * R_pad + r];
    int inc = 0, dec = 0;
    for (int k = 1; k < E.len; ++k) {
      const uint32_t cur = keys[(int64_t)E.cols[k] * R_pad + r];
      inc += cur > prev;
      dec += cur < prev;
      prev = cur;
    }
    acc = inc >= t || (neg && dec >= t);
  }
  const uint32_t m = __ballot_sync(kFull, acc);
  if (lane == 0) out[(int64_t)e * Wst + w] = m;
}

__global__ void k_rehash(const uint64_t *old_keys, uint32_t old_cap, uint64_t *keys,
                         uint32_t mask) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < old_cap && old_keys[i]) tabu_insert(keys, mask, old_keys[i]);
}

__global__ void k_tabu_load(const uint64_t *list, int64_t n, uint64_t *keys, uint32_t mask) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) tabu_insert(keys, mask, list[i]);
}

}  // namespace

// ------------------------------------------------------------------------------ host state

struct GenState {
  ebic_params p{};
  int P = 0, K = 0, C = 0, eval_mode = EBIC_MODE_DIRECT;
  bool initialised = false;
  bool reset_pending = false;          // the run state must be cleared before the next run
  const void *graph_buf = nullptr;  // codes or bitmap the captured graphs read (null: keys)
  const void *graph_cnt = nullptr;  // pair-count table the captured graphs read (or null)
  DevBuf cols[2], len[2], att_hits[2], rows[2], att_dead[2], dead[2], hash[2], fit[2];
  DevBuf dkeys[2], dslot[2];
  DevBuf rows_scr, work, tabu, top, ctl, usage, cand_f, cand_h, cand_s, extract, todo;
  uint32_t tcap = 0, dcap = 0, ccap = 0;
  int fuse_np = 0;  // pair limit of the evaluation inside the evolve kernel (0: none)
  int seq_blocks = 1;  // blocks of the persistent k_evolve_seq launch
  int32_t sort_cap = 0;
  int finish_blocks = 1;
  size_t top_smem = 0;
  // [parity][0]: the plain generation graph; [parity][1]: the same with event-record nodes
  // between the kernels, used while kernel statistics are on (its source graph is kept alive,
  // because the event nodes are re-pointed at fresh events before each replay)
  cudaGraphExec_t graph[2][2] = {};
  cudaGraph_t graph_src[2][2] = {};
  // kGraphGenerations consecutive generations in one graph, by the parity of the first one (the
  // kernels of successive generations then overlap through programmatic launches, which a graph
  // launch per generation would not allow)
  cudaGraphExec_t multi[2] = {};
  cudaGraphNode_t mark_node[2][4] = {};
  cudaEvent_t cap_ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaStream_t cap_stream = nullptr;

  void drop_graphs() {
    for (int k = 0; k < 2; ++k) {
      if (multi[k]) cudaGraphExecDestroy(multi[k]);
      multi[k] = nullptr;
    }
    for (int k = 0; k < 2; ++k)
      for (int v = 0; v < 2; ++v) {
        if (graph[k][v]) cudaGraphExecDestroy(graph[k][v]);
        if (graph_src[k][v]) cudaGraphDestroy(graph_src[k][v]);
        graph[k][v] = nullptr;
        graph_src[k][v] = nullptr;
      }
  }
  ~GenState() {
    drop_graphs();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    for (cudaEvent_t e : cap_ev)
      if (e) cudaEventDestroy(e);
    DevBuf *all[] = {&rows_scr, &work, &tabu, &dkeys[0], &dslot[0], &dkeys[1], &dslot[1], &top,
                     &ctl, &usage, &cand_f, &cand_h, &cand_s, &extract, &todo};
    for (DevBuf *b : all) b->release();
    for (int k = 0; k < 2; ++k) {
      DevBuf *bs[] = {&cols[k], &len[k], &att_hits[k], &rows[k], &att_dead[k], &dead[k],
                      &hash[k], &fit[k]};
      for (DevBuf *b : bs) b->release();
    }
  }
  Buf buf(int k) {
    Buf b;
    b.cols = cols[k].as<int32_t>();
    b.len = len[k].as<int32_t>();
    b.att_hits = att_hits[k].as<int32_t>();
    b.rows = rows[k].as<int32_t>();
    b.att_dead = att_dead[k].as<uint8_t>();
    b.dead = dead[k].as<uint8_t>();
    b.hash = hash[k].as<uint64_t>();
    b.fit = fit[k].as<uint64_t>();
    return b;
  }
};

void gen_state_free(GenState *g) { delete g; }

void gen_mark_reset(GenState *g) {
  g->initialised = false;
  g->reset_pending = true;
}

void gen_drop_graphs(GenState *g) {
  if (g) g->drop_graphs();
}

namespace {

bool same_run_params(const ebic_params &a, const ebic_params &b) {
  ebic_params x = a, y = b;
  x.mode = y.mode = 0;
  x.use_graph = y.use_graph = 0;
  x.ipw = y.ipw = 0;  // (performance choices, like the two above)
  x.fuse_pairs = y.fuse_pairs = 0;
  return memcmp(&x, &y, sizeof(x)) == 0;
}

GenArgs gen_args(ebic_ctx *ctx, GenState *g) {
  GenArgs ga{};
  ga.ctl = g->ctl.as<GenCtl>();
  ga.top = g->top.as<TopEntry>();
  ga.usage = g->usage.as<int32_t>();
  ga.tabu = g->tabu.as<uint64_t>();
  ga.tmask = g->tcap - 1;
  for (int k = 0; k < 2; ++k) {
    ga.dkeys[k] = g->dkeys[k].as<uint64_t>();
    ga.dslot[k] = g->dslot[k].as<uint32_t>();
  }
  ga.dmask = g->dcap - 1;
  ga.rows_scr = g->rows_scr.as<int32_t>();
  ga.work = g->work.as<int32_t>();
  ga.cand_f = g->cand_f.as<uint64_t>();
  ga.cand_h = g->cand_h.as<uint64_t>();
  ga.cand_s = g->cand_s.as<int32_t>();
  ga.cand_cap = (int32_t)g->ccap;
  ga.sort_cap = g->sort_cap;
  const ebic_params &p = g->p;
  ga.seed = p.seed;
  ga.P = p.pop_size;
  ga.C = ctx->C;
  ga.K = p.n_biclusters;
  ga.E = p.elite;
  ga.T = p.tournament;
  ga.A = p.max_attempts;
  ga.max_len = p.max_len;
  ga.init_min = p.init_min_len;
  ga.init_max = p.init_max_len;
  ga.min_rows = p.min_rows;
  ga.col_cap = p.col_cap;
  ga.ov_num = p.overlap_num;
  ga.ov_den = p.overlap_den;
  ga.tabu_limit = p.tabu_hit_limit;
  if (g->fuse_np > 0) {
    ga.bitmap = ctx->bitmap.as<uint32_t>();
    ga.pair_cnt = ctx->pair_cnt_ok ? ctx->pair_cnt.as<unsigned long long>() : nullptr;
    ga.Wst = ctx->Wst;
    ga.R = ctx->R;
    ga.neg = p.neg_trends;
    ga.ns = p.non_strict;
    ga.rnum = p.ratio_num;
    ga.rden = p.ratio_den;
    ga.fuse_np = g->fuse_np;
    ga.todo = g->todo.as<int32_t>();
  }
  return ga;
}

EvalArgs gen_eval_args(ebic_ctx *ctx, GenState *g, int k, bool has_prev) {
  EvalArgs a = eval_args_for(ctx);
  // generation g-1's live keys (population buffer k ^ 1) join the hashed tabu list meanwhile,
  // and its duplicate table is cleared (there is none before the initial population)
  if (has_prev) {
    a.mv_hash = g->hash[k ^ 1].as<uint64_t>();
    a.mv_dead = g->att_dead[k ^ 1].as<uint8_t>();
    a.mv_len = g->len[k ^ 1].as<int32_t>();
    a.mv_n = (uint32_t)g->P;
    a.mv_table = g->tabu.as<uint64_t>();
    a.mv_tmask = g->tcap - 1;
    a.mv_count = reinterpret_cast<unsigned long long *>(&g->ctl.as<GenCtl>()->tabu_count);
    a.clr_keys = g->dkeys[k ^ 1].as<uint64_t>();
    a.clr_slots = g->dslot[k ^ 1].as<uint32_t>();
    a.clr_n = g->dcap;
  }
  a.neg = g->p.neg_trends;
  a.non_strict = g->p.non_strict;
  a.last_kept = g->p.last_kept;
  a.rnum = g->p.ratio_num;
  a.rden = g->p.ratio_den;
  a.min_rows = g->p.min_rows;
  a.col_cap = g->p.col_cap;
  a.rows_pos = g->rows_scr.as<int32_t>();
  a.rows_neg = a.rows_pos + g->P;
  a.rows_any = a.rows_neg + g->P;
  a.fitness = nullptr;
  a.work = g->work.as<int32_t>();
  // (the autotuner's loop sizes were measured in the loop, with the form it chose)
  const bool tuned = ctx->tuned && g->eval_mode == ctx->tuned_mode;
  a.seg_passes = tuned ? ctx->seg_loop : 0;
  a.ipw = g->p.ipw > 0 ? g->p.ipw : (tuned ? ctx->ipw_loop : 1);
  return a;
}

// The population of buffer k; with `listed`, only the slots the evolve kernel left to the
// evaluation launch.
PopView gen_view(GenState *g, int k, bool listed) {
  PopView v{};
  v.cols = g->cols[k].as<int32_t>();
  v.len = g->len[k].as<int32_t>();
  v.dead = g->att_dead[k].as<uint8_t>();
  v.stride = kS;
  v.n = g->P;
  v.stop = &g->ctl.as<GenCtl>()->stopped;
  v.hash = g->hash[k].as<uint64_t>();
  v.dkeys = g->dkeys[k].as<uint64_t>();
  v.dslot = g->dslot[k].as<uint32_t>();
  v.dmask = g->dcap - 1;
  if (listed) {
    v.list = g->todo.as<int32_t>();
    v.list_n = &g->ctl.as<GenCtl>()->n_todo;
  }
  return v;
}

// Launch with programmatic stream serialisation: the kernel may be scheduled while the previous
// kernel of the stream drains; it waits (griddepcontrol.wait) before reading that kernel's results.
template <class... Args>
cudaError_t launch_pdl(void (*kern)(Args...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Event marks between the kernels of one generation: 0 before k_evolve, 1 before the evaluation,
// 2 before k_finish, 3 after it.  While a graph is captured they become event-record nodes whose
// events are swapped before each profiled replay.
struct Marks {
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphNode_t node[4] = {nullptr, nullptr, nullptr, nullptr};
  bool capture = false;
};

cudaError_t mark(cudaStream_t s, Marks *m, int i) {
  if (!m || !m->ev[i]) return cudaSuccess;
  if (!m->capture) return cudaEventRecord(m->ev[i], s);
  return cudaEventRecordWithFlags(m->ev[i], s, cudaEventRecordExternal);
}

// The event-record nodes of a captured generation, matched to marks by the event they record.
cudaError_t find_mark_nodes(cudaGraph_t graph, const cudaEvent_t ev[4], cudaGraphNode_t node[4]) {
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(graph, nullptr, &n);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> nodes(n);
  if ((e = cudaGraphGetNodes(graph, nodes.data(), &n)) != cudaSuccess) return e;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if ((e = cudaGraphNodeGetType(nd, &t)) != cudaSuccess) return e;
    if (t != cudaGraphNodeTypeEventRecord) continue;
    cudaEvent_t ev_n = nullptr;
    if ((e = cudaGraphEventRecordNodeGetEvent(nd, &ev_n)) != cudaSuccess) return e;
    for (int i = 0; i < 4; ++i)
      if (ev[i] == ev_n) node[i] = nd;
  }
  for (int i = 0; i < 4; ++i)
    if (!node[i]) return cudaErrorInvalidValue;
  return cudaSuccess;
}

// Scoring kernels shared by initialisation and every generation (buffer k was just built;
// has_prev: a previous generation sits in buffer k ^ 1).
cudaError_t launch_scoring(ebic_ctx *ctx, GenState *g, int k, bool has_prev, cudaStream_t s,
                           Marks *m) {
  cudaError_t e;
  if ((e = mark(s, m, 1)) != cudaSuccess) return e;
  // (the initial population has no evolve step: all of it is evaluated here)
  const bool listed = has_prev && g->fuse_np > 0;
  if ((e = launch_eval_kernel(g->eval_mode, gen_eval_args(ctx, g, k, has_prev),
                              gen_view(g, k, listed), ctx->num_sms, s, true)) != cudaSuccess)
    return e;
  if ((e = mark(s, m, 2)) != cudaSuccess) return e;
  if ((e = launch_pdl(k_finish, dim3(g->finish_blocks), dim3(kTopThreads), g->top_smem, s,
                      gen_args(ctx, g), g->buf(k), k)) != cudaSuccess)
    return e;
  return mark(s, m, 3);
}

cudaError_t launch_generation(ebic_ctx *ctx, GenState *g, int parity, cudaStream_t s, Marks *m) {
  int G = 1;
  while (G < g->p.max_attempts) G <<= 1;
  cudaError_t e = mark(s, m, 0);
  if (e != cudaSuccess) return e;
  // A block of G attempt warps per slot while every slot's block fits on the GPU at once (the
  // slot's latency is then the launch's); beyond that a warp per slot, attempts in turn.
  if ((int64_t)g->P * G <= (int64_t)ctx->num_sms * kEvolveResidentWarps) {
    e = launch_pdl(k_evolve, dim3((unsigned)g->P), dim3(G * 32), evolve_smem(G, g->C), s,
                   gen_args(ctx, g), g->buf(parity ^ 1), g->buf(parity), parity);
  } else {
    e = launch_pdl(k_evolve_seq, dim3((unsigned)g->seq_blocks),
                   dim3(kSeqWarps * 32), evolve_smem(kSeqWarps, g->C), s, gen_args(ctx, g),
                   g->buf(parity ^ 1), g->buf(parity), parity);
  }
  if (e != cudaSuccess) return e;
  return launch_scoring(ctx, g, parity, true, s, m);
}

// Queues the event pairs of one profiled generation (evolve, evaluation, finish).
void push_generation_timing(ebic_ctx *ctx, const Marks &m, bool with_evolve) {
  if (with_evolve) prof_push(ctx, m.ev[0], m.ev[1], EBIC_KERNEL_EVOLVE, 0, 0, 0, true, false);
  prof_push(ctx, m.ev[1], m.ev[2], EBIC_KERNEL_EVAL, 0, 0, 0, true, false);
  prof_push(ctx, m.ev[2], m.ev[3], EBIC_KERNEL_FINISH, 0, 0, 0, true, true);
}

bool take_marks(ebic_ctx *ctx, Marks *m, bool with_evolve) {
  for (int i = with_evolve ? 0 : 1; i < 4; ++i) {
    m->ev[i] = prof_event(ctx);
    if (!m->ev[i]) {
      for (int j = 0; j < i; ++j)
        if (m->ev[j]) ctx->ev_pool.push_back(m->ev[j]);
      return false;
    }
  }
  return true;
}

int check_run_params(ebic_ctx *ctx, const ebic_params *p) {
  EBIC_TRY(ebic_check_eval_params(ctx, p));
  const int maxlen_cap = std::min(EBIC_MAX_LEN, ctx->C);
  if (!(2 <= p->init_min_len && p->init_min_len <= p->init_max_len &&
        p->init_max_len <= p->max_len && p->max_len <= maxlen_cap))
    return ebic_fail(ctx, EBIC_EINVAL,
                     "need 2 <= init_min_len <= init_max_len <= max_len <= min(64, cols)");
  if (!(p->overlap_den > 0 && p->overlap_num >= 0 && p->overlap_num <= p->overlap_den))
    return ebic_fail(ctx, EBIC_EINVAL, "need 0 <= overlap_num <= overlap_den, overlap_den > 0");
  if (p->n_biclusters < 1 || p->n_biclusters > EBIC_MAX_BICLUSTERS)
    return ebic_fail(ctx, EBIC_EINVAL, "n_biclusters must be in [1, 256]");
  if (p->pop_size < 2 || p->pop_size > (1 << 20))
    return ebic_fail(ctx, EBIC_EINVAL, "pop_size must be in [2, 2^20]");
  if (p->elite < 0 || p->elite > p->n_biclusters || p->elite >= p->pop_size)
    return ebic_fail(ctx, EBIC_EINVAL, "elite must be in [0, min(n_biclusters, pop_size - 1)]");
  if (p->tournament < 1 || p->tournament > 16 || p->max_attempts < 1 || p->max_attempts > 16)
    return ebic_fail(ctx, EBIC_EINVAL, "tournament and max_attempts must be in [1, 16]");
  if (p->mode == EBIC_MODE_PLAIN)
    return ebic_fail(ctx, EBIC_EINVAL,
                     "the generation loop evaluates with the DIRECT, STAGED or BITMAP form");
  return EBIC_OK;
}

}  // namespace

int ebic_check_loop_params(ebic_ctx *ctx, const ebic_params *p) { return check_run_params(ctx, p); }

namespace {

#define GEN_ALLOC(buf, bytes) EBIC_CHECK_CUDA(ctx, (buf).ensure(bytes, ctx->stream))

// Clears the run state of g (population, duplicate tables, tabu list, top list, column usage,
// counters) on the context stream; buffers and graphs stay.
int gen_reset(ebic_ctx *ctx, GenState *g) {
  const size_t P = (size_t)g->P;
  for (int k = 0; k < 2; ++k) {
    EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(g->cols[k].p, 0, P * kS * 4, ctx->stream));
    EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(g->len[k].p, 0, P * 4, ctx->stream));
    EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(g->fit[k].p, 0, P * 8, ctx->stream));
    EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(g->dkeys[k].p, 0, (size_t)g->dcap * 8, ctx->stream));
    EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(g->dslot[k].p, 0, (size_t)g->dcap * 4, ctx->stream));
  }
  EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(g->rows_scr.p, 0, P * 3 * 4, ctx->stream));
  EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(g->work.p, 0, 64, ctx->stream));
  EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(g->usage.p, 0, (size_t)g->C * 4, ctx->stream));
  EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(g->top.p, 0, (size_t)g->K * sizeof(TopEntry), ctx->stream));
  if (g->tcap) EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(g->tabu.p, 0, (size_t)g->tcap * 8, ctx->stream));
  GenCtl c0{};
  c0.gen = -1;
  // (a copy from pageable memory has taken its source before the call returns)
  EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(g->ctl.p, &c0, sizeof(c0), cudaMemcpyHostToDevice,
                                       ctx->stream));
  g->initialised = false;
  g->reset_pending = false;
  return EBIC_OK;
}

int gen_create(ebic_ctx *ctx, const ebic_params *p) {
  gen_state_free(ctx->gen);
  ctx->gen = nullptr;
  GenState *g = new (std::nothrow) GenState();
  if (!g) return ebic_fail(ctx, EBIC_ENOMEM, "host allocation failed");
  ctx->gen = g;
  g->p = *p;
  g->P = p->pop_size;
  g->K = p->n_biclusters;
  g->C = ctx->C;
  const size_t P = (size_t)g->P;
  for (int k = 0; k < 2; ++k) {
    GEN_ALLOC(g->cols[k], P * kS * 4);
    GEN_ALLOC(g->len[k], P * 4);
    GEN_ALLOC(g->att_hits[k], P * 4);
    GEN_ALLOC(g->rows[k], P * 3 * 4);
    GEN_ALLOC(g->att_dead[k], P);
    GEN_ALLOC(g->dead[k], P);
    GEN_ALLOC(g->hash[k], P * 8);
    GEN_ALLOC(g->fit[k], P * 8);
  }
  GEN_ALLOC(g->rows_scr, P * 3 * 4);
  GEN_ALLOC(g->todo, P * 4);
  GEN_ALLOC(g->work, 64);
  g->dcap = (uint32_t)dedup_capacity(P);
  for (int k = 0; k < 2; ++k) {
    GEN_ALLOC(g->dkeys[k], (size_t)g->dcap * 8);
    GEN_ALLOC(g->dslot[k], (size_t)g->dcap * 4);
  }
  g->ccap = (uint32_t)pow2_at_least(P);
  GEN_ALLOC(g->cand_f, (size_t)g->ccap * 8);
  GEN_ALLOC(g->cand_h, (size_t)g->ccap * 8);
  GEN_ALLOC(g->cand_s, (size_t)g->ccap * 4);
  GEN_ALLOC(g->top, (size_t)g->K * sizeof(TopEntry));
  GEN_ALLOC(g->ctl, sizeof(GenCtl));
  GEN_ALLOC(g->usage, (size_t)ctx->C * 4);
  const int cw = (ctx->C + 31) / 32;
  g->sort_cap = (int32_t)std::min<uint64_t>(kSortSmemMax, pow2_at_least(P));
  g->top_smem = (size_t)(g->K + 1) * sizeof(TopEntry) + (size_t)g->sort_cap * 16 +
                (size_t)cw * 4 + (size_t)g->sort_cap * 4 + (size_t)(g->K + 1) * 12 +
                (size_t)kChunk * (kS + 4) * 4 + (size_t)(g->K + 1) + 16;
  // One fixed upper bound for every context (contexts on other threads set the same value, so no
  // context can lower another's limit): K = 256, 65,535 columns, the largest sort buffer.
  static_assert((size_t)(EBIC_MAX_BICLUSTERS + 1) * sizeof(TopEntry) + kSortSmemMax * 20 +
                        2048 * 4 + (EBIC_MAX_BICLUSTERS + 1) * 13 + kChunk * (kS + 4) * 4 + 16 <=
                    kFinishSmemMax,
                "k_finish shared memory bound");
  if (g->top_smem > kFinishSmemMax) return ebic_fail(ctx, EBIC_EINVAL, "top-list workspace too large");
  EBIC_CHECK_CUDA(ctx, cudaFuncSetAttribute(k_finish, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kFinishSmemMax));
  EBIC_CHECK_CUDA(ctx, cudaFuncSetAttribute(k_evolve, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)evolve_smem(kMaxAttemptWarps, kUsageSmemMax)));
  EBIC_CHECK_CUDA(ctx, cudaFuncSetAttribute(k_evolve_seq,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)evolve_smem(kSeqWarps, kUsageSmemMax)));
  int seq_per_sm = 0;
  EBIC_CHECK_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                           &seq_per_sm, k_evolve_seq, kSeqWarps * 32,
                           evolve_smem(kSeqWarps, ctx->C)));
  g->seq_blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>((g->P + kSeqWarps - 1) / kSeqWarps,
                           (int64_t)ctx->num_sms * std::max(seq_per_sm, 1)));

  // one block per 1,024 slots (a slot per thread): the slot loop spread, few blocks to meet at
  // the end (measured: one block for P = 800, 8.4 against 10.2 us with two; with the evaluation
  // inside the evolve kernel, 16.3 against 18.6 us at P = 8,192 and 12.0 against 14.6 us at
  // P = 4,096 over one block per 2,048 slots)
  g->finish_blocks = (int)std::max<int64_t>(
      1, std::min<int64_t>((g->P + kTopThreads - 1) / kTopThreads, ctx->num_sms));
  EBIC_CHECK_CUDA(ctx, cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
  for (cudaEvent_t &e : g->cap_ev) EBIC_CHECK_CUDA(ctx, cudaEventCreate(&e));
  return gen_reset(ctx, g);
}

int read_ctl(ebic_ctx *ctx, GenState *g, GenCtl *out) {
  EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(out, g->ctl.p, sizeof(GenCtl), cudaMemcpyDeviceToHost,
                                       ctx->stream));
  EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return EBIC_OK;
}

// Grows the tabu table to hold `need` keys at load factor <= 1 / kTableSpread (rehashing live
// keys).
int ensure_tabu(ebic_ctx *ctx, GenState *g, int64_t need) {
  const uint64_t want = tabu_capacity(need);
  if (want > (1ull << 31)) return ebic_fail(ctx, EBIC_ENOMEM, "tabu list beyond 2^31 slots");
  if (g->tcap >= want) return EBIC_OK;
  DevBuf fresh;
  EBIC_CHECK_CUDA(ctx, fresh.ensure(want * 8, ctx->stream));
  EBIC_CHECK_CUDA(ctx, cudaMemsetAsync(fresh.p, 0, want * 8, ctx->stream));
  if (g->tcap) {
    k_rehash<<<(g->tcap + 255) / 256, 256, 0, ctx->stream>>>(g->tabu.as<uint64_t>(), g->tcap,
                                                           fresh.as<uint64_t>(),
                                                           (uint32_t)want - 1);
    EBIC_CHECK_CUDA(ctx, cudaGetLastError());
    prof_count(ctx, -1, 1);
  }
  EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  g->tabu.release();
  g->tabu = fresh;
  fresh.p = nullptr;
  fresh.bytes = 0;
  g->tcap = (uint32_t)want;
  g->drop_graphs();
  return EBIC_OK;
}

// Pair limit of the evaluation inside the evolve kernel (0: none): the caller's, else the
// autotuner's, else none for the block-per-slot form (whose launch lasts one slot's latency,
// which an evaluation would lengthen: measured slower on 10,000 x 100, P = 800) and, for the
// warp-per-slot form, the largest pair count whose staged units (pairs x directions x passes of
// 128 words) stay within kFuseDefaultUnits, so that evaluating a child keeps its warp about as
// long as building it did.  Only the bitmap form has it.
constexpr int64_t kFuseDefaultUnits = 64;

int fuse_limit(const ebic_ctx *ctx, int mode, const ebic_params *p) {
  if (mode != EBIC_MODE_BITMAP || p->fuse_pairs < 0 || p->last_kept) return 0;
  if (p->fuse_pairs > 0) return p->fuse_pairs;
  // (the autotuner's limit, measured in the loop with this form)
  if (ctx->tuned && ctx->tuned_mode == mode && ctx->fuse_loop != 0)
    return ctx->fuse_loop > 0 ? ctx->fuse_loop : 0;
  int G = 1;
  while (G < p->max_attempts) G <<= 1;
  if ((int64_t)p->pop_size * G <= (int64_t)ctx->num_sms * kEvolveResidentWarps) return 0;
  const int64_t per_pair = (ctx->Wst + 127) / 128 * (p->neg_trends ? 2 : 1);
  return (int)std::min<int64_t>(EBIC_MAX_LEN - 1, kFuseDefaultUnits / per_pair);
}

int ensure_eval_ready(ebic_ctx *ctx, GenState *g, const ebic_params *p, int n_gen) {
  int mode = choose_mode(ctx, p->mode, g->P, 0.5 * (p->init_min_len + p->max_len), n_gen + 1,
                         p->last_kept);
  if (mode == EBIC_MODE_PLAIN) mode = EBIC_MODE_DIRECT;
  if (mode == EBIC_MODE_BITMAP && !ctx->bitmap_ok) EBIC_TRY(ebic_build_bitmap(ctx));
  const bool direct = direct_form_used(ctx, mode, p);
  if (direct) EBIC_TRY(ensure_codes(ctx));
  // the captured graphs hold the evaluation kernel's data buffer: recapture when it changed
  const void *buf = mode == EBIC_MODE_BITMAP ? ctx->bitmap.p
                    : (direct && ctx->codes_ready ? ctx->codes.p : nullptr);
  // (and the fusion limit, which the captured evolve launches hold)
  const int fuse = fuse_limit(ctx, mode, p);
  const void *cnt = fuse > 0 && ctx->pair_cnt_ok ? ctx->pair_cnt.p : nullptr;
  if (mode != g->eval_mode || buf != g->graph_buf || fuse != g->fuse_np ||
      cnt != g->graph_cnt) {
    g->drop_graphs();
    g->graph_buf = buf;
    g->graph_cnt = cnt;
  }
  g->eval_mode = mode;
  g->fuse_np = fuse;
  return EBIC_OK;
}

int capture_graph(ebic_ctx *ctx, GenState *g, int parity, int profiled) {
  cudaGraph_t graph = nullptr;
  EBIC_CHECK_CUDA(ctx, cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
  Marks m;
  m.capture = true;
  if (profiled)
    for (int i = 0; i < 4; ++i) m.ev[i] = g->cap_ev[i];
  cudaError_t e = launch_generation(ctx, g, parity, g->cap_stream, profiled ? &m : nullptr);
  cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return ebic_fail_cuda(ctx, e, "generation capture", __FILE__, __LINE__);
  }
  EBIC_CHECK_CUDA(ctx, e2);
  if (profiled) {
    for (int i = 0; i < 4; ++i) g->mark_node[parity][i] = nullptr;
    e = find_mark_nodes(graph, g->cap_ev, g->mark_node[parity]);
    if (e != cudaSuccess) {
      cudaGraphDestroy(graph);
      return ebic_fail_cuda(ctx, e, "event nodes of the generation graph", __FILE__, __LINE__);
    }
  }
  e = cudaGraphInstantiate(&g->graph[parity][profiled], graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return ebic_fail_cuda(ctx, e, "cudaGraphInstantiate", __FILE__, __LINE__);
  }
  if (profiled)
    g->graph_src[parity][profiled] = graph;
  else
    cudaGraphDestroy(graph);
  return EBIC_OK;
}

constexpr int kGraphGenerations = 16;  // even: a chunk ends on the parity it started with

// The graph of kGraphGenerations generations starting at `parity` (no event marks).
int capture_multi(ebic_ctx *ctx, GenState *g, int parity) {
  cudaGraph_t graph = nullptr;
  EBIC_CHECK_CUDA(ctx, cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < kGraphGenerations && e == cudaSuccess; ++j)
    e = launch_generation(ctx, g, parity ^ (j & 1), g->cap_stream, nullptr);
  cudaError_t e2 = cudaStreamEndCapture(g->cap_stream, &graph);
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return ebic_fail_cuda(ctx, e, "generation capture", __FILE__, __LINE__);
  }
  EBIC_CHECK_CUDA(ctx, e2);
  e = cudaGraphInstantiate(&g->multi[parity], graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return ebic_fail_cuda(ctx, e, "cudaGraphInstantiate", __FILE__, __LINE__);
  return EBIC_OK;
}

}  // namespace

extern "C" {

int ebic_run_generations(ebic_ctx *ctx, const ebic_params *p, int32_t n_gen,
                         ebic_run_report *rep) {
  if (!ctx) return EBIC_EINVAL;
  if (!ctx->have_matrix) return ebic_fail(ctx, EBIC_ESTATE, "no matrix loaded");
  EBIC_TRY(check_run_params(ctx, p));
  if (n_gen < 0) return ebic_fail(ctx, EBIC_EINVAL, "n_gen must be >= 0");
  int prev_dev = -1;
  cudaGetDevice(&prev_dev);
  cudaSetDevice(ctx->device);
  struct Restore {
    int d;
    ~Restore() {
      if (d >= 0) cudaSetDevice(d);
    }
  } restore{prev_dev};
  GenState *g = ctx->gen;
  if (!g || !same_run_params(g->p, *p)) {
    EBIC_TRY(gen_create(ctx, p));
    g = ctx->gen;
  } else if (g->reset_pending) {
    EBIC_TRY(gen_reset(ctx, g));
  }
  g->p.mode = p->mode;
  g->p.use_graph = p->use_graph;
  if (g->p.ipw != p->ipw) g->drop_graphs();  // (the captured launches hold the group size)
  g->p.ipw = p->ipw;
  g->p.fuse_pairs = p->fuse_pairs;
  EBIC_TRY(ensure_eval_ready(ctx, g, p, n_gen));
  GenCtl c{};
  EBIC_TRY(read_ctl(ctx, g, &c));
  EBIC_TRY(ensure_tabu(ctx, g, c.tabu_count + (int64_t)g->P * ((int64_t)n_gen + 2)));
  cudaStream_t s = ctx->stream;
  const GenCtl c_start = c;
  if (!g->initialised) {
    Marks m;
    const bool timed = ctx->prof && take_marks(ctx, &m, false);
    k_init<<<(unsigned)((g->P + kInitWarps - 1) / kInitWarps), kInitWarps * 32, 0, s>>>(
        gen_args(ctx, g), g->buf(0));
    EBIC_CHECK_CUDA(ctx, cudaGetLastError());
    EBIC_CHECK_CUDA(ctx, launch_scoring(ctx, g, 0, false, s, timed ? &m : nullptr));
    if (timed) push_generation_timing(ctx, m, false);
    prof_count(ctx, EBIC_KERNEL_EVAL, 1);
    prof_count(ctx, EBIC_KERNEL_FINISH, 1);
    prof_count(ctx, -1, 1);
    g->initialised = true;
    EBIC_TRY(read_ctl(ctx, g, &c));
  }
  if (!c.stopped) {
    for (int i = 0; i < n_gen; ++i) {
      const int gnext = c.gen + 1 + i;
      const int parity = gnext & 1;
      if (p->use_graph && !ctx->prof && n_gen - i >= kGraphGenerations) {
        if (!g->multi[parity]) EBIC_TRY(capture_multi(ctx, g, parity));
        EBIC_CHECK_CUDA(ctx, cudaGraphLaunch(g->multi[parity], s));
        prof_count(ctx, EBIC_KERNEL_EVOLVE, kGraphGenerations);
        prof_count(ctx, EBIC_KERNEL_EVAL, kGraphGenerations);
        prof_count(ctx, EBIC_KERNEL_FINISH, kGraphGenerations);
        i += kGraphGenerations - 1;
        continue;
      }
      Marks m;
      const bool timed = ctx->prof && take_marks(ctx, &m, true);
      if (p->use_graph) {
        const int v = timed ? 1 : 0;
        if (!g->graph[parity][v]) EBIC_TRY(capture_graph(ctx, g, parity, v));
        if (timed) {
          // point the graph's event nodes at this replay's events
          for (int k = 0; k < 4; ++k)
            EBIC_CHECK_CUDA(ctx, cudaGraphExecEventRecordNodeSetEvent(
                                     g->graph[parity][1], g->mark_node[parity][k], m.ev[k]));
        }
        EBIC_CHECK_CUDA(ctx, cudaGraphLaunch(g->graph[parity][v], s));
      } else {
        EBIC_CHECK_CUDA(ctx, launch_generation(ctx, g, parity, s, timed ? &m : nullptr));
      }
      if (timed) push_generation_timing(ctx, m, true);
      prof_count(ctx, EBIC_KERNEL_EVOLVE, 1);
      prof_count(ctx, EBIC_KERNEL_EVAL, 1);
      prof_count(ctx, EBIC_KERNEL_FINISH, 1);
      if (!p->use_graph) {
        GenCtl cc{};
        EBIC_TRY(read_ctl(ctx, g, &cc));
        if (cc.stopped) break;
      }
    }
  }
  // the counters and the kernels' error word, in one synchronisation
  int32_t kerr = 0;
  EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(&c, g->ctl.p, sizeof(GenCtl), cudaMemcpyDeviceToHost,
                                       ctx->stream));
  EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(&kerr, ctx->d_kerr.p, 4, cudaMemcpyDeviceToHost,
                                       ctx->stream));
  EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (kerr) {
    cudaMemset(ctx->d_kerr.p, 0, 4);
    return ebic_fail(ctx, EBIC_ETIMEOUT, "a bounded device wait expired in the generation loop");
  }
  if (ctx->prof) {
    // algorithmic work of the evaluations run by this call (live slots only)
    // (split between the evaluation launches and the evolve kernel's own evaluations)
    const double flen = (double)(c.fused_len - c_start.fused_len);
    const double flive = (double)(c.n_fused - c_start.n_fused);
    const double dlen = (double)(c.sum_len - c_start.sum_len) - flen;
    const double dlive = (double)(c.n_evaluated - c_start.n_evaluated) - flive;
    const double nd = g->p.neg_trends ? 2.0 : 1.0;
    KStats &k = ctx->kst[EBIC_KERNEL_EVAL];
    k.bytes += eval_bytes(ctx, g->eval_mode, (int64_t)dlen, (int64_t)dlive, g->p.neg_trends);
    k.ops += (dlen - dlive) * (double)ctx->R * nd;
    k.units += dlive * (double)ctx->R;
    // (a one-pair slot scored from the pair-count table reads one count per direction)
    const double ntab = (double)(c.n_table - c_start.n_table);
    KStats &kf = ctx->kst[EBIC_KERNEL_EVOLVE];
    kf.bytes += eval_bytes(ctx, g->eval_mode, (int64_t)(flen - 2.0 * ntab),
                           (int64_t)(flive - ntab), g->p.neg_trends) + ntab * 4.0 * nd;
    kf.ops += (flen - flive) * (double)ctx->R * nd;
    kf.units += flive * (double)ctx->R;
    prof_collect(ctx);
  }
  if (rep) {
    memset(rep, 0, sizeof(*rep));
    rep->gens_done = c.gen;
    rep->stopped = c.stopped;
    rep->last_hits = c.hits_last;
    rep->n_top = c.n_top;
    rep->n_evaluated = c.n_evaluated;
    rep->eval_mode = g->eval_mode;
    rep->fuse_pairs = g->fuse_np;
    rep->n_fused = c.n_fused;
    rep->n_table = c.n_table;
  }
  return EBIC_OK;
}

int ebic_get_toplist(ebic_ctx *ctx, int32_t capacity, int32_t *n_top, int32_t *cols,
                     int32_t *lens, uint64_t *fitness, uint64_t *keys, int32_t *rows) {
  if (!ctx) return EBIC_EINVAL;
  GenState *g = ctx->gen;
  if (!g || !g->initialised) return ebic_fail(ctx, EBIC_ESTATE, "no run");
  cudaSetDevice(ctx->device);
  GenCtl c{};
  EBIC_TRY(read_ctl(ctx, g, &c));
  if (capacity < c.n_top) return ebic_fail(ctx, EBIC_EINVAL, "capacity below the list size");
  std::vector<TopEntry> host(c.n_top > 0 ? c.n_top : 1);
  if (c.n_top > 0)
    EBIC_CHECK_CUDA(ctx, cudaMemcpy(host.data(), g->top.p, sizeof(TopEntry) * c.n_top,
                                    cudaMemcpyDeviceToHost));
  std::vector<int32_t> hc((size_t)c.n_top * kS, 0), hl(c.n_top), hr((size_t)c.n_top * 3);
  std::vector<uint64_t> hf(c.n_top), hk(c.n_top);
  for (int e = 0; e < c.n_top; ++e) {
    for (int k = 0; k < host[e].len; ++k) hc[(size_t)e * kS + k] = host[e].cols[k];
    hl[e] = host[e].len;
    hf[e] = host[e].f;
    hk[e] = host[e].h;
    hr[e * 3] = host[e].rp;
    hr[e * 3 + 1] = host[e].rn;
    hr[e * 3 + 2] = host[e].ra;
  }
  if (n_top) *n_top = c.n_top;
  if (c.n_top > 0) {
    if (cols) EBIC_CHECK_CUDA(ctx, cudaMemcpy(cols, hc.data(), hc.size() * 4, cudaMemcpyDefault));
    if (lens) EBIC_CHECK_CUDA(ctx, cudaMemcpy(lens, hl.data(), hl.size() * 4, cudaMemcpyDefault));
    if (fitness)
      EBIC_CHECK_CUDA(ctx, cudaMemcpy(fitness, hf.data(), hf.size() * 8, cudaMemcpyDefault));
    if (keys) EBIC_CHECK_CUDA(ctx, cudaMemcpy(keys, hk.data(), hk.size() * 8, cudaMemcpyDefault));
    if (rows) EBIC_CHECK_CUDA(ctx, cudaMemcpy(rows, hr.data(), hr.size() * 4, cudaMemcpyDefault));
  }
  return EBIC_OK;
}

int ebic_get_population(ebic_ctx *ctx, int32_t capacity, int32_t *cols, int32_t *lens,
                        uint8_t *dead, uint64_t *fitness) {
  if (!ctx) return EBIC_EINVAL;
  GenState *g = ctx->gen;
  if (!g || !g->initialised) return ebic_fail(ctx, EBIC_ESTATE, "no run");
  if (capacity < g->P) return ebic_fail(ctx, EBIC_EINVAL, "capacity below pop_size");
  cudaSetDevice(ctx->device);
  GenCtl c{};
  EBIC_TRY(read_ctl(ctx, g, &c));
  const int k = c.gen & 1;
  const size_t P = (size_t)g->P;
  if (cols) EBIC_CHECK_CUDA(ctx, cudaMemcpy(cols, g->cols[k].p, P * kS * 4, cudaMemcpyDefault));
  if (lens) EBIC_CHECK_CUDA(ctx, cudaMemcpy(lens, g->len[k].p, P * 4, cudaMemcpyDefault));
  if (dead) EBIC_CHECK_CUDA(ctx, cudaMemcpy(dead, g->dead[k].p, P, cudaMemcpyDefault));
  if (fitness) EBIC_CHECK_CUDA(ctx, cudaMemcpy(fitness, g->fit[k].p, P * 8, cudaMemcpyDefault));
  return EBIC_OK;
}

int ebic_extract_biclusters(ebic_ctx *ctx, int32_t capacity, uint32_t *rowmask, int32_t *n_out) {
  if (!ctx) return EBIC_EINVAL;
  GenState *g = ctx->gen;
  if (!g || !g->initialised) return ebic_fail(ctx, EBIC_ESTATE, "no run");
  if (!rowmask) return ebic_fail(ctx, EBIC_EINVAL, "rowmask is NULL");
  cudaSetDevice(ctx->device);
  GenCtl c{};
  EBIC_TRY(read_ctl(ctx, g, &c));
  if (capacity < c.n_top) return ebic_fail(ctx, EBIC_EINVAL, "capacity below the list size");
  const size_t words = (size_t)c.n_top * ctx->Wst;
  const bool dev = ebic_is_device_ptr(rowmask);
  uint32_t *dst = rowmask;
  if (!dev) {
    EBIC_CHECK_CUDA(ctx, g->extract.ensure(words * 4 + 4, ctx->stream));
    dst = g->extract.as<uint32_t>();
  }
  if (words) {
    const int64_t threads = (int64_t)words * 32;
    k_extract<<<(unsigned)((threads + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->keys.as<uint32_t>(), ctx->R, ctx->R_pad, ctx->Wst, g->top.as<TopEntry>(),
        g->ctl.as<GenCtl>(), g->p.neg_trends, g->p.ratio_num, g->p.ratio_den, dst);
    EBIC_CHECK_CUDA(ctx, cudaGetLastError());
    prof_count(ctx, -1, 1);
    if (!dev)
      EBIC_CHECK_CUDA(ctx, cudaMemcpyAsync(rowmask, dst, words * 4, cudaMemcpyDeviceToHost,
                                           ctx->stream));
  }
  EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (n_out) *n_out = c.n_top;
  return EBIC_OK;
}

// Checkpoint blob: header, GenCtl, current buffer (cols, len, dead, hash, fit, rows, att_dead),
// top list, then the tabu list as sorted keys (the hashed table plus the last scored
// generation's keys, which still sit in its duplicate table).
struct StateHeader {
  uint64_t magic;
  int64_t rows;
  int32_t cols, P, K, k;
  int64_t n_tabu;
  ebic_params p;
};

static const uint64_t kMagic = 0x4542494347423332ull;  // "EBICGB32"

static int64_t state_fixed_size(const GenState *g) {
  const int64_t P = g->P;
  return (int64_t)sizeof(StateHeader) + (int64_t)sizeof(GenCtl) + P * kS * 4 + P * 4 + P + P * 8 +
         P * 8 + P * 12 + P + (int64_t)g->K * (int64_t)sizeof(TopEntry);
}

static int collect_tabu(ebic_ctx *ctx, GenState *g, int k, std::vector<uint64_t> *keys) {
  std::vector<uint64_t> table(g->tcap), pend(g->dcap);
  EBIC_CHECK_CUDA(ctx, cudaMemcpy(table.data(), g->tabu.p, (size_t)g->tcap * 8,
                                  cudaMemcpyDeviceToHost));
  EBIC_CHECK_CUDA(ctx, cudaMemcpy(pend.data(), g->dkeys[k].p, (size_t)g->dcap * 8,
                                  cudaMemcpyDeviceToHost));
  keys->clear();
  for (uint64_t v : table)
    if (v) keys->push_back(v);
  for (uint64_t v : pend)
    if (v) keys->push_back(v);
  std::sort(keys->begin(), keys->end());
  keys->erase(std::unique(keys->begin(), keys->end()), keys->end());
  return EBIC_OK;
}

int64_t ebic_state_bytes(ebic_ctx *ctx) {
  if (!ctx || !ctx->gen || !ctx->gen->initialised) return 0;
  cudaSetDevice(ctx->device);
  GenCtl c{};
  if (read_ctl(ctx, ctx->gen, &c) != EBIC_OK) return 0;
  std::vector<uint64_t> keys;
  if (collect_tabu(ctx, ctx->gen, c.gen & 1, &keys) != EBIC_OK) return 0;
  return state_fixed_size(ctx->gen) + (int64_t)keys.size() * 8;
}

int ebic_save_state(ebic_ctx *ctx, void *blob, int64_t size) {
  if (!ctx) return EBIC_EINVAL;
  GenState *g = ctx->gen;
  if (!g || !g->initialised) return ebic_fail(ctx, EBIC_ESTATE, "no run");
  cudaSetDevice(ctx->device);
  GenCtl c{};
  EBIC_TRY(read_ctl(ctx, g, &c));
  const int k = c.gen & 1;
  std::vector<uint64_t> keys;
  EBIC_TRY(collect_tabu(ctx, g, k, &keys));
  const int64_t need = state_fixed_size(g) + (int64_t)keys.size() * 8;
  if (!blob || size < need) return ebic_fail(ctx, EBIC_EINVAL, "blob too small");
  unsigned char *o = static_cast<unsigned char *>(blob);
  StateHeader h{};
  h.magic = kMagic;
  h.rows = ctx->R;
  h.cols = ctx->C;
  h.P = g->P;
  h.K = g->K;
  h.k = k;
  h.n_tabu = (int64_t)keys.size();
  h.p = g->p;
  memcpy(o, &h, sizeof(h));
  o += sizeof(h);
  memcpy(o, &c, sizeof(c));
  o += sizeof(c);
  const size_t P = (size_t)g->P;
  struct Part {
    DevBuf *b;
    size_t n;
  } parts[] = {{&g->cols[k], P * kS * 4}, {&g->len[k], P * 4},  {&g->dead[k], P},
               {&g->hash[k], P * 8},      {&g->fit[k], P * 8},  {&g->rows[k], P * 12},
               {&g->att_dead[k], P},      {&g->top, (size_t)g->K * sizeof(TopEntry)}};
  for (const Part &pt : parts) {
    EBIC_CHECK_CUDA(ctx, cudaMemcpy(o, pt.b->p, pt.n, cudaMemcpyDeviceToHost));
    o += pt.n;
  }
  memcpy(o, keys.data(), keys.size() * 8);
  return EBIC_OK;
}

int ebic_load_state(ebic_ctx *ctx, const ebic_params *p, const void *blob, int64_t size) {
  if (!ctx) return EBIC_EINVAL;
  if (!ctx->have_matrix) return ebic_fail(ctx, EBIC_ESTATE, "no matrix loaded");
  EBIC_TRY(check_run_params(ctx, p));
  if (!blob || size < (int64_t)sizeof(StateHeader))
    return ebic_fail(ctx, EBIC_EINVAL, "blob too small");
  StateHeader h;
  memcpy(&h, blob, sizeof(h));
  if (h.magic != kMagic || h.rows != ctx->R || h.cols != ctx->C || h.P != p->pop_size ||
      h.K != p->n_biclusters || !same_run_params(h.p, *p) || h.n_tabu < 0)
    return ebic_fail(ctx, EBIC_EINVAL, "state blob does not match this matrix and parameters");
  cudaSetDevice(ctx->device);
  EBIC_TRY(gen_create(ctx, p));
  GenState *g = ctx->gen;
  if (size < state_fixed_size(g) + h.n_tabu * 8)
    return ebic_fail(ctx, EBIC_EINVAL, "blob truncated");
  const unsigned char *o = static_cast<const unsigned char *>(blob) + sizeof(h);
  GenCtl c;
  memcpy(&c, o, sizeof(c));
  o += sizeof(c);
  const int k = c.gen & 1;
  const size_t P = (size_t)g->P;
  struct Part {
    DevBuf *b;
    size_t n;
  } parts[] = {{&g->cols[k], P * kS * 4}, {&g->len[k], P * 4},  {&g->dead[k], P},
               {&g->hash[k], P * 8},      {&g->fit[k], P * 8},  {&g->rows[k], P * 12},
               {&g->att_dead[k], P},      {&g->top, (size_t)g->K * sizeof(TopEntry)}};
  for (const Part &pt : parts) {
    EBIC_CHECK_CUDA(ctx, cudaMemcpy(pt.b->p, o, pt.n, cudaMemcpyHostToDevice));
    o += pt.n;
  }
  EBIC_TRY(ensure_tabu(ctx, g, h.n_tabu + (int64_t)g->P));
  if (h.n_tabu > 0) {
    DevBuf list;
    EBIC_CHECK_CUDA(ctx, list.ensure((size_t)h.n_tabu * 8, ctx->stream));
    EBIC_CHECK_CUDA(ctx, cudaMemcpy(list.p, o, (size_t)h.n_tabu * 8, cudaMemcpyHostToDevice));
    k_tabu_load<<<(unsigned)((h.n_tabu + 255) / 256), 256, 0, ctx->stream>>>(
        list.as<uint64_t>(), h.n_tabu, g->tabu.as<uint64_t>(), g->tcap - 1);
    EBIC_CHECK_CUDA(ctx, cudaGetLastError());
    EBIC_CHECK_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    list.release();
  }
  c.tabu_count = h.n_tabu;
  c.hits_cur = 0;
  c.live_cur = 0;
  c.n_cand = 0;
  c.done = 0;
  EBIC_CHECK_CUDA(ctx, cudaMemcpy(g->ctl.p, &c, sizeof(c), cudaMemcpyHostToDevice));
  // column usage of the restored top list
  std::vector<TopEntry> top(g->K);
  memcpy(top.data(), static_cast<const unsigned char *>(blob) + sizeof(h) + sizeof(GenCtl) +
                         P * kS * 4 + P * 4 + P + P * 8 + P * 8 + P * 12 + P,
         sizeof(TopEntry) * g->K);
  std::vector<int32_t> usage(ctx->C, 0);
  for (int e = 0; e < c.n_top; ++e)
    for (int q = 0; q < top[e].len; ++q) usage[top[e].cols[q]] += 1;
  EBIC_CHECK_CUDA(ctx, cudaMemcpy(g->usage.p, usage.data(), usage.size() * 4,
                                  cudaMemcpyHostToDevice));
  g->initialised = true;
  return EBIC_OK;
}

}  // extern "C"
