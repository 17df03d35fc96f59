// Population evaluation kernels (Sec. 2.4, steps 2-3 and 7 of the EBIC.jl paper: score every
// individual by the number of rows that follow its column order; trend definition of Sec. 2.3).
//
// For individual i with columns c_0..c_{L-1} and row r:
//   inc = #{k : key(r, c_{k+1}) > key(r, c_k)},  dec = #{k : key(r, c_{k+1}) < key(r, c_k)}
//   pos = inc >= t(L), neg = neg_trends && dec >= t(L), t(L) = ceil(ratio * (L-1)),
// and rows_pos / rows_neg / rows_any count the rows with pos / neg / (pos || neg).
//
// Three forms compute the same counts:
//   direct  keys gathered per row (4 rows per lane, 16-byte loads of the column-major keys);
//           with up to 1,024 columns the per-row rank codes of codes.cu stand in for the keys;
//   bitmap  32 rows per word from the pair bitmap: an AND of the L-1 pair words for the exact
//           trend, a bit-sliced carry-save counter compared with t(L) for approximate trends;
//   plain   one kernel launch per individual, one row per thread (the reference GPU form).
// The direct and bitmap kernels are persistent: warps pull (individual, row segment) work items
// from an atomic counter, segment-major (every individual of a row segment before the next
// segment, so the segment's data stays in L2 while all individuals read it), then the chunks of
// the generation loop's side task (items.cuh), and add their partial counts with one atomic per
// item.
#include <mutex>
#include <type_traits>

#include "internal.h"
#include "tables.cuh"
#include "items.cuh"
#include "trend.cuh"

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kMaxDevices = 64;

__device__ __forceinline__ int threshold(int L, int num, int den) {
  return (num * (L - 1) + den - 1) / den;
}

__device__ __forceinline__ int pv_len(const PopView &v, int i) {
  return v.off ? (v.off[i + 1] - v.off[i]) : v.len[i];
}

__device__ __forceinline__ bool pv_dead(const PopView &v, int i) {
  if (v.dead && v.dead[i]) return true;
  if (v.dkeys) return dedup_is_dup(v.dkeys, v.dslot, v.dmask, v.hash[i], i);
  return false;
}

// Waits for the preceding kernel of a programmatic launch (no-op otherwise).
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ uint4 ldg4(const uint32_t *p) {
  return __ldg(reinterpret_cast<const uint4 *>(p));
}

// ------------------------------------------------------------------------------- validation

// One warp per individual: lane k holds columns k and k + 32 (sentinels that no column and no
// other lane's sentinel equals past the length); a column out of range, a repeated column, a
// start below 0 or a length outside [2, 64] sets bit 2 of *err.
__global__ void k_validate_csr(const int32_t *__restrict__ cols, const int32_t *__restrict__ off,
                               int32_t n, int32_t C, int32_t *__restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= n) return;  // (whole warps)
  const int s = off[i], e = off[i + 1];
  const int L = e - s;
  bool bad = (s < 0) || L < 2 || L > EBIC_MAX_LEN;  // (warp-uniform)
  if (!bad) {
    const bool in0 = lane < L, in1 = lane + 32 < L;
    const int c0 = in0 ? cols[s + lane] : -1 - lane;
    const int c1 = in1 ? cols[s + 32 + lane] : -33 - lane;
    // (every lane takes part in each collective: none sits in a short-circuited operand)
    const unsigned m0 = __match_any_sync(kFull, c0), m1 = __match_any_sync(kFull, c1);
    bad = (in0 && (c0 < 0 || c0 >= C)) || (in1 && (c1 < 0 || c1 >= C));
    bad = bad || __popc(m0) > 1 || __popc(m1) > 1;
    for (int j = 0; j < 32; ++j) {
      const int b = __shfl_sync(kFull, c0, j);
      bad = bad || c1 == b;
    }
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(err, 2);
}

// ------------------------------------------------------------------------------- direct form

// NS / LK: the pair-test variants of trend.cuh (ties count for both directions / compare with
// the last value kept).  With ties counting, the pad rows past R (key 0 everywhere) would pass,
// so they are masked out.
template <bool NEG, bool NS, bool LK>
__global__ void __launch_bounds__(kThreads, 4) k_eval_direct(EvalArgs a, PopView pv) {
  __shared__ int64_t s_base[kWarps][EBIC_MAX_LEN];
  wait_prior_grid();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t passes_total = a.R_pad / 128;
  const int32_t n_side = items::move_chunks(a), n_all = n_side + pv.n * a.n_seg;
  for (int q = items::first(); q < n_all; q = items::next(a.work, lane, q, n_all)) {
    if (q < n_side) {
      if (items::stopped(pv)) return;  // a stopped run changes nothing
      items::move_chunk(a, q, lane);
      continue;
    }
    const int seg = (q - n_side) / pv.n, i = (q - n_side) - seg * pv.n;  // segment-major
    const items::Meta m = items::load_meta(pv, i, lane);
    if (items::stopped(pv)) return;  // (read with the item's loads; before any store)
    if (m.dead || m.L < 2) continue;
    const items::Insert ins = items::insert_start(pv, seg, m.h, lane);
    const int L = m.L;
    __syncwarp();
    s_base[warp][lane] = (int64_t)m.c0 * a.R_pad;
    s_base[warp][lane + 32] = (int64_t)m.c1 * a.R_pad;
    __syncwarp();
    const int t = threshold(L, a.rnum, a.rden);
    const int64_t p0 = (int64_t)seg * a.seg_passes;
    const int64_t p1 = min(p0 + a.seg_passes, passes_total);
    int cp = 0, cn = 0, ca = 0;
    for (int64_t pass = p0; pass < p1; ++pass) {
      const int64_t r = pass * 128 + lane * 4;
      const uint4 v0 = ldg4(a.keys + s_base[warp][0] + r);
      RowTrend<uint32_t, NEG, NS, LK> tr[4];
      tr[0].start(v0.x);
      tr[1].start(v0.y);
      tr[2].start(v0.z);
      tr[3].start(v0.w);
#pragma unroll 4
      for (int k = 1; k < L; ++k) {
        const uint4 cur = ldg4(a.keys + s_base[warp][k] + r);
        tr[0].step(cur.x);
        tr[1].step(cur.y);
        tr[2].step(cur.z);
        tr[3].step(cur.w);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const bool valid = !NS || r + j < a.R;
        const bool po = valid && tr[j].inc >= t, ne = valid && NEG && tr[j].dec >= t;
        cp += po;
        cn += ne;
        ca += po | ne;
      }
    }
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

// ------------------------------------------------------------------------------- bitmap form

// Bit-sliced 6-bit counter of up to 63 one-bit inputs per bit position (one word = 32 rows).
struct Cnt6 {
  uint32_t b0, b1, b2, b3, b4, b5;
};

__device__ __forceinline__ void cnt_zero(Cnt6 &c) { c.b0 = c.b1 = c.b2 = c.b3 = c.b4 = c.b5 = 0u; }

__device__ __forceinline__ uint32_t maj3(uint32_t x, uint32_t y, uint32_t z) {
  return (x & y) | (z & (x ^ y));
}

__device__ __forceinline__ void cnt_ripple2(Cnt6 &c, uint32_t k) {
  uint32_t t = c.b2 & k;
  c.b2 ^= k;
  k = t;
  t = c.b3 & k;
  c.b3 ^= k;
  k = t;
  t = c.b4 & k;
  c.b4 ^= k;
  k = t;
  c.b5 ^= k;
}

// Adds four inputs: two full adders into the ones, one into the twos, ripple from the fours.
__device__ __forceinline__ void cnt_add4(Cnt6 &c, uint32_t x0, uint32_t x1, uint32_t x2,
                                         uint32_t x3) {
  const uint32_t tA = maj3(c.b0, x0, x1);
  c.b0 ^= x0 ^ x1;
  const uint32_t tB = maj3(c.b0, x2, x3);
  c.b0 ^= x2 ^ x3;
  const uint32_t f = maj3(c.b1, tA, tB);
  c.b1 ^= tA ^ tB;
  cnt_ripple2(c, f);
}

// Bits where the count is >= t (1 <= t <= 63), most significant bit first.
__device__ __forceinline__ uint32_t cnt_ge(const Cnt6 &c, int t) {
  const uint32_t b[6] = {c.b0, c.b1, c.b2, c.b3, c.b4, c.b5};
  uint32_t gt = 0u, eq = kFull;
#pragma unroll
  for (int k = 5; k >= 0; --k) {
    if ((t >> k) & 1) {
      eq &= b[k];
    } else {
      gt |= eq & b[k];
      eq &= ~b[k];
    }
  }
  return gt | eq;
}

__device__ __forceinline__ uint4 and4(uint4 a, uint4 b) {
  return make_uint4(a.x & b.x, a.y & b.y, a.z & b.z, a.w & b.w);
}

__device__ __forceinline__ int popc4(uint4 v) {
  return __popc(v.x) + __popc(v.y) + __popc(v.z) + __popc(v.w);
}

// Rows of word w that exist (bit j = row 32 w + j < R).
__device__ __forceinline__ uint32_t valid_bits(int64_t w, int64_t R) {
  const int64_t n = R - 32 * w;
  return n >= 32 ? kFull : (n <= 0 ? 0u : ((1u << n) - 1u));
}

// A pass covers 128 words (4096 rows) of a column pair; lane l holds words 4l..4l+3.
constexpr int kPassWords = 128;

// Staged form: each warp has kStageBytes of shared memory, two halves of NB / 2 pair rows per
// direction.  The lanes copy the pair words of a unit (up to NB / 2 rows: one pass of a batch of
// pairs, or several passes of a short chromosome's pairs) with asynchronous copies (cp.async, 16
// bytes each, no registers held while they are in flight) into one half while the other half's
// unit is counted, so two units are in flight per warp.  Each lane reads back only the bytes it
// copied, so the hardware's own per-thread wait is the only synchronisation.
constexpr uint32_t kStageBytes = 12 * 1024;
template <bool NEG>
__host__ __device__ constexpr int stage_pairs() {
  return (int)(kStageBytes / (kPassWords * 4u)) / (NEG ? 2 : 1);  // 12 with NEG, else 24
}
constexpr size_t kBitmapSmem = (size_t)kWarps * kStageBytes;
constexpr int kMaxIpw = 4;  // individuals per work item of the grouped staged form, at most

__device__ __forceinline__ uint4 not4(uint4 v) { return make_uint4(~v.x, ~v.y, ~v.z, ~v.w); }

// A pair word where `on`, else `fill` (the identity of the operation it feeds), from global
// (ldb) or staged shared memory (lds).  With ties counting (NS) the word is the complement of the
// opposite direction's word: key(d) >= key(c) = not key(c) > key(d).  The complement follows the
// same predicated load as in the strict form (fill complemented beforehand): selecting between a
// loaded word's complement and a constant instead made the NS forms 1.6-2.8x slower.
template <bool NS>
__device__ __forceinline__ uint4 ldb(bool on, const uint32_t *p, uint4 fill) {
  uint4 v = NS ? not4(fill) : fill;
  if (on) v = ldg4(p);
  return NS ? not4(v) : v;
}

template <bool NS>
__device__ __forceinline__ uint4 lds(bool on, const uint32_t *p, uint4 fill) {
  uint4 v = NS ? not4(fill) : fill;
  if (on) v = *reinterpret_cast<const uint4 *>(p);
  return NS ? not4(v) : v;
}

__device__ __forceinline__ void cp_async16(uint32_t *dst, const uint32_t *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"((uint64_t)__cvta_generic_to_global(src))
               : "memory");
}

// Closes this thread's current group of asynchronous copies.
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Waits until at most N of this thread's committed copy groups are pending (a hardware wait).
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Adds four pair words per direction to the bit-sliced counters.
template <bool NEG>
__device__ __forceinline__ void cnt_add_group(Cnt6 (&P)[4], Cnt6 (&N)[4], const uint4 (&v)[4],
                                              const uint4 (&u)[4]) {
  cnt_add4(P[0], v[0].x, v[1].x, v[2].x, v[3].x);
  cnt_add4(P[1], v[0].y, v[1].y, v[2].y, v[3].y);
  cnt_add4(P[2], v[0].z, v[1].z, v[2].z, v[3].z);
  cnt_add4(P[3], v[0].w, v[1].w, v[2].w, v[3].w);
  if (NEG) {
    cnt_add4(N[0], u[0].x, u[1].x, u[2].x, u[3].x);
    cnt_add4(N[1], u[0].y, u[1].y, u[2].y, u[3].y);
    cnt_add4(N[2], u[0].z, u[1].z, u[2].z, u[3].z);
    cnt_add4(N[3], u[0].w, u[1].w, u[2].w, u[3].w);
  }
}

// NS: ties count for both directions (complemented opposite words; pad rows masked out).  The
// last-kept variant has no pair-word form (its reference value differs from row to row).
// STAGE: pair words staged in shared memory, for bitmaps larger than L2 whose words stream from
// HBM (more bytes in flight per warp), unless every item is exact (ratio 1: the AND needs no
// counter registers, so rounds of 8 pairs fit in registers).  Otherwise rounds of register loads.
// Staging measured slower where L2 holds the bitmap and with ratio 1; register loads inside the
// staged kernel measured slower still (its shared memory leaves the L1 too little room for the
// loads in flight), so that kernel stages every item.
// The counts of one pass (4 words per lane) of an individual with threshold t into cp / cn /
// ca: the AND of the pair words (exact) or the bit-sliced counters against t.
template <bool NEG, bool NS>
__device__ __forceinline__ void pass_counts(const EvalArgs &a, int64_t w, bool act, bool exact,
                                            int t, uint4 ap, uint4 an, const Cnt6 (&P)[4],
                                            const Cnt6 (&N)[4], int &cp, int &cn, int &ca) {
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
  uint4 pos, neg = zero4;
  if (exact) {
    pos = act ? ap : zero4;
    if (NEG) neg = act ? an : zero4;
  } else {
    pos = make_uint4(cnt_ge(P[0], t), cnt_ge(P[1], t), cnt_ge(P[2], t), cnt_ge(P[3], t));
    if (NEG) neg = make_uint4(cnt_ge(N[0], t), cnt_ge(N[1], t), cnt_ge(N[2], t), cnt_ge(N[3], t));
  }
  if (NS) {  // pad rows (and inactive lanes) hold complemented zeros: mask them out
    const uint4 vm = act ? make_uint4(valid_bits(w, a.R), valid_bits(w + 1, a.R),
                                      valid_bits(w + 2, a.R), valid_bits(w + 3, a.R))
                         : zero4;
    pos = and4(pos, vm);
    if (NEG) neg = and4(neg, vm);
  }
  cp += popc4(pos);
  if (NEG) {
    cn += popc4(neg);
    ca += popc4(make_uint4(pos.x | neg.x, pos.y | neg.y, pos.z | neg.z, pos.w | neg.w));
  } else {
    ca += popc4(pos);
  }
}

// Staged form (the bitmap exceeds L2, ratio below 1).  A work item is a group of a.ipw
// consecutive individuals (1 <= ipw <= kMaxIpw) and one row segment.  The group's bookkeeping
// loads in one round (lane j holds individual j's length, dead flag and key; the columns of
// every individual go to shared memory), and the pair words of all its live individuals form
// one stream of units staged two at a time: the copies of the next unit, of the same individual
// or of the next, are in flight while the current unit is counted.  A unit holds up to H pair
// rows per direction: several consecutive passes of all pairs when the chromosome is short
// (np <= H: H / np passes per unit), else one pass of a batch of up to H pairs.  Grouping
// individuals keeps the stream full across the short chromosomes of the generation loop, whose
// items are otherwise one unit each with a round trip for their bookkeeping before it.  The
// individuals' pair-row indices (c * C + d) are computed once per item into shared memory.
template <bool NEG, bool NS>
__device__ __forceinline__ void bitmap_staged_items(const EvalArgs &a, const PopView &pv,
                                                    int lane, uint32_t *sp, uint32_t *sn,
                                                    uint32_t *pidx) {
  constexpr int NB = stage_pairs<NEG>();
  constexpr int H = NB / 2;
  const int64_t Wst = a.Wst;
  const int64_t passes_total = (Wst + kPassWords - 1) / kPassWords;
  const int ipw = a.ipw;
  const int32_t n_ind = items::count(pv);
  const int32_t n_grp = (n_ind + ipw - 1) / ipw;
  const int32_t n_side = items::move_chunks(a), n_all = n_side + n_grp * a.n_seg;
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
  const uint4 ones = make_uint4(kFull, kFull, kFull, kFull);
  for (int q = items::first(); q < n_all; q = items::next(a.work, lane, q, n_all)) {
    if (q < n_side) {
      if (items::stopped(pv)) return;  // a stopped run changes nothing
      items::move_chunk(a, q, lane);
      continue;
    }
    const int seg = (q - n_side) / n_grp, grp = (q - n_side) - seg * n_grp;  // segment-major
    const int i0 = grp * ipw, cnt = min(ipw, n_ind - i0);
    // lane j < cnt: individual i0 + j's bookkeeping (its slot myi)
    int myL = 0, myst = 0, myi = 0;
    bool mydead = true;
    uint64_t myh = 0ull;
    if (lane < cnt) myi = items::slot(pv, i0 + lane);
    if (lane < cnt) {
      const int i = myi;
      if (pv.off) {
        myst = pv.off[i];
        myL = pv.off[i + 1] - myst;
      } else {
        myst = i * pv.stride;
        myL = pv.len[i];
      }
      mydead = pv.dead && pv.dead[i];
      myh = pv.dkeys ? pv.hash[i] : 0ull;
    }
    __syncwarp();  // (the previous item's reads of pidx are done)
#pragma unroll
    for (int j = 0; j < kMaxIpw; ++j) {
      if (j < cnt) {  // (cnt is the same in every lane)
        int c0, c1;
        if (!pv.off) {  // fixed-stride rows: the column words load with the lengths
          const int st = __shfl_sync(kFull, myi, j) * pv.stride;
          c0 = pv.cols[st + lane];
          c1 = pv.cols[st + 32 + lane];
        } else {
          const int st = __shfl_sync(kFull, myst, j), L = __shfl_sync(kFull, myL, j);
          c0 = lane < L ? pv.cols[st + lane] : 0;
          c1 = lane + 32 < L ? pv.cols[st + 32 + lane] : 0;
        }
        // pair k = (column k, column k + 1): lane k holds pairs k and 32 + k; the index of the
        // pair word row is c * C + d for the positive direction, d * C + c for the negative
        // (swapped when ties count both ways), below 2^32 since C <= 65,535
        const int n0 = __shfl_down_sync(kFull, c0, 1), n1 = __shfl_down_sync(kFull, c1, 1);
        const int c32 = __shfl_sync(kFull, c1, 0);
        const uint32_t C = (uint32_t)a.C;
        const uint32_t ka = (uint32_t)c0, kb = (uint32_t)(lane < 31 ? n0 : c32);
        const uint32_t la = (uint32_t)c1, lb = (uint32_t)(lane < 31 ? n1 : 0);
        uint32_t *pj = pidx + j * 2 * EBIC_MAX_LEN;
        pj[lane] = NS ? kb * C + ka : ka * C + kb;
        pj[EBIC_MAX_LEN + lane] = NS ? ka * C + kb : kb * C + ka;
        pj[32 + lane] = NS ? lb * C + la : la * C + lb;
        pj[EBIC_MAX_LEN + 32 + lane] = NS ? la * C + lb : lb * C + la;
      }
    }
    if (items::stopped(pv)) return;  // (read with the item's loads; before any store)
    const bool mylive = lane < cnt && !mydead && myL >= 2;
    const unsigned live = __ballot_sync(kFull, mylive);
    if (!live) continue;
    // each live individual's key enters the duplicate table from its first segment's item
    items::Insert myins{0ull, 0u, pv.dkeys != nullptr && seg == 0 && mylive};
    if (myins.on) {
      myins.idx = table_index(myh, pv.dmask);
      myins.prev = atomicCAS(reinterpret_cast<unsigned long long *>(pv.dkeys + myins.idx), 0ull,
                             (unsigned long long)myh);
    }
    __syncwarp();  // pidx is written
    const int64_t p0 = (int64_t)seg * a.seg_passes;
    const int64_t p1 = min(p0 + a.seg_passes, passes_total);
    const int n_pass = (int)(p1 - p0);
    // lane j: individual j's unit plan
    const int mynp = myL - 1;
    const bool mypacked = mynp <= H;
    const int myppu = mypacked ? H / max(mynp, 1) : 1;   // passes per unit
    const int mynbat = mypacked ? 1 : (mynp + H - 1) / H;  // batches per pass
    const int myunits = !mylive ? 0 : (mypacked ? (n_pass + myppu - 1) / myppu : n_pass * mynbat);
    auto next_live = [&](int from) -> int {  // the first live individual >= from, or kMaxIpw
      const unsigned m = from >= 32 ? 0u : (live >> from) << from;
      return m ? __ffs(m) - 1 : kMaxIpw;
    };
    auto advance = [&](int &j, int &u) {
      if (++u >= __shfl_sync(kFull, myunits, j)) {
        j = next_live(j + 1);
        u = 0;
      }
    };
    // copies of unit u of individual j into half b
    auto issue = [&](int j, int u, int b) {
      const int np = __shfl_sync(kFull, mynp, j), ppu = __shfl_sync(kFull, myppu, j);
      const int nbat = __shfl_sync(kFull, mynbat, j);
      const uint32_t *pj = pidx + j * 2 * EBIC_MAX_LEN;
      uint32_t *bp = sp + b * H * kPassWords, *bn = sn + b * H * kPassWords;
      int64_t qa, qb;
      int k0, nb;
      if (np <= H) {
        qa = p0 + (int64_t)u * ppu;
        qb = min(p1, qa + ppu);
        k0 = 0;
        nb = np;
      } else {
        qa = p0 + u / nbat;
        qb = qa + 1;
        k0 = (u % nbat) * H;
        nb = min(H, np - k0);
      }
      for (int64_t qq = qa; qq < qb; ++qq) {
        const int64_t w = qq * kPassWords + lane * 4;
        if (w < Wst) {
          const uint32_t *G = a.bitmap + w;
          const int slot0 = (int)(qq - qa) * nb;
          for (int k = 0; k < nb; ++k) {
            cp_async16(bp + (slot0 + k) * kPassWords, G + (int64_t)pj[k0 + k] * Wst);
            if (NEG)
              cp_async16(bn + (slot0 + k) * kPassWords,
                         G + (int64_t)pj[EBIC_MAX_LEN + k0 + k] * Wst);
          }
        }
      }
      cp_async_commit();
    };
    int ji = next_live(0), ui = 0, jc = ji, uc = 0, gi = 0, gc = 0;
    int cp = 0, cn = 0, ca = 0;
    uint4 ap = ones, an = ones;
    Cnt6 P[4], N[4];
    issue(ji, ui, 0);
    ++gi;
    advance(ji, ui);
    while (jc < kMaxIpw) {
      if (ji < kMaxIpw) {
        issue(ji, ui, gi & 1);
        ++gi;
        advance(ji, ui);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      // count unit uc of individual jc from half gc & 1
      const int np = __shfl_sync(kFull, mynp, jc), ppu = __shfl_sync(kFull, myppu, jc);
      const int nbat = __shfl_sync(kFull, mynbat, jc), nu = __shfl_sync(kFull, myunits, jc);
      const int t = threshold(np + 1, a.rnum, a.rden);
      const bool exact = (t == np);
      const uint32_t *bp = sp + (gc & 1) * H * kPassWords, *bn = sn + (gc & 1) * H * kPassWords;
      ++gc;
      int64_t qa, qb;
      int k0, nb;
      if (np <= H) {
        qa = p0 + (int64_t)uc * ppu;
        qb = min(p1, qa + ppu);
        k0 = 0;
        nb = np;
      } else {
        qa = p0 + uc / nbat;
        qb = qa + 1;
        k0 = (uc % nbat) * H;
        nb = min(H, np - k0);
      }
      for (int64_t qq = qa; qq < qb; ++qq) {
        const int64_t w = qq * kPassWords + lane * 4;
        const bool act = w < Wst;  // (Wst is a multiple of 4: a lane's 4 words all exist or not)
        const int s0 = (int)(qq - qa) * nb;
        if (k0 == 0) {
          ap = ones;
          an = ones;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            cnt_zero(P[j]);
            cnt_zero(N[j]);
          }
        }
        if (exact) {
          for (int j = 0; j < nb; ++j) {
            ap = and4(ap, lds<NS>(act, bp + (s0 + j) * kPassWords, ones));
            if (NEG) an = and4(an, lds<NS>(act, bn + (s0 + j) * kPassWords, ones));
          }
        } else {
          for (int h = 0; h < nb; h += 4) {  // (the last group padded with zeros)
            uint4 v[4], uu[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const bool in = act && h + j < nb;
              v[j] = lds<NS>(in, bp + (s0 + h + j) * kPassWords, zero4);
              uu[j] = NEG ? lds<NS>(in, bn + (s0 + h + j) * kPassWords, zero4) : zero4;
            }
            cnt_add_group<NEG>(P, N, v, uu);
          }
        }
        if (k0 + nb == np) pass_counts<NEG, NS>(a, w, act, exact, t, ap, an, P, N, cp, cn, ca);
      }
      if (uc + 1 == nu) {  // the individual's last unit: its counts
        cp = __reduce_add_sync(kFull, cp);
        cn = __reduce_add_sync(kFull, cn);
        ca = __reduce_add_sync(kFull, ca);
        const int i = __shfl_sync(kFull, myi, jc);
        if (lane == 0) {
          if (cp) atomicAdd(a.rows_pos + i, cp);
          if (cn) atomicAdd(a.rows_neg + i, cn);
          if (ca) atomicAdd(a.rows_any + i, ca);
        }
        cp = cn = ca = 0;
      }
      advance(jc, uc);
    }
    items::insert_finish(pv, myins, myh, myi);
  }
}

// GROUP (with STAGE only): work items of a.ipw > 1 individuals (bitmap_staged_items); else one
// individual per item.  Each form declares only its own shared arrays.
template <bool NEG, bool NS, bool STAGE, bool GROUP>
__global__ void __launch_bounds__(kThreads, 2) k_eval_bitmap(EvalArgs a, PopView pv) {
  extern __shared__ __align__(128) uint32_t s_stage[];  // kStageBytes per warp (STAGE)
  __shared__ int64_t s_pos[GROUP ? 1 : kWarps][EBIC_MAX_LEN];
  __shared__ int64_t s_neg[GROUP ? 1 : kWarps][EBIC_MAX_LEN];
  __shared__ int32_t s_col[GROUP ? 1 : kWarps][EBIC_MAX_LEN];
  __shared__ uint32_t s_pidx[GROUP ? kWarps * kMaxIpw * 2 : 1][EBIC_MAX_LEN];
  constexpr int NB = stage_pairs<NEG>();
  static_assert(NB % 4 == 0, "staged batches are read in groups of four pairs");
  static_assert(STAGE || !GROUP, "groups of individuals are a form of the staged kernel");
  wait_prior_grid();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *sp = s_stage + (size_t)warp * (kStageBytes / 4) + lane * 4;  // pair j: sp + 128 j
  uint32_t *sn = sp + NB * kPassWords;                                    // negative direction
  if (GROUP) {
    bitmap_staged_items<NEG, NS>(a, pv, lane, sp, sn, &s_pidx[warp * kMaxIpw * 2][0]);
    return;
  }
  const int64_t Wst = a.Wst;
  const int64_t passes_total = (Wst + kPassWords - 1) / kPassWords;
  const int32_t n_ind = items::count(pv);
  const int32_t n_side = items::move_chunks(a), n_all = n_side + n_ind * a.n_seg;
  const uint4 zero4 = make_uint4(0u, 0u, 0u, 0u);
  const uint4 ones = make_uint4(kFull, kFull, kFull, kFull);
  for (int q = items::first(); q < n_all; q = items::next(a.work, lane, q, n_all)) {
    if (q < n_side) {
      if (items::stopped(pv)) return;  // a stopped run changes nothing
      items::move_chunk(a, q, lane);
      continue;
    }
    const int seg = (q - n_side) / n_ind;  // segment-major
    const int i = items::slot(pv, (q - n_side) - seg * n_ind);
    const items::Meta m = items::load_meta(pv, i, lane);
    if (items::stopped(pv)) return;  // (read with the item's loads; before any store)
    if (m.dead || m.L < 2) continue;
    const items::Insert ins = items::insert_start(pv, seg, m.h, lane);
    const int L = m.L, np = L - 1;
    __syncwarp();
    s_col[warp][lane] = m.c0;
    s_col[warp][lane + 32] = m.c1;
    __syncwarp();
    for (int k = lane; k < np; k += 32) {
      const int64_t c = s_col[warp][k], d = s_col[warp][k + 1];
      s_pos[warp][k] = NS ? (d * a.C + c) * Wst : (c * a.C + d) * Wst;
      s_neg[warp][k] = NS ? (c * a.C + d) * Wst : (d * a.C + c) * Wst;
    }
    __syncwarp();
    const int t = threshold(L, a.rnum, a.rden);
    const bool exact_item = (t == np);
    const int64_t p0 = (int64_t)seg * a.seg_passes;
    const int64_t p1 = min(p0 + a.seg_passes, passes_total);
    int cp = 0, cn = 0, ca = 0;
    // The item's passes, compiled twice: for the exact test (the AND of the pair words, no
    // counters) and for the counting one, so that neither carries the other's work.
    auto run = [&](auto ex) {
      const bool exact = decltype(ex)::value;
      // The counts of one pass's 4 words per lane, added to cp / cn / ca.
      auto finish_pass = [&](int64_t w, bool act, uint4 ap, uint4 an, Cnt6 (&P)[4],
                             Cnt6 (&N)[4]) {
        uint4 pos, neg = zero4;
        if (exact) {
          pos = act ? ap : zero4;
          if (NEG) neg = act ? an : zero4;
        } else {
          pos = make_uint4(cnt_ge(P[0], t), cnt_ge(P[1], t), cnt_ge(P[2], t), cnt_ge(P[3], t));
          if (NEG)
            neg = make_uint4(cnt_ge(N[0], t), cnt_ge(N[1], t), cnt_ge(N[2], t), cnt_ge(N[3], t));
        }
        if (NS) {  // pad rows (and inactive lanes) hold complemented zeros: mask them out
          const uint4 vm = act ? make_uint4(valid_bits(w, a.R), valid_bits(w + 1, a.R),
                                            valid_bits(w + 2, a.R), valid_bits(w + 3, a.R))
                               : zero4;
          pos = and4(pos, vm);
          if (NEG) neg = and4(neg, vm);
        }
        cp += popc4(pos);
        if (NEG) {
          cn += popc4(neg);
          ca += popc4(make_uint4(pos.x | neg.x, pos.y | neg.y, pos.z | neg.z, pos.w | neg.w));
        } else {
          ca += popc4(pos);
        }
      };
      if (STAGE) {
        // Units staged two at a time: the copies of the next unit are in flight while the current
        // unit is counted.  A unit holds up to H pair rows per direction: several consecutive
        // passes of all pairs when the chromosome is short (np <= H: H / np passes per unit), else
        // one pass of a batch of up to H pairs.  So a warp keeps about H rows per direction in
        // flight however short its chromosome (the loop's evolved population is mostly one- and
        // two-pair chromosomes).
        constexpr int H = NB / 2;
        const bool packed = np <= H;
        const int ppu = packed ? H / np : 1;                  // passes per unit
        const int nbat = packed ? 1 : (np + H - 1) / H;       // batches per pass
        const int n_pass = (int)(p1 - p0);
        const int n_units = packed ? (n_pass + ppu - 1) / ppu : n_pass * nbat;
        auto issue = [&](int u) {
          uint32_t *bp = sp + (u & 1) * H * kPassWords, *bn = sn + (u & 1) * H * kPassWords;
          if (packed) {
            const int64_t qa = p0 + (int64_t)u * ppu, qb = min(p1, qa + ppu);
            for (int64_t q = qa; q < qb; ++q) {
              const int64_t w = q * kPassWords + lane * 4;
              if (w < Wst) {
                const uint32_t *G = a.bitmap + w;
                const int slot0 = (int)(q - qa) * np;
                for (int j = 0; j < np; ++j) {
                  cp_async16(bp + (slot0 + j) * kPassWords, G + s_pos[warp][j]);
                  if (NEG) cp_async16(bn + (slot0 + j) * kPassWords, G + s_neg[warp][j]);
                }
              }
            }
          } else {
            const int64_t pass = p0 + u / nbat;
            const int k0 = (u % nbat) * H, nb = min(H, np - k0);
            const int64_t w = pass * kPassWords + lane * 4;
            if (w < Wst) {
              const uint32_t *G = a.bitmap + w;
              for (int j = 0; j < nb; ++j) {
                cp_async16(bp + j * kPassWords, G + s_pos[warp][k0 + j]);
                if (NEG) cp_async16(bn + j * kPassWords, G + s_neg[warp][k0 + j]);
              }
            }
          }
          cp_async_commit();
        };
        uint4 ap = ones, an = ones;
        Cnt6 P[4], N[4];
        // counts slots [s0, s0 + nb) of a half into the running pass
        auto count = [&](const uint32_t *bp, const uint32_t *bn, int s0, int nb, bool act) {
          if (exact) {
            for (int j = 0; j < nb; ++j) {
              ap = and4(ap, lds<NS>(act, bp + (s0 + j) * kPassWords, ones));
              if (NEG) an = and4(an, lds<NS>(act, bn + (s0 + j) * kPassWords, ones));
            }
          } else {
            for (int h = 0; h < nb; h += 4) {  // (the last group padded with zeros)
              uint4 v[4], uu[4];
  #pragma unroll
              for (int j = 0; j < 4; ++j) {
                const bool in = act && h + j < nb;
                v[j] = lds<NS>(in, bp + (s0 + h + j) * kPassWords, zero4);
                uu[j] = NEG ? lds<NS>(in, bn + (s0 + h + j) * kPassWords, zero4) : zero4;
              }
              cnt_add_group<NEG>(P, N, v, uu);
            }
          }
        };
        auto start_pass = [&]() {
          ap = ones;
          an = ones;
  #pragma unroll
          for (int j = 0; j < 4; ++j) {
            cnt_zero(P[j]);
            cnt_zero(N[j]);
          }
        };
        if (n_units > 0) issue(0);
        for (int u = 0; u < n_units; ++u) {
          if (u + 1 < n_units) {
            issue(u + 1);
            cp_async_wait<1>();
          } else {
            cp_async_wait<0>();
          }
          const uint32_t *bp = sp + (u & 1) * H * kPassWords, *bn = sn + (u & 1) * H * kPassWords;
          if (packed) {
            const int64_t qa = p0 + (int64_t)u * ppu, qb = min(p1, qa + ppu);
            for (int64_t q = qa; q < qb; ++q) {
              const int64_t w = q * kPassWords + lane * 4;
              const bool act = w < Wst;  // (Wst is a multiple of 4: a lane's 4 words all exist or not)
              start_pass();
              count(bp, bn, (int)(q - qa) * np, np, act);
              finish_pass(w, act, ap, an, P, N);
            }
          } else {
            const int64_t pass = p0 + u / nbat;
            const int k0 = (u % nbat) * H, nb = min(H, np - k0);
            const int64_t w = pass * kPassWords + lane * 4;
            const bool act = w < Wst;
            if (k0 == 0) start_pass();
            count(bp, bn, 0, nb, act);
            if (k0 + nb == np) finish_pass(w, act, ap, an, P, N);
          }
        }
      } else {
        for (int64_t pass = p0; pass < p1; ++pass) {
          const int64_t w = pass * kPassWords + lane * 4;
          const bool act = w < Wst;  // (Wst is a multiple of 4: a lane's 4 words all exist or not)
          const uint32_t *G = a.bitmap + w;
          uint4 ap = ones, an = ones;
          Cnt6 P[4], N[4];
  #pragma unroll
          for (int j = 0; j < 4; ++j) {
            cnt_zero(P[j]);
            cnt_zero(N[j]);
          }
          if (exact) {
            // The pair words of a round are loaded together, the last round padded with the
            // operation's identity, so np pairs cost ceil(np / 8) dependent load rounds.
            for (int k = 0; k < np; k += 8) {
              uint4 v[8], u[8];
  #pragma unroll
              for (int j = 0; j < 8; ++j) {
                const bool in = k + j < np;
                v[j] = ldb<NS>(act && in, G + (in ? s_pos[warp][k + j] : 0), ones);
                if (NEG) u[j] = ldb<NS>(act && in, G + (in ? s_neg[warp][k + j] : 0), ones);
              }
  #pragma unroll
              for (int j = 0; j < 8; ++j) {
                ap = and4(ap, v[j]);
                if (NEG) an = and4(an, u[j]);
              }
            }
          } else {
            constexpr int RC = NEG ? 4 : 8;  // pairs per round (the counters of both directions
                                             // and 8 pairs' words exceed the register budget)
            for (int k = 0; k < np; k += RC) {
              uint4 v[RC], u[RC];
  #pragma unroll
              for (int j = 0; j < RC; ++j) {
                const bool in = k + j < np;
                v[j] = ldb<NS>(act && in, G + (in ? s_pos[warp][k + j] : 0), zero4);
                if (NEG) u[j] = ldb<NS>(act && in, G + (in ? s_neg[warp][k + j] : 0), zero4);
              }
  #pragma unroll
              for (int h = 0; h < RC; h += 4) {
                const uint4 vv[4] = {v[h], v[h + 1], v[h + 2], v[h + 3]};
                const uint4 uu[4] = {NEG ? u[h] : zero4, NEG ? u[h + 1] : zero4,
                                     NEG ? u[h + 2] : zero4, NEG ? u[h + 3] : zero4};
                cnt_add_group<NEG>(P, N, vv, uu);
              }
            }
          }
          finish_pass(w, act, ap, an, P, N);
        }
      }
    };
    if (exact_item)
      run(std::true_type{});
    else
      run(std::false_type{});
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

// ------------------------------------------------------------------------------- plain form

// One launch per individual; one row per thread; block counts by __syncthreads_count and one
// atomic per block and output (the paper's Sec. 2.4 kernel: atomics, no intermediate buffer).
template <bool NEG, bool NS, bool LK>
__global__ void k_eval_plain(EvalArgs a, const int32_t *__restrict__ cols, int L, int i) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool po = false, ne = false;
  if (r < a.R) {
    const int t = threshold(L, a.rnum, a.rden);
    RowTrend<uint32_t, NEG, NS, LK> tr;
    tr.start(a.keys[(int64_t)cols[0] * a.R_pad + r]);
    for (int k = 1; k < L; ++k) tr.step(a.keys[(int64_t)cols[k] * a.R_pad + r]);
    po = tr.inc >= t;
    ne = NEG && tr.dec >= t;
  }
  const int np = __syncthreads_count(po);
  const int nn = __syncthreads_count(ne);
  const int na = __syncthreads_count(po || ne);
  if (threadIdx.x == 0) {
    if (np) atomicAdd(a.rows_pos + i, np);
    if (nn) atomicAdd(a.rows_neg + i, nn);
    if (na) atomicAdd(a.rows_any + i, na);
  }
}

// ------------------------------------------------------------------------------- fitness

// f = 0 when dead or rows_any < min_rows, else rows_any * 2^min(L, col_cap) (exact uint64).
__global__ void k_fitness(EvalArgs a, PopView pv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= pv.n) return;
  const int ra = a.rows_any[i];
  const bool dead = pv_dead(pv, i);
  const int L = pv_len(pv, i);
  const int sh = L < a.col_cap ? L : a.col_cap;
  a.fitness[i] = (dead || ra < a.min_rows) ? 0ull : ((uint64_t)ra << sh);
}

int blocks_per_sm_for(const void *kernel, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    nb = 1;
  }
  return nb < 1 ? 1 : nb;
}

}  // namespace

cudaError_t launch_validate_csr(const int32_t *cols, const int32_t *off, int32_t n, int32_t C,
                                int32_t *err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_validate_csr<<<(unsigned)((n + 7) / 8), 256, 0, s>>>(cols, off, n, C, err);
  return cudaGetLastError();
}

cudaError_t launch_fitness(const EvalArgs &a, const PopView &pv, cudaStream_t s) {
  if (pv.n <= 0 || !a.fitness) return cudaSuccess;
  k_fitness<<<(pv.n + 255) / 256, 256, 0, s>>>(a, pv);
  return cudaGetLastError();
}

// Launches `kern` with programmatic stream serialisation when `pdl` is set (the kernel calls
// griddepcontrol.wait before it reads what the previous kernel wrote).
template <class... Args>
cudaError_t launch_maybe_pdl(void (*kern)(Args...), dim3 grid, dim3 block, size_t smem,
                             cudaStream_t s, bool pdl, Args... args) {
  if (!pdl) {
    kern<<<grid, block, smem, s>>>(args...);
    return cudaGetLastError();
  }
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

using EvalKernel = void (*)(EvalArgs, PopView);

// The instantiation for (negative trends, ties counting, last kept).
static EvalKernel direct_kernel(bool neg, bool ns, bool lk) {
  static const EvalKernel t[8] = {
      k_eval_direct<false, false, false>, k_eval_direct<false, false, true>,
      k_eval_direct<false, true, false>,  k_eval_direct<false, true, true>,
      k_eval_direct<true, false, false>,  k_eval_direct<true, false, true>,
      k_eval_direct<true, true, false>,   k_eval_direct<true, true, true>};
  return t[(neg ? 4 : 0) + (ns ? 2 : 0) + (lk ? 1 : 0)];
}

static EvalKernel bitmap_kernel(bool neg, bool ns, bool stage, bool group) {
  static const EvalKernel t[12] = {
      k_eval_bitmap<false, false, false, false>, k_eval_bitmap<false, false, true, false>,
      k_eval_bitmap<false, true, false, false>,  k_eval_bitmap<false, true, true, false>,
      k_eval_bitmap<true, false, false, false>,  k_eval_bitmap<true, false, true, false>,
      k_eval_bitmap<true, true, false, false>,   k_eval_bitmap<true, true, true, false>,
      k_eval_bitmap<false, false, true, true>,   k_eval_bitmap<false, true, true, true>,
      k_eval_bitmap<true, false, true, true>,    k_eval_bitmap<true, true, true, true>};
  if (group) return t[8 + (neg ? 2 : 0) + (ns ? 1 : 0)];
  return t[(neg ? 4 : 0) + (ns ? 2 : 0) + (stage ? 1 : 0)];
}

cudaError_t prepare_bitmap_eval() {
  // one fixed limit for every context (no call lowers another's), set once per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  static std::mutex mu;
  static bool attr_set[kMaxDevices] = {};
  std::lock_guard<std::mutex> lock(mu);
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (attr_set[dev]) return cudaSuccess;
  for (int k = 0; k < 8; ++k)
    if ((e = cudaFuncSetAttribute(bitmap_kernel(k & 2, k & 1, true, k & 4),
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kBitmapSmem)) != cudaSuccess)
      return e;
  attr_set[dev] = true;
  return cudaSuccess;
}

cudaError_t launch_eval_kernel(int mode, const EvalArgs &a0, const PopView &pv, int num_sms,
                               cudaStream_t s, bool pdl) {
  if (pv.n <= 0) return cudaSuccess;
  if (mode == EBIC_MODE_STAGED) {
    // the staged kernel implements the default pair test and needs its tiles to fit
    if (a0.dtma && a0.dtma->ok && !a0.non_strict && !a0.last_kept)
      return launch_eval_direct_tma(*a0.dtma, a0, pv, num_sms, s, pdl);
    mode = EBIC_MODE_DIRECT;
  }
  if (mode == EBIC_MODE_BITMAP && a0.last_kept) return cudaErrorInvalidValue;  // no word form
  if (pv.list && mode != EBIC_MODE_BITMAP) return cudaErrorInvalidValue;  // (bitmap kernels only)
  if (mode == EBIC_MODE_DIRECT && a0.codes) return launch_eval_codes(a0, pv, num_sms, s, pdl);
  EvalArgs a = a0;
  const bool bitmap = (mode == EBIC_MODE_BITMAP);
  const int64_t passes_total = bitmap ? (a.Wst + 127) / 128 : a.R_pad / 128;
  const bool stage = bitmap && a.stage_bitmap && a.rnum < a.rden;  // (ratio 1: all exact)
  // Individuals per work item: groups (ipw > 1) are a form of the staged kernel.
  a.ipw = stage ? std::max(1, std::min(a0.ipw, kMaxIpw)) : 1;
  const EvalKernel kern = bitmap ? bitmap_kernel(a.neg, a.non_strict, stage, a.ipw > 1)
                                 : direct_kernel(a.neg, a.non_strict, a.last_kept);
  const size_t smem = stage ? kBitmapSmem : 0;
  if (stage) {
    const cudaError_t e = prepare_bitmap_eval();
    if (e != cudaSuccess) return e;
  }
  const int bps = blocks_per_sm_for((const void *)kern, smem);
  const int64_t warps = (int64_t)num_sms * bps * kWarps;
  const int64_t n_grp = ((int64_t)pv.n + a.ipw - 1) / a.ipw;
  // Segments: the autotuner's size when it set one, else enough work items for ~8 per
  // resident warp; at most 2^30 items in total.
  int64_t seg = a0.seg_passes > 0 ? a0.seg_passes : (n_grp * passes_total) / (8 * warps);
  if (seg < 1) seg = 1;
  if (seg > passes_total) seg = passes_total;
  int64_t n_seg = (passes_total + seg - 1) / seg;
  while (n_grp * n_seg > (1LL << 30)) {
    seg *= 2;
    n_seg = (passes_total + seg - 1) / seg;
  }
  a.seg_passes = (int32_t)seg;
  a.n_seg = (int32_t)n_seg;
  // (the side task's chunks count too: with a warp for every item they run beside the others)
  const int64_t items = n_grp * n_seg + (a.mv_table ? (a.mv_n + 31) / 32 : 0);
  int64_t grid = (int64_t)num_sms * bps;
  const int64_t need = (items + kWarps - 1) / kWarps;
  if (grid > need) grid = need;
  return launch_maybe_pdl(kern, dim3((unsigned)grid), dim3(kThreads), smem, s, pdl, a, pv);
}

cudaError_t launch_eval(int mode, const EvalArgs &a, const PopView &pv, int num_sms,
                        cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
  cudaError_t e;
  const size_t nb = (size_t)(pv.n > 0 ? pv.n : 0) * sizeof(int32_t);
  if ((e = cudaMemsetAsync(a.rows_pos, 0, nb, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.rows_neg, 0, nb, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.rows_any, 0, nb, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(a.work, 0, sizeof(int32_t), s)) != cudaSuccess) return e;
  if (ev0 && (e = cudaEventRecord(ev0, s)) != cudaSuccess) return e;
  if ((e = launch_eval_kernel(mode, a, pv, num_sms, s)) != cudaSuccess) return e;
  if (ev1 && (e = cudaEventRecord(ev1, s)) != cudaSuccess) return e;
  return launch_fitness(a, pv, s);
}

cudaError_t launch_eval_plain(const EvalArgs &a, const int32_t *d_cols, int32_t L, int32_t i,
                              cudaStream_t s) {
  using PlainKernel = void (*)(EvalArgs, const int32_t *, int, int);
  static const PlainKernel t[8] = {
      k_eval_plain<false, false, false>, k_eval_plain<false, false, true>,
      k_eval_plain<false, true, false>,  k_eval_plain<false, true, true>,
      k_eval_plain<true, false, false>,  k_eval_plain<true, false, true>,
      k_eval_plain<true, true, false>,   k_eval_plain<true, true, true>};
  const PlainKernel k = t[(a.neg ? 4 : 0) + (a.non_strict ? 2 : 0) + (a.last_kept ? 1 : 0)];
  const unsigned grid = (unsigned)((a.R + 255) / 256);
  k<<<grid, 256, 0, s>>>(a, d_cols, L, i);
  return cudaGetLastError();
}
