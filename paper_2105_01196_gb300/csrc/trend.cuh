// The pair test of the trend counts (Sec. 2.3) for one row along a series of columns, in the
// library's three variants:
//   strict ties (default)  a positive pair holds when the next value is greater, a negative pair
//                          when it is smaller; a tie holds for neither direction;
//   NS (non-strict)        greater-or-equal / smaller-or-equal: a tie holds for both;
//   LK (last kept)         each direction compares a value with the last value that kept that
//                          direction (the series' first value to begin with) instead of with its
//                          predecessor; a value that breaks the direction is skipped.
// Works on order keys (uint32) and on float32 values alike.
#pragma once

#include <stdint.h>

template <bool NS, typename T>
__device__ __forceinline__ bool pair_up(T cur, T ref) {
  return NS ? cur >= ref : cur > ref;
}

template <bool NS, typename T>
__device__ __forceinline__ bool pair_down(T cur, T ref) {
  return NS ? cur <= ref : cur < ref;
}

template <typename T, bool NEG, bool NS, bool LK>
struct RowTrend {
  T up_ref, down_ref;  // predecessor, or the last value each direction kept
  int inc, dec;
  __device__ __forceinline__ void start(T v) {
    up_ref = v;
    down_ref = v;
    inc = 0;
    dec = 0;
  }
  __device__ __forceinline__ void step(T v) {
    const bool u = pair_up<NS>(v, up_ref);
    inc += u;
    if (NEG) {
      const bool d = pair_down<NS>(v, down_ref);
      dec += d;
      if (LK && d) down_ref = v;
    }
    if (LK) {
      if (u) up_ref = v;
    } else {
      up_ref = v;
      down_ref = v;
    }
  }
};
