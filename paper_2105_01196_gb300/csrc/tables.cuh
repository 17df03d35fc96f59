// Device hash tables of the generation loop: the tabu list (set of chromosome keys) and the
// per-generation duplicate table (key -> lowest slot).  Open addressing with linear probing over a
// power-of-two capacity that is kept at least eight times the number of keys, so every probe
// sequence meets an empty slot; loops are still bounded by the capacity.  Each probe step is a
// dependent round trip to L2 (an atomic for insertions), and the slowest of a launch's probes
// sets the launch's length: at load factor 1/2 the longest runs of linear probing cost several
// microseconds per generation, at 1/8 they are short.  Key 0 marks an empty slot (the
// chromosome key never is 0: a zero FNV-1a hash is replaced by a fixed constant).
#pragma once

#include <stdint.h>

__device__ __forceinline__ uint32_t table_index(uint64_t h, uint32_t mask) {
  return (uint32_t)(h ^ (h >> 32)) & mask;
}

__device__ __forceinline__ bool tabu_contains(const uint64_t *keys, uint32_t mask, uint64_t h) {
  uint32_t i = table_index(h, mask);
  for (uint32_t n = 0; n <= mask; ++n) {
    const uint64_t k = keys[i];
    if (k == h) return true;
    if (k == 0ull) return false;
    i = (i + 1) & mask;
  }
  return false;
}

// Returns true when h was not present and has been inserted.
__device__ __forceinline__ bool tabu_insert(uint64_t *keys, uint32_t mask, uint64_t h) {
  uint32_t i = table_index(h, mask);
  for (uint32_t n = 0; n <= mask; ++n) {
    const unsigned long long prev =
        atomicCAS(reinterpret_cast<unsigned long long *>(keys + i), 0ull, (unsigned long long)h);
    if (prev == 0ull) return true;
    if (prev == h) return false;
    i = (i + 1) & mask;
  }
  return false;
}

// Duplicate table: slot word holds 0xFFFFFFFF - s so that atomicMax keeps the lowest slot and a
// zero-filled table is empty.
__device__ __forceinline__ void dedup_insert(uint64_t *keys, uint32_t *slot, uint32_t mask,
                                             uint64_t h, int s) {
  uint32_t i = table_index(h, mask);
  for (uint32_t n = 0; n <= mask; ++n) {
    const unsigned long long prev =
        atomicCAS(reinterpret_cast<unsigned long long *>(keys + i), 0ull, (unsigned long long)h);
    if (prev == 0ull || prev == h) {
      atomicMax(slot + i, 0xFFFFFFFFu - (uint32_t)s);
      return;
    }
    i = (i + 1) & mask;
  }
}

// True when h was inserted by a lower slot than s.  (A position's key and slot word are loaded
// together, so each probe step is one round trip.)
__device__ __forceinline__ bool dedup_is_dup(const uint64_t *keys, const uint32_t *slot,
                                             uint32_t mask, uint64_t h, int s) {
  uint32_t i = table_index(h, mask);
  for (uint32_t n = 0; n <= mask; ++n) {
    const uint64_t k = keys[i];
    const uint32_t w = slot[i];
    if (k == h) return w != 0xFFFFFFFFu - (uint32_t)s;
    if (k == 0ull) return false;
    i = (i + 1) & mask;
  }
  return false;
}
