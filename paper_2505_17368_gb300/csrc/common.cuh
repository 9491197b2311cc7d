// common.cuh -- shared device helpers of libhenn (sm_103a).
//
// Counter-based random numbers (SplitMix64, Steele, Lea & Flood 2014), the
// keyed permutation that fixes each layer's NSW insertion order, sortable
// keys for (distance, index) pairs, and warp utilities.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/henn.h"

namespace henn {

constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;
constexpr int kWarp = 32;
constexpr int kMmax = 32;  // adjacency row width: one 128-byte line of int32

// ------------------------------------------------------------------ RNG

// SplitMix64 output finaliser.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Output w (0-based) of a SplitMix64 generator whose state starts at h.
__host__ __device__ __forceinline__ uint64_t derive(uint64_t h, uint64_t w) {
  return mix64(h + (w + 1ull) * kGolden);
}

// floor(u * s / 2^64): an unbiased-enough index in [0, s).
__host__ __device__ __forceinline__ uint64_t bounded(uint64_t u, uint64_t s) {
#ifdef __CUDA_ARCH__
  return __umul64hi(u, s);
#else
  return (uint64_t)(((unsigned __int128)u * (unsigned __int128)s) >> 64);
#endif
}

// Keyed permutation of [0, n): balanced 4-round Feistel network on 2*half
// bits with a SplitMix64 round function (Luby-Rackoff construction), folded
// onto [0, n) by cycle walking (Black & Rogaway 2002).  perm(j) is the
// insertion rank of layer-local point j.
struct Feistel {
  uint64_t key;
  uint64_t n;
  int half;

  __host__ __device__ static Feistel make(uint64_t seed, int layer, uint64_t n) {
    Feistel f;
    f.key = derive(derive(seed, HENN_TAG_ORDER), (uint64_t)layer);
    f.n = n;
    int bits = 2;
    while ((1ull << bits) < n) ++bits;
    if (bits & 1) ++bits;
    f.half = bits / 2;
    return f;
  }
  __host__ __device__ __forceinline__ uint64_t round_trip(uint64_t x) const {
    const uint64_t mask = (1ull << half) - 1ull;
    uint64_t l = x >> half, r = x & mask;
#pragma unroll
    for (uint64_t k = 0; k < 4; ++k) {
      uint64_t f = derive(derive(key, k), r) & mask;
      uint64_t nr = l ^ f;
      l = r;
      r = nr;
    }
    return (l << half) | r;
  }
  __host__ __device__ __forceinline__ uint64_t perm(uint64_t x) const {
    if (n <= 1) return 0;
    uint64_t y = round_trip(x);
    while (y >= n) y = round_trip(y);  // ends: x lies on a cycle that re-enters [0, n)
    return y;
  }
};

// ---------------------------------------------------------- sortable keys

// Order-preserving map float -> uint32 (total order for non-NaN floats).
__host__ __device__ __forceinline__ uint32_t float_key(float f) {
  uint32_t u;
#ifdef __CUDA_ARCH__
  u = __float_as_uint(f);
#else
  __builtin_memcpy(&u, &f, 4);
#endif
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ __forceinline__ float key_float(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k;
  float f;
#ifdef __CUDA_ARCH__
  f = __uint_as_float(u);
#else
  __builtin_memcpy(&f, &u, 4);
#endif
  return f;
}
__host__ __device__ __forceinline__ uint64_t double_key(double v) {
  uint64_t u;
#ifdef __CUDA_ARCH__
  u = (uint64_t)__double_as_longlong(v);
#else
  __builtin_memcpy(&u, &v, 8);
#endif
  return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

// (distance, index) pair as one 64-bit key: the uint64 order is the
// lexicographic (distance, index) order.  Empty = all ones.
constexpr uint64_t kEmpty = ~0ull;
__device__ __forceinline__ uint64_t pack(float d, uint32_t i) {
  return ((uint64_t)float_key(d) << 32) | i;
}
__device__ __forceinline__ float key_dist(uint64_t k) { return key_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ uint32_t key_index(uint64_t k) { return (uint32_t)k; }

// ------------------------------------------------------------ warp utils

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
  return __shfl_sync(0xffffffffu, v, src);
}
__device__ __forceinline__ uint64_t shfl_xor64(uint64_t v, int m) {
  return __shfl_xor_sync(0xffffffffu, v, m);
}

// Bitonic sort of one uint64 per lane, ascending across lanes 0..31.
__device__ __forceinline__ uint64_t warp_sort_asc(uint64_t v) {
  const int lane = lane_id();
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      uint64_t o = shfl_xor64(v, stride);
      bool up = ((lane & size) == 0);
      bool lower = ((lane & stride) == 0);
      bool take_min = (up == lower);
      v = take_min ? (o < v ? o : v) : (o > v ? o : v);
    }
  }
  return v;
}

__device__ __forceinline__ uint64_t warp_min64(uint64_t v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    uint64_t o = shfl_xor64(v, m);
    v = o < v ? o : v;
  }
  return v;
}

// Sorted list of KP (distance, index) keys spread over a warp: element
// g = r * 32 + lane lives in register r of lane `lane`, ascending in g.
template <int KP>
struct WarpList {
  static constexpr int R = KP / 32;
  uint64_t v[R];

  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = kEmpty;
  }
  // largest kept key (the admission threshold)
  __device__ __forceinline__ uint64_t worst() const { return shfl64(v[R - 1], 31); }
  // Insert key x (warp-uniform) keeping the KP smallest; duplicates of a
  // kept key are ignored.
  __device__ __forceinline__ void insert(uint64_t x) {
    const int lane = lane_id();
    uint64_t up[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      uint64_t a = __shfl_up_sync(0xffffffffu, v[r], 1);
      uint64_t b = (r > 0) ? shfl64(v[r > 0 ? r - 1 : 0], 31) : kEmpty;
      up[r] = (lane == 0) ? b : a;
    }
    bool dup = false;
#pragma unroll
    for (int r = 0; r < R; ++r) dup |= (v[r] == x);
    if (__any_sync(0xffffffffu, dup)) return;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      // element g keeps v if v < x; takes x if it is the first >= x; else shifts
      bool keep = v[r] < x;
      bool prev_less = (up[r] < x) || (r == 0 && lane == 0);
      if (r == 0 && lane == 0) prev_less = true;
      if (!keep) v[r] = prev_less ? x : up[r];
    }
  }
};

}  // namespace henn
