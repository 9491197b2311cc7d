// layers.cu -- eps-net layer construction (Alg. 1 membership, Alg. 2).
//
//  * draws: ceil(s/2^m) samples with replacement of the previous layer's
//    positions (Alg. 2; App. D parallel sampling: one thread per draw)
//  * compaction: the distinct positions in ascending order (= the new
//    layer, and its down pointers into the previous layer)
//  * IsEpsNet with r sampled ring ranges (App. B practical implementation):
//    FP32 distances from each ring centre to every point of the previous
//    layer, radix selection of the ring's two boundary order statistics,
//    and a certified decision per ring; a ring whose FP32 decision is not
//    certain is re-decided with FP64 distances computed operation by
//    operation in the same order as an FP64 reference (no FMA contraction).
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.cuh"

namespace henn {

// ---------------------------------------------------------------- draws

__global__ void k_sample_draws(uint64_t base, uint64_t s, int64_t t, uint8_t* __restrict__ flags) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < t;
       j += (int64_t)gridDim.x * blockDim.x) {
    flags[bounded(derive(base, (uint64_t)j), s)] = 1;
  }
}

// ------------------------------------------------------------ compaction

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;  // items per thread: 4096 per block
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t s = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kScanThreads / 32) warp_sums[lane] = s;
  }
  __syncthreads();
  int64_t before = (w > 0 ? warp_sums[w - 1] : 0) + x - v;
  if (total) *total = warp_sums[kScanThreads / 32 - 1];
  __syncthreads();
  return before;
}

// per-tile count of nonzero flags
__global__ void k_count_flags(const uint8_t* __restrict__ flags, int64_t s, int64_t* __restrict__ tile_counts) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t c = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int64_t p = base + (int64_t)threadIdx.x * kScanItems + i;
    if (p < s) c += flags[p] != 0;
  }
  int64_t total;
  block_exclusive_scan<int64_t>(c, &total);
  if (threadIdx.x == 0) tile_counts[blockIdx.x] = total;
}

// exclusive scan of an int64 array in one block (tiles <= a few thousand)
__global__ void k_scan_small(int64_t* __restrict__ a, int64_t count, int64_t* __restrict__ total) {
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < count; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < count ? a[i] : 0;
    int64_t chunk;
    int64_t ex = block_exclusive_scan<int64_t>(v, &chunk);
    if (i < count) a[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += chunk;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// write ascending positions of set flags; out_ids[j] = prev_ids[pos] (or pos)
__global__ void k_write_positions(const uint8_t* __restrict__ flags, int64_t s,
                                  const int64_t* __restrict__ tile_offsets,
                                  const int32_t* __restrict__ prev_ids, int32_t* __restrict__ out_pos,
                                  int32_t* __restrict__ out_ids) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t c = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int64_t p = base + i;
    if (p < s) c += flags[p] != 0;
  }
  int64_t at = tile_offsets[blockIdx.x] + block_exclusive_scan<int64_t>(c, nullptr);
  for (int i = 0; i < kScanItems; ++i) {
    int64_t p = base + i;
    if (p < s && flags[p]) {
      out_pos[at] = (int32_t)p;
      out_ids[at] = prev_ids ? prev_ids[p] : (int32_t)p;
      ++at;
    }
  }
}

// generic exclusive scan of int32 counts into int64 offsets (same tiling)
__global__ void k_count_ints(const int32_t* __restrict__ v, int64_t s, int64_t* __restrict__ tile_sums) {
  int64_t base = (int64_t)blockIdx.x * kScanTile;
  int64_t c = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int64_t p = base + (int64_t)threadIdx.x * kScanItems + i;
    if (p < s) c += v[p];
  }
  int64_t total;
  block_exclusive_scan<int64_t>(c, &total);
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

__global__ void k_write_offsets(const int32_t* __restrict__ v, int64_t s,
                                const int64_t* __restrict__ tile_offsets, int64_t* __restrict__ out) {
  int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t c = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int64_t p = base + i;
    if (p < s) c += v[p];
  }
  int64_t at = tile_offsets[blockIdx.x] + block_exclusive_scan<int64_t>(c, nullptr);
  for (int i = 0; i < kScanItems; ++i) {
    int64_t p = base + i;
    if (p < s) {
      out[p] = at;
      at += v[p];
    }
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == kScanThreads - 1) out[s] = at;
}

void launch_sample(const LayerSampleArgs& a, cudaStream_t st) {
  int grid = (int)((a.t + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  if (grid < 1) grid = 1;
  k_sample_draws<<<grid, 256, 0, st>>>(a.base, (uint64_t)a.s, a.t, a.flags);
}

void launch_compact(const uint8_t* flags, int64_t s, const int32_t* prev_ids, int64_t* tile_buf,
                    int64_t* d_total, int32_t* out_pos, int32_t* out_ids, cudaStream_t st) {
  int tiles = (int)((s + kScanTile - 1) / kScanTile);
  k_count_flags<<<tiles, kScanThreads, 0, st>>>(flags, s, tile_buf);
  k_scan_small<<<1, kScanThreads, 0, st>>>(tile_buf, tiles, d_total);
  k_write_positions<<<tiles, kScanThreads, 0, st>>>(flags, s, tile_buf, prev_ids, out_pos, out_ids);
}

int64_t scan_tiles(int64_t s) { return (s + kScanTile - 1) / kScanTile; }

void launch_offsets(const int32_t* counts, int64_t s, int64_t* tile_buf, int64_t* out_offsets,
                    cudaStream_t st) {
  int tiles = (int)((s + kScanTile - 1) / kScanTile);
  if (tiles < 1) tiles = 1;
  k_count_ints<<<tiles, kScanThreads, 0, st>>>(counts, s, tile_buf);
  k_scan_small<<<1, kScanThreads, 0, st>>>(tile_buf, tiles, nullptr);
  k_write_offsets<<<tiles, kScanThreads, 0, st>>>(counts, s, tile_buf, out_offsets);
}

// ------------------------------------------------------ halving (Alg. 3)

// One halving step of BuildEpsNetDiscV2: the current list (in, c entries;
// nullptr = positions 0..c-1) is matched in consecutive pairs, pair j keeps
// in[2j + coin], coin = bounded(derive(base, j), 2); an unmatched last entry
// is kept.  out[j] for j < ceil(c / 2).
__global__ void k_halve_step(const int32_t* __restrict__ in, int64_t c, uint64_t base, int32_t* __restrict__ out) {
  const int64_t half = (c + 1) / 2;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < half; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pick = 2 * j + 1 < c ? 2 * j + (int64_t)bounded(derive(base, (uint64_t)j), 2) : 2 * j;
    out[j] = in ? in[pick] : (int32_t)pick;
  }
}

__global__ void k_positions_to_ids(const int32_t* __restrict__ pos, int64_t cnt, const int32_t* __restrict__ prev_ids,
                                   int32_t* __restrict__ ids) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < cnt; j += (int64_t)gridDim.x * blockDim.x)
    ids[j] = prev_ids ? prev_ids[pos[j]] : pos[j];
}

int64_t launch_halving(uint64_t seed, int32_t layer, int64_t s, int32_t m, const int32_t* prev_ids, int32_t* tmp,
                       int32_t* pos, int32_t* ids, cudaStream_t st) {
  // ping-pong so that the last step lands in pos
  int64_t c = s;
  const int32_t* in = nullptr;
  for (int32_t step = 0; step < m; ++step) {
    int32_t* out = ((m - 1 - step) & 1) ? tmp : pos;
    const uint64_t base = derive(derive(derive(seed, HENN_TAG_HALVE), (uint64_t)layer), (uint64_t)step);
    const int64_t half = (c + 1) / 2;
    int grid = (int)((half + 255) / 256);
    if (grid > 152 * 16) grid = 152 * 16;
    if (grid < 1) grid = 1;
    k_halve_step<<<grid, 256, 0, st>>>(in, c, base, out);
    in = out;
    c = half;
  }
  int grid = (int)((c + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  if (grid < 1) grid = 1;
  k_positions_to_ids<<<grid, 256, 0, st>>>(pos, c, prev_ids, ids);
  return c;
}

// ---------------------------------------------------------- ring ranges

__global__ void k_ring_params(uint64_t bc, uint64_t bs, int32_t r, uint64_t s, uint64_t span,
                              int32_t* __restrict__ centre, int64_t* __restrict__ start) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < r) {
    centre[q] = (int32_t)bounded(derive(bc, (uint64_t)q), s);
    start[q] = (int64_t)bounded(derive(bs, (uint64_t)q), span);
  }
}

// FP32 distance from ring centres to the points of the previous layer.
// One warp per point; each lane holds dpad/32 coordinates (zero padded);
// the centres of the current chunk sit in shared memory.  L2: sum of
// squared differences; angular: 1 - <c,x> * inv|c| * inv|x|.
__global__ void k_ring_dist(const float* __restrict__ x32, int32_t dpad, const int32_t* __restrict__ prev_ids,
                            int64_t s, const int32_t* __restrict__ centre, int32_t r0, int32_t rc,
                            int32_t metric, const float* __restrict__ inv_norm, float* __restrict__ D) {
  extern __shared__ float sc[];  // rc * dpad
  for (int i = threadIdx.x; i < rc * dpad; i += blockDim.x) {
    int q = i / dpad, k = i % dpad;
    int64_t g = prev_ids ? prev_ids[centre[r0 + q]] : centre[r0 + q];
    sc[i] = x32[g * dpad + k];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const int warps = blockDim.x >> 5;
  for (int64_t x = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); x < s; x += (int64_t)gridDim.x * warps) {
    int64_t g = prev_ids ? prev_ids[x] : x;
    const float* row = x32 + g * dpad;
    float v[kMaxDimPerLane];
    int per = dpad / 32;
#pragma unroll
    for (int t = 0; t < kMaxDimPerLane; ++t) v[t] = t < per ? row[t * 32 + lane] : 0.f;
    float invx = metric == HENN_ANGULAR ? inv_norm[g] : 0.f;
    for (int q = 0; q < rc; ++q) {
      const float* c = sc + q * dpad;
      float acc = 0.f;
      if (metric == HENN_ANGULAR) {
#pragma unroll
        for (int t = 0; t < kMaxDimPerLane; ++t)
          if (t < per) acc = fmaf(v[t], c[t * 32 + lane], acc);
      } else {
#pragma unroll
        for (int t = 0; t < kMaxDimPerLane; ++t)
          if (t < per) {
            float df = v[t] - c[t * 32 + lane];
            acc = fmaf(df, df, acc);
          }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        float out = acc;
        if (metric == HENN_ANGULAR) {
          int64_t gc = prev_ids ? prev_ids[centre[r0 + q]] : centre[r0 + q];
          out = 1.f - acc * inv_norm[gc] * invx;
        }
        D[(int64_t)(r0 + q) * s + x] = out;
      }
    }
  }
}

// Radix selection of two order statistics (ranks k0 <= k1) of one row of
// keys, 8 bits per pass, one block per row.
template <typename K, int PASSES>
__device__ void block_select2(const K* __restrict__ keys_or_null, const float* __restrict__ fvals,
                              const double* __restrict__ dvals, int64_t s, int64_t k0, int64_t k1,
                              K* out0, K* out1) {
  __shared__ unsigned int hist[2][256];
  __shared__ K prefix[2];
  __shared__ int64_t rank[2];
  if (threadIdx.x == 0) {
    prefix[0] = prefix[1] = 0;
    rank[0] = k0;
    rank[1] = k1;
  }
  __syncthreads();
  for (int pass = 0; pass < PASSES; ++pass) {
    const int shift = (PASSES - 1 - pass) * 8;
    for (int i = threadIdx.x; i < 512; i += blockDim.x) (&hist[0][0])[i] = 0;
    __syncthreads();
    const K p0 = prefix[0], p1 = prefix[1];
    const K hmask = (shift + 8 >= (int)(sizeof(K) * 8)) ? (K)0 : (~(K)0) << (shift + 8);
    for (int64_t i = threadIdx.x; i < s; i += blockDim.x) {
      K key;
      if (sizeof(K) == 4)
        key = (K)float_key(fvals[i]);
      else
        key = (K)double_key(dvals[i]);
      unsigned b = (unsigned)((key >> shift) & 0xFF);
      if ((key & hmask) == p0) atomicAdd(&hist[0][b], 1u);
      if ((key & hmask) == p1) atomicAdd(&hist[1][b], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      int w = threadIdx.x;
      int64_t rem = rank[w];
      int b = 0;
      for (; b < 256; ++b) {
        if (rem < (int64_t)hist[w][b]) break;
        rem -= hist[w][b];
      }
      if (b > 255) b = 255;  // unreachable for 0 <= rank < s
      prefix[w] |= ((K)b) << shift;
      rank[w] = rem;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out0 = prefix[0];
    *out1 = prefix[1];
  }
}

__global__ void k_ring_select32(const float* __restrict__ D, int64_t s, const int64_t* __restrict__ start,
                                int64_t w, float* __restrict__ lo, float* __restrict__ hi) {
  const int q = blockIdx.x;
  uint32_t a, b;
  block_select2<uint32_t, 4>(nullptr, D + (int64_t)q * s, nullptr, s, start[q], start[q] + w - 1, &a, &b);
  if (threadIdx.x == 0) {
    lo[q] = key_float(a);
    hi[q] = key_float(b);
  }
}

// Certified FP32 decision.  With |v32 - v64| <= eta_rel*|v64| + eta_abs for
// every point, f(v) = v(1+er)+ea and g(v) = v(1-er)-ea bound v32 from both
// sides; f and g are increasing, so the order statistics obey the same
// bounds.  A candidate is surely inside when its lowest possible FP64 value
// is >= the highest possible lower end and its highest possible value is <=
// the lowest possible upper end; surely outside when it misses the widest
// possible interval.  Everything else is ambiguous.
__device__ __forceinline__ double finv(double y, double er, double ea) { return (y - ea) / (1.0 + er); }
__device__ __forceinline__ double ginv(double y, double er, double ea) { return (y + ea) / (1.0 - er); }

__global__ void k_ring_decide(const float* __restrict__ D, int64_t s, const int32_t* __restrict__ net_pos,
                              const int64_t* __restrict__ nnet_ptr, const float* __restrict__ lo,
                              const float* __restrict__ hi, double er, double ea, int32_t* __restrict__ status) {
  const int q = blockIdx.x;
  const int64_t nnet = *nnet_ptr;  // written by the compaction on the device
  __shared__ int any_in, any_amb;
  if (threadIdx.x == 0) any_in = any_amb = 0;
  __syncthreads();
  const double l = lo[q], h = hi[q];
  const double l_hi = ginv(l, er, ea), l_lo = finv(l, er, ea);
  const double h_hi = ginv(h, er, ea), h_lo = finv(h, er, ea);
  int in = 0, amb = 0;
  for (int64_t j = threadIdx.x; j < nnet; j += blockDim.x) {
    double v = D[(int64_t)q * s + net_pos[j]];
    double v_lo = finv(v, er, ea), v_hi = ginv(v, er, ea);
    if (v_lo >= l_hi && v_hi <= h_lo)
      in = 1;
    else if (!(v_hi < l_lo || v_lo > h_hi))
      amb = 1;
  }
  if (in) atomicOr(&any_in, 1);
  if (amb) atomicOr(&any_amb, 1);
  __syncthreads();
  if (threadIdx.x == 0) status[q] = any_in ? kRingPass : (any_amb ? kRingAmbiguous : kRingFail);
}

// ---------------------------------------------------- FP64 re-decision

// Same operation sequence as the FP64 reference: per coordinate one
// subtraction, one multiplication, one addition, in index order, every
// operation rounded to nearest (explicit intrinsics: no FMA contraction).
__device__ double dist64(const float* __restrict__ a, const float* __restrict__ b, int d, int metric) {
  if (metric == HENN_ANGULAR) {
    double ab = 0.0, aa = 0.0, bb = 0.0;
    for (int k = 0; k < d; ++k) {
      double x = (double)a[k], y = (double)b[k];
      ab = __dadd_rn(ab, __dmul_rn(x, y));
      aa = __dadd_rn(aa, __dmul_rn(x, x));
      bb = __dadd_rn(bb, __dmul_rn(y, y));
    }
    return __dsub_rn(1.0, __ddiv_rn(ab, __dmul_rn(__dsqrt_rn(aa), __dsqrt_rn(bb))));
  }
  double acc = 0.0;
  for (int k = 0; k < d; ++k) {
    double t = __dsub_rn((double)a[k], (double)b[k]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

__global__ void k_ring_dist64(const float* __restrict__ x32, int32_t d, int32_t dpad,
                              const int32_t* __restrict__ prev_ids, int64_t s, int64_t centre_pos,
                              int32_t metric, double* __restrict__ D64) {
  int64_t gc = prev_ids ? prev_ids[centre_pos] : centre_pos;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < s; x += (int64_t)gridDim.x * blockDim.x) {
    int64_t g = prev_ids ? prev_ids[x] : x;
    D64[x] = dist64(x32 + gc * dpad, x32 + g * dpad, d, metric);
  }
}

__global__ void k_ring_select64(const double* __restrict__ D64, int64_t s, int64_t k0, int64_t k1,
                                double* __restrict__ out) {
  uint64_t a, b;
  block_select2<uint64_t, 8>(nullptr, nullptr, D64, s, k0, k1, &a, &b);
  if (threadIdx.x == 0) {
    uint64_t ua = (a & 0x8000000000000000ull) ? (a & 0x7FFFFFFFFFFFFFFFull) : ~a;
    uint64_t ub = (b & 0x8000000000000000ull) ? (b & 0x7FFFFFFFFFFFFFFFull) : ~b;
    out[0] = __longlong_as_double((long long)ua);
    out[1] = __longlong_as_double((long long)ub);
  }
}

__global__ void k_ring_decide64(const double* __restrict__ D64, const int32_t* __restrict__ net_pos,
                                int64_t nnet, const double* __restrict__ bounds, int32_t* __restrict__ status,
                                int32_t q) {
  __shared__ int any_in;
  if (threadIdx.x == 0) any_in = 0;
  __syncthreads();
  const double l = bounds[0], h = bounds[1];
  int in = 0;
  for (int64_t j = threadIdx.x; j < nnet; j += blockDim.x) {
    double v = D64[net_pos[j]];
    if (l <= v && v <= h) in = 1;
  }
  if (in) atomicOr(&any_in, 1);
  __syncthreads();
  if (threadIdx.x == 0) status[q] = any_in ? kRingPass : kRingFail;
}

void launch_ring_params(uint64_t bc, uint64_t bs, int32_t r, int64_t s, int64_t span, int32_t* centre,
                        int64_t* start, cudaStream_t st) {
  k_ring_params<<<(r + 127) / 128, 128, 0, st>>>(bc, bs, r, (uint64_t)s, (uint64_t)span, centre, start);
}

void launch_ring_dist(const float* x32, int32_t dpad, const int32_t* prev_ids, int64_t s,
                      const int32_t* centre, int32_t r, int32_t metric, const float* inv_norm, float* D,
                      cudaStream_t st) {
  int rc_max = (int)(40960 / (dpad * 4));
  if (rc_max < 1) rc_max = 1;
  for (int r0 = 0; r0 < r; r0 += rc_max) {
    int rc = r - r0 < rc_max ? r - r0 : rc_max;
    int64_t warps = (s + 0) / 1;
    int grid = (int)((warps + 7) / 8);
    if (grid > 152 * 8) grid = 152 * 8;
    if (grid < 1) grid = 1;
    k_ring_dist<<<grid, 256, (size_t)rc * dpad * 4, st>>>(x32, dpad, prev_ids, s, centre, r0, rc, metric,
                                                          inv_norm, D);
  }
}

void launch_ring_select_decide(const float* D, int64_t s, const int64_t* start, int64_t w, int32_t r,
                               const int32_t* net_pos, const int64_t* nnet_dev, double er, double ea, float* lo,
                               float* hi, int32_t* status, cudaStream_t st) {
  k_ring_select32<<<r, 512, 0, st>>>(D, s, start, w, lo, hi);
  k_ring_decide<<<r, 256, 0, st>>>(D, s, net_pos, nnet_dev, lo, hi, er, ea, status);
}

void launch_ring_recheck(const float* x32, int32_t d, int32_t dpad, const int32_t* prev_ids, int64_t s,
                         int64_t centre_pos, int64_t a0, int64_t w, int32_t metric, const int32_t* net_pos,
                         int64_t nnet, double* D64, double* bounds, int32_t* status, int32_t q,
                         cudaStream_t st) {
  int grid = (int)((s + 255) / 256);
  if (grid > 152 * 8) grid = 152 * 8;
  k_ring_dist64<<<grid, 256, 0, st>>>(x32, d, dpad, prev_ids, s, centre_pos, metric, D64);
  k_ring_select64<<<1, 1024, 0, st>>>(D64, s, a0, a0 + w - 1, bounds);
  k_ring_decide64<<<1, 256, 0, st>>>(D64, net_pos, nnet, bounds, status, q);
}

}  // namespace henn
