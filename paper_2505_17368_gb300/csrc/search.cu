// search.cu -- batched HENN query (Alg. 4 + layer-0 beam), one persistent
// launch per batch, one warp per query.
//
// Per query:
//   S1  entry = node bounded(derive(derive(seed, ENTR), key), |L_L|) of the
//       top layer (Alg. 4 starts from a random node of the root layer)
//   S2  layers L..1: GreedySearch of Alg. 4 (move to the closest
//       neighbour, ties by index, while strictly closer), or a beam of width
//       ef_upper, then down to the copy of the result in the layer below
//   S3  layer 0: best-first beam of width ef' = max(ef, k) (Sec. 2.2: a set
//       of candidates for k > 1).  The beam list W is kept sorted in shared
//       memory; "candidate set C" = the entries of W not yet expanded.  The
//       next node to expand is the first unexpanded entry of W; the search
//       ends when every entry of W is expanded.  This is the classic
//       two-queue loop: a candidate that fell out of W is farther than every
//       entry of W, so popping it would end that loop.
//   S4  BF16 / FP8 storage: exact FP32 distances for the best
//       rerank_mult * k entries, sorted by (distance, index).
// The visited set is a fixed-size open-addressing table in shared memory
// that may forget entries when full.  A forgotten node that is seen again
// is re-evaluated but cannot enter W twice: a candidate equal to an entry
// of W is dropped, and a node that is not in W any more is farther than the
// current worst entry (the worst entry only decreases), so it is rejected
// exactly as a visited node would be.  Results therefore equal those of an
// exact visited set.  On layers of at most 32 << hash_bits points the same
// shared memory holds an exact bitmap instead (one bit per point).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"
#include "search.cuh"

namespace henn {

// Occupancy / memory-parallelism trade-off of the search kernels: blocks
// of 4 warps guaranteed per SM (caps registers per thread at
// 65536 / (128 * min_blocks)) and 16-byte chunks in flight per lane.
#ifndef HENN_SEARCH_MIN_BLOCKS
#define HENN_SEARCH_MIN_BLOCKS 6
#endif
#ifndef HENN_SEARCH_CHUNKS_IN_FLIGHT
#define HENN_SEARCH_CHUNKS_IN_FLIGHT 4
#endif
// The beam's shared-memory pointers re-derived from the dynamic shared
// memory base (1) or used as passed (0).
#ifndef HENN_SEARCH_SMEM32
#define HENN_SEARCH_SMEM32 1
#endif


constexpr int kStageBytes = 32 * 8;     // per-warp staging of one neighbour list

// The kernels' dynamic shared memory (every extern __shared__ array names
// its start).  Pointers a non-inlined function re-derives from it (base +
// offset) are known to be shared-memory addresses: 32-bit, read and written
// without the generic-address translation.
extern __shared__ __align__(16) unsigned char dyn_smem[];
template <typename T>
__device__ __forceinline__ T* as_shared(T* p) {
#if HENN_SEARCH_SMEM32
  const size_t off = reinterpret_cast<const unsigned char*>(p) - dyn_smem;
  return reinterpret_cast<T*>(dyn_smem + off);
#else
  return p;
#endif
}

// A team of warps answering one query (team_size > 1): the leader warp runs
// the query; for the neighbour rows of each beam expansion it posts a job
// (the row ids) and every warp of the team computes the distances of rows
// rank, rank + T, ...  The team synchronises on its own named barrier.
struct alignas(16) TeamJob {
  int32_t ids[32];
  float dist[32];
  const void* vec;
  const float* scale;
  int64_t qi;     // the team's current query
  int32_t count;  // rows of this job
  int32_t cmd;    // 0: rows, 1: the query is done
};

struct Team {
  TeamJob* job;  // nullptr for a single warp
  int bar;       // named barrier of the team (1 + team index)
  int threads;   // 32 * size
  int size;      // warps per query
};

// A single warp's "team": nothing to pass.
struct Solo {};

__device__ __forceinline__ void team_sync(const Team& tm) {
  asm volatile("bar.sync %0, %1;" ::"r"(tm.bar), "r"(tm.threads) : "memory");
}
constexpr uint64_t kFlag = 1ull << 31;  // "expanded" bit inside the index word
constexpr uint64_t kKeyMask = ~kFlag;

// -------------------------------------------------- row distance engine

// (a0, a1) += (x0 - q0)^2, (x1 - q1)^2 with paired FP32 operations
// (sub / fma on f32x2, each element rounded as its scalar form).
__device__ __forceinline__ void sqdiff2(float x0, float x1, float q0, float q1, float& a0, float& a1) {
  asm("{\n\t.reg .b64 xx, qq, tt, aa;\n\t"
      "mov.b64 xx, {%2, %3};\n\t"
      "mov.b64 qq, {%4, %5};\n\t"
      "mov.b64 aa, {%0, %1};\n\t"
      "sub.rn.f32x2 tt, xx, qq;\n\t"
      "fma.rn.f32x2 aa, tt, tt, aa;\n\t"
      "mov.b64 {%0, %1}, aa;\n\t}"
      : "+f"(a0), "+f"(a1)
      : "f"(x0), "f"(x1), "f"(q0), "f"(q1));
}

// 16-byte chunk -> squared-difference partial sums (two accumulators, even
// and odd elements) against the query chunk q (16-byte aligned, shared
// memory).
template <typename VT>
struct Chunk;

template <>
struct Chunk<float> {
  static constexpr int kElems = 4;
  __device__ __forceinline__ static void acc(const uint4& raw, const float* q, float, float& a0, float& a1) {
    const float4 v = *reinterpret_cast<const float4*>(&raw);
    const float4 qv = *reinterpret_cast<const float4*>(q);
    sqdiff2(v.x, v.y, qv.x, qv.y, a0, a1);
    sqdiff2(v.z, v.w, qv.z, qv.w, a0, a1);
  }
  __device__ __forceinline__ static void to_float(const uint4& raw, float, float* out) {
    out[0] = __uint_as_float(raw.x);
    out[1] = __uint_as_float(raw.y);
    out[2] = __uint_as_float(raw.z);
    out[3] = __uint_as_float(raw.w);
  }
};

template <>
struct Chunk<__nv_bfloat16> {
  static constexpr int kElems = 8;
  __device__ __forceinline__ static void acc(const uint4& raw, const float* q, float, float& a0, float& a1) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
    const float4 q0 = *reinterpret_cast<const float4*>(q);
    const float4 q1 = *reinterpret_cast<const float4*>(q + 4);
    const float qq[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
    for (int i = 0; i < 4; ++i)
      sqdiff2(__uint_as_float(w[i] << 16), __uint_as_float(w[i] & 0xFFFF0000u), qq[2 * i], qq[2 * i + 1], a0, a1);
  }
  __device__ __forceinline__ static void to_float(const uint4& raw, float, float* out) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      out[2 * i] = __uint_as_float(w[i] << 16);
      out[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
  }
};

template <>
struct Chunk<__nv_fp8_e4m3> {
  static constexpr int kElems = 16;
  __device__ __forceinline__ static void acc(const uint4& raw, const float* q, float scale, float& a0, float& a1) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float4 qv = *reinterpret_cast<const float4*>(q + 4 * i);
      __half2_raw h0 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] & 0xFFFF), __NV_E4M3);
      __half2_raw h1 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] >> 16), __NV_E4M3);
      float2 f0 = __half22float2(*reinterpret_cast<__half2*>(&h0));
      float2 f1 = __half22float2(*reinterpret_cast<__half2*>(&h1));
      sqdiff2(f0.x * scale, f0.y * scale, qv.x, qv.y, a0, a1);
      sqdiff2(f1.x * scale, f1.y * scale, qv.z, qv.w, a0, a1);
    }
  }
  __device__ __forceinline__ static void to_float(const uint4& raw, float scale, float* out) {
    const uint32_t w[4] = {raw.x, raw.y, raw.z, raw.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      __half2_raw h0 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] & 0xFFFF), __NV_E4M3);
      __half2_raw h1 = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[i] >> 16), __NV_E4M3);
      float2 f0 = __half22float2(*reinterpret_cast<__half2*>(&h0));
      float2 f1 = __half22float2(*reinterpret_cast<__half2*>(&h1));
      out[4 * i] = f0.x * scale;
      out[4 * i + 1] = f0.y * scale;
      out[4 * i + 2] = f1.x * scale;
      out[4 * i + 3] = f1.y * scale;
    }
  }
};

// One 16-byte chunk of a row.  Rows are read once per query: they skip L1
// (no allocation there), which keeps the adjacency lines that the beam
// prefetches, and the lines of rows still in flight, resident.
__device__ __forceinline__ uint4 load_row_chunk(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// Distances from the query (in shared memory) to up to 32 rows whose ids
// are held one per lane in lanes 0..count-1.  G lanes cooperate on a row
// (16-byte chunks lane, lane+G, ...), 32/G rows per pass.  The loads of PB
// passes are all issued before any arithmetic, so one neighbour list costs
// one or two memory round trips instead of one per pass.  Returns, in lane
// j < count, the squared distance of row j.
template <typename VT, int G, int CPL>
__device__ __forceinline__ float rows_dist(const VT* __restrict__ vec, const float* __restrict__ scale, int64_t stride_bytes,
                                           int32_t my_id, int count, const float* __restrict__ qs, int nchunk) {
  const int lane = lane_id();
  constexpr int RP = 32 / G;
  constexpr int PB0 = HENN_SEARCH_CHUNKS_IN_FLIGHT / CPL;  // passes per batch
  constexpr int PB = PB0 < 1 ? 1 : (PB0 > 32 / RP ? 32 / RP : PB0);
  const int g = lane % G, slot_in_pass = lane / G;
  float mine = 0.f;
  const char* base = reinterpret_cast<const char*>(vec);
  for (int p0 = 0; p0 * RP < count; p0 += PB) {
    uint4 raw[PB][CPL];
    float sc[PB];
#pragma unroll
    for (int pb = 0; pb < PB; ++pb) {
      const int slot = (p0 + pb) * RP + slot_in_pass;
      const int32_t id = __shfl_sync(0xffffffffu, my_id, slot < count ? slot : 0);
      sc[pb] = 1.f;
      if (slot < count) {
        const uint4* row = reinterpret_cast<const uint4*>(base + (int64_t)id * stride_bytes);
        if (scale) sc[pb] = __ldg(scale + id);
#pragma unroll
        for (int t = 0; t < CPL; ++t) {
          const int c = g + t * G;
          if (c < nchunk) raw[pb][t] = load_row_chunk(row + c);
        }
      }
    }
#pragma unroll
    for (int pb = 0; pb < PB; ++pb) {
      const int slot = (p0 + pb) * RP + slot_in_pass;
      float a0 = 0.f, a1 = 0.f;
      if (slot < count) {
#pragma unroll
        for (int t = 0; t < CPL; ++t) {
          const int c = g + t * G;
          if (c < nchunk) Chunk<VT>::acc(raw[pb][t], qs + c * Chunk<VT>::kElems, sc[pb], a0, a1);
        }
      }
      float a = a0 + a1;
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      const float got = __shfl_sync(0xffffffffu, a, (lane % RP) * G);
      if (lane / RP == p0 + pb) mine = got;
    }
  }
  return mine;
}

// rows_dist shared by a team: the leader (all its lanes) posts the ids and
// takes rows 0, T, 2T, ...; the other warps take theirs in team_helper.
// Each row's distance is computed by the same lane arithmetic as in
// rows_dist alone, so the result does not depend on the team size.
template <typename VT, int G, int CPL>
__device__ __forceinline__ float team_rows(const Team& tm, const VT* __restrict__ vec, const float* __restrict__ scale,
                                           int64_t stride_bytes, int32_t my_id, int count,
                                           const float* __restrict__ qs, int nchunk) {
  const int lane = lane_id();
  TeamJob* job = tm.job;
  if (lane < count) job->ids[lane] = my_id;
  if (lane == 0) {
    job->vec = vec;
    job->scale = scale;
    job->count = count;
    job->cmd = 0;
  }
  __syncwarp();
  team_sync(tm);
  const int mine = (count + tm.size - 1) / tm.size;
  const int32_t id = lane < mine ? job->ids[lane * tm.size] : 0;
  const float d = rows_dist<VT, G, CPL>(vec, scale, stride_bytes, id, mine, qs, nchunk);
  if (lane < mine) job->dist[lane * tm.size] = d;
  team_sync(tm);
  return lane < count ? job->dist[lane] : 0.f;
}

// The other warps of a team: rows jobs until the leader ends the query.
template <typename VT, int G, int CPL>
__device__ __noinline__ void team_helper(const Team& tm, int rank, int64_t stride_bytes, int nchunk,
                                         const float* __restrict__ qs) {
  const int lane = lane_id();
  TeamJob* job = tm.job;
  for (;;) {
    team_sync(tm);
    if (job->cmd != 0) break;
    const int count = job->count;
    const int mine = (count - rank + tm.size - 1) / tm.size;  // rows rank, rank + T, ...
    const int32_t id = lane < mine ? job->ids[rank + lane * tm.size] : 0;
    const float d = rows_dist<VT, G, CPL>(static_cast<const VT*>(job->vec), job->scale, stride_bytes, id, mine, qs,
                                          nchunk);
    if (lane < mine) job->dist[rank + lane * tm.size] = d;
    team_sync(tm);
  }
}

// ------------------------------------------------------ visited table

__device__ __forceinline__ bool visit(int32_t* table, int HB, int32_t id, int& evictions) {
  const uint32_t mask = (1u << HB) - 1u;
  uint32_t h = ((uint32_t)id * 0x9E3779B1u) >> (32 - HB);
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const uint32_t s = (h + p) & mask;
    const int32_t old = atomicCAS(table + s, -1, id);  // lanes of one row never share an id
    if (old == -1) return true;
    if (old == id) return false;
  }
  table[h] = id;  // full neighbourhood: forget the resident entry
  ++evictions;
  return true;
}

// Layers of at most 32 << HB points: an exact visited bitmap in the
// table's space (one atomic OR per node, nothing forgotten).
__device__ __forceinline__ bool visit_bit(int32_t* table, int32_t id) {
  const unsigned bit = 1u << (id & 31);
  return (atomicOr(reinterpret_cast<unsigned*>(table) + (id >> 5), bit) & bit) == 0u;
}

// number of entries of sorted W[0..nw) (masked) strictly below key
__device__ __forceinline__ int lower_bound_w(const uint64_t* W, int nw, uint64_t key) {
  int lo = 0, hi = nw;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if ((W[mid] & kKeyMask) < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Best-first beam of width ef on one layer from `entry` (S3).  Leaves W
// sorted ascending (with expanded flags) and returns its length.
// nseed > 0: W[0..nseed) already holds sorted, unexpanded entries (the
// copies of the layer above's candidates) and `entry` is ignored.
// The layer comes as its arrays and size (not a reference to a descriptor,
// which would put a memory load before every adjacency-row address).
template <typename VT, int G, int CPL, typename TM>
__device__ __noinline__ int beam(const int32_t* __restrict__ adj, const void* vec_, const float* __restrict__ scale,
                                 int64_t size, int64_t stride, int nchunk, int32_t entry, int ef, uint64_t* W,
                                 int32_t* table, int HB, uint64_t* stage, const float* qs, int& evals_out,
                                 int& expansions_out, int& evictions_out, int nseed, const TM tm) {
  constexpr bool TEAM = std::is_same<TM, Team>::value;
  W = as_shared(W);
  table = as_shared(table);
  stage = as_shared(stage);
  qs = as_shared(qs);
  const int lane = lane_id();
  const unsigned below = (1u << lane) - 1u;  // lanes under this one
  int32_t* stage32 = reinterpret_cast<int32_t*>(stage);
  const VT* vec = reinterpret_cast<const VT*>(vec_);
  const bool bitmap = size <= ((int64_t)32 << HB);
  // the counters stay in registers here (the caller's live in its frame)
  int evals = 0, expansions = 0, evictions = evictions_out;
  auto mark = [&](int32_t id) { return bitmap ? visit_bit(table, id) : visit(table, HB, id, evictions); };
  const int words = bitmap ? (int)((size + 31) >> 5) : (1 << HB);
  for (int s = lane; s < words; s += 32) table[s] = bitmap ? 0 : -1;
  __syncwarp();
  int nw;
  if (nseed > 0) {
    nw = min(nseed, ef);
    // the seeds are distinct points: each lane marks its own
    for (int j = lane; j < nw; j += 32) mark((int32_t)key_index(W[j] & kKeyMask));
  } else {
    if (lane == 0) mark(entry);
    float d0 = rows_dist<VT, G, CPL>(vec, scale, stride, entry, 1, qs, nchunk);
    d0 = __shfl_sync(0xffffffffu, d0, 0);
    ++evals;
    if (lane == 0) W[0] = pack(d0, (uint32_t)entry);
    nw = 1;
  }
  __syncwarp();
  int first = 0;
  for (;;) {
    // next unexpanded entry (and the one after it, for the prefetch)
    int pos = -1, after = -1;
    for (int base = first; base < nw; base += 32) {
      int i = base + lane;
      bool un = i < nw && !(W[i] & kFlag);
      unsigned m = __ballot_sync(0xffffffffu, un);
      if (m) {
        pos = base + __ffs(m) - 1;
        m &= m - 1;
        if (m) after = base + __ffs(m) - 1;
        break;
      }
    }
    if (pos < 0) break;
    uint64_t e = W[pos];
    __syncwarp();
    if (lane == 0) W[pos] = e | kFlag;
    first = pos + 1;
    ++expansions;
    const int32_t c = (int32_t)key_index(e & kKeyMask);
    int32_t nb = adj[(int64_t)c * kMmax + lane];
    // the next unexpanded entry is the likely next expansion: pull its
    // adjacency line towards the SM while this one is processed (the exact
    // next node, known once the new candidates are sorted, measured no
    // faster: the extra work on the critical path outweighs the later hit)
    if (lane == 0 && after >= 0) {
      const int32_t* nxt = adj + (int64_t)key_index(W[after] & kKeyMask) * kMmax;
      asm volatile("prefetch.global.L1 [%0];" ::"l"(nxt));
    }
    __syncwarp();
    bool fresh = nb >= 0 && mark(nb);
    unsigned fm = __ballot_sync(0xffffffffu, fresh);
    int cnt = __popc(fm);
    if (cnt == 0) continue;
    // compact fresh ids into lanes 0..cnt-1 (lane j gets the j-th fresh one)
    if (fresh) stage32[__popc(fm & below)] = nb;
    __syncwarp();
    const int32_t packed_id = lane < cnt ? stage32[lane] : -1;
    float dn;
    if constexpr (TEAM)
      dn = team_rows<VT, G, CPL>(tm, vec, scale, stride, packed_id, cnt, qs, nchunk);
    else
      dn = rows_dist<VT, G, CPL>(vec, scale, stride, packed_id, cnt, qs, nchunk);
    evals += cnt;
    const uint64_t worst = nw < ef ? kEmpty : (W[nw - 1] & kKeyMask);
    uint64_t kk = lane < cnt ? pack(dn, (uint32_t)packed_id) : kEmpty;
    bool take = kk < worst;
    // a node can reach W twice only if the visited table forgot it
    if (__any_sync(0xffffffffu, evictions > 0) && take) {
      const int lb = lower_bound_w(W, nw, kk);
      if (lb < nw && (W[lb] & kKeyMask) == kk) take = false;
    }
    const unsigned cm = __ballot_sync(0xffffffffu, take);
    const int ccnt = __popc(cm);
    if (ccnt == 0) continue;
    if (nw <= 64) {
      // W in two chunks: one pass over the candidates (compacted, unsorted)
      // counts, for each entry of W, the candidates below it (its shift),
      // and for each candidate the candidates and the entries of W below it
      // (its position); then every moved entry and every candidate is
      // written once
      __syncwarp();
      if (take) stage[__popc(cm & below)] = kk;
      __syncwarp();
      const bool v0 = lane < nw, v1 = lane + 32 < nw;
      const uint64_t w0 = v0 ? W[lane] : kEmpty, w1 = v1 ? W[lane + 32] : kEmpty;
      const uint64_t m0 = w0 & kKeyMask, m1 = w1 & kKeyMask;
      const uint64_t cand = lane < ccnt ? stage[lane] : kEmpty;
      int cl0 = 0, cl1 = 0, rk = 0, lb = 0;
      for (int j = 0; j < ccnt; ++j) {
        const uint64_t cj = stage[j];
        const bool below0 = cj < m0, below1 = cj < m1;  // keys are distinct
        cl0 += below0;
        cl1 += below1;
        rk += cj < cand;
        const int nb = __popc(__ballot_sync(0xffffffffu, v0 && !below0)) +
                       __popc(__ballot_sync(0xffffffffu, v1 && !below1));
        if (lane == j) lb = nb;
      }
      const int cpos = lane < ccnt ? lb + rk : 0x7fffffff;
      const int p0 = __reduce_min_sync(0xffffffffu, cpos);
      __syncwarp();
      if (v0 && cl0 > 0 && lane + cl0 < ef) W[lane + cl0] = w0;
      if (v1 && cl1 > 0 && lane + 32 + cl1 < ef) W[lane + 32 + cl1] = w1;
      if (lane < ccnt && cpos < ef) W[cpos] = cand;
      __syncwarp();
      nw = min(ef, nw + ccnt);
      first = min(first, p0);
      continue;
    }
    // candidates, compacted, then sorted into stage[0..ccnt); lane j < ccnt
    // holds the j-th smallest and its position in the new W
    __syncwarp();
    if (take) stage[__popc(cm & below)] = kk;
    __syncwarp();
    uint64_t cand = lane < ccnt ? stage[lane] : kEmpty;
    int rank = 0;
    for (int j = 0; j < ccnt; ++j) rank += stage[j] < cand;
    __syncwarp();
    if (lane < ccnt) stage[rank] = cand;
    __syncwarp();
    cand = lane < ccnt ? stage[lane] : kEmpty;
    const int cpos = lane < ccnt ? lower_bound_w(W, nw, cand) + lane : 0x7fffffff;
    const int p0 = __shfl_sync(0xffffffffu, cpos, 0);
    // entries at or after p0 shift right by the number of smaller candidates
    for (int base = ((nw - 1) >> 5) << 5; base >= (p0 & ~31); base -= 32) {
      const int i = base + lane;
      const bool mv = i < nw && i >= p0;
      const uint64_t w = mv ? W[i] : kEmpty;
      int cl = 0;
      for (int j = 0; j < ccnt; ++j) cl += stage[j] < (w & kKeyMask);
      __syncwarp();
      if (mv && i + cl < ef) W[i + cl] = w;
      __syncwarp();
    }
    if (lane < ccnt && cpos < ef) W[cpos] = cand;
    __syncwarp();
    nw = min(ef, nw + ccnt);
    first = min(first, p0);
  }
  evals_out += evals;
  expansions_out += expansions;
  evictions_out = evictions;
  return nw;
}

// The exact candidate set of an upper layer for exact_method 1 / 2: the
// keys (traversal distance, layer position) of its 32 nearest points,
// ascending, one per lane (kEmpty past the layer's size).  Method 1 starts
// from the query's 32 tile candidates, rescored here: a point outside them
// has a tile distance >= thr (the 32nd candidate's, rounded down to its
// 16-bit key's bucket by the selection), so a true distance >=
// thr - beta, beta bounding the tile error for this query; if that exceeds
// the need-th rescored distance (widened for its own rounding), no outside
// point belongs to the first `need` keys.  Otherwise, and for method 2,
// every point of the layer is evaluated into a running top 32 (warp
// bitonic merge of each sorted batch of 32).
template <typename VT, int G, int CPL>
__device__ __noinline__ uint64_t exact_top32(const SearchArgs& a, const void* vec_, const float* __restrict__ scale,
                                             int64_t size, int64_t stride, int nchunk, const float* qs,
                                             const uint64_t* pre_row, float pre_qn, int need, int& evals) {
  qs = as_shared(qs);
  const int lane = lane_id();
  const VT* vec = reinterpret_cast<const VT*>(vec_);
  const int s = (int)size;
  if (pre_row && *a.pre_err == 0) {
    const uint64_t tk = pre_row[lane];
    const int cnt = __popc(__ballot_sync(0xffffffffu, tk != kEmpty));
    const int32_t id = tk != kEmpty ? (int32_t)key_index(tk) : 0;
    const float dn = rows_dist<VT, G, CPL>(vec, scale, stride, id, cnt, qs, nchunk);
    evals += cnt;
    const uint64_t mine = warp_sort_asc(lane < cnt ? pack(dn, (uint32_t)id) : kEmpty);
    bool ok = cnt == s;  // the candidates are the whole layer
    if (!ok && cnt == 32) {
      const double thr = (double)key_dist(shfl64(tk, 31));
      const double dw = (double)key_dist(shfl64(mine, need - 1));
      // rounding of the rescored distances (FMA chains of <= dpad / 16
      // steps per accumulator, pairing and butterfly), doubled
      const double slack = (double)(a.dpad / 16 + 16) * 0x1p-23;
      // points that can come within dw of the query lie within sqrt(dw)
      // of it: their centred norm is capped by (|q| + sqrt(dw))^2
      const double nr = (double)pre_qn;
      const double rad = sqrt(nr) * (1.0 + 1e-3) + sqrt(dw * (1.0 + 2.0 * slack)) * (1.0 + 1e-3);
      const double nc = fmin((double)*a.pre_nmax, rad * rad);
      const double beta = a.pre_tile_u * 4.0 * (nr + nc) + 1e-30;
      ok = thr - beta > dw * (1.0 + slack);
    }
    if (ok) return mine;
    if (lane == 0 && a.pre_scans) atomicAdd(a.pre_scans, 1);
  }
  uint64_t mine = kEmpty;
  for (int c0 = 0; c0 < s; c0 += 32) {
    const int cnt = min(32, s - c0);
    const float dn = rows_dist<VT, G, CPL>(vec, scale, stride, c0 + lane, cnt, qs, nchunk);
    uint64_t kk = lane < cnt ? pack(dn, (uint32_t)(c0 + lane)) : kEmpty;
    if (!__any_sync(0xffffffffu, kk < shfl64(mine, 31))) continue;
    // the running list and the reversed sorted batch: their element-wise
    // minimum holds the 32 smallest as a bitonic sequence
    kk = shfl64(warp_sort_asc(kk), 31 - lane);
    uint64_t r = mine < kk ? mine : kk;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
      const uint64_t o = shfl_xor64(r, j);
      r = (lane & j) == 0 ? (o < r ? o : r) : (o > r ? o : r);
    }
    mine = r;
  }
  evals += s;
  return mine;
}

// ------------------------------------------------------- the kernel

// G lanes per row (8 for rows of <= 32 chunks of 16 bytes, else 32) and
// CPL chunks per lane, for the traversal rows (VT) and the FP32 rows.
template <typename VT, int DMAX>
struct RowShape {
  static constexpr int kChunks = DMAX * (int)sizeof(VT) / 16;
  static constexpr int G = kChunks <= 32 ? 8 : 32;
  static constexpr int CPL = (kChunks + G - 1) / G;
};

// S4 + output: exact FP32 rerank of the best rerank_mult * k entries
// (BF16 / FP8 storage), then the first k of W in (distance, index) order.
template <int G32, int CPL32>
__device__ __noinline__ void finish_query(const SearchArgs& a, uint64_t* W, int nw, int k, const float* qs,
                                          int64_t* out_ids, float* out_d) {
  W = as_shared(W);
  qs = as_shared(qs);
  const int lane = lane_id();
  const int dpad = a.dpad;
  const int out_k = min(k, a.out_stride);
  if (a.dead) {
    // deleted points carried the walk but leave the list (order kept)
    int live = 0;
    for (int base = 0; base < nw; base += 32) {
      const int i = base + lane;
      const uint64_t e = i < nw ? W[i] : kEmpty;
      const bool keep = i < nw && !a.dead[key_index(e & kKeyMask)];
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      __syncwarp();
      if (keep) W[live + __popc(m & ((1u << lane) - 1u))] = e;
      __syncwarp();
      live += __popc(m);
    }
    nw = live;
  }
  if (a.rerank && nw > 0) {
    int R = min(nw, max(k, a.rerank_mult * k));
    // exact FP32 distances for W[0..R), then sort in place
    for (int b = 0; b < R; b += 32) {
      int i = b + lane;
      int32_t id = i < R ? (int32_t)key_index(W[i] & kKeyMask) : 0;
      int cntb = min(32, R - b);
      float dx = rows_dist<float, G32, CPL32>(a.x32, nullptr, (int64_t)dpad * 4, id, cntb, qs, dpad / 4);
      __syncwarp();
      if (i < R) W[i] = pack(dx, (uint32_t)id);
      __syncwarp();
    }
    // bitonic sort of W[0..P), P = next pow2 >= R, padded with kEmpty
    int P = 1;
    while (P < R) P <<= 1;
    for (int i = R + lane; i < P; i += 32) W[i] = kEmpty;
    __syncwarp();
    for (int size = 2; size <= P; size <<= 1)
      for (int stride2 = size >> 1; stride2 > 0; stride2 >>= 1) {
        for (int i = lane; i < P; i += 32) {
          int j = i ^ stride2;
          if (j > i) {
            uint64_t x = W[i], y = W[j];
            bool up = (i & size) == 0;
            if ((x > y) == up) {
              W[i] = y;
              W[j] = x;
            }
          }
        }
        __syncwarp();
      }
    nw = R;
  }
  for (int j = lane; j < a.out_stride; j += 32) {
    bool ok = j < out_k && j < nw;
    uint64_t e = ok ? (W[j] & kKeyMask) : kEmpty;
    float dv = ok ? key_dist(e) : __int_as_float(0x7f800000);
    if (ok) dv = a.metric == HENN_ANGULAR ? 0.5f * dv : sqrtf(dv);
    out_ids[j] = ok ? (int64_t)key_index(e) : -1;
    out_d[j] = dv;
  }
}

// One query, one warp: S1-S4 for the query row `qg` (d floats), writing
// out_stride results to out_ids / out_d and 4 counters to stats (optional).
// `my` is this warp's shared-memory slice.
template <typename VT, int DMAX, typename TM>
__device__ __forceinline__ void run_query(const SearchArgs& a, unsigned char* my, const float* __restrict__ qg, int k,
                                          int ef, uint64_t key, int64_t* out_ids, float* out_d, int32_t* stats,
                                          const uint64_t* pre_row, float pre_qn, const TM tm) {
  constexpr int G = RowShape<VT, DMAX>::G, CPL = RowShape<VT, DMAX>::CPL;
  constexpr int G32 = RowShape<float, DMAX>::G, CPL32 = RowShape<float, DMAX>::CPL;
  const int lane = lane_id();
  const int dpad = a.dpad;
  const int EFCAP = a.ef_cap, HB = a.hash_bits;
  uint64_t* W = reinterpret_cast<uint64_t*>(my);
  int32_t* table = reinterpret_cast<int32_t*>(my + EFCAP * 8);
  uint64_t* stage = reinterpret_cast<uint64_t*>(my + EFCAP * 8 + (4 << HB));
  float* qs = reinterpret_cast<float*>(my + EFCAP * 8 + (4 << HB) + kStageBytes);
  const int64_t stride = (int64_t)dpad * sizeof(VT);
  const int nchunk = (int)(stride / 16);

  ef = max(ef, k);
  ef = min(ef, EFCAP);
  int evals = 0, expansions = 0, moves = 0, evictions = 0;

  // query into shared memory (normalised for the angular metric)
  {
    float ss = 0.f;
    for (int c = lane; c < dpad; c += 32) {
      float v = c < a.d ? __ldcg(qg + c) : 0.f;  // L2 read: serving rings are rewritten
      qs[c] = v;
      ss = fmaf(v, v, ss);
    }
    if (a.metric == HENN_ANGULAR) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      float inv = ss > 0.f ? __fdiv_rn(1.f, __fsqrt_rn(ss)) : 0.f;
      __syncwarp();
      for (int c = lane; c < dpad; c += 32) qs[c] *= inv;
    }
    __syncwarp();
  }

  // S1: random node of the top layer
  int32_t cur = (int32_t)bounded(derive(a.entry_key, key), (uint64_t)a.layers[a.L].size);
  // S2: upper layers: GreedySearch of Alg. 4, or a beam of width ef_upper
  int nseed = 0;
  // the lowest exact layer's set does not depend on the layers above it:
  // the walk starts there (exact_method 1 / 2 first, so that nothing of it
  // stays live across the beams)
  int li = a.top_exact;
  if (a.exact_method != 0) {
    const SearchLayer Ly = a.layers[li];
    const int width = (li == 1 && a.ef_l1 > 0) ? a.ef_l1 : a.ef_upper;
    // the host keeps width <= 32 when the candidates seed the next layer
    const bool seeds = a.descend_all && width > 1;
    const int nw = seeds ? min(min(width, 32), (int)Ly.size) : 1;
    const uint64_t mine = exact_top32<VT, G, CPL>(a, Ly.vec, Ly.scale, Ly.size, stride, nchunk, qs,
                                                  a.exact_method == 1 ? pre_row : nullptr, pre_qn, nw, evals);
    if (lane < nw) W[lane] = seeds ? ((mine & 0xFFFFFFFF00000000ull) | (uint32_t)Ly.down[key_index(mine)]) : mine;
    cur = Ly.down[key_index(shfl64(mine, 0))];
    if (seeds) nseed = nw;
    __syncwarp();
    --li;
  }
  for (; li >= 1; --li) {
    const SearchLayer Ly = a.layers[li];
    const int width = (li == 1 && a.ef_l1 > 0) ? a.ef_l1 : a.ef_upper;
    if (Ly.size <= a.exact_upper) {
      // a small layer: its exact candidate set, the nearest max(width, 1)
      // points by (distance, index), every point evaluated; the keys sit in
      // the visited table's space (the next walk clears it)
      const int s = (int)Ly.size;
      uint64_t* keys = reinterpret_cast<uint64_t*>(table);
      const VT* vec = reinterpret_cast<const VT*>(Ly.vec);
      for (int c0 = 0; c0 < s; c0 += 32) {
        const int cnt = min(32, s - c0);
        const float dn = rows_dist<VT, G, CPL>(vec, Ly.scale, stride, c0 + lane, cnt, qs, nchunk);
        if (lane < cnt) keys[c0 + lane] = pack(dn, (uint32_t)(c0 + lane));
      }
      evals += s;
      int P = 1;
      while (P < s) P <<= 1;
      for (int i = s + lane; i < P; i += 32) keys[i] = kEmpty;
      __syncwarp();
      for (int size = 2; size <= P; size <<= 1)
        for (int half = size >> 1; half > 0; half >>= 1) {
          for (int i = lane; i < P; i += 32) {
            const int j = i ^ half;
            if (j > i) {
              const uint64_t x = keys[i], y = keys[j];
              if ((x > y) == ((i & size) == 0)) {
                keys[i] = y;
                keys[j] = x;
              }
            }
          }
          __syncwarp();
        }
      const int nw = min(min(max(width, 1), EFCAP), s);
      for (int j = lane; j < nw; j += 32) W[j] = keys[j];
      __syncwarp();
      cur = (int32_t)key_index(W[0]);
      if (a.descend_all && width > 1) {
        for (int j = lane; j < nw; j += 32) {
          const uint64_t e = W[j];
          W[j] = (e & 0xFFFFFFFF00000000ull) | (uint32_t)Ly.down[key_index(e)];
        }
        nseed = nw;
      }
      __syncwarp();
    } else if (width > 1) {
      int ex = 0;
      int nw = beam<VT, G, CPL, TM>(Ly.adj, Ly.vec, Ly.scale, Ly.size, stride, nchunk, cur, min(width, EFCAP), W,
                                    table, HB, stage, qs, evals, ex, evictions, nseed, tm);
      moves += ex;
      cur = (int32_t)key_index(W[0] & kKeyMask);
      if (a.descend_all) {
        // the layer below is entered at the copies of every candidate;
        // down pointers are increasing, so the (distance, index) order holds
        for (int j = lane; j < nw; j += 32) {
          uint64_t e = W[j] & kKeyMask;
          W[j] = (e & 0xFFFFFFFF00000000ull) | (uint32_t)Ly.down[key_index(e)];
        }
        nseed = nw;
      }
      __syncwarp();
    } else {
      const VT* vec = reinterpret_cast<const VT*>(Ly.vec);
      float dc = rows_dist<VT, G, CPL>(vec, Ly.scale, stride, cur, 1, qs, nchunk);
      dc = __shfl_sync(0xffffffffu, dc, 0);
      ++evals;
      for (;;) {
        int32_t nb = Ly.adj[(int64_t)cur * kMmax + lane];
        unsigned valid = __ballot_sync(0xffffffffu, nb >= 0);
        int cnt = __popc(valid);
        // neighbours are packed at the front of each row (-1 padding after)
        float dn = rows_dist<VT, G, CPL>(vec, Ly.scale, stride, nb, cnt, qs, nchunk);
        evals += cnt;
        uint64_t kk = lane < cnt ? pack(dn, (uint32_t)nb) : kEmpty;
        uint64_t best = warp_min64(kk);
        if (best == kEmpty || !(key_dist(best) < dc)) break;
        cur = (int32_t)key_index(best);
        dc = key_dist(best);
        ++moves;
      }
    }
    cur = Ly.down[cur];
  }

  // S3: layer-0 beam
  const SearchLayer B = a.layers[0];
  int nw = beam<VT, G, CPL, TM>(B.adj, B.vec, B.scale, B.size, stride, nchunk, cur, ef, W, table, HB, stage, qs,
                                evals, expansions, evictions, nseed, tm);

  // S4 + output
  finish_query<G32, CPL32>(a, W, nw, k, qs, out_ids, out_d);
  if (stats && lane == 0) {
    stats[0] = evals;
    stats[1] = expansions;
    stats[2] = moves;
    stats[3] = evictions;
  }
  __syncwarp();
  if constexpr (std::is_same<TM, Team>::value) {
    // the query is done: release the team's other warps
    if (lane == 0) tm.job->cmd = 1;
    __syncwarp();
    team_sync(tm);
  }
}

// TM = Solo: one warp per query.  TM = Team: teams of a.team warps.
template <typename VT, int DMAX, typename TM>
__global__ void __launch_bounds__(128, HENN_SEARCH_MIN_BLOCKS) k_search(const __grid_constant__ SearchArgs a) {
  constexpr int G = RowShape<VT, DMAX>::G, CPL = RowShape<VT, DMAX>::CPL;
  constexpr bool TEAM = std::is_same<TM, Team>::value;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = lane_id();
  const int T = TEAM ? a.team : 1;
  const int warp = threadIdx.x >> 5, team = warp / T, rank = warp - team * T;
  unsigned char* my = smem + (size_t)team * a.warp_smem;
  TM tm;
  if constexpr (TEAM) {
    tm.size = T;
    tm.bar = 1 + team;
    tm.threads = 32 * T;
    tm.job = reinterpret_cast<TeamJob*>(my + a.warp_smem - sizeof(TeamJob));
  }
  for (;;) {
    int64_t qi = 0;
    if constexpr (!TEAM) {
      if (lane == 0) qi = atomicAdd(reinterpret_cast<unsigned long long*>(a.counter), 1ull);
      qi = (int64_t)__shfl_sync(0xffffffffu, (unsigned long long)qi, 0);
    } else {
      // the leader takes the team's next query; the others read it after
      // the barrier (the leader writes it again only after the query's end
      // barrier, which every warp of the team has reached by then)
      if (rank == 0 && lane == 0)
        tm.job->qi = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(a.counter), 1ull);
      team_sync(tm);
      qi = tm.job->qi;
    }
    if (qi >= a.nq) break;
    if constexpr (TEAM) {
      if (rank != 0) {
        const int64_t stride = (int64_t)a.dpad * sizeof(VT);
        const float* qs = reinterpret_cast<const float*>(my + a.ef_cap * 8 + (4 << a.hash_bits) + kStageBytes);
        team_helper<VT, G, CPL>(tm, rank, stride, (int)(stride / 16), qs);
        continue;
      }
    }
    if (a.order) qi = a.order[qi];
    const int k = a.kq ? a.kq[qi] : a.k_uniform;
    const int ef = a.efq ? a.efq[qi] : a.ef_uniform;
    const uint64_t key = a.keys ? a.keys[qi] : (uint64_t)qi;
    run_query<VT, DMAX>(a, my, a.Q + qi * a.d, k, ef, key, a.out_ids + qi * a.out_stride,
                        a.out_d + qi * a.out_stride, a.stats ? a.stats + qi * 4 : nullptr,
                        a.pre_keys ? a.pre_keys + qi * 32 : nullptr, a.pre_qnorm ? a.pre_qnorm[qi] : 0.f, tm);
  }
}

// ------------------------------------------------------ serving loop

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ long long ld_acquire_gpu(const long long* p) {
  long long v;
  asm volatile("ld.acquire.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Persistent serving kernel.  Work items (one per query) are numbered in
// arrival order; the host publishes a prefix by raising `published` (device
// memory, written by a copy after the item's query row and descriptor).  A
// warp takes the next item only if it is already published (CAS on
// `taken`), so no warp ever waits while holding an item.  With nothing to
// take, a warp polls with back-off until `stop` is raised or it has been
// idle for idle_ns, then leaves; the host relaunches the kernel when new
// items are published and it has ended.  A finished query bumps its
// request's counter in mapped host memory after a system-scope fence.
template <typename VT, int DMAX>
__global__ void __launch_bounds__(128, HENN_SEARCH_MIN_BLOCKS) k_serve(const __grid_constant__ ServeArgs s) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = lane_id();
  unsigned char* my = smem + (size_t)(threadIdx.x >> 5) * s.base.warp_smem;
  for (;;) {
    long long t = -1;
    if (lane == 0) {
      unsigned backoff = 256;
      for (long long spin = 0; spin < (1ll << 26); ++spin) {
        const long long p = ld_acquire_gpu(s.published);
        const unsigned long long tk = *reinterpret_cast<volatile unsigned long long*>(s.taken);
        if ((long long)tk < p) {
          if (atomicCAS(s.taken, tk, tk + 1ull) == tk) {
            t = (long long)tk;
            atomicMax(s.last_active, (unsigned long long)global_ns());
            break;
          }
          continue;
        }
        if (*reinterpret_cast<const volatile int*>(s.stop)) break;
        // leave only when the whole kernel has been without work for
        // idle_ns, so that all warps leave together and the host relaunches
        // a full grid next time
        unsigned long long last = *reinterpret_cast<volatile unsigned long long*>(s.last_active);
        if (last == ~0ull) {  // first look of a fresh launch: start its clock now
          atomicCAS(s.last_active, ~0ull, (unsigned long long)global_ns());
          continue;
        }
        if (global_ns() > last + (uint64_t)s.idle_ns) break;
        __nanosleep(backoff);
        if (backoff < 8192) backoff <<= 1;
      }
    }
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t < 0) break;
    const int64_t slot = t % s.cap;
    const int32_t req = __ldcg(&s.desc[slot].slot);
    const int32_t k = __ldcg(&s.desc[slot].k);
    const int32_t ef = __ldcg(&s.desc[slot].ef);
    const uint64_t key = __ldcg(&s.desc[slot].key);
    run_query<VT, DMAX>(s.base, my, s.qring + slot * s.base.d, k, ef, key, s.out_ids + slot * s.base.out_stride,
                        s.out_d + slot * s.base.out_stride, nullptr, nullptr, 0.f, Solo());
    __syncwarp();
    if (lane == 0) {
      __threadfence_system();
      atomicAdd_system(s.done + req, 1);
    }
  }
}

// ------------------------------------------------------ greedy probes

// GreedySearch of Alg. 4 on one layer from a given start node, one warp
// per (query, start): move to the closest neighbour (ties by index) while it
// is strictly closer.  The local minimum it ends at is what the recall
// bound rho_delta of Def. 3 ranks among the query's true neighbours.
template <typename VT, int DMAX>
__global__ void __launch_bounds__(128) k_greedy_probe(const __grid_constant__ GreedyProbeArgs a) {
  constexpr int G = RowShape<VT, DMAX>::G, CPL = RowShape<VT, DMAX>::CPL;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = lane_id();
  float* qs = reinterpret_cast<float*>(smem) + (threadIdx.x >> 5) * a.dpad;
  const int64_t stride = (int64_t)a.dpad * sizeof(VT);
  const int nchunk = (int)(stride / 16);
  const VT* vec = reinterpret_cast<const VT*>(a.layer.vec);
  const int64_t total = a.nq * a.S;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; p < total; p += warps) {
    const int64_t qi = p / a.S;
    const float* qg = a.Q + qi * a.d;
    float ss = 0.f;
    __syncwarp();
    for (int c = lane; c < a.dpad; c += 32) {
      const float v = c < a.d ? qg[c] : 0.f;
      qs[c] = v;
      ss = fmaf(v, v, ss);
    }
    if (a.metric == HENN_ANGULAR) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      const float inv = ss > 0.f ? __fdiv_rn(1.f, __fsqrt_rn(ss)) : 0.f;
      __syncwarp();
      for (int c = lane; c < a.dpad; c += 32) qs[c] *= inv;
    }
    __syncwarp();
    int32_t cur = a.starts[p];
    if (cur < 0 || cur >= a.layer.size) {
      if (lane == 0) {
        a.out_node[p] = -1;
        a.out_dist[p] = __int_as_float(0x7f800000);
        if (a.out_hops) a.out_hops[p] = 0;
      }
      continue;
    }
    float dc = rows_dist<VT, G, CPL>(vec, a.layer.scale, stride, cur, 1, qs, nchunk);
    dc = __shfl_sync(0xffffffffu, dc, 0);
    int32_t moves = 0;
    for (;;) {
      const int32_t nb = a.layer.adj[(int64_t)cur * kMmax + lane];
      const int cnt = __popc(__ballot_sync(0xffffffffu, nb >= 0));
      // neighbours are packed at the front of each row (-1 padding after)
      const float dn = rows_dist<VT, G, CPL>(vec, a.layer.scale, stride, nb, cnt, qs, nchunk);
      const uint64_t kk = lane < cnt ? pack(dn, (uint32_t)nb) : kEmpty;
      const uint64_t best = warp_min64(kk);
      if (best == kEmpty || !(key_dist(best) < dc)) break;
      cur = (int32_t)key_index(best);
      dc = key_dist(best);
      ++moves;
    }
    if (lane == 0) {
      a.out_node[p] = cur;
      a.out_dist[p] = dc;
      if (a.out_hops) a.out_hops[p] = moves;
    }
  }
}

template <typename VT, int DMAX>
static cudaError_t launch_probe_t(const GreedyProbeArgs& a, cudaStream_t st) {
  const int64_t warps_needed = a.nq * a.S;
  int64_t blocks = (warps_needed + 3) / 4;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_greedy_probe<VT, DMAX><<<(int)blocks, 128, (size_t)4 * a.dpad * sizeof(float), st>>>(a);
  return cudaGetLastError();
}

template <typename VT>
static cudaError_t launch_probe_vt(const GreedyProbeArgs& a, cudaStream_t st) {
  if (a.dpad <= 32) return launch_probe_t<VT, 32>(a, st);
  if (a.dpad <= 64) return launch_probe_t<VT, 64>(a, st);
  if (a.dpad <= 128) return launch_probe_t<VT, 128>(a, st);
  if (a.dpad <= 512) return launch_probe_t<VT, 512>(a, st);
  return launch_probe_t<VT, 1024>(a, st);
}

cudaError_t launch_greedy_probe(const GreedyProbeArgs& a, int storage, cudaStream_t st) {
  if (storage == HENN_BF16) return launch_probe_vt<__nv_bfloat16>(a, st);
  if (storage == HENN_FP8E4M3) return launch_probe_vt<__nv_fp8_e4m3>(a, st);
  return launch_probe_vt<float>(a, st);
}

// ------------------------------------------- exact-layer preparation

template <typename VT>
__global__ void k_layer_rows_f32(const VT* __restrict__ vec, const float* __restrict__ scale, int64_t s, int32_t dpad,
                                 float* __restrict__ out) {
  constexpr int E = Chunk<VT>::kElems;
  const int nchunk = dpad / E;
  const int64_t total = s * nchunk;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / nchunk;
    const int c = (int)(i - r * nchunk);
    const uint4 raw = reinterpret_cast<const uint4*>(vec + r * dpad)[c];
    float v[E];
    Chunk<VT>::to_float(raw, scale ? scale[r] : 1.f, v);
#pragma unroll
    for (int e = 0; e < E; ++e) out[r * dpad + c * E + e] = v[e];
  }
}

cudaError_t launch_layer_rows_f32(const void* vec, const float* scale, int64_t s, int storage, int32_t dpad, float* out,
                                  cudaStream_t st) {
  if (storage == HENN_BF16)
    k_layer_rows_f32<__nv_bfloat16><<<152 * 8, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(vec), scale, s, dpad,
                                                             out);
  else if (storage == HENN_FP8E4M3)
    k_layer_rows_f32<__nv_fp8_e4m3><<<152 * 8, 256, 0, st>>>(static_cast<const __nv_fp8_e4m3*>(vec), scale, s, dpad,
                                                             out);
  else
    k_layer_rows_f32<float><<<152 * 8, 256, 0, st>>>(static_cast<const float*>(vec), scale, s, dpad, out);
  return cudaGetLastError();
}

// One warp per query: the row exactly as run_query stages it (the angular
// normalisation in the same order), minus the layer's centre.  The row is
// read once into shared memory (16-byte loads where the rows allow: the
// rows may sit in page-locked host memory, read over the host link) and,
// with qraw, also written there as read (a device copy for the search
// kernel).
constexpr int kEntryMaxD = 1024;

__global__ void __launch_bounds__(256) k_entry_queries(const float* __restrict__ Q, int64_t nq, int32_t d,
                                                       int32_t dpad, int32_t metric, const float* __restrict__ mean,
                                                       float* __restrict__ xo, __nv_bfloat16* __restrict__ hi,
                                                       __nv_bfloat16* __restrict__ lo, int32_t dk,
                                                       float* __restrict__ norms, float* __restrict__ qraw) {
  __shared__ __align__(16) float rows[8][kEntryMaxD];
  const int lane = threadIdx.x & 31;
  float* r = rows[threadIdx.x >> 5];
  const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(Q) & 15) == 0) &&
                   (!qraw || (reinterpret_cast<uintptr_t>(qraw) & 15) == 0);
  for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < nq;
       q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const float* qg = Q + q * d;
    if (vec) {
      for (int c4 = lane; c4 < d / 4; c4 += 32) {
        const float4 v = __ldcs(reinterpret_cast<const float4*>(qg) + c4);
        reinterpret_cast<float4*>(r)[c4] = v;
        if (qraw) reinterpret_cast<float4*>(qraw + q * d)[c4] = v;
      }
    } else {
      for (int c = lane; c < d; c += 32) {
        const float v = __ldcs(qg + c);
        r[c] = v;
        if (qraw) qraw[q * d + c] = v;
      }
    }
    __syncwarp();
    float inv = 1.f;
    if (metric == HENN_ANGULAR) {
      float ss = 0.f;
      for (int c = lane; c < dpad; c += 32) {
        const float v = c < d ? r[c] : 0.f;
        ss = fmaf(v, v, ss);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
      inv = ss > 0.f ? __fdiv_rn(1.f, __fsqrt_rn(ss)) : 0.f;
    }
    float acc = 0.f;
    for (int c = lane; c < dk; c += 32) {
      float v = 0.f;
      if (c < dpad) {
        float x = c < d ? r[c] : 0.f;
        if (metric == HENN_ANGULAR) x *= inv;
        v = x - mean[c];
        acc = fmaf(v, v, acc);
        if (xo) xo[q * dpad + c] = v;
      }
      if (hi) {
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[q * dk + c] = h;
        lo[q * dk + c] = __float2bfloat16_rn(v - __bfloat162float(h));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) norms[q] = acc;
    __syncwarp();  // r is rewritten by the next query of this warp
  }
}

void launch_entry_queries(const float* Q, int64_t nq, int32_t d, int32_t dpad, int32_t metric, const float* mean,
                          float* xo, void* hi, void* lo, int32_t dk, float* norms, float* qraw, cudaStream_t st) {
  int64_t blocks = (nq + 7) / 8;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  k_entry_queries<<<(int)blocks, 256, 0, st>>>(Q, nq, d, dpad, metric, mean, xo, static_cast<__nv_bfloat16*>(hi),
                                               static_cast<__nv_bfloat16*>(lo), hi ? dk : dpad, norms, qraw);
}

// Bitonic sort of one float per lane across the warp, ascending.
__device__ __forceinline__ float warp_sort_asc_f32(float v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int size = 2; size <= 32; size <<= 1)
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const float o = __shfl_xor_sync(0xffffffffu, v, stride);
      const bool up = (lane & size) == 0;
      const bool lower = (lane & stride) == 0;
      v = (lower == up) ? fminf(v, o) : fmaxf(v, o);
    }
  return v;
}

// One warp per query: the 32 smallest (distance, column) keys of its row of
// a tile distance matrix (+inf entries never enter), ascending, one per
// lane.  The matrix holds 16-bit keys, each the distance rounded down to 8
// mantissa bits (its float bits 30..15); an entry's distance here is the
// lower end of its key's bucket (the key shifted back), so every column
// outside the 32 has a tile distance at or above the 32nd's.  The tile
// launch also wrote each row's minimum over every 32-column chunk (cmin,
// rows of ldc floats, the same rounding).  T = the 32nd smallest of those
// chunk minima bounds the row's 32nd smallest value (32 distinct columns lie
// at or below it), and a column at or below T lies in a chunk whose minimum
// is at or below T: only those chunks (32 of them, plus ties) are read, four
// 64-byte chunks at a time, and their entries <= T merged into the running
// list -- a few by shuffle insertion, many by sorting the batch and a
// bitonic merge.  The result is the row's 32 smallest keys, as a full scan
// would give; with `discard` each line read is dropped from L2 afterwards.
#ifndef HENN_SELECT_ONE_TRIP
#define HENN_SELECT_ONE_TRIP 1
#endif
constexpr int kSelChunks = 128;  // candidate chunks listed per row
constexpr int kSelKeys = 256;    // entries <= T staged per row

// the lower end of a 16-bit distance key's bucket
__device__ __forceinline__ float key16_dist(uint32_t k) { return __uint_as_float(k << 15); }

__global__ void __launch_bounds__(256) k_select_top32(const uint16_t* __restrict__ D, const float* __restrict__ cmin,
                                                      int64_t nq, int64_t s, int64_t ldo, int64_t ldc,
                                                      uint64_t* __restrict__ out, int32_t discard) {
#if HENN_SELECT_ONE_TRIP
  __shared__ int sel_chunks[8][kSelChunks];
  __shared__ uint64_t sel_keys[8][kSelKeys];
#endif
  const int lane = threadIdx.x & 31;
  const float kInf = __int_as_float(0x7f800000);
  const int nch = (int)(ldo / 32);
  for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < nq;
       q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const float* cm = cmin + q * ldc;
    // T = the 32nd smallest chunk minimum.  Rows of up to 128 chunks hold
    // the minima as keys (each minimum is the lower end of its key's
    // bucket, so the key is exact) and find T's key bit by bit from the top:
    // the largest key t with at most 31 minima below it.  Longer rows keep
    // the 32 smallest minima sorted across the warp.
    const bool few = nch <= 128;
    uint32_t mk[4];
    uint32_t pk = 0;  // T's key (few rows)
    float T;
    if (few) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = 32 * j + lane;
        mk[j] = c < nch ? (__float_as_uint(__ldg(cm + c)) >> 15) & 0xFFFFu : 0xFFFFu;
      }
      // fewer than 32 chunks: T = +inf (key 0xFF00; no minimum is NaN).
      // Else T's key lies between the smallest and the largest minimum, so
      // their common leading bits are its own and the search starts below
      uint32_t p = 0xFFFFu;
      if (nch >= 32) {
        uint32_t lo = 0xFFFFu, hi = 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          lo = min(lo, mk[j]);
          if (32 * j + lane < nch) hi = max(hi, mk[j]);
        }
        lo = __reduce_min_sync(0xffffffffu, lo);
        hi = __reduce_max_sync(0xffffffffu, hi);
        const int free_bits = lo == hi ? 0 : 32 - __clz(lo ^ hi);  // bits below the common prefix
        p = lo & ~((1u << free_bits) - 1u);
#pragma unroll 1
        for (int b = free_bits - 1; b >= 0; --b) {
          const uint32_t t = p | (1u << b);
          int cnt = 0;
#pragma unroll
          for (int j = 0; j < 4; ++j) cnt += __popc(__ballot_sync(0xffffffffu, mk[j] < t));
          if (cnt <= 31) p = t;
        }
      }
      pk = min(p, 0xFF00u);
      T = pk == 0xFF00u ? kInf : __uint_as_float(pk << 15);
    } else {
      float best = kInf;
      for (int g = 0; g < nch; g += 32) {
        float v = g + lane < nch ? __ldg(cm + g + lane) : kInf;
        v = __shfl_sync(0xffffffffu, warp_sort_asc_f32(v), 31 - lane);
        float r = fminf(best, v);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float x = __shfl_xor_sync(0xffffffffu, r, o);
          r = (lane & o) == 0 ? fminf(x, r) : fmaxf(x, r);
        }
        best = r;
      }
      T = __shfl_sync(0xffffffffu, best, 31);
    }
    uint64_t mine = kEmpty, worst = kEmpty;
    const uint16_t* row = D + q * ldo;
#if HENN_SELECT_ONE_TRIP
    // the chunks that can hold an entry <= T (usually exactly 32): their ids
    // listed, then each lane loads one whole chunk, so that every chunk of
    // the row is in flight at once; the entries <= T are staged as keys and
    // merged 32 at a time.  Longer lists take the loop below.
    // whole chunks as 16-byte loads: rows 16-byte aligned
    bool fast = ((reinterpret_cast<uintptr_t>(D) & 15) == 0) && (ldo % 8 == 0);
    if (fast) {
      int* chl = sel_chunks[threadIdx.x >> 5];
      uint64_t* stg = sel_keys[threadIdx.x >> 5];
      int nc = 0;
      if (few) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const bool in = 32 * j + lane < nch && mk[j] <= pk;
          const unsigned bm = __ballot_sync(0xffffffffu, in);
          const int pos = nc + __popc(bm & ((1u << lane) - 1u));
          if (in) chl[pos] = 32 * j + lane;
          nc += __popc(bm);
        }
      } else {
        for (int g = 0; g < nch; g += 32) {
          const bool in = g + lane < nch && __ldg(cm + g + lane) <= T;
          const unsigned bm = __ballot_sync(0xffffffffu, in);
          const int pos = nc + __popc(bm & ((1u << lane) - 1u));
          if (in && pos < kSelChunks) chl[pos] = g + lane;
          nc += __popc(bm);
        }
      }
      fast = nc <= kSelChunks;
      __syncwarp();
      int n = 0;
      // the keys <= T as integers: T is the lower end of a key's bucket,
      // and keys of +inf or NaN (0xFF00 and above) never enter
      const uint32_t Tk = min((__float_as_uint(T) >> 15) & 0xFFFFu, 0xFEFFu);
      for (int r0 = 0; fast && r0 < nc; r0 += 32) {
        const int ch = r0 + lane < nc ? chl[r0 + lane] : -1;
        uint32_t w[16];  // the chunk's 32 keys, two per word (the lower column in the low half)
        unsigned keep = 0;
        if (ch >= 0) {
          const uint4* src = reinterpret_cast<const uint4*>(row + (int64_t)ch * 32);
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint4 x = __ldcs(src + i);
            w[4 * i] = x.x;
            w[4 * i + 1] = x.y;
            w[4 * i + 2] = x.z;
            w[4 * i + 3] = x.w;
          }
#pragma unroll
          for (int i = 0; i < 16; ++i)
            keep |= ((w[i] & 0xFFFFu) <= Tk ? 1u : 0u) << (2 * i) | ((w[i] >> 16) <= Tk ? 2u : 0u) << (2 * i);
        }
        const int c = __popc(keep);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int t = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += t;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        if (n + tot > kSelKeys) {
          fast = false;
          break;
        }
        int at = n + incl - c;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (!(keep & (3u << (2 * i)))) continue;
          if (keep & (1u << (2 * i))) stg[at++] = pack(key16_dist(w[i] & 0xFFFFu), (uint32_t)(ch * 32 + 2 * i));
          if (keep & (2u << (2 * i))) stg[at++] = pack(key16_dist(w[i] >> 16), (uint32_t)(ch * 32 + 2 * i + 1));
        }
        n += tot;
      }
      if (fast) {
        __syncwarp();
        for (int b = 0; b < n; b += 32) {
          uint64_t kk = b + lane < n ? stg[b + lane] : kEmpty;
          if (b == 0) {
            // the first batch is the running list itself, sorted
            mine = warp_sort_asc(kk);
            worst = shfl64(mine, 31);
            continue;
          }
          if (!__any_sync(0xffffffffu, kk < worst)) continue;
          // the running list and the reversed sorted batch: their
          // element-wise minimum holds the 32 smallest as a bitonic sequence
          kk = shfl64(warp_sort_asc(kk), 31 - lane);
          uint64_t r = mine < kk ? mine : kk;
#pragma unroll
          for (int j = 16; j > 0; j >>= 1) {
            const uint64_t o = shfl_xor64(r, j);
            r = (lane & j) == 0 ? (o < r ? o : r) : (o > r ? o : r);
          }
          mine = r;
          worst = shfl64(mine, 31);
        }
      }
      __syncwarp();
    }
    for (int g = 0; !fast && g < nch; g += 32) {
#else
    for (int g = 0; g < nch; g += 32) {
#endif
      const bool in = g + lane < nch && __ldg(cm + g + lane) <= T;
      unsigned m = __ballot_sync(0xffffffffu, in);
      while (m) {
        // up to four of the chunks at a time: their loads in flight together
        int ch[4];
        float dv[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          ch[b] = m ? g + __ffs(m) - 1 : -1;
          if (m) m &= m - 1;
          dv[b] = ch[b] >= 0 ? key16_dist(__ldcs(row + (int64_t)ch[b] * 32 + lane)) : kInf;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          if (ch[b] < 0) continue;  // warp-uniform
          const float x = dv[b];
          uint64_t kk = (x <= T && !isinf(x)) ? pack(x, (uint32_t)(ch[b] * 32 + lane)) : kEmpty;
          unsigned bm = __ballot_sync(0xffffffffu, kk < worst);
          if (!bm) continue;
          if (__popc(bm) > 6) {
            kk = shfl64(warp_sort_asc(kk), 31 - lane);
            uint64_t r = mine < kk ? mine : kk;
#pragma unroll
            for (int j = 16; j > 0; j >>= 1) {
              const uint64_t o = shfl_xor64(r, j);
              r = (lane & j) == 0 ? (o < r ? o : r) : (o > r ? o : r);
            }
            mine = r;
          } else {
            do {
              const int src = __ffs(bm) - 1;
              bm &= bm - 1;
              const uint64_t x64 = shfl64(kk, src);
              if (x64 < worst) {
                const int pos = __popc(__ballot_sync(0xffffffffu, mine < x64));
                const uint64_t up = shfl64(mine, lane > 0 ? lane - 1 : 0);
                mine = lane < pos ? mine : (lane == pos ? x64 : up);
                worst = shfl64(mine, 31);
              }
            } while (bm);
          }
          worst = shfl64(mine, 31);
        }
      }
    }
    out[q * 32 + lane] = mine;
    // the row is not read again: drop its lines from L2 without writing
    // them back (the buffer is rewritten or freed next)
    __syncwarp();
    if (discard) {
      const char* rb = reinterpret_cast<const char*>(row);
      for (int64_t l = lane; l < ldo / 64; l += 32) asm volatile("discard.global.L2 [%0], 128;" ::"l"(rb + l * 128) : "memory");
    }
  }
}

void launch_select_top32(const uint16_t* D, const float* cmin, int64_t nq, int64_t s, int64_t ldo, int64_t ldc,
                         uint64_t* out, bool discard, cudaStream_t st) {
  int64_t blocks = (nq + 7) / 8;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (blocks < 1) blocks = 1;
  // discard works on whole 128-byte lines: rows must start on one
  const bool lines = (reinterpret_cast<uintptr_t>(D) & 127) == 0 && ldo % 64 == 0;
  k_select_top32<<<(int)blocks, 256, 0, st>>>(D, cmin, nq, s, ldo, ldc, out, discard && lines ? 1 : 0);
}

// ------------------------------------------------------------ dispatch

size_t search_warp_smem(int ef_cap, int hash_bits, int dpad) {
  size_t b = (size_t)ef_cap * 8 + ((size_t)4 << hash_bits) + kStageBytes + (size_t)dpad * 4;
  return (b + 15) & ~(size_t)15;
}

size_t search_team_smem(int ef_cap, int hash_bits, int dpad, int team) {
  const size_t b = search_warp_smem(ef_cap, hash_bits, dpad);
  return team > 1 ? b + sizeof(TeamJob) : b;
}

int search_beam_cap(int k, int ef, int ef_upper, int ef_l1, bool rerank, int rerank_mult) {
  int need = max(max(k, ef), max(ef_upper, ef_l1));
  if (rerank) need = max(need, min(ef, rerank_mult * k));
  int c = 32;
  while (c < need) c <<= 1;
  return c;
}

int search_hash_bits(int ef_cap) {
  int hb = 10;
  while (hb < 12 && (1 << hb) < ef_cap * 8) ++hb;
  return hb;
}

cudaError_t search_persistent_grid(int device, int warps, size_t smem, int* grid) {
  int sms = 0;
  const cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return e;
  int per_sm = (int)((200 * 1024) / (smem > 0 ? smem : 1));
  if (per_sm < 1) per_sm = 1;
  if (per_sm > 64 / warps) per_sm = 64 / warps;
  *grid = sms * per_sm;
  return cudaSuccess;
}

template <typename VT, int DMAX>
static cudaError_t launch_t(const SearchArgs& a, int warps, int grid, size_t smem, cudaStream_t st) {
  auto kern = a.team > 1 ? k_search<VT, DMAX, Team> : k_search<VT, DMAX, Solo>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename VT>
static cudaError_t launch_vt(const SearchArgs& a, int warps, int grid, size_t smem, cudaStream_t st) {
  if (a.dpad <= 32) return launch_t<VT, 32>(a, warps, grid, smem, st);
  if (a.dpad <= 64) return launch_t<VT, 64>(a, warps, grid, smem, st);
  if (a.dpad <= 128) return launch_t<VT, 128>(a, warps, grid, smem, st);
  if (a.dpad <= 512) return launch_t<VT, 512>(a, warps, grid, smem, st);
  return launch_t<VT, 1024>(a, warps, grid, smem, st);
}

template <typename VT, int DMAX>
static cudaError_t launch_serve_t(const ServeArgs& a, int warps, int grid, size_t smem, cudaStream_t st) {
  auto kern = k_serve<VT, DMAX>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <typename VT>
static cudaError_t launch_serve_vt(const ServeArgs& a, int warps, int grid, size_t smem, cudaStream_t st) {
  if (a.base.dpad <= 32) return launch_serve_t<VT, 32>(a, warps, grid, smem, st);
  if (a.base.dpad <= 64) return launch_serve_t<VT, 64>(a, warps, grid, smem, st);
  if (a.base.dpad <= 128) return launch_serve_t<VT, 128>(a, warps, grid, smem, st);
  if (a.base.dpad <= 512) return launch_serve_t<VT, 512>(a, warps, grid, smem, st);
  return launch_serve_t<VT, 1024>(a, warps, grid, smem, st);
}

cudaError_t launch_serve(const ServeArgs& a, int warps_per_block, int grid, cudaStream_t st) {
  ServeArgs b = a;
  b.base.warp_smem = (int32_t)search_warp_smem(a.base.ef_cap, a.base.hash_bits, a.base.dpad);
  size_t smem = (size_t)b.base.warp_smem * warps_per_block;
  if (a.base.storage == HENN_BF16) return launch_serve_vt<__nv_bfloat16>(b, warps_per_block, grid, smem, st);
  if (a.base.storage == HENN_FP8E4M3) return launch_serve_vt<__nv_fp8_e4m3>(b, warps_per_block, grid, smem, st);
  return launch_serve_vt<float>(b, warps_per_block, grid, smem, st);
}

cudaError_t launch_search(const SearchArgs& a, int warps_per_block, int grid, cudaStream_t st) {
  SearchArgs b = a;
  const int team = a.team > 1 ? a.team : 1;
  if (warps_per_block % team != 0) return cudaErrorInvalidValue;
  b.team = team;
  b.warp_smem = (int32_t)search_team_smem(a.ef_cap, a.hash_bits, a.dpad, team);
  size_t smem = (size_t)b.warp_smem * (warps_per_block / team);
  if (a.storage == HENN_BF16) return launch_vt<__nv_bfloat16>(b, warps_per_block, grid, smem, st);
  if (a.storage == HENN_FP8E4M3) return launch_vt<__nv_fp8_e4m3>(b, warps_per_block, grid, smem, st);
  return launch_vt<float>(b, warps_per_block, grid, smem, st);
}

}  // namespace henn
