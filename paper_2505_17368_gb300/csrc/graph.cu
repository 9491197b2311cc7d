// graph.cu -- the edge rule that turns forward lists into adjacency rows.
//
// NSW links are undirected at insertion (App. B): a point sees its own
// forward links and the later points that linked to it (reverse links).
// Each row of width Mmax = 32 keeps the nearest predecessor pred(j) =
// fwd(j)[0] first (so every point keeps a path towards the first inserted
// point and the graph stays connected), then the Mmax - 1 nearest of
// fwd(j) U rev(j) \ {pred(j)} by (distance, index).  For the kNN graph no
// slot is reserved.  Reverse lists are built with a count / scan / scatter;
// their order does not matter because each row is selected by sorted key.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.cuh"

namespace henn {

__global__ void k_rev_count(const int32_t* __restrict__ fwd, int64_t total, int32_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = fwd[i];
    if (v >= 0) atomicAdd(&cnt[v], 1);
  }
}

__global__ void k_rev_fill(const int32_t* __restrict__ fwd, const float* __restrict__ fwd_d, int64_t total, int32_t M,
                           const int64_t* __restrict__ off, int32_t* __restrict__ fill, uint64_t* __restrict__ rev) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t v = fwd[i];
    if (v < 0) continue;
    int32_t p = (int32_t)(i / M);
    int32_t slot = atomicAdd(&fill[v], 1);
    rev[off[v] + slot] = pack(fwd_d[i], (uint32_t)p);
  }
}

// one warp per node
__global__ void k_select_adj(const int32_t* __restrict__ fwd, const float* __restrict__ fwd_d, int64_t s, int32_t M,
                             const int64_t* __restrict__ off, const uint64_t* __restrict__ rev, int32_t graph,
                             int32_t* __restrict__ adj) {
  const int lane = threadIdx.x & 31;
  for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; v < s;
       v += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int32_t pred = (graph == HENN_GRAPH_NSW) ? fwd[v * M] : -1;
    WarpList<32> list;
    list.clear();
    // forward links (M <= 32 entries, one per lane)
    {
      uint64_t key = kEmpty;
      if (lane < M) {
        int32_t u = fwd[v * M + lane];
        if (u >= 0 && u != pred) key = pack(fwd_d[v * M + lane], (uint32_t)u);
      }
      unsigned m = __ballot_sync(0xffffffffu, key != kEmpty);
      while (m) {
        int src = __ffs(m) - 1;
        m &= m - 1;
        uint64_t x = shfl64(key, src);
        if (x < list.worst()) list.insert(x);
      }
    }
    // reverse links, 32 at a time
    const int64_t b = off[v], e = off[v + 1];
    for (int64_t c = b; c < e; c += 32) {
      uint64_t key = kEmpty;
      if (c + lane < e) {
        key = rev[c + lane];
        if ((int32_t)key_index(key) == pred) key = kEmpty;
      }
      uint64_t thr = list.worst();
      unsigned m = __ballot_sync(0xffffffffu, key < thr);
      while (m) {
        int src = __ffs(m) - 1;
        m &= m - 1;
        uint64_t x = shfl64(key, src);
        if (x < list.worst()) list.insert(x);
      }
    }
    // row: [pred] + first 31, or first 32 for the kNN graph
    int32_t out;
    if (pred >= 0) {
      uint64_t prev = __shfl_up_sync(0xffffffffu, list.v[0], 1);
      out = lane == 0 ? pred : (prev == kEmpty ? -1 : (int32_t)key_index(prev));
    } else {
      out = list.v[0] == kEmpty ? -1 : (int32_t)key_index(list.v[0]);
    }
    adj[v * kMmax + lane] = out;
  }
}

void launch_rev_count(const int32_t* fwd, int64_t s, int32_t M, int32_t* cnt, cudaStream_t st) {
  k_rev_count<<<152 * 8, 256, 0, st>>>(fwd, s * M, cnt);
}

void launch_rev_fill(const int32_t* fwd, const float* fwd_d, int64_t s, int32_t M, const int64_t* off, int32_t* fill,
                     uint64_t* rev, cudaStream_t st) {
  k_rev_fill<<<152 * 8, 256, 0, st>>>(fwd, fwd_d, s * M, M, off, fill, rev);
}

void launch_select_adj(const int32_t* fwd, const float* fwd_d, int64_t s, int32_t M, const int64_t* off,
                       const uint64_t* rev, int32_t graph, int32_t* adj, cudaStream_t st) {
  int grid = (int)((s + 7) / 8);
  if (grid > 152 * 32) grid = 152 * 32;
  if (grid < 1) grid = 1;
  k_select_adj<<<grid, 256, 0, st>>>(fwd, fwd_d, s, M, off, rev, graph, adj);
}

}  // namespace henn
