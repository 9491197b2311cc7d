// search.cuh -- arguments of the persistent search kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace henn {

constexpr int kSearchWarps = 4;  // warps (queries in flight) per block

// One layer as the search kernel sees it (device memory, layer order).
struct SearchLayer {
  const int32_t* adj;   // size x 32 layer-local neighbour indices, -1 padded at the end
  const void* vec;      // size x dpad traversal vectors (FP32 / BF16 / FP8 codes)
  const float* scale;   // FP8: per-row scale, else nullptr
  const int32_t* down;  // layers >= 1: position of each point in the layer below
  int64_t size;
};

struct SearchArgs {
  const SearchLayer* layers;  // device array, L + 1 entries
  int32_t L;
  int32_t dpad, d;
  int32_t metric, storage;
  int32_t rerank, rerank_mult;
  const float* x32;  // FP32 layer-0 rows (unit length for angular), for the rerank
  const uint8_t* dead;  // nullptr, or 1 per deleted point (global id): kept out of results
  const float* Q;    // nq x d queries
  int64_t nq;
  const int32_t* kq;
  const int32_t* efq;
  int32_t k_uniform, ef_uniform;
  int32_t ef_upper;           // beam width on layers >= 1 (<= 1: greedy)
  int32_t descend_all;        // enter each layer at all candidates of the layer above
  int32_t ef_l1;              // beam width on layer 1 (0: ef_upper)
  int32_t exact_upper;        // upper layers of at most this many points: exact candidate set
  int32_t top_exact;          // the lowest such layer (the layers above it are skipped), else L
  int32_t exact_method;       // its set by: 0 sort in the visited table, 1 tile candidates, 2 scan
  const uint64_t* pre_keys;   // method 1: nq x 32 tile keys (distance, layer position), ascending
  const float* pre_qnorm;     // method 1: squared norm of each centred query
  const float* pre_nmax;      // method 1: largest squared norm of the layer's centred points
  const int32_t* pre_err;     // method 1: tile error flags (nonzero: every query scans)
  int32_t* pre_scans;         // method 1: queries whose certificate failed (nullable)
  double pre_tile_u;          // method 1: unit error of the tile distances
  int32_t ef_cap, hash_bits;  // beam capacity and log2 visited slots per warp
  const uint64_t* keys;
  uint64_t entry_key;  // derive(seed, ENTR)
  int64_t* out_ids;
  float* out_d;
  int32_t out_stride;
  int32_t* stats;
  unsigned long long* counter;  // work counter, zero at launch
  const int32_t* order;         // nullptr, or the query of each work slot
  int32_t warp_smem;            // bytes of shared memory per team (per warp when team = 1)
  int32_t team;                 // warps per query (1, 2 or 4)
};

// One published work item of the serving loop (one query).
struct ServeDesc {
  int32_t slot;  // request slot whose counter the query bumps
  int32_t k, ef, pad;
  uint64_t key;  // entry-node key
};

struct ServeArgs {
  SearchArgs base;               // index, shapes, beam parameters, out_stride
  const float* qring;            // cap x d query rows (device)
  const ServeDesc* desc;         // cap descriptors (device)
  int64_t cap;                   // ring capacity (items)
  int64_t* out_ids;              // cap x out_stride (device)
  float* out_d;                  // cap x out_stride (device)
  const long long* published;    // items published so far (device, written by copies)
  unsigned long long* taken;     // items taken so far (device)
  const int* stop;               // raised to end the loop (device)
  int* done;                     // per request slot: finished queries (mapped host memory)
  unsigned long long* last_active;  // globaltimer of the last item taken (device)
  long long idle_ns;             // the kernel leaves after this long without work
};

// GreedySearch probes on one layer (henn_greedy_probe).
struct GreedyProbeArgs {
  SearchLayer layer;
  int32_t dpad, d, metric;
  const float* Q;        // nq x d queries
  int64_t nq;
  const int32_t* starts;  // nq x S start positions in the layer
  int32_t S;
  int32_t* out_node;     // nq x S local minima (layer positions), -1 for a bad start
  float* out_dist;       // their distances in traversal precision
  int32_t* out_hops;     // moves per probe, or nullptr
};

size_t search_warp_smem(int ef_cap, int hash_bits, int dpad);
// Shared memory of one query's team of `team` warps: the leader's slice as
// above plus, for team > 1, the job area the team's warps exchange rows in.
size_t search_team_smem(int ef_cap, int hash_bits, int dpad, int team);
// Launch shape of k_search, shared by every entry point that runs it.
// Beam capacity of a query: the power of two (at least 32) that holds its
// widest list -- k, ef, the upper-layer widths, and with a rerank the
// min(ef, rerank_mult * k) reranked entries.
int search_beam_cap(int k, int ef, int ef_upper, int ef_l1, bool rerank, int rerank_mult);
// log2 of the visited-table slots per query for a beam capacity: at least
// 2^10 and about 8 per beam entry, at most 2^12 (the table may forget
// entries without changing results, so it is sized for occupancy).
int search_hash_bits(int ef_cap);
// Blocks of `warps` warps using `smem` bytes of shared memory each that
// stay resident together on every SM of `device` (a persistent launch).
cudaError_t search_persistent_grid(int device, int warps, size_t smem, int* grid);
// Exact-layer preparation for exact_method 1 (tile candidates).
// Layer rows in traversal precision, as FP32 (dequantised BF16 / FP8 codes).
cudaError_t launch_layer_rows_f32(const void* vec, const float* scale, int64_t s, int storage, int32_t dpad, float* out,
                                  cudaStream_t st);
// Queries as the search kernel sees them (angular: normalised the same
// way), minus `mean`: squared norms, and FP32 rows (xo, dpad wide) and / or
// split BF16 planes (hi, lo, dk wide), each output nullable; qraw
// (nullable, nq x d): the rows as read (d <= 1024).
void launch_entry_queries(const float* Q, int64_t nq, int32_t d, int32_t dpad, int32_t metric, const float* mean,
                          float* xo, void* hi, void* lo, int32_t dk, float* norms, float* qraw, cudaStream_t st);
// Per query, the 32 smallest keys of its row of a distance-key matrix (nq
// rows of ldo 16-bit keys as the tile launch's mode 3 writes them, s
// columns), guided by the rows' 32-column chunk minima (cmin, rows of ldc
// floats): the tile candidates of exact_method 1, each as (the lower end of
// its key's bucket, column).  With discard, each row's cache lines are
// dropped from L2 after it is read (its contents are undefined afterwards).
void launch_select_top32(const uint16_t* D, const float* cmin, int64_t nq, int64_t s, int64_t ldo, int64_t ldc,
                         uint64_t* out, bool discard, cudaStream_t st);
cudaError_t launch_greedy_probe(const GreedyProbeArgs& a, int storage, cudaStream_t st);
cudaError_t launch_serve(const ServeArgs& a, int warps_per_block, int grid, cudaStream_t st);
cudaError_t launch_search(const SearchArgs& a, int warps_per_block, int grid, cudaStream_t st);

}  // namespace henn
