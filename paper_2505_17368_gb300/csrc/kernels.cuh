// kernels.cuh -- launch interfaces between the host orchestration
// (henn_abi.cu) and the kernels of libhenn.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace henn {

constexpr int kMaxDimPerLane = 32;  // dpad <= 1024 (dpad = d rounded up to 32)
constexpr int kMaxD = 1024;

enum RingStatus : int32_t { kRingPass = 1, kRingFail = 2, kRingAmbiguous = 3 };

struct LayerSampleArgs {
  uint64_t base;   // derive(derive(derive(seed, SAMP), layer), attempt)
  int64_t s;       // size of the previous layer
  int64_t t;       // number of draws
  uint8_t* flags;  // s bytes, zeroed by the caller
};

// layers.cu
void launch_sample(const LayerSampleArgs& a, cudaStream_t st);
int64_t scan_tiles(int64_t s);
void launch_compact(const uint8_t* flags, int64_t s, const int32_t* prev_ids, int64_t* tile_buf,
                    int64_t* d_total, int32_t* out_pos, int32_t* out_ids, cudaStream_t st);
void launch_offsets(const int32_t* counts, int64_t s, int64_t* tile_buf, int64_t* out_offsets,
                    cudaStream_t st);
void launch_ring_params(uint64_t bc, uint64_t bs, int32_t r, int64_t s, int64_t span, int32_t* centre,
                        int64_t* start, cudaStream_t st);
void launch_ring_dist(const float* x32, int32_t dpad, const int32_t* prev_ids, int64_t s,
                      const int32_t* centre, int32_t r, int32_t metric, const float* inv_norm, float* D,
                      cudaStream_t st);
// Alg. 3 halving: m steps over positions 0..s-1; the survivors (ascending)
// land in pos and their global ids in ids; returns their count.  tmp holds
// ceil(s/2) entries.
int64_t launch_halving(uint64_t seed, int32_t layer, int64_t s, int32_t m, const int32_t* prev_ids, int32_t* tmp,
                       int32_t* pos, int32_t* ids, cudaStream_t st);
void launch_ring_select_decide(const float* D, int64_t s, const int64_t* start, int64_t w, int32_t r,
                               const int32_t* net_pos, const int64_t* nnet_dev, double er, double ea, float* lo,
                               float* hi, int32_t* status, cudaStream_t st);
void launch_ring_recheck(const float* x32, int32_t d, int32_t dpad, const int32_t* prev_ids, int64_t s,
                         int64_t centre_pos, int64_t a0, int64_t w, int32_t metric, const int32_t* net_pos,
                         int64_t nnet, double* D64, double* bounds, int32_t* status, int32_t q,
                         cudaStream_t st);

// prep.cu: vector copies and per-layer preparation
void launch_pad_copy(const float* X, int64_t n, int32_t d, int32_t dpad, float* x32, cudaStream_t st);
void launch_inv_norms(const float* x32, int64_t n, int32_t dpad, float* inv_norm, cudaStream_t st);
void launch_normalise(const float* x32, const float* inv_norm, int64_t n, int32_t dpad, float* xn,
                      cudaStream_t st);
// mean over the rows listed in ids (or rows 0..s-1): partial buffer of
// ceil(s/4096) * dpad floats
void launch_layer_mean(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, float* partial,
                       float* mean, cudaStream_t st);
// insertion order: rank[j] = perm(j), inv[rank] = j; xo[rank] = xw[ids[j]] - mean; norms
void launch_order_gather(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, uint64_t seed,
                         int32_t layer, int32_t graph, const float* mean, int32_t* inv, float* xo,
                         float* norms, cudaStream_t st);
void launch_gather_rows32(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, float* out,
                          cudaStream_t st);
void launch_quantize(const float* x, int64_t n, int32_t d, int32_t dpad_in, int32_t dpad_out,
                     int32_t storage, void* out, float* scales, cudaStream_t st);

// knn.cu: tiles (approximate distances) + running top-KP per row
//   mode 0: causal (column c valid iff c < row), A == B
//   mode 1: all other rows (c != row), A == B
//   mode 2: rows of A against all rows of B
void launch_tile_topk_simt(const float* A, const float* An, int64_t na, const float* B, const float* Bn,
                           int64_t nb, int32_t dpad, int32_t mode, int32_t KP, int32_t splits,
                           uint64_t* out, cudaStream_t st);
void launch_merge_splits(const uint64_t* in, int64_t rows, int32_t KP, int32_t splits, uint64_t* out,
                         cudaStream_t st);
// knn_tc.cu: the same tiles on tcgen05 tensor cores (split BF16, KP = 32,
// dpad <= 128); scratch_hi / scratch_lo hold s * roundup(dpad, 64) BF16
bool tc_tiles_supported(int32_t dpad, int32_t KP);
cudaError_t launch_tile_topk_tc(const float* xo, const float* norms, int64_t s, int32_t dpad, int32_t mode,
                                uint64_t* out, void* scratch_hi, void* scratch_lo, int32_t* err, cudaStream_t st);
// FP32 rows (dpad wide) -> BF16 planes hi = bf16(x), lo = bf16(x - hi), dk wide (zero padded)
void launch_split_bf16(const float* x, int64_t s, int32_t dpad, int32_t dk, void* hi, void* lo, cudaStream_t st);
// mode 2 on tensor cores from pre-split planes: na rows (queries) against nb
// columns (a layer's points), out = na x 32 keys (distance, column); with
// out_d (mode 3) every distance instead, as a 16-bit order-preserving key
// (the distance's float bits 30..15: rounded down to 8 mantissa bits), na
// rows of ldo keys (ldo a multiple of 64, >= nb, out_d 128-byte aligned;
// the key of +inf past column nb)
// b_maps: the four tensor maps of make_column_maps, 128 bytes each;
// tile_n: columns per tile, 128 or 256 (0 = 256), the same results
// out_cmin (mode 3, nullable): each row's minimum over every 32-column chunk,
// as the lower end of its key's bucket, rows of ldc floats (ldc a multiple
// of 8 covering every tile, 16-byte aligned)
cudaError_t launch_tile_cross_tc(const void* a_hi, const void* a_lo, const float* a_norms, int64_t na,
                                 const void* b_maps, const float* b_norms, int64_t nb, int32_t dk, uint64_t* out,
                                 uint16_t* out_d, int64_t ldo, float* out_cmin, int64_t ldc, int32_t* err,
                                 int32_t tile_n, cudaStream_t st);
// Tensor maps of the column operand (hi, lo planes of nb rows, dk wide) for
// launch_tile_cross_tc -- hi and lo for tiles of 256 columns, then for 128 --
// written to maps (4 x 128 bytes); false if not encodable.
bool make_column_maps(const void* b_hi, const void* b_lo, int64_t nb, int32_t dk, void* maps);
// exact FP32 rerank of layer candidates -> forward lists (layer-local ids)
void launch_rerank_fwd(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, int32_t metric,
                       const int32_t* inv, const uint64_t* cand, int32_t KP, int32_t M, const float* norms,
                       const float* norm_max, double tile_u, int32_t* fwd, float* fwd_d, int32_t* uncertified,
                       cudaStream_t st);
void launch_max_nonneg(const float* v, int64_t n, float* out, cudaStream_t st);
// exact recompute of the forward list of uncertified rows
void launch_exact_rows(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, int32_t metric,
                       const int32_t* inv, int32_t mode, const int32_t* rows, int32_t nrows, int32_t M,
                       int32_t* fwd, float* fwd_d, cudaStream_t st);
// exact rerank of query candidates -> k results
void launch_rerank_queries(const float* Q, int64_t nq, const float* X, int32_t dpad, int32_t metric,
                           const uint64_t* cand, int32_t KP, int32_t k, int64_t* out_ids, float* out_d,
                           cudaStream_t st);

// graph.cu: edge rule
void launch_rev_count(const int32_t* fwd, int64_t s, int32_t M, int32_t* cnt, cudaStream_t st);
void launch_rev_fill(const int32_t* fwd, const float* fwd_d, int64_t s, int32_t M, const int64_t* off,
                     int32_t* fill, uint64_t* rev, cudaStream_t st);
void launch_select_adj(const int32_t* fwd, const float* fwd_d, int64_t s, int32_t M, const int64_t* off,
                       const uint64_t* rev, int32_t graph, int32_t* adj, cudaStream_t st);

}  // namespace henn
