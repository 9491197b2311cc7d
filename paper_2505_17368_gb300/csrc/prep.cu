// prep.cu -- vector copies kept in HBM and per-layer preparation.
//
//  * padded FP32 master copy (rows of dpad = roundup(d, 32) floats, zero
//    tail, so every row is a whole number of 128-byte lines)
//  * inverse norms and unit-length copies for the angular metric (App. G:
//    cosine similarity works on vectors normalised to the unit sphere)
//  * insertion order of a layer (keyed Feistel permutation) and the layer's
//    centred vectors in that order, the operand of the distance tiles
//  * BF16 / FP8-E4M3 precision copies of the traversal vectors
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.cuh"

namespace henn {

__global__ void k_pad_copy(const float* __restrict__ X, int64_t n, int32_t d, int32_t dpad, float* __restrict__ x32) {
  int64_t total = n * dpad;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / dpad;
    int32_t k = (int32_t)(i - r * dpad);
    x32[i] = k < d ? X[r * d + k] : 0.f;
  }
}

void launch_pad_copy(const float* X, int64_t n, int32_t d, int32_t dpad, float* x32, cudaStream_t st) {
  k_pad_copy<<<152 * 8, 256, 0, st>>>(X, n, d, dpad, x32);
}

// one warp per row: 1/sqrt(sum x^2), correctly rounded division and sqrt
__global__ void k_inv_norms(const float* __restrict__ x32, int64_t n, int32_t dpad, float* __restrict__ inv) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const float* row = x32 + r * dpad;
    float acc = 0.f;
    for (int k = lane; k < dpad; k += 32) acc = fmaf(row[k], row[k], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) inv[r] = acc > 0.f ? __fdiv_rn(1.f, __fsqrt_rn(acc)) : 0.f;
  }
}

void launch_inv_norms(const float* x32, int64_t n, int32_t dpad, float* inv_norm, cudaStream_t st) {
  k_inv_norms<<<152 * 8, 256, 0, st>>>(x32, n, dpad, inv_norm);
}

__global__ void k_normalise(const float* __restrict__ x32, const float* __restrict__ inv, int64_t n, int32_t dpad,
                            float* __restrict__ xn) {
  int64_t total = n * dpad;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    xn[i] = x32[i] * inv[i / dpad];
}

void launch_normalise(const float* x32, const float* inv_norm, int64_t n, int32_t dpad, float* xn,
                      cudaStream_t st) {
  k_normalise<<<152 * 8, 256, 0, st>>>(x32, inv_norm, n, dpad, xn);
}

// Deterministic column means: fixed 4096-row chunks summed in row order,
// then chunk partials summed in chunk order (FP64 for the second stage).
constexpr int kMeanChunk = 4096;

__global__ void k_mean_partial(const float* __restrict__ xw, const int32_t* __restrict__ ids, int64_t s,
                               int32_t dpad, float* __restrict__ partial) {
  const int64_t c = blockIdx.x;
  const int64_t r0 = c * kMeanChunk, r1 = min(s, r0 + kMeanChunk);
  for (int k = threadIdx.x; k < dpad; k += blockDim.x) {
    float acc = 0.f;
    for (int64_t r = r0; r < r1; ++r) {
      int64_t g = ids ? ids[r] : r;
      acc += xw[g * dpad + k];
    }
    partial[c * dpad + k] = acc;
  }
}

__global__ void k_mean_final(const float* __restrict__ partial, int64_t chunks, int64_t s, int32_t dpad,
                             float* __restrict__ mean) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= dpad) return;
  double acc = 0.0;
  for (int64_t c = 0; c < chunks; ++c) acc += (double)partial[c * dpad + k];
  mean[k] = (float)(acc / (double)s);
}

void launch_layer_mean(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, float* partial, float* mean,
                       cudaStream_t st) {
  int64_t chunks = (s + kMeanChunk - 1) / kMeanChunk;
  k_mean_partial<<<(unsigned)chunks, 128, 0, st>>>(xw, ids, s, dpad, partial);
  k_mean_final<<<(dpad + 127) / 128, 128, 0, st>>>(partial, chunks, s, dpad, mean);
}

// Insertion order of a layer: point j (layer-local) is inserted at rank
// perm(j); the tiles work in rank order so that "inserted earlier" is
// "lower row index" (causal lower triangle).  For the kNN graph the order
// is irrelevant and the identity is used.
__global__ void k_order_gather(const float* __restrict__ xw, const int32_t* __restrict__ ids, int64_t s,
                               int32_t dpad, Feistel f, int32_t identity, const float* __restrict__ mean,
                               int32_t* __restrict__ inv, float* __restrict__ xo, float* __restrict__ norms) {
  const int lane = threadIdx.x & 31;
  for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < s;
       j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    int64_t rank = identity ? j : (int64_t)f.perm((uint64_t)j);
    int64_t g = ids ? ids[j] : j;
    const float* src = xw + g * dpad;
    float* dst = xo + rank * dpad;
    float acc = 0.f;
    for (int k = lane; k < dpad; k += 32) {
      float v = src[k] - mean[k];
      dst[k] = v;
      acc = fmaf(v, v, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      inv[rank] = (int32_t)j;
      norms[rank] = acc;
    }
  }
}

void launch_order_gather(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, uint64_t seed, int32_t layer,
                         int32_t graph, const float* mean, int32_t* inv, float* xo, float* norms, cudaStream_t st) {
  Feistel f = Feistel::make(seed, layer, (uint64_t)s);
  k_order_gather<<<152 * 8, 256, 0, st>>>(xw, ids, s, dpad, f, graph == HENN_GRAPH_KNN ? 1 : 0, mean, inv, xo,
                                          norms);
}

__global__ void k_gather_rows32(const float* __restrict__ xw, const int32_t* __restrict__ ids, int64_t s,
                                int32_t dpad, float* __restrict__ out) {
  int64_t total = s * dpad;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / dpad;
    out[i] = xw[(int64_t)ids[r] * dpad + (i - r * dpad)];
  }
}

void launch_gather_rows32(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, float* out, cudaStream_t st) {
  k_gather_rows32<<<152 * 8, 256, 0, st>>>(xw, ids, s, dpad, out);
}

// BF16: round to nearest even.  FP8: scale = max|x|/448 per row (FP32),
// code = E4M3(x / scale) rounded to nearest even with saturation.
__global__ void k_quant_bf16(const float* __restrict__ x, int64_t n, int32_t d, int32_t din, int32_t dout,
                             __nv_bfloat16* __restrict__ out) {
  int64_t total = n * dout;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / dout;
    int32_t k = (int32_t)(i - r * dout);
    out[i] = __float2bfloat16_rn(k < d ? x[r * din + k] : 0.f);
  }
}

__global__ void k_quant_fp8(const float* __restrict__ x, int64_t n, int32_t d, int32_t din, int32_t dout,
                            __nv_fp8_storage_t* __restrict__ out, float* __restrict__ scales) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < n;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const float* row = x + r * din;
    float m = 0.f;
    for (int k = lane; k < d; k += 32) m = fmaxf(m, fabsf(row[k]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    float scale = m > 0.f ? __fdiv_rn(m, 448.f) : 1.f;
    for (int k = lane; k < dout; k += 32) {
      float v = k < d ? __fdiv_rn(row[k], scale) : 0.f;
      out[r * dout + k] = __nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    }
    if (lane == 0) scales[r] = scale;
  }
}

void launch_quantize(const float* x, int64_t n, int32_t d, int32_t dpad_in, int32_t dpad_out, int32_t storage,
                     void* out, float* scales, cudaStream_t st) {
  if (storage == HENN_BF16)
    k_quant_bf16<<<152 * 8, 256, 0, st>>>(x, n, d, dpad_in, dpad_out, (__nv_bfloat16*)out);
  else if (storage == HENN_FP8E4M3)
    k_quant_fp8<<<152 * 8, 256, 0, st>>>(x, n, d, dpad_in, dpad_out, (__nv_fp8_storage_t*)out, scales);
}

}  // namespace henn
