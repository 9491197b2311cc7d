// knn.cu -- construction distance tiles with a running top-KP per row, the
// exact FP32 rerank that turns the KP candidates into forward lists, and
// the exact k-NN of a query batch (k-NN query of Sec. 2).
//
// Tile distances use |a|^2 + |b|^2 - 2<a,b> on centred vectors: a dense
// contraction.  This file holds the CUDA-core (SIMT FP32) engine; the
// tcgen05 tensor-core engine lives in knn_tc.cu and feeds the same
// candidate format.  Candidates are (distance, column) keys packed into
// uint64 so the integer order is the (distance, index) order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "kernels.cuh"

namespace henn {

constexpr int kBM = 64, kBN = 64, kBK = 32;

template <int KP>
__global__ void __launch_bounds__(256) k_tile_topk_simt(const float* __restrict__ A, const float* __restrict__ An,
                                                        int64_t na, const float* __restrict__ B,
                                                        const float* __restrict__ Bn, int64_t nb, int32_t dpad,
                                                        int32_t mode, int32_t splits, uint64_t* __restrict__ out) {
  __shared__ __align__(16) float As[kBK][kBM + 4];
  __shared__ __align__(16) float Bs[kBK][kBN + 4];
  __shared__ float S[kBM][kBN + 1];

  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int warp = tid >> 5;
  const int64_t nblocks = (na + kBM - 1) / kBM;
  // causal rows: heaviest row blocks first
  const int64_t rb = (mode == 0) ? (nblocks - 1 - blockIdx.x) : blockIdx.x;
  const int64_t r0 = rb * kBM;
  const int split = blockIdx.y;

  int64_t cend = (mode == 0) ? min(nb, r0 + kBM) : nb;
  // columns of this split
  int64_t ctiles = (cend + kBN - 1) / kBN;
  int64_t per = (ctiles + splits - 1) / splits;
  int64_t ct0 = split * per, ct1 = min(ctiles, ct0 + per);

  WarpList<KP> lists[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) lists[i].clear();

  for (int64_t ct = ct0; ct < ct1; ++ct) {
    const int64_t c0 = ct * kBN;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int k0 = 0; k0 < dpad; k0 += kBK) {
      // load A rows r0..r0+63, dims k0..k0+31 (8 threads per row, float4 each)
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        int idx = tid + p * 256;  // 0..511
        int row = idx >> 3, kq = (idx & 7) * 4;
        int64_t gr = r0 + row;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gr < na) v = *reinterpret_cast<const float4*>(A + gr * dpad + k0 + kq);
        As[kq + 0][row] = v.x;
        As[kq + 1][row] = v.y;
        As[kq + 2][row] = v.z;
        As[kq + 3][row] = v.w;
        int64_t gc = c0 + row;
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gc < nb) w = *reinterpret_cast<const float4*>(B + gc * dpad + k0 + kq);
        Bs[kq + 0][row] = w.x;
        Bs[kq + 1][row] = w.y;
        Bs[kq + 2][row] = w.z;
        Bs[kq + 3][row] = w.w;
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < kBK; ++k) {
        float4 a = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
        float4 b = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
        float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
    // epilogue: approximate distances with the validity mask
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int64_t gr = r0 + ty * 4 + i;
      float an = gr < na ? An[gr] : 0.f;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int64_t gc = c0 + tx * 4 + j;
        bool valid = gr < na && gc < nb;
        if (mode == 0) valid = valid && gc < gr;
        if (mode == 1) valid = valid && gc != gr;
        float dv = valid ? fmaxf(an + Bn[gc] - 2.f * acc[i][j], 0.f) : __int_as_float(0x7f800000);
        S[ty * 4 + i][tx * 4 + j] = dv;
      }
    }
    __syncthreads();
    // running top-KP: warp w owns rows w*8 .. w*8+7
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = warp * 8 + i;
      const int lane = tid & 31;
      uint64_t thr = lists[i].worst();
      float d0 = S[row][lane], d1 = S[row][lane + 32];
      uint64_t k0v = isinf(d0) ? kEmpty : pack(d0, (uint32_t)(c0 + lane));
      uint64_t k1v = isinf(d1) ? kEmpty : pack(d1, (uint32_t)(c0 + lane + 32));
      unsigned m0 = __ballot_sync(0xffffffffu, k0v < thr);
      unsigned m1 = __ballot_sync(0xffffffffu, k1v < thr);
      while (m0 | m1) {
        uint64_t x;
        if (m0) {
          int src = __ffs(m0) - 1;
          m0 &= m0 - 1;
          x = shfl64(k0v, src);
        } else {
          int src = __ffs(m1) - 1;
          m1 &= m1 - 1;
          x = shfl64(k1v, src);
        }
        if (x < thr) {
          lists[i].insert(x);
          thr = lists[i].worst();
        }
      }
    }
    __syncthreads();
  }
  // write lists
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    int64_t gr = r0 + warp * 8 + i;
    if (gr < na) {
      uint64_t* dst = out + ((int64_t)split * na + gr) * KP;
#pragma unroll
      for (int r = 0; r < KP / 32; ++r) dst[r * 32 + (tid & 31)] = lists[i].v[r];
    }
  }
}

void launch_tile_topk_simt(const float* A, const float* An, int64_t na, const float* B, const float* Bn, int64_t nb,
                           int32_t dpad, int32_t mode, int32_t KP, int32_t splits, uint64_t* out, cudaStream_t st) {
  dim3 grid((unsigned)((na + kBM - 1) / kBM), (unsigned)splits);
  switch (KP) {
    case 32: k_tile_topk_simt<32><<<grid, 256, 0, st>>>(A, An, na, B, Bn, nb, dpad, mode, splits, out); break;
    case 64: k_tile_topk_simt<64><<<grid, 256, 0, st>>>(A, An, na, B, Bn, nb, dpad, mode, splits, out); break;
    case 128: k_tile_topk_simt<128><<<grid, 256, 0, st>>>(A, An, na, B, Bn, nb, dpad, mode, splits, out); break;
    default: k_tile_topk_simt<256><<<grid, 256, 0, st>>>(A, An, na, B, Bn, nb, dpad, mode, splits, out); break;
  }
}

// merge per-split lists of one row into one list of KP
template <int KP>
__global__ void k_merge_splits(const uint64_t* __restrict__ in, int64_t rows, int32_t splits, uint64_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < rows;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    WarpList<KP> list;
    list.clear();
    for (int s = 0; s < splits; ++s) {
      const uint64_t* src = in + ((int64_t)s * rows + r) * KP;
      for (int c = 0; c < KP; c += 32) {
        uint64_t v = src[c + lane];
        uint64_t thr = list.worst();
        unsigned m = __ballot_sync(0xffffffffu, v < thr);
        while (m) {
          int sl = __ffs(m) - 1;
          m &= m - 1;
          uint64_t x = shfl64(v, sl);
          if (x < list.worst()) list.insert(x);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < KP / 32; ++q) out[r * KP + q * 32 + lane] = list.v[q];
  }
}

void launch_merge_splits(const uint64_t* in, int64_t rows, int32_t KP, int32_t splits, uint64_t* out, cudaStream_t st) {
  int grid = (int)((rows + 7) / 8);
  if (grid > 152 * 16) grid = 152 * 16;
  switch (KP) {
    case 32: k_merge_splits<32><<<grid, 256, 0, st>>>(in, rows, splits, out); break;
    case 64: k_merge_splits<64><<<grid, 256, 0, st>>>(in, rows, splits, out); break;
    case 128: k_merge_splits<128><<<grid, 256, 0, st>>>(in, rows, splits, out); break;
    default: k_merge_splits<256><<<grid, 256, 0, st>>>(in, rows, splits, out); break;
  }
}

// Exact FP32 distance, warp cooperative: lane k handles coordinates k, k+32,
// ... (coalesced 128-byte lines), xor-tree reduction.  The operation order is
// symmetric in (a, b), so dist(a,b) and dist(b,a) are bitwise equal.
// L2: squared distance; angular (unit vectors): |a-b|^2 / 2 = 1 - cos.
__device__ __forceinline__ float warp_exact_dist(const float* __restrict__ a, const float* __restrict__ b,
                                                 int32_t dpad, int32_t metric) {
  const int lane = threadIdx.x & 31;
  float acc = 0.f;
  for (int k = lane; k < dpad; k += 32) {
    float t = a[k] - b[k];
    acc = fmaf(t, t, acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  return metric == HENN_ANGULAR ? 0.5f * acc : acc;
}

// Forward lists from the KP tile candidates of each row (rank space).
// Certification: the tile distance of any non-candidate column is >= the
// row's KP-th tile distance thr; its true distance is >= thr - beta where
// beta bounds the tile error for this row.  If thr - beta exceeds the M-th
// exact distance, no column outside the pool can enter the forward list;
// otherwise the row is flagged for an exact recompute.
template <int KP>
__global__ void k_rerank_fwd(const float* __restrict__ xw, const int32_t* __restrict__ ids, int64_t s, int32_t dpad,
                             int32_t metric, const int32_t* __restrict__ inv, const uint64_t* __restrict__ cand,
                             int32_t M, const float* __restrict__ norms, const float* __restrict__ norm_max, double tile_u,
                             int32_t* __restrict__ fwd, float* __restrict__ fwd_d, int32_t* __restrict__ uncertified) {
  const int lane = threadIdx.x & 31;
  for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < s;
       r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t j = inv[r];
    const int64_t gj = ids ? ids[j] : j;
    const float* xj = xw + gj * dpad;
    WarpList<KP> list;
    list.clear();
    const uint64_t* row = cand + r * KP;
    uint64_t thr_key = kEmpty;
    int count = 0;
    for (int c = 0; c < KP; ++c) {
      uint64_t key = row[c];  // warp-uniform broadcast load
      if (key == kEmpty) break;
      ++count;
      thr_key = key;
      int64_t qj = inv[key_index(key)];
      int64_t gq = ids ? ids[qj] : qj;
      float dv = warp_exact_dist(xj, xw + gq * dpad, dpad, metric);
      list.insert(pack(dv, (uint32_t)qj));
    }
    // certification (every lane evaluates it; lane 0 records)
    uint64_t mkey = shfl64(list.v[(M - 1) >> 5], (M - 1) & 31);
    if (count == KP && uncertified) {
      double thr = (double)key_dist(thr_key);
      double dm = (mkey == kEmpty) ? 1e300 : (double)key_dist(mkey);
      // exact distances here are of raw vectors; tile distances of centred
      // ones: identical in exact arithmetic.  Angular: tile values are 2x.
      if (metric == HENN_ANGULAR) dm *= 2.0;
      // relative error bound of the exact FP32 distances (dpad / 32 FMA
      // steps per lane, five butterfly additions), doubled
      const double slack = (dpad / 32 + 8) * 0x1p-23;
      // Only columns whose true distance can reach dm matter, and those lie
      // within sqrt(dm) of this row, so their centred norm is at most
      // (|x_r| + sqrt(dm))^2 (widened for the centring rounding); the tile
      // error bound needs the column norm only up to that cap.
      const double nr = (double)norms[r];
      const double rad = sqrt(nr) * (1.0 + 1e-3) + sqrt(dm * (1.0 + 2.0 * slack)) * (1.0 + 1e-3);
      const double nc = fmin((double)*norm_max, rad * rad);
      const double beta = tile_u * 4.0 * (nr + nc) + 1e-30;
      if (!(thr - beta > dm * (1.0 + slack))) {
        if (lane == 0) {
          int at = atomicAdd(uncertified, 1);
          uncertified[1 + at] = (int32_t)r;
        }
      }
    }
    // output first M of the list, layer-local ids
#pragma unroll
    for (int q = 0; q < KP / 32; ++q) {
      int g = q * 32 + lane;
      if (g < M) {
        uint64_t key = list.v[q];
        fwd[j * M + g] = key == kEmpty ? -1 : (int32_t)key_index(key);
        fwd_d[j * M + g] = key == kEmpty ? __int_as_float(0x7f800000) : key_dist(key);
      }
    }
  }
}

void launch_rerank_fwd(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, int32_t metric, const int32_t* inv,
                       const uint64_t* cand, int32_t KP, int32_t M, const float* norms, const float* norm_max, double tile_u,
                       int32_t* fwd, float* fwd_d, int32_t* uncertified, cudaStream_t st) {
  int grid = (int)((s + 7) / 8);
  if (grid > 152 * 32) grid = 152 * 32;
  if (grid < 1) grid = 1;
  switch (KP) {
    case 32:
      k_rerank_fwd<32><<<grid, 256, 0, st>>>(xw, ids, s, dpad, metric, inv, cand, M, norms, norm_max, tile_u, fwd,
                                             fwd_d, uncertified);
      break;
    case 64:
      k_rerank_fwd<64><<<grid, 256, 0, st>>>(xw, ids, s, dpad, metric, inv, cand, M, norms, norm_max, tile_u, fwd,
                                             fwd_d, uncertified);
      break;
    default:
      k_rerank_fwd<128><<<grid, 256, 0, st>>>(xw, ids, s, dpad, metric, inv, cand, M, norms, norm_max, tile_u, fwd,
                                              fwd_d, uncertified);
      break;
  }
}

// Exact forward lists of flagged rows, batched: a block takes RT flagged
// rows (kept in shared memory) and streams every candidate column once for
// all of them, so the columns are read once per RT rows instead of once per
// row.  Each distance is formed exactly as warp_exact_dist forms it (lane
// l sums the squared differences of elements l, l+32, ... in order with
// FMA, then the xor butterfly over the 32 lanes), so a flagged row gets the
// list the certified path would give it.  Column validity: mode 0 (causal,
// NSW) columns before the row in insertion order, mode 1 (kNN) all other
// columns.  inv maps insertion ranks to layer positions (nullptr: the
// identity, as for points appended by an insertion).  KD = dpad / 32 when dpad <= 128 (the loads of CPG columns are
// issued together), else 0 (any dpad, one column at a time, read once).
template <int KM, int RT, int KD>
__global__ void __launch_bounds__(256, 2) k_exact_rows(const float* __restrict__ xw, const int32_t* __restrict__ ids,
                                                       int64_t s, int32_t dpad, int32_t metric,
                                                       const int32_t* __restrict__ inv, int32_t mode,
                                                       const int32_t* __restrict__ rows, int32_t nrows, int32_t M,
                                                       int32_t* __restrict__ fwd, float* __restrict__ fwd_d) {
  constexpr int CPG = KD > 0 ? 4 : 1;  // columns whose loads are in flight together
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* qrows = reinterpret_cast<float*>(smem_raw);                   // RT x dpad
  uint64_t* merged = reinterpret_cast<uint64_t*>(qrows + RT * dpad);  // warps x RT x KM
  __shared__ int64_t rank_of[RT];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int warps = blockDim.x >> 5;
  const int64_t t0 = (int64_t)blockIdx.x * RT;
  for (int i = 0; i < RT; ++i) {
    const int64_t r = t0 + i < nrows ? (int64_t)rows[t0 + i] : -1;
    if (threadIdx.x == 0) rank_of[i] = r;
    if (r >= 0) {
      const int64_t j = inv ? (int64_t)inv[r] : r;
      const float* src = xw + (ids ? (int64_t)ids[j] : j) * dpad;
      for (int k = threadIdx.x; k < dpad; k += blockDim.x) qrows[i * dpad + k] = src[k];
    }
  }
  __syncthreads();
  int64_t rr[RT];
  int64_t cend = 0;
#pragma unroll
  for (int i = 0; i < RT; ++i) {
    rr[i] = rank_of[i];
    if (rr[i] >= 0) cend = max(cend, mode == 0 ? rr[i] : s);
  }
  WarpList<KM> lists[RT];
#pragma unroll
  for (int i = 0; i < RT; ++i) lists[i].clear();
  const int kd = KD > 0 ? KD : dpad / 32;

  for (int64_t c0 = (int64_t)w * 32; c0 < cend; c0 += (int64_t)warps * 32) {
    // this chunk's 32 columns: lane cc owns column c0 + cc
    const int64_t mycol = c0 + lane;
    int32_t myq = -1;
    const float* myrow = xw;
    if (mycol < cend) {
      myq = inv ? inv[mycol] : (int32_t)mycol;
      myrow = xw + (int64_t)(ids ? ids[myq] : myq) * dpad;
    }
    float dist[RT];
#pragma unroll
    for (int i = 0; i < RT; ++i) dist[i] = 0.f;
    const int ncols = (int)min((int64_t)32, cend - c0);
    for (int cc = 0; cc < ncols; cc += CPG) {
      if constexpr (KD > 0) {
        float v[CPG][KD];
#pragma unroll
        for (int g = 0; g < CPG; ++g) {
          const float* p = reinterpret_cast<const float*>(
              __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(myrow), (cc + g) & 31));
          const bool ok = cc + g < ncols;
#pragma unroll
          for (int k = 0; k < KD; ++k) v[g][k] = ok ? __ldg(p + lane + 32 * k) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < RT; ++i) {
          float q[KD];
#pragma unroll
          for (int k = 0; k < KD; ++k) q[k] = qrows[i * dpad + lane + 32 * k];
#pragma unroll
          for (int g = 0; g < CPG; ++g) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < KD; ++k) {
              const float t = q[k] - v[g][k];
              acc = fmaf(t, t, acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == cc + g) dist[i] = acc;
          }
        }
      } else {
        // any width: the column is read once, 8 elements per lane at a time,
        // into every row's running sum (same element order per row)
        const float* p = reinterpret_cast<const float*>(
            __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(myrow), cc & 31));
        float acc[RT];
#pragma unroll
        for (int i = 0; i < RT; ++i) acc[i] = 0.f;
        for (int k0 = 0; k0 < kd; k0 += 8) {
          float v[8];
#pragma unroll
          for (int t = 0; t < 8; ++t) v[t] = k0 + t < kd ? __ldg(p + lane + 32 * (k0 + t)) : 0.f;
#pragma unroll
          for (int i = 0; i < RT; ++i)
#pragma unroll
            for (int t = 0; t < 8; ++t)
              if (k0 + t < kd) {
                const float u = qrows[i * dpad + lane + 32 * (k0 + t)] - v[t];
                acc[i] = fmaf(u, u, acc[i]);
              }
        }
#pragma unroll
        for (int i = 0; i < RT; ++i) {
          float r = acc[i];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
          if (lane == cc) dist[i] = r;
        }
      }
    }
    // lane cc holds column c0 + cc's distance to every row of the tile
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      const bool valid = mycol < cend && rr[i] >= 0 && (mode == 0 ? mycol < rr[i] : mycol != rr[i]);
      const float dv = metric == HENN_ANGULAR ? 0.5f * dist[i] : dist[i];
      const uint64_t key = valid ? pack(dv, (uint32_t)myq) : kEmpty;
      unsigned m = __ballot_sync(0xffffffffu, key < lists[i].worst());
      while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const uint64_t k2 = shfl64(key, src);
        if (k2 < lists[i].worst()) lists[i].insert(k2);
      }
    }
  }
  // merge the warps' lists row by row
#pragma unroll
  for (int i = 0; i < RT; ++i)
#pragma unroll
    for (int q = 0; q < KM / 32; ++q) merged[((int64_t)w * RT + i) * KM + q * 32 + lane] = lists[i].v[q];
  __syncthreads();
  for (int i = w; i < RT; i += warps) {
    if (rank_of[i] < 0) continue;
    WarpList<KM> all;
    all.clear();
    for (int o = 0; o < warps; ++o)
      for (int c = 0; c < KM; ++c) {
        const uint64_t key = merged[((int64_t)o * RT + i) * KM + c];
        if (key < all.worst()) all.insert(key);
      }
    const int64_t j = inv ? (int64_t)inv[rank_of[i]] : rank_of[i];
#pragma unroll
    for (int q = 0; q < KM / 32; ++q) {
      const int g = q * 32 + lane;
      if (g < M) {
        const uint64_t key = all.v[q];
        fwd[j * M + g] = key == kEmpty ? -1 : (int32_t)key_index(key);
        fwd_d[j * M + g] = key == kEmpty ? __int_as_float(0x7f800000) : key_dist(key);
      }
    }
  }
}

template <int KM, int KD>
static void launch_exact_rows_t(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, int32_t metric,
                                const int32_t* inv, int32_t mode, const int32_t* rows, int32_t nrows, int32_t M,
                                int32_t* fwd, float* fwd_d, cudaStream_t st) {
  constexpr int RT = 8;
  const int threads = 256;
  const size_t smem = (size_t)RT * dpad * sizeof(float) + (size_t)(threads / 32) * RT * KM * sizeof(uint64_t);
  auto kern = k_exact_rows<KM, RT, KD>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int grid = (int)((nrows + RT - 1) / RT);
  kern<<<grid, threads, smem, st>>>(xw, ids, s, dpad, metric, inv, mode, rows, nrows, M, fwd, fwd_d);
}

void launch_exact_rows(const float* xw, const int32_t* ids, int64_t s, int32_t dpad, int32_t metric, const int32_t* inv,
                       int32_t mode, const int32_t* rows, int32_t nrows, int32_t M, int32_t* fwd, float* fwd_d,
                       cudaStream_t st) {
  if (nrows <= 0) return;
  const int kd = dpad / 32;
  if (M <= 32) {
    if (kd == 1) return launch_exact_rows_t<32, 1>(xw, ids, s, dpad, metric, inv, mode, rows, nrows, M, fwd, fwd_d, st);
    if (kd == 2) return launch_exact_rows_t<32, 2>(xw, ids, s, dpad, metric, inv, mode, rows, nrows, M, fwd, fwd_d, st);
    if (kd == 3) return launch_exact_rows_t<32, 3>(xw, ids, s, dpad, metric, inv, mode, rows, nrows, M, fwd, fwd_d, st);
    if (kd == 4) return launch_exact_rows_t<32, 4>(xw, ids, s, dpad, metric, inv, mode, rows, nrows, M, fwd, fwd_d, st);
    return launch_exact_rows_t<32, 0>(xw, ids, s, dpad, metric, inv, mode, rows, nrows, M, fwd, fwd_d, st);
  }
  if (kd == 4) return launch_exact_rows_t<64, 4>(xw, ids, s, dpad, metric, inv, mode, rows, nrows, M, fwd, fwd_d, st);
  return launch_exact_rows_t<64, 0>(xw, ids, s, dpad, metric, inv, mode, rows, nrows, M, fwd, fwd_d, st);
}

// Query candidates -> exact k results (int64 ids, reported distances).
template <int KP>
__global__ void k_rerank_queries(const float* __restrict__ Q, int64_t nq, const float* __restrict__ X, int32_t dpad,
                                 int32_t metric, const uint64_t* __restrict__ cand, int32_t k,
                                 int64_t* __restrict__ out_ids, float* __restrict__ out_d) {
  const int lane = threadIdx.x & 31;
  for (int64_t q = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; q < nq;
       q += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    WarpList<KP> list;
    list.clear();
    for (int c = 0; c < KP; ++c) {
      uint64_t key = cand[q * KP + c];
      if (key == kEmpty) break;
      uint32_t col = key_index(key);
      float dv = warp_exact_dist(Q + q * dpad, X + (int64_t)col * dpad, dpad, metric);
      list.insert(pack(dv, col));
    }
#pragma unroll
    for (int r = 0; r < KP / 32; ++r) {
      int g = r * 32 + lane;
      if (g < k) {
        uint64_t key = list.v[r];
        bool e = key == kEmpty;
        float dv = e ? __int_as_float(0x7f800000) : key_dist(key);
        out_ids[q * k + g] = e ? -1 : (int64_t)key_index(key);
        out_d[q * k + g] = e ? dv : (metric == HENN_ANGULAR ? dv : sqrtf(dv));
      }
    }
  }
}

void launch_rerank_queries(const float* Q, int64_t nq, const float* X, int32_t dpad, int32_t metric, const uint64_t* cand,
                           int32_t KP, int32_t k, int64_t* out_ids, float* out_d, cudaStream_t st) {
  int grid = (int)((nq + 7) / 8);
  if (grid > 152 * 32) grid = 152 * 32;
  if (grid < 1) grid = 1;
  switch (KP) {
    case 32: k_rerank_queries<32><<<grid, 256, 0, st>>>(Q, nq, X, dpad, metric, cand, k, out_ids, out_d); break;
    case 64: k_rerank_queries<64><<<grid, 256, 0, st>>>(Q, nq, X, dpad, metric, cand, k, out_ids, out_d); break;
    case 128: k_rerank_queries<128><<<grid, 256, 0, st>>>(Q, nq, X, dpad, metric, cand, k, out_ids, out_d); break;
    default: k_rerank_queries<256><<<grid, 256, 0, st>>>(Q, nq, X, dpad, metric, cand, k, out_ids, out_d); break;
  }
}

// max of non-negative floats (bit patterns order like the values)
__global__ void k_max_nonneg(const float* __restrict__ v, int64_t n, float* __restrict__ out) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, v[i]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int*>(out), __float_as_int(m));
}

void launch_max_nonneg(const float* v, int64_t n, float* out, cudaStream_t st) {
  cudaMemsetAsync(out, 0, sizeof(float), st);
  k_max_nonneg<<<152 * 2, 256, 0, st>>>(v, n, out);
}

}  // namespace henn
