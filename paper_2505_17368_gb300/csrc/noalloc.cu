// noalloc.cu -- henn_search_host_noalloc: the batched search for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a process whose device memory is
// owned entirely by another allocator (a serving framework's arena, a
// deep-learning framework's caching pool), or code that must not allocate
// while it runs.  henn_search with host buffers allocates device staging
// and a work counter on every call; this entry point instead uses one
// file-scope device array, kNoAllocScratchBytes large, that every GPU
// loading the library holds until the process exits.  The caller passes
// host queries and host result arrays; the call copies the queries into
// the array, runs the same search kernel, copies the results out and
// synchronises the stream.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>

#include "../../include/henn.h"
#include "common.cuh"
#include "search.cuh"

namespace henn {
void index_search_args(const henn_index* idx, SearchArgs& a, int* device);
void set_last_error(const std::string& msg);
}

using namespace henn;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(16) << 20;  // 16 MiB per GPU
constexpr int kMaxDevices = 64;

// Work counter at offset 0, then query rows, result ids, result distances
// (each region 256-byte aligned).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

henn_status fail(henn_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

}  // namespace

extern "C" henn_status henn_search_host_noalloc(const henn_index* idx, const float* Q, int64_t nq, int32_t k,
                                                int32_t ef, int32_t ef_upper, int64_t* out_ids, float* out_dists,
                                                int32_t out_stride, void* stream) {
  set_last_error("");
  if (!idx || !Q || !out_ids || !out_dists) return fail(HENN_ERR_INVALID_ARG, "NULL argument");
  if (nq < 0) return fail(HENN_ERR_INVALID_ARG, "nq must be >= 0");
  if (k < 1 || k > 1024) return fail(HENN_ERR_INVALID_ARG, "k must be in [1, 1024]");
  if (ef < 1 || ef > 4096) return fail(HENN_ERR_INVALID_ARG, "ef must be in [1, 4096]");
  if (ef_upper < 0 || ef_upper > 4096) return fail(HENN_ERR_INVALID_ARG, "ef_upper must be in [0, 4096]");
  if (out_stride < k) return fail(HENN_ERR_INVALID_ARG, "out_stride must be >= k");
  if (nq == 0) return HENN_OK;
  cudaStream_t st = (cudaStream_t)stream;

  SearchArgs a;
  int device = 0;
  index_search_args(idx, a, &device);
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != device)
    return fail(HENN_ERR_INVALID_ARG, "the index's device must be current");
  if (device < 0 || device >= kMaxDevices) return fail(HENN_ERR_UNSUPPORTED, "device ordinal too large");

  // scratch layout and the size limit
  const size_t q_off = 256;
  const size_t q_bytes = align256((size_t)nq * a.d * sizeof(float));
  const size_t id_off = q_off + q_bytes;
  const size_t id_bytes = align256((size_t)nq * out_stride * sizeof(int64_t));
  const size_t d_off = id_off + id_bytes;
  const size_t d_bytes = align256((size_t)nq * out_stride * sizeof(float));
  if (d_off + d_bytes > kNoAllocScratchBytes)
    return fail(HENN_ERR_INVALID_ARG, "batch needs " + std::to_string(d_off + d_bytes) +
                                          " bytes of scratch; this entry point has " +
                                          std::to_string(kNoAllocScratchBytes) +
                                          " (nq * (4 d + 12 out_stride) must stay below about that)");

  // once per device, with that device current: the array's device address
  // (in host code the symbol itself is only a host-side stand-in)
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[device]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return fail(HENN_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_scratch_addr[device] = p;
    }
    base = static_cast<unsigned char*>(g_scratch_addr[device]);
  }
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(base);
  float* dq = reinterpret_cast<float*>(base + q_off);
  int64_t* dids = reinterpret_cast<int64_t*>(base + id_off);
  float* dd = reinterpret_cast<float*>(base + d_off);

  // beam capacity, visited table and grid by the rules henn_search uses
  // (search.cuh), with henn_search's default rerank multiplier
  henn_search_params defaults;
  henn_search_params_default(&defaults);
  const int ef_cap = search_beam_cap(k, ef, ef_upper, 0, a.rerank != 0, defaults.rerank_mult);
  const int hb = search_hash_bits(ef_cap);
  a.rerank_mult = defaults.rerank_mult;
  a.Q = dq;
  a.nq = nq;
  a.kq = nullptr;
  a.efq = nullptr;
  a.k_uniform = k;
  a.ef_uniform = ef;
  a.ef_upper = ef_upper;
  a.descend_all = 0;
  a.ef_cap = ef_cap;
  a.hash_bits = hb;
  a.keys = nullptr;
  a.out_ids = dids;
  a.out_d = dd;
  a.out_stride = out_stride;
  a.stats = nullptr;
  a.counter = counter;

  const int warps = kSearchWarps;
  const size_t smem = search_warp_smem(ef_cap, hb, a.dpad) * warps;
  int grid = 0;
  cudaError_t e = search_persistent_grid(device, warps, smem, &grid);
  if (e != cudaSuccess) return fail(HENN_ERR_CUDA, cudaGetErrorString(e));
  const long long blocks = (nq + warps - 1) / warps;
  if (blocks < grid) grid = (int)blocks;

  // the work counter must start at zero on every call; everything else is
  // overwritten before it is read
  if ((e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(dq, Q, (size_t)nq * a.d * sizeof(float), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = launch_search(a, warps, grid, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(out_ids, dids, (size_t)nq * out_stride * sizeof(int64_t), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(out_dists, dd, (size_t)nq * out_stride * sizeof(float), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(HENN_ERR_CUDA, cudaGetErrorString(e));
  return HENN_OK;
}
