// henn_abi.cu -- host orchestration behind the C ABI of include/henn.h.
//
// BuildHENN (Alg. 1) runs layer by layer: membership first (Alg. 2 draws,
// ring-range verification, Las-Vegas retries; the only device->host reads
// are the layer size and the ring verdicts of each attempt), then every
// layer's navigable graph (tiles + top-KP, exact FP32 rerank, edge rule) and
// its traversal copy.  Search is one persistent kernel per batch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <exception>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/henn.h"
#include "common.cuh"
#include "kernels.cuh"
#include "search.cuh"

using namespace henn;

namespace {

thread_local std::string g_error;

struct Failure : std::exception {
  henn_status status;
  std::string msg;
  Failure(henn_status s, std::string m) : status(s), msg(std::move(m)) {}
};

void check(cudaError_t e, const char* what, int line) {
  if (e == cudaSuccess) return;
  henn_status s = (e == cudaErrorMemoryAllocation) ? HENN_ERR_OOM : HENN_ERR_CUDA;
  throw Failure(s, std::string(what) + " (line " + std::to_string(line) + "): " + cudaGetErrorString(e));
}
#define CK(x) check((x), #x, __LINE__)
#define CKL(what) check(cudaGetLastError(), what, __LINE__)

void require(bool ok, const std::string& msg) {
  if (!ok) throw Failure(HENN_ERR_INVALID_ARG, msg);
}

// The device address of a host buffer in page-locked memory the device can
// address (cudaHostAlloc / cudaMallocHost, or registered with mapping), else
// nullptr (pageable memory, which has to be staged).
static void* mapped_host(const void* p) {
  cudaPointerAttributes at;
  if (p == nullptr || cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // clear the failed query's error
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Stream-ordered scratch allocation, released when the owner goes out of
// scope (also on failure).
struct Scratch {
  cudaStream_t st;
  cudaMemPool_t pool;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s, cudaMemPool_t p = nullptr) : st(s), pool(p) {}
  template <typename T>
  T* get(size_t count) {
    void* p = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = 16;
    if (pool)
      CK(cudaMallocFromPoolAsync(&p, bytes, pool, st));
    else
      CK(cudaMallocAsync(&p, bytes, st));
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
};

// Build tracing: with HENN_TRACE=1 in the environment, henn_build prints the
// wall time of each step to stderr, measured after synchronising the build
// stream (so the steps no longer overlap while tracing), and the number of
// rows that needed the exact recompute.
struct BuildTrace {
  bool on = false;
  cudaStream_t st = nullptr;
  std::chrono::steady_clock::time_point t;
  explicit BuildTrace(cudaStream_t s) : st(s), t(std::chrono::steady_clock::now()) {
    const char* e = std::getenv("HENN_TRACE");
    on = e && std::atoi(e) > 0;
  }
  void mark(const char* what, int32_t layer, int64_t count = -1) {
    if (!on) return;
    cudaStreamSynchronize(st);
    auto n = std::chrono::steady_clock::now();
    std::fprintf(stderr, "[henn build] layer %d %-22s %9.3f ms", layer, what,
                 std::chrono::duration<double, std::milli>(n - t).count());
    if (count >= 0) std::fprintf(stderr, "  (%lld)", (long long)count);
    std::fprintf(stderr, "\n");
    t = n;
  }
};

// One build step run as a CUDA graph, again and again: each run captures
// the launches f() enqueues on st (not the legacy default stream; device
// memory used inside is allocated before the capture) and launches them as
// one graph.  The executable graph is kept: a capture with the same
// topology (the next epsilon-net attempt, the next layer -- only kernel
// arguments, grid sizes and copy sizes differ) updates it in place, which
// costs far less than instantiating; a different topology instantiates anew.
struct CapturedGraph {
  cudaGraphExec_t exec = nullptr;
  int32_t instantiations = 0, updates = 0;
  CapturedGraph() = default;
  CapturedGraph(const CapturedGraph&) = delete;
  CapturedGraph& operator=(const CapturedGraph&) = delete;
  ~CapturedGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
  template <class F>
  void run(cudaStream_t st, F&& f) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      f();
    } catch (...) {
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    CK(cudaStreamEndCapture(st, &g));
    bool updated = false;
    if (exec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(exec, g, &info) == cudaSuccess) {
        updated = true;
      } else {
        cudaGetLastError();  // an update refused for topology is not an error
        cudaGraphExecDestroy(exec);
        exec = nullptr;
      }
    }
    cudaError_t e = cudaSuccess;
    if (updated) {
      ++updates;
    } else {
      e = cudaGraphInstantiate(&exec, g, 0);
      if (e == cudaSuccess) ++instantiations;
      else exec = nullptr;
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    cudaGraphDestroy(g);
    CK(e);
  }
};

int64_t ring_window(double c0, int32_t d, int64_t s, int32_t m) {
  // eps(s) * s with eps from Eq. 1 (natural log), evaluated as
  // ((c0 * d) * log(s)) * 2^m; heavy rings hold floor(eps*s)+1 points.
  volatile double es = c0 * (double)d;
  es = es * std::log((double)s);
  es = es * (double)(1LL << m);
  if (!(es < (double)s)) return s + 1;
  return (int64_t)std::floor(es) + 1;
}

int32_t round_up(int32_t v, int32_t m) { return (v + m - 1) / m * m; }

// Relative error bound (per unit of sum |a_i b_i|) of a split-BF16 tile dot
// product over dk values: each product hi.hi + lo.hi + hi.lo misses lo.lo
// and the rounding of lo, 3 * 2^-18 of |a_i b_i|; the products themselves
// are exact in FP32 (8-bit significands).  The tensor core sums them as a
// blocked sum: 16 products per MMA (at most 15 additions inside a block),
// then one accumulation into the FP32 accumulator per MMA, 3 * dk / 16 MMAs
// in all, each addition with a relative error of at most 2^-24, doubled to
// allow for truncation instead of rounding inside the tensor core.
double tc_tile_unit_error(int32_t dk) {
  return 3.0 * std::ldexp(1.0, -18) + 2.0 * (15.0 + 3.0 * dk / 16.0 + 8.0) * std::ldexp(1.0, -24);
}

}  // namespace

// ----------------------------------------------------------- the index

struct LayerDev {
  int64_t size = 0;
  int64_t cap = 0;          // rows the arrays below hold (insertions grow it)
  int32_t* ids = nullptr;   // global ids (layers >= 1)
  int32_t* down = nullptr;  // positions in the layer below (layers >= 1)
  int32_t* adj = nullptr;   // size x 32
  int32_t* fwd = nullptr;   // size x M
  float* fwd_d = nullptr;   // size x M
  void* vec = nullptr;      // traversal vectors, layer order
  float* vscale = nullptr;  // FP8 per-row scales
};

struct henn_index {
  int64_t n = 0;
  int64_t cap_n = 0;  // rows x32 / xw / inv_norm hold
  int32_t m = 4;      // layer decay 2^m of the build
  int32_t d = 0, dpad = 0, metric = 0, storage = 0, graph = 0, M = 16, Mmax = 32;
  uint64_t seed = 0;
  int32_t L = 0;
  std::vector<LayerDev> layers;
  std::vector<int32_t> attempts, ambiguous;
  float* x32 = nullptr;  // raw vectors, rows of dpad
  float* xw = nullptr;   // working vectors: x32 (l2) or unit rows (angular)
  float* inv_norm = nullptr;
  uint8_t* dead = nullptr;  // 1 per deleted point (allocated at the first delete)
  int64_t n_dead = 0;
  SearchLayer* d_layers = nullptr;
  std::vector<void*> allocs;
  int64_t bytes = 0;
  int64_t uncertified = 0;
  double build_seconds = 0.0;
  double tile_seconds = 0.0, tile_flops = 0.0;
  int32_t tile_engine = 0;
  int32_t graph_instantiations = 0, graph_updates = 0;
  henn_build_params params;  // as the build validated them (delete's resampling reuses them)
  int device = 0;

  template <typename T>
  T* alloc(size_t count) {
    void* p = nullptr;
    size_t b = count * sizeof(T);
    if (b == 0) b = 16;
    CK(cudaMalloc(&p, b));
    allocs.push_back(p);
    bytes += (int64_t)b;
    return static_cast<T*>(p);
  }
  // frees one allocation made by alloc() (device idle for it)
  void release(void* p) {
    if (!p) return;
    for (size_t i = 0; i < allocs.size(); ++i)
      if (allocs[i] == p) {
        cudaFree(p);
        allocs.erase(allocs.begin() + (long)i);
        return;
      }
  }
  // side streams for the concurrent per-class launches of one batch
  // (created on first use)
  mutable std::mutex side_mu;
  mutable std::vector<cudaStream_t> side;
  // Tile operands of an exact upper layer (exact_method TILES), made at its
  // first use: the layer's traversal rows as FP32 minus their mean, split
  // into BF16 planes (tcgen05) or kept as FP32 rows (SIMT), their squared
  // norms and the largest of them.
  struct EntryOps {
    int64_t size = 0;    // 0: not made
    int32_t engine = 0;  // HENN_TILES_TCGEN05 or HENN_TILES_SIMT
    void* hi = nullptr;
    void* lo = nullptr;
    alignas(64) unsigned char maps[512];  // tensor maps of hi / lo for 256- and 128-column tiles (tcgen05)
    float* xo = nullptr;
    float* mean = nullptr;
    float* norms = nullptr;
    float* nmax = nullptr;
    std::vector<void*> mem;
  };
  mutable std::mutex entry_mu;
  mutable std::vector<EntryOps> entry;
  void drop_entry_ops() const {
    std::lock_guard<std::mutex> lk(entry_mu);
    for (EntryOps& e : entry)
      for (void* p : e.mem) cudaFree(p);
    entry.clear();
  }
  // search scratch comes from this pool, which keeps its memory between
  // calls (created on first use)
  mutable std::mutex pool_mu;
  mutable cudaMemPool_t pool = nullptr;
  cudaMemPool_t search_pool() const {
    std::lock_guard<std::mutex> lk(pool_mu);
    if (!pool) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = device;
      CK(cudaMemPoolCreate(&pool, &props));
      uint64_t keep = UINT64_MAX;
      CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
    }
    return pool;
  }
  // events of the last search with time_kernel = 1
  mutable std::mutex time_mu;
  mutable cudaEvent_t tev[2] = {nullptr, nullptr};
  mutable int32_t t_launches = 0;
  mutable bool t_valid = false;
  ~henn_index() {
    drop_entry_ops();
    if (pool) {
      cudaDeviceSynchronize();
      cudaMemPoolDestroy(pool);
    }
    for (cudaEvent_t e : tev)
      if (e) cudaEventDestroy(e);
    for (cudaStream_t t : side) cudaStreamDestroy(t);
    for (void* p : allocs) cudaFree(p);
  }
};

// ------------------------------------------------------------ defaults

extern "C" void henn_build_params_default(henn_build_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(henn_build_params);
  p->metric = HENN_L2;
  p->storage = HENN_F32;
  p->graph = HENN_GRAPH_NSW;
  p->m = 4;
  p->max_layers = 0;
  p->eps_c0 = 1.0;
  p->num_ranges = 100;
  p->max_attempts = 64;
  p->M = 16;
  p->Mmax = 32;
  p->tiles = HENN_TILES_AUTO;
  p->seed = 0;
  p->sampler = HENN_SAMPLER_SAMPLING;
  p->resample_share = 0.5;
}

extern "C" void henn_search_params_default(henn_search_params* sp) {
  if (!sp) return;
  std::memset(sp, 0, sizeof(*sp));
  sp->struct_size = sizeof(henn_search_params);
  sp->k_uniform = 10;
  sp->ef_uniform = 64;
  sp->rerank_mult = 4;
  sp->ef_upper = 1;
}

extern "C" const char* henn_last_error(void) { return g_error.c_str(); }

// --------------------------------------------------------------- build

namespace {

// Alg. 2 for one layer: returns the accepted attempt; fills pos/ids.
int32_t build_layer_membership(henn_index* ix, const henn_build_params& p, int32_t layer, int64_t s,
                               const int32_t* prev_ids, Scratch& sc, uint8_t* flags, int64_t* tile_buf,
                               int64_t* d_total, int32_t* pos, int32_t* ids, int64_t* out_count,
                               int32_t* out_ambiguous, CapturedGraph& graph, cudaStream_t st) {
  const int64_t decay = 1LL << p.m;
  const int64_t t = (s + decay - 1) / decay;
  const int64_t w = ring_window(p.eps_c0, ix->d, s, p.m);
  const int32_t r = p.num_ranges;
  int32_t* centre = sc.get<int32_t>(r);
  int64_t* start = sc.get<int64_t>(r);
  float* lo = sc.get<float>(r);
  float* hi = sc.get<float>(r);
  int32_t* status = sc.get<int32_t>(r);
  float* D = (w <= s) ? sc.get<float>((size_t)r * s) : nullptr;
  double* D64 = nullptr;
  double* bounds = sc.get<double>(2);
  // certified FP32 error model of the ring distances (see layers.cu)
  const double u = std::ldexp(1.0, -24);
  double er = 0.0, ea = 0.0;
  if (ix->metric == HENN_ANGULAR)
    ea = (4.0 * ix->dpad + 64.0) * u;
  else
    er = (ix->dpad + 16.0) * u + 1e-12;
  std::vector<int32_t> h_status(r), h_centre(r);
  std::vector<int64_t> h_start(r);
  int32_t ambiguous = 0;
  for (int32_t a = 0; a < p.max_attempts; ++a) {
    // one attempt of Alg. 2 as one captured graph: draws, compaction and,
    // when heavy rings exist, the r ring checks; then one read-back
    const uint64_t base = derive(derive(derive(ix->seed, HENN_TAG_SAMPLE), (uint64_t)layer), (uint64_t)a);
    const uint64_t bc = derive(derive(derive(ix->seed, HENN_TAG_RCENTRE), (uint64_t)layer), (uint64_t)a);
    const uint64_t bs = derive(derive(derive(ix->seed, HENN_TAG_RSTART), (uint64_t)layer), (uint64_t)a);
    graph.run(st, [&] {
      CK(cudaMemsetAsync(flags, 0, (size_t)s, st));
      LayerSampleArgs la;
      la.base = base;
      la.s = s;
      la.t = t;
      la.flags = flags;
      launch_sample(la, st);
      launch_compact(flags, s, prev_ids, tile_buf, d_total, pos, ids, st);
      CKL("sample/compact");
      if (w <= s) {
        launch_ring_params(bc, bs, r, s, s - w + 1, centre, start, st);
        launch_ring_dist(ix->x32, ix->dpad, prev_ids, s, centre, r, ix->metric, ix->inv_norm, D, st);
        launch_ring_select_decide(D, s, start, w, r, pos, d_total, er, ea, lo, hi, status, st);
        CKL("ring checks");
      }
    });
    int64_t count = 0;
    CK(cudaMemcpyAsync(&count, d_total, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    bool pass = true;
    if (w <= s) {
      CK(cudaMemcpyAsync(h_status.data(), status, sizeof(int32_t) * r, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      for (int32_t q = 0; q < r; ++q)
        if (h_status[q] == kRingFail) pass = false;
      if (pass) {
        bool fetched = false;
        for (int32_t q = 0; q < r && pass; ++q) {
          if (h_status[q] != kRingAmbiguous) continue;
          if (!fetched) {
            CK(cudaMemcpyAsync(h_centre.data(), centre, sizeof(int32_t) * r, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(h_start.data(), start, sizeof(int64_t) * r, cudaMemcpyDeviceToHost, st));
            if (!D64) D64 = sc.get<double>((size_t)s);
            fetched = true;
          }
          ++ambiguous;
          launch_ring_recheck(ix->x32, ix->d, ix->dpad, prev_ids, s, h_centre[q], h_start[q], w, ix->metric, pos,
                              count, D64, bounds, status, q, st);
          CKL("ring FP64 recheck");
          int32_t v = 0;
          CK(cudaMemcpyAsync(&v, status + q, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
          CK(cudaStreamSynchronize(st));
          if (v != kRingPass) pass = false;
        }
      }
    } else {
      CK(cudaStreamSynchronize(st));
    }
    if (pass) {
      *out_count = count;
      *out_ambiguous = ambiguous;
      return a;
    }
  }
  return -1;
}

// Membership of layers first_layer, first_layer + 1, ... (Alg. 1 with Alg. 2
// or Alg. 3) on top of a layer of s0 points whose global ids are prev_ids
// (device, ascending; nullptr: the points 0..s0-1), appended to ix->layers
// with their down pointers (positions in prev_ids for the first); stops as
// the build does (|L| < 2^m or max_layers).
void build_membership(henn_index* ix, const henn_build_params& p, int32_t first_layer, const int32_t* prev_ids,
                      int64_t s0, CapturedGraph& attempt_graph, BuildTrace& tr, cudaStream_t st) {
  Scratch sc(st);
  uint8_t* flags = sc.get<uint8_t>(s0);
  int64_t* tile_buf = sc.get<int64_t>((size_t)scan_tiles(s0) + 1);
  int64_t* d_total = sc.get<int64_t>(1);
  int32_t* pos = sc.get<int32_t>(s0);
  int32_t* ids = sc.get<int32_t>(s0);
  const int64_t decay = 1LL << p.m;
  const int32_t* prev = prev_ids;
  int64_t s = s0;
  for (int32_t layer = first_layer; layer < HENN_MAX_LAYERS; ++layer) {
    if (p.max_layers > 0 && layer > p.max_layers) break;
    if (s < decay) break;
    int64_t count = 0;
    int32_t amb = 0;
    int32_t a = 0;
    if (p.sampler == HENN_SAMPLER_HALVING) {
      // Alg. 3 (BuildEpsNetDiscV2): m halving steps, no verification;
      // `ids` doubles as the ping-pong buffer until the ids are written
      count = launch_halving(ix->seed, layer, s, p.m, prev, ids, pos, ids, st);
      CKL("halving");
    } else {
      a = build_layer_membership(ix, p, layer, s, prev, sc, flags, tile_buf, d_total, pos, ids, &count, &amb,
                                 attempt_graph, st);
    }
    if (a < 0)
      throw Failure(HENN_ERR_EPSNET_NOT_FOUND, "no eps-net for layer " + std::to_string(layer) + " within max_attempts");
    LayerDev Ly;
    Ly.size = count;
    Ly.ids = ix->alloc<int32_t>(count);
    Ly.down = ix->alloc<int32_t>(count);
    CK(cudaMemcpyAsync(Ly.ids, ids, sizeof(int32_t) * count, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(Ly.down, pos, sizeof(int32_t) * count, cudaMemcpyDeviceToDevice, st));
    ix->layers.push_back(Ly);
    ix->attempts.push_back(a);
    ix->ambiguous.push_back(amb);
    tr.mark("membership", layer);
    prev = Ly.ids;
    s = count;
  }
  CK(cudaStreamSynchronize(st));
}

void build_layer_graph(henn_index* ix, const henn_build_params& p, int32_t li, CapturedGraph& graph, cudaStream_t st,
                       BuildTrace& tr) {
  LayerDev& Ly = ix->layers[li];
  const int64_t s = Ly.size;
  const int32_t dpad = ix->dpad, M = ix->M;
  Scratch sc(st);
  // insertion order and centred operand
  int64_t chunks = (s + 4095) / 4096;
  float* partial = sc.get<float>((size_t)chunks * dpad);
  float* mean = sc.get<float>(dpad);
  launch_layer_mean(ix->xw, Ly.ids, s, dpad, partial, mean, st);
  int32_t* inv = sc.get<int32_t>(s);
  float* xo = sc.get<float>((size_t)s * dpad);
  float* norms = sc.get<float>(s);
  launch_order_gather(ix->xw, Ly.ids, s, dpad, ix->seed, li, ix->graph, mean, inv, xo, norms, st);
  CKL("order/gather");
  float* nmax = sc.get<float>(1);
  launch_max_nonneg(norms, s, nmax, st);
  tr.mark("mean/order/norms", li);
  // tiles + top-KP
  const int32_t KP = M <= 16 ? 32 : (M <= 48 ? 64 : 128);
  uint64_t* cand = sc.get<uint64_t>((size_t)s * KP);
  const int32_t mode = ix->graph == HENN_GRAPH_KNN ? 1 : 0;
  const bool tc_ok = tc_tiles_supported(dpad, KP);
  if (p.tiles == HENN_TILES_TCGEN05 && !tc_ok)
    throw Failure(HENN_ERR_UNSUPPORTED, "tcgen05 tiles need M <= 16");
  const bool use_tc = tc_ok && p.tiles != HENN_TILES_SIMT;
  double tile_u;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  CK(cudaEventCreate(&ev0));
  CK(cudaEventCreate(&ev1));
  CK(cudaEventRecord(ev0, st));
  if (use_tc) {
    const int32_t dk = (dpad + 63) / 64 * 64;
    void* hi = sc.get<uint16_t>((size_t)s * dk);
    void* lo = sc.get<uint16_t>((size_t)s * dk);
    int32_t* err = sc.get<int32_t>(1);
    CK(cudaMemsetAsync(err, 0, sizeof(int32_t), st));
    CK(launch_tile_topk_tc(xo, norms, s, dpad, mode, cand, hi, lo, err, st));
    int32_t herr = 0;
    CK(cudaMemcpyAsync(&herr, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr) throw Failure(HENN_ERR_TIMEOUT, "tensor-core tile pipeline wait timed out (code " + std::to_string(herr) + ")");
    tile_u = tc_tile_unit_error(dk);
  } else {
    launch_tile_topk_simt(xo, norms, s, xo, norms, s, dpad, mode, KP, 1, cand, st);
    CKL("distance tiles");
    tile_u = (dpad + 8.0) * std::ldexp(1.0, -24);
  }
  CK(cudaEventRecord(ev1, st));
  CK(cudaEventSynchronize(ev1));
  float tile_ms = 0.f;
  CK(cudaEventElapsedTime(&tile_ms, ev0, ev1));
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  ix->tile_seconds += tile_ms * 1e-3;
  const double pairs = mode == 0 ? 0.5 * (double)s * (double)(s - 1) : (double)s * (double)(s - 1);
  ix->tile_flops += pairs * 2.0 * ix->d;
  if (li == 0) ix->tile_engine = use_tc ? HENN_TILES_TCGEN05 : HENN_TILES_SIMT;
  tr.mark("tiles + top-k", li);
  int32_t* unc = sc.get<int32_t>((size_t)s + 1);
  CK(cudaMemsetAsync(unc, 0, sizeof(int32_t), st));
  launch_rerank_fwd(ix->xw, Ly.ids, s, dpad, ix->metric, inv, cand, KP, M, norms, nmax, tile_u, Ly.fwd, Ly.fwd_d, unc,
                    st);
  CKL("rerank");
  int32_t nunc = 0;
  CK(cudaMemcpyAsync(&nunc, unc, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (nunc > 0) {
    launch_exact_rows(ix->xw, Ly.ids, s, dpad, ix->metric, inv, mode, unc + 1, nunc, M, Ly.fwd, Ly.fwd_d, st);
    CKL("exact rows");
    ix->uncertified += nunc;
  }
  tr.mark("rerank/certify", li, nunc);
  // edge rule and traversal copy (layer order) as one captured graph;
  // every buffer is allocated before the capture
  int32_t* cnt = sc.get<int32_t>(s);
  int32_t* fill = sc.get<int32_t>(s);
  int64_t* off = sc.get<int64_t>((size_t)s + 1);
  int64_t* tiles = sc.get<int64_t>((size_t)scan_tiles(s) + 1);
  uint64_t* rev = sc.get<uint64_t>((size_t)s * M);
  float* gathered = nullptr;
  if (li > 0)
    gathered = (ix->storage == HENN_F32) ? ix->alloc<float>((size_t)s * dpad) : sc.get<float>((size_t)s * dpad);
  if (ix->storage == HENN_F32) {
    Ly.vec = li > 0 ? (void*)gathered : (void*)ix->xw;
  } else if (ix->storage == HENN_BF16) {
    Ly.vec = ix->alloc<uint16_t>((size_t)s * dpad);
  } else {
    Ly.vec = ix->alloc<uint8_t>((size_t)s * dpad);
    Ly.vscale = ix->alloc<float>(s);
  }
  graph.run(st, [&] {
    CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * s, st));
    CK(cudaMemsetAsync(fill, 0, sizeof(int32_t) * s, st));
    launch_rev_count(Ly.fwd, s, M, cnt, st);
    launch_offsets(cnt, s, tiles, off, st);
    launch_rev_fill(Ly.fwd, Ly.fwd_d, s, M, off, fill, rev, st);
    launch_select_adj(Ly.fwd, Ly.fwd_d, s, M, off, rev, ix->graph, Ly.adj, st);
    CKL("edge rule");
    const float* src = ix->xw;
    if (li > 0) {
      launch_gather_rows32(ix->xw, Ly.ids, s, dpad, gathered, st);
      src = gathered;
    }
    if (ix->storage == HENN_BF16)
      launch_quantize(src, s, dpad, dpad, dpad, HENN_BF16, Ly.vec, nullptr, st);
    else if (ix->storage == HENN_FP8E4M3)
      launch_quantize(src, s, dpad, dpad, dpad, HENN_FP8E4M3, Ly.vec, Ly.vscale, st);
    CKL("traversal copy");
  });
  CK(cudaStreamSynchronize(st));
  tr.mark("edge rule + copy", li);
}

}  // namespace

extern "C" henn_status henn_build(const float* X, int64_t n, int32_t d, int32_t x_on_device, const henn_build_params* pp,
                                  void* stream, henn_index** out) {
  g_error.clear();
  if (out) *out = nullptr;
  henn_index* ix = nullptr;
  try {
    auto t0 = std::chrono::steady_clock::now();
    require(out != nullptr, "out is NULL");
    require(X != nullptr, "X is NULL");
    require(n >= 1 && n < (1LL << 31), "n must be in [1, 2^31)");
    require(d >= 1 && d <= kMaxD, "d must be in [1, 1024]");
    henn_build_params p;
    henn_build_params_default(&p);
    if (pp) {
      require(pp->struct_size == sizeof(henn_build_params), "henn_build_params.struct_size mismatch");
      p = *pp;
    }
    require(p.metric == HENN_L2 || p.metric == HENN_ANGULAR, "metric");
    require(p.storage >= HENN_F32 && p.storage <= HENN_FP8E4M3, "storage");
    require(p.graph == HENN_GRAPH_NSW || p.graph == HENN_GRAPH_KNN, "graph");
    require(p.m >= 1 && p.m <= 8, "m must be in [1, 8]");
    require(p.sampler == HENN_SAMPLER_SAMPLING || p.sampler == HENN_SAMPLER_HALVING, "sampler");
    require(p.max_layers >= 0 && p.max_layers < HENN_MAX_LAYERS, "max_layers");
    require(p.eps_c0 > 0.0 && std::isfinite(p.eps_c0), "eps_c0 must be > 0");
    require(p.num_ranges >= 1 && p.num_ranges <= 4096, "num_ranges must be in [1, 4096]");
    require(p.max_attempts >= 1 && p.max_attempts <= 100000, "max_attempts");
    require(p.M >= 1 && p.M <= 32, "M must be in [1, 32]");
    require(std::isfinite(p.resample_share), "resample_share must be finite");
    require(p.Mmax == 32, "Mmax must be 32");
    // The build runs on its own non-blocking stream (the legacy default
    // stream cannot be captured into graphs), after the caller's stream
    // has produced X; it synchronises before returning.
    cudaStream_t ust = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(ust));
    struct OwnStream {
      cudaStream_t s = nullptr;
      ~OwnStream() {
        if (s) {
          cudaStreamSynchronize(s);
          cudaStreamDestroy(s);
        }
      }
    } own;
    CK(cudaStreamCreateWithFlags(&own.s, cudaStreamNonBlocking));
    cudaStream_t st = own.s;
    BuildTrace tr(st);

    ix = new henn_index();
    ix->params = p;
    CK(cudaGetDevice(&ix->device));
    ix->n = n;
    ix->d = d;
    ix->dpad = round_up(d, 32);
    ix->metric = p.metric;
    ix->storage = p.storage;
    ix->graph = p.graph;
    ix->M = p.M;
    ix->Mmax = p.Mmax;
    ix->seed = p.seed;
    ix->m = p.m;
    const int32_t dpad = ix->dpad;

    // FP32 master copy with zero padding
    ix->x32 = ix->alloc<float>((size_t)n * dpad);
    ix->cap_n = n;
    CK(cudaMemsetAsync(ix->x32, 0, sizeof(float) * (size_t)n * dpad, st));
    CK(cudaMemcpy2DAsync(ix->x32, sizeof(float) * dpad, X, sizeof(float) * d, sizeof(float) * d, (size_t)n,
                         x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    ix->xw = ix->x32;
    if (p.metric == HENN_ANGULAR) {
      ix->inv_norm = ix->alloc<float>(n);
      launch_inv_norms(ix->x32, n, dpad, ix->inv_norm, st);
      ix->xw = ix->alloc<float>((size_t)n * dpad);
      launch_normalise(ix->x32, ix->inv_norm, n, dpad, ix->xw, st);
      CKL("normalise");
    }

    tr.mark("input copy", 0);
    // ---- layer membership (Alg. 1 + Alg. 2)
    ix->layers.push_back(LayerDev());
    ix->layers[0].size = n;
    ix->attempts.push_back(0);
    ix->ambiguous.push_back(0);
    CapturedGraph attempt_graph, layer_graph;
    build_membership(ix, p, 1, nullptr, n, attempt_graph, tr, st);
    ix->L = (int32_t)ix->layers.size() - 1;

    // ---- navigable graph + traversal copy per layer
    for (int32_t li = 0; li <= ix->L; ++li) {
      LayerDev& Ly = ix->layers[li];
      Ly.cap = Ly.size;
      Ly.adj = ix->alloc<int32_t>((size_t)Ly.size * kMmax);
      Ly.fwd = ix->alloc<int32_t>((size_t)Ly.size * ix->M);
      Ly.fwd_d = ix->alloc<float>((size_t)Ly.size * ix->M);
      build_layer_graph(ix, p, li, layer_graph, st, tr);
      tr.mark("scratch release", li);
    }
    ix->graph_instantiations = attempt_graph.instantiations + layer_graph.instantiations;
    ix->graph_updates = attempt_graph.updates + layer_graph.updates;

    // ---- search-side layer table
    std::vector<SearchLayer> h(ix->L + 1);
    for (int32_t li = 0; li <= ix->L; ++li) {
      h[li].adj = ix->layers[li].adj;
      h[li].vec = ix->layers[li].vec;
      h[li].scale = ix->layers[li].vscale;
      h[li].down = ix->layers[li].down;
      h[li].size = ix->layers[li].size;
    }
    ix->d_layers = ix->alloc<SearchLayer>(h.size());
    CK(cudaMemcpyAsync(ix->d_layers, h.data(), sizeof(SearchLayer) * h.size(), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    ix->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = ix;
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    delete ix;
    return f.status;
  } catch (const std::exception& e) {
    g_error = e.what();
    delete ix;
    return HENN_ERR_CUDA;
  }
}

extern "C" void henn_free(henn_index* idx) { delete idx; }

// ---------------------------------------------------------------- delete

namespace {

// The search-side layer table of ix (device), rewritten from ix->layers;
// reallocated when the number of layers changed.
void upload_layer_table(henn_index* ix, cudaStream_t st) {
  std::vector<SearchLayer> h(ix->L + 1);
  for (int32_t li = 0; li <= ix->L; ++li) {
    h[li].adj = ix->layers[li].adj;
    h[li].vec = ix->layers[li].vec;
    h[li].scale = ix->layers[li].vscale;
    h[li].down = ix->layers[li].down;
    h[li].size = ix->layers[li].size;
  }
  ix->release(ix->d_layers);
  ix->d_layers = ix->alloc<SearchLayer>(h.size());
  CK(cudaMemcpyAsync(ix->d_layers, h.data(), sizeof(SearchLayer) * h.size(), cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));
}

// Layer i resampled from the live points of layer i - 1 (global ids
// liveids, at positions livepos of layer i - 1) and every layer above it
// rebuilt: membership (Alg. 1 + Alg. 2 or Alg. 3, the build's seed and
// layer numbers), down pointers into layer i - 1's arrays (which keep
// their dead entries), graphs and traversal copies.
void rebuild_from(henn_index* ix, int32_t i, const std::vector<int32_t>& liveids, const std::vector<int32_t>& livepos) {
  const henn_build_params& p = ix->params;
  struct OwnStream {
    cudaStream_t s = nullptr;
    ~OwnStream() {
      if (s) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    }
  } own;
  CK(cudaStreamCreateWithFlags(&own.s, cudaStreamNonBlocking));
  cudaStream_t st = own.s;
  BuildTrace tr(st);
  ix->drop_entry_ops();
  for (int32_t li = ix->L; li >= i; --li) {
    LayerDev& Ly = ix->layers[li];
    for (void* q : {(void*)Ly.ids, (void*)Ly.down, (void*)Ly.adj, (void*)Ly.fwd, (void*)Ly.fwd_d, Ly.vec,
                    (void*)Ly.vscale})
      ix->release(q);
  }
  ix->layers.resize(i);
  ix->attempts.resize(i);
  ix->ambiguous.resize(i);
  {
    Scratch sc(st);
    int32_t* prev = sc.get<int32_t>(liveids.size());
    CK(cudaMemcpyAsync(prev, liveids.data(), sizeof(int32_t) * liveids.size(), cudaMemcpyHostToDevice, st));
    CapturedGraph attempt_graph;
    build_membership(ix, p, i, prev, (int64_t)liveids.size(), attempt_graph, tr, st);
  }
  if ((int32_t)ix->layers.size() > i) {
    // the first new layer's down pointers: positions in the live list -> in layer i - 1
    LayerDev& F = ix->layers[i];
    std::vector<int32_t> dn((size_t)F.size);
    CK(cudaMemcpyAsync(dn.data(), F.down, sizeof(int32_t) * dn.size(), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int32_t& v : dn) v = livepos[(size_t)v];
    CK(cudaMemcpyAsync(F.down, dn.data(), sizeof(int32_t) * dn.size(), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
  }
  ix->L = (int32_t)ix->layers.size() - 1;
  CapturedGraph layer_graph;
  for (int32_t li = i; li <= ix->L; ++li) {
    LayerDev& Ly = ix->layers[li];
    Ly.cap = Ly.size;
    Ly.adj = ix->alloc<int32_t>((size_t)Ly.size * kMmax);
    Ly.fwd = ix->alloc<int32_t>((size_t)Ly.size * ix->M);
    Ly.fwd_d = ix->alloc<float>((size_t)Ly.size * ix->M);
    build_layer_graph(ix, p, li, layer_graph, st, tr);
  }
  upload_layer_table(ix, st);
}

// Delete of App. C after the tombstones are set: the lowest upper layer i
// whose live points number fewer than resample_share * ceil(live(L_{i-1}) /
// 2^m) is resampled from the live points of layer i - 1 and the hierarchy
// rebuilt above it.  Reads the tombstones and the layers' ids to the host.
void resample_after_delete(henn_index* ix) {
  const henn_build_params& p = ix->params;
  if (!(p.resample_share > 0.0) || ix->L < 1 || !ix->dead) return;
  std::vector<uint8_t> dead((size_t)ix->n);
  CK(cudaMemcpy(dead.data(), ix->dead, (size_t)ix->n, cudaMemcpyDeviceToHost));
  std::vector<int32_t> below((size_t)ix->n), cur;
  for (int64_t j = 0; j < ix->n; ++j) below[(size_t)j] = (int32_t)j;
  for (int32_t i = 1; i <= ix->L; ++i) {
    cur.resize((size_t)ix->layers[i].size);
    CK(cudaMemcpy(cur.data(), ix->layers[i].ids, sizeof(int32_t) * cur.size(), cudaMemcpyDeviceToHost));
    std::vector<int32_t> livepos, liveids;
    for (size_t j = 0; j < below.size(); ++j)
      if (!dead[(size_t)below[j]]) {
        livepos.push_back((int32_t)j);
        liveids.push_back(below[j]);
      }
    int64_t live_i = 0;
    for (int32_t v : cur) live_i += dead[(size_t)v] ? 0 : 1;
    const int64_t need = ((int64_t)liveids.size() + (1LL << p.m) - 1) >> p.m;
    if ((double)live_i < p.resample_share * (double)need) {
      rebuild_from(ix, i, liveids, livepos);
      return;
    }
    below.swap(cur);
  }
}

__global__ void k_mark_dead(const int64_t* __restrict__ ids, int64_t n, uint8_t* __restrict__ dead) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dead[ids[i]] = 1;
}
}  // namespace

extern "C" henn_status henn_delete(henn_index* ix, const int64_t* ids, int64_t n, void* stream) {
  g_error.clear();
  try {
    require(ix != nullptr, "index is NULL");
    require(n >= 0, "n must be >= 0");
    if (n == 0) return HENN_OK;
    require(ids != nullptr, "ids is NULL");
    for (int64_t i = 0; i < n; ++i) require(ids[i] >= 0 && ids[i] < ix->n, "id out of range");
    cudaStream_t st = (cudaStream_t)stream;
    if (!ix->dead) {
      ix->dead = ix->alloc<uint8_t>((size_t)ix->cap_n);
      CK(cudaMemsetAsync(ix->dead, 0, (size_t)ix->cap_n, st));
    }
    Scratch sc(st);
    int64_t* d_ids = sc.get<int64_t>((size_t)n);
    CK(cudaMemcpyAsync(d_ids, ids, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st));
    int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
    k_mark_dead<<<grid, 256, 0, st>>>(d_ids, n, ix->dead);
    CKL("delete");
    CK(cudaStreamSynchronize(st));
    ix->n_dead += n;  // an upper bound: a point deleted twice counts twice
    resample_after_delete(ix);
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    return f.status;
  } catch (const std::exception& e) {
    g_error = e.what();
    return HENN_ERR_CUDA;
  }
}

// ------------------------------------------------------------- insertion

namespace {

// Reallocates a tracked device array to `cap` elements keeping the first
// `used` (the stream is synchronised before the old one is freed).
template <typename T>
T* regrow(henn_index* ix, T* old, size_t used, size_t cap, cudaStream_t st) {
  T* p = ix->alloc<T>(cap);
  if (old && used) CK(cudaMemcpyAsync(p, old, sizeof(T) * used, cudaMemcpyDeviceToDevice, st));
  if (old) {
    CK(cudaStreamSynchronize(st));
    ix->release(old);
  }
  return p;
}

}  // namespace

extern "C" henn_status henn_insert(henn_index* ix, const float* X, int64_t n_new, int32_t x_on_device, void* stream) {
  g_error.clear();
  try {
    require(ix != nullptr, "index is NULL");
    require(n_new >= 0, "n_new must be >= 0");
    if (n_new == 0) return HENN_OK;
    require(X != nullptr, "X is NULL");
    if (ix->graph != HENN_GRAPH_NSW) throw Failure(HENN_ERR_UNSUPPORTED, "insertion supports NSW graphs only");
    require(ix->n + n_new < (int64_t)INT32_MAX, "too many points");
    CK(cudaStreamSynchronize((cudaStream_t)stream));
    ix->drop_entry_ops();  // upper layers may grow
    struct OwnStream {
      cudaStream_t s = nullptr;
      ~OwnStream() {
        if (s) {
          cudaStreamSynchronize(s);
          cudaStreamDestroy(s);
        }
      }
    } own;
    CK(cudaStreamCreateWithFlags(&own.s, cudaStreamNonBlocking));
    cudaStream_t st = own.s;
    const int64_t n0 = ix->n, n1 = n0 + n_new;
    const int32_t dpad = ix->dpad, d = ix->d, M = ix->M;
    const bool angular = ix->metric == HENN_ANGULAR;

    // ---- vectors (FP32 master copy, unit rows for angular)
    if (n1 > ix->cap_n) {
      const int64_t cap = std::max(n1, 2 * ix->cap_n);
      const bool aliased = ix->xw == ix->x32;
      ix->x32 = regrow(ix, ix->x32, (size_t)n0 * dpad, (size_t)cap * dpad, st);
      if (angular) {
        ix->xw = regrow(ix, ix->xw, (size_t)n0 * dpad, (size_t)cap * dpad, st);
        ix->inv_norm = regrow(ix, ix->inv_norm, (size_t)n0, (size_t)cap, st);
      } else if (aliased) {
        ix->xw = ix->x32;
      }
      if (ix->dead) ix->dead = regrow(ix, ix->dead, (size_t)n0, (size_t)cap, st);
      ix->cap_n = cap;
    }
    if (ix->dead) CK(cudaMemsetAsync(ix->dead + n0, 0, (size_t)n_new, st));
    float* xrow = ix->x32 + (size_t)n0 * dpad;
    CK(cudaMemsetAsync(xrow, 0, sizeof(float) * (size_t)n_new * dpad, st));
    CK(cudaMemcpy2DAsync(xrow, sizeof(float) * dpad, X, sizeof(float) * d, sizeof(float) * d, (size_t)n_new,
                         x_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    if (angular) {
      launch_inv_norms(xrow, n_new, dpad, ix->inv_norm + n0, st);
      launch_normalise(xrow, ix->inv_norm + n0, n_new, dpad, ix->xw + (size_t)n0 * dpad, st);
      CKL("normalise");
    }

    // ---- layers each new point joins (App. C, Insert)
    std::vector<std::vector<int32_t>> add(ix->L + 1);
    for (int64_t j = 0; j < n_new; ++j) {
      const uint64_t pid = (uint64_t)(n0 + j);
      add[0].push_back((int32_t)pid);
      for (int32_t i = 1; i <= ix->L; ++i) {
        if (bounded(derive(derive(derive(ix->seed, HENN_TAG_INSERT), pid), (uint64_t)i), 1ull << ix->m) != 0) break;
        add[i].push_back((int32_t)pid);
      }
    }

    // ---- per layer: append members, their traversal rows, forward lists, edge rule
    for (int32_t li = 0; li <= ix->L; ++li) {
      LayerDev& Ly = ix->layers[li];
      const int64_t s0 = Ly.size, c = (int64_t)add[li].size(), s1 = s0 + c;
      if (c == 0) continue;
      const size_t elem = ix->storage == HENN_BF16 ? 2 : (ix->storage == HENN_FP8E4M3 ? 1 : 4);
      const bool vec_aliased = li == 0 && ix->storage == HENN_F32;
      if (s1 > Ly.cap) {
        const int64_t cap = std::max(s1, 2 * Ly.cap);
        if (li >= 1) {
          Ly.ids = regrow(ix, Ly.ids, (size_t)s0, (size_t)cap, st);
          Ly.down = regrow(ix, Ly.down, (size_t)s0, (size_t)cap, st);
        }
        Ly.adj = regrow(ix, Ly.adj, (size_t)s0 * kMmax, (size_t)cap * kMmax, st);
        Ly.fwd = regrow(ix, Ly.fwd, (size_t)s0 * M, (size_t)cap * M, st);
        Ly.fwd_d = regrow(ix, Ly.fwd_d, (size_t)s0 * M, (size_t)cap * M, st);
        if (!vec_aliased)
          Ly.vec = regrow(ix, static_cast<uint8_t*>(Ly.vec), (size_t)s0 * dpad * elem, (size_t)cap * dpad * elem, st);
        if (ix->storage == HENN_FP8E4M3) Ly.vscale = regrow(ix, Ly.vscale, (size_t)s0, (size_t)cap, st);
        Ly.cap = cap;
      }
      if (vec_aliased) Ly.vec = ix->xw;
      Scratch sc(st);
      if (li >= 1) {
        // global ids, and positions in the layer below (appended there in this call)
        std::vector<int32_t> dn(c);
        const LayerDev& Lb = ix->layers[li - 1];
        const int64_t below_first = Lb.size - (int64_t)add[li - 1].size();
        size_t at = 0;
        for (int64_t j = 0; j < c; ++j) {
          while (add[li - 1][at] != add[li][j]) ++at;
          dn[j] = (int32_t)(below_first + (int64_t)at);
        }
        CK(cudaMemcpyAsync(Ly.ids + s0, add[li].data(), sizeof(int32_t) * c, cudaMemcpyHostToDevice, st));
        CK(cudaMemcpyAsync(Ly.down + s0, dn.data(), sizeof(int32_t) * c, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));  // host vectors go out of scope
      }
      // traversal rows of the new members
      const float* src = ix->xw + (size_t)n0 * dpad;  // layer 0: the appended rows in order
      if (li >= 1) {
        float* g = ix->storage == HENN_F32 ? static_cast<float*>(Ly.vec) + (size_t)s0 * dpad
                                           : sc.get<float>((size_t)c * dpad);
        launch_gather_rows32(ix->xw, Ly.ids + s0, c, dpad, g, st);
        src = g;
      }
      if (ix->storage == HENN_BF16)
        launch_quantize(src, c, dpad, dpad, dpad, HENN_BF16, static_cast<uint16_t*>(Ly.vec) + (size_t)s0 * dpad,
                        nullptr, st);
      else if (ix->storage == HENN_FP8E4M3)
        launch_quantize(src, c, dpad, dpad, dpad, HENN_FP8E4M3, static_cast<uint8_t*>(Ly.vec) + (size_t)s0 * dpad,
                        Ly.vscale + s0, st);
      CKL("traversal rows");
      // forward lists: the new rows, inserted last in this order
      std::vector<int32_t> rows(c);
      for (int64_t j = 0; j < c; ++j) rows[j] = (int32_t)(s0 + j);
      int32_t* drows = sc.get<int32_t>(c);
      CK(cudaMemcpyAsync(drows, rows.data(), sizeof(int32_t) * c, cudaMemcpyHostToDevice, st));
      launch_exact_rows(ix->xw, li >= 1 ? Ly.ids : nullptr, s1, dpad, ix->metric, nullptr, 0, drows, (int32_t)c, M,
                        Ly.fwd, Ly.fwd_d, st);
      CKL("forward lists");
      // edge rule over the layer's updated forward lists
      int32_t* cnt = sc.get<int32_t>(s1);
      int32_t* fill = sc.get<int32_t>(s1);
      int64_t* off = sc.get<int64_t>((size_t)s1 + 1);
      int64_t* tiles = sc.get<int64_t>((size_t)scan_tiles(s1) + 1);
      uint64_t* rev = sc.get<uint64_t>((size_t)s1 * M);
      CK(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * s1, st));
      CK(cudaMemsetAsync(fill, 0, sizeof(int32_t) * s1, st));
      launch_rev_count(Ly.fwd, s1, M, cnt, st);
      launch_offsets(cnt, s1, tiles, off, st);
      launch_rev_fill(Ly.fwd, Ly.fwd_d, s1, M, off, fill, rev, st);
      launch_select_adj(Ly.fwd, Ly.fwd_d, s1, M, off, rev, ix->graph, Ly.adj, st);
      CKL("edge rule");
      CK(cudaStreamSynchronize(st));  // rows vector goes out of scope
      Ly.size = s1;
    }
    ix->n = n1;

    // ---- search-side layer table
    std::vector<SearchLayer> h(ix->L + 1);
    for (int32_t li = 0; li <= ix->L; ++li) {
      h[li].adj = ix->layers[li].adj;
      h[li].vec = ix->layers[li].vec;
      h[li].scale = ix->layers[li].vscale;
      h[li].down = ix->layers[li].down;
      h[li].size = ix->layers[li].size;
    }
    CK(cudaMemcpyAsync(ix->d_layers, h.data(), sizeof(SearchLayer) * h.size(), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    return f.status;
  } catch (const std::exception& e) {
    g_error = e.what();
    return HENN_ERR_CUDA;
  }
}

// -------------------------------------------------------------- search

namespace {

// Visited-table slots per query (search_hash_bits): sized for occupancy,
// since the table may forget entries without changing results.
int pick_hash_bits(int ef_cap) { return search_hash_bits(ef_cap); }

}  // namespace

namespace {

void fill_search_args(const henn_index* idx, SearchArgs& a) {
  std::memset(&a, 0, sizeof(a));
  a.layers = idx->d_layers;
  a.L = idx->L;
  a.dpad = idx->dpad;
  a.d = idx->d;
  a.metric = idx->metric;
  a.storage = idx->storage;
  a.rerank = idx->storage != HENN_F32;
  a.x32 = idx->xw;
  a.dead = idx->dead;
  a.entry_key = derive(idx->seed, HENN_TAG_ENTRY);
  a.top_exact = idx->L;
  a.exact_method = HENN_EXACT_SORT;
}

// The tile operands of upper layer li (exact_method TILES), made on first
// use on stream st and waited for, so that any stream may use them after.
const henn_index::EntryOps& entry_ops(const henn_index* idx, int32_t li, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(idx->entry_mu);
  if ((int)idx->entry.size() <= li) idx->entry.resize(li + 1);
  henn_index::EntryOps& e = idx->entry[li];
  const LayerDev& Ly = idx->layers[li];
  if (e.size == Ly.size) return e;
  for (void* p : e.mem) cudaFree(p);
  e = henn_index::EntryOps();
  const int64_t s = Ly.size;
  const int32_t dpad = idx->dpad;
  auto get = [&](size_t bytes) {
    void* p = nullptr;
    CK(cudaMalloc(&p, bytes > 0 ? bytes : 16));
    e.mem.push_back(p);
    return p;
  };
  Scratch sc(st);
  float* rows = sc.get<float>((size_t)s * dpad);
  CK(launch_layer_rows_f32(Ly.vec, Ly.vscale, s, idx->storage, dpad, rows, st));
  e.mean = static_cast<float*>(get(sizeof(float) * dpad));
  float* partial = sc.get<float>((size_t)((s + 4095) / 4096) * dpad);
  launch_layer_mean(rows, nullptr, s, dpad, partial, e.mean, st);
  int32_t* inv = sc.get<int32_t>(s);
  float* xo = sc.get<float>((size_t)s * dpad);
  e.norms = static_cast<float*>(get(sizeof(float) * s));
  launch_order_gather(rows, nullptr, s, dpad, 0, 0, HENN_GRAPH_KNN, e.mean, inv, xo, e.norms, st);
  e.nmax = static_cast<float*>(get(sizeof(float)));
  launch_max_nonneg(e.norms, s, e.nmax, st);
  if (tc_tiles_supported(dpad, 32)) {
    const int32_t dk = round_up(dpad, 64);
    e.hi = get((size_t)s * dk * 2);
    e.lo = get((size_t)s * dk * 2);
    launch_split_bf16(xo, s, dpad, dk, e.hi, e.lo, st);
    require(make_column_maps(e.hi, e.lo, s, dk, e.maps), "tensor maps of the exact layer");
    e.engine = HENN_TILES_TCGEN05;
  } else {
    e.xo = static_cast<float*>(get(sizeof(float) * s * dpad));
    CK(cudaMemcpyAsync(e.xo, xo, sizeof(float) * s * dpad, cudaMemcpyDeviceToDevice, st));
    e.engine = HENN_TILES_SIMT;
  }
  CKL("exact-layer operands");
  CK(cudaStreamSynchronize(st));
  e.size = s;
  return e;
}

// exact_method TILES: layers up to this size go through the distance
// matrix instead of in-epilogue lists, in chunks of whole 128-query blocks
// whose matrix takes at most a third of L2 (written by the tile launch, read
// by the selection from L2 and dropped there, so it never reaches DRAM)
constexpr int64_t kDenseExactMax = 16384;

#ifndef HENN_EXACT_L2_SHARE
#define HENN_EXACT_L2_SHARE 0  // a chunk's matrix takes at most L2 / this (0: up to 1 GiB, one chunk here)
#endif

int persistent_grid(int device, int warps, size_t smem) {
  int grid = 0;
  CK(search_persistent_grid(device, warps, smem, &grid));
  return grid;
}

}  // namespace

extern "C" henn_status henn_search(const henn_index* idx, const float* Q, int64_t nq, int32_t q_on_device,
                                   const henn_search_params* spp, int64_t* out_ids, float* out_dists, int32_t out_stride,
                                   void* stream) {
  g_error.clear();
  try {
    require(idx != nullptr, "index is NULL");
    require(nq >= 0, "nq must be >= 0");
    if (nq == 0) return HENN_OK;
    require(Q && out_ids && out_dists, "Q / out_ids / out_dists must not be NULL");
    henn_search_params sp;
    henn_search_params_default(&sp);
    if (spp) {
      require(spp->struct_size == sizeof(henn_search_params), "henn_search_params.struct_size mismatch");
      sp = *spp;
      if (sp.rerank_mult <= 0) sp.rerank_mult = 4;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // per-query k / ef bounds (host view needed for the kernel shape)
    int32_t kmax = sp.k_uniform, efmax = sp.ef_uniform;
    std::vector<int32_t> hk, hef;
    if (sp.k) {
      hk.resize(nq);
      CK(cudaMemcpy(hk.data(), sp.k, sizeof(int32_t) * nq, q_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
      kmax = 0;
      for (int32_t v : hk) {
        require(v >= 1 && v <= 1024, "k must be in [1, 1024]");
        kmax = std::max(kmax, v);
      }
    } else {
      require(kmax >= 1 && kmax <= 1024, "k must be in [1, 1024]");
    }
    if (sp.ef) {
      hef.resize(nq);
      CK(cudaMemcpy(hef.data(), sp.ef, sizeof(int32_t) * nq, q_on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost));
      efmax = 0;
      for (int32_t v : hef) {
        require(v >= 1 && v <= 4096, "ef must be in [1, 4096]");
        efmax = std::max(efmax, v);
      }
    } else {
      require(efmax >= 1 && efmax <= 4096, "ef must be in [1, 4096]");
    }
    require(out_stride >= kmax, "out_stride must be >= max k");
    const int rerank = idx->storage != HENN_F32;
    require(sp.ef_upper >= 0 && sp.ef_upper <= 4096, "ef_upper must be in [0, 4096]");
    require(sp.ef_l1 >= 0 && sp.ef_l1 <= 4096, "ef_l1 must be in [0, 4096]");
    require(sp.exact_upper >= 0, "exact_upper must be >= 0");
    require(sp.exact_method >= HENN_EXACT_SORT && sp.exact_method <= HENN_EXACT_SCAN, "exact_method must be 0, 1 or 2");
    // the lowest upper layer with at most exact_upper points (sizes shrink
    // upwards); the layers above it are skipped
    int32_t top_exact = idx->L;
    bool has_exact = false;
    for (int32_t li = 1; sp.exact_upper > 0 && li <= idx->L; ++li)
      if (idx->layers[li].size <= sp.exact_upper) {
        top_exact = li;
        has_exact = true;
        break;
      }
    const int32_t exact_width = (top_exact == 1 && sp.ef_l1 > 0) ? sp.ef_l1 : sp.ef_upper;
    if (has_exact && sp.exact_method != HENN_EXACT_SORT)
      require(!(sp.descend_all && exact_width > 32),
              "exact_method TILES / SCAN with descend_all needs the exact layer's width (ef_upper, or ef_l1 on layer 1) <= 32");
    // beam capacity of a query: the power of two holding its widest list
    auto cap_of = [&](int32_t kq, int32_t efq) {
      return search_beam_cap(kq, efq, sp.ef_upper, sp.ef_l1, rerank != 0, sp.rerank_mult);
    };
    const int ef_cap = cap_of(kmax, efmax);
    int hb = sp.hash_bits > 0 ? sp.hash_bits : pick_hash_bits(ef_cap);
    require(hb >= 8 && hb <= 15, "hash_bits must be in [8, 15]");
    // the exact layers' keys sit in the visited table; capacity-group launches
    // (default table sizes) use at least 2^10 slots
    const int hb_min = sp.hash_bits > 0 ? hb : 10;
    if (has_exact && sp.exact_method == HENN_EXACT_SORT)
      require(idx->layers[top_exact].size <= (1 << (hb_min - 1)),
              "exact_method SORT: the exact layer must have <= 2^(hash_bits - 1) points (512 by default)");
    int warps = sp.warps_per_block > 0 ? sp.warps_per_block : kSearchWarps;
    require(warps >= 1 && warps <= kSearchWarps, "warps_per_block must be in [1, 4]");
    const int team = sp.team_size > 0 ? sp.team_size : 1;
    require(team == 1 || team == 2 || team == 4, "team_size must be 1, 2 or 4");
    require(sp.tile_n == 0 || sp.tile_n == 128 || sp.tile_n == 256, "tile_n must be 0, 128 or 256");
    require(warps % team == 0, "team_size must divide warps_per_block");
    const int teams = warps / team;  // queries in flight per block

    Scratch sc(st, idx->search_pool());
    const float* dQ = Q;
    const int32_t* dk = sp.k;
    const int32_t* def = sp.ef;
    const uint64_t* dkeys = sp.query_keys;
    int64_t* dids = out_ids;
    float* dd = out_dists;
    int32_t* dstats = sp.stats;
    bool out_in_place = q_on_device != 0;
    bool q_in_host = false;  // the kernels read the queries from page-locked host memory
    if (!q_on_device) {
      // page-locked queries and outputs are used in place (the kernels read
      // and write them over the host link); other host buffers are staged
      if (const void* qm = mapped_host(Q)) {
        dQ = static_cast<const float*>(qm);
        q_in_host = true;
      } else {
        float* q = sc.get<float>((size_t)nq * idx->d);
        CK(cudaMemcpyAsync(q, Q, sizeof(float) * nq * idx->d, cudaMemcpyHostToDevice, st));
        dQ = q;
      }
      if (sp.k) {
        int32_t* t = sc.get<int32_t>(nq);
        CK(cudaMemcpyAsync(t, hk.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
        dk = t;
      }
      if (sp.ef) {
        int32_t* t = sc.get<int32_t>(nq);
        CK(cudaMemcpyAsync(t, hef.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
        def = t;
      }
      if (sp.query_keys) {
        uint64_t* t = sc.get<uint64_t>(nq);
        CK(cudaMemcpyAsync(t, sp.query_keys, sizeof(uint64_t) * nq, cudaMemcpyHostToDevice, st));
        dkeys = t;
      }
      void* im = mapped_host(out_ids);
      void* dm = mapped_host(out_dists);
      out_in_place = im != nullptr && dm != nullptr;
      dids = out_in_place ? static_cast<int64_t*>(im) : sc.get<int64_t>((size_t)nq * out_stride);
      dd = out_in_place ? static_cast<float*>(dm) : sc.get<float>((size_t)nq * out_stride);
      if (sp.stats) dstats = sc.get<int32_t>((size_t)nq * 4);
    }
    // Per-query k / ef: queries are grouped by beam capacity and each group
    // runs as its own persistent launch, sized (shared memory per warp,
    // visited table, resident warps) for that capacity; the launches run
    // concurrently on side streams.  Results do not depend on the grouping.
    std::vector<int> caps;                  // distinct capacities, widest first
    std::vector<int64_t> begin, count;      // their ranges in `order`
    const int32_t* d_order = nullptr;
    if ((sp.k || sp.ef) && sp.hash_bits <= 0) {
      std::vector<int> qcap(nq);
      for (int64_t q = 0; q < nq; ++q) qcap[q] = cap_of(sp.k ? hk[q] : kmax, sp.ef ? hef[q] : efmax);
      for (int c = ef_cap; c >= 32; c >>= 1) {
        int64_t n = 0;
        for (int64_t q = 0; q < nq; ++q) n += qcap[q] == c;
        if (n > 0) {
          caps.push_back(c);
          count.push_back(n);
        }
      }
      if (caps.size() > 1) {
        std::vector<int32_t> h_order;
        h_order.reserve(nq);
        for (size_t g = 0; g < caps.size(); ++g) {
          begin.push_back((int64_t)h_order.size());
          for (int64_t q = 0; q < nq; ++q)
            if (qcap[q] == caps[g]) h_order.push_back((int32_t)q);
        }
        int32_t* o = sc.get<int32_t>(nq);
        CK(cudaMemcpyAsync(o, h_order.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));  // h_order is a local vector
        d_order = o;
      } else {
        caps.clear();
        count.clear();
      }
    }
    const int groups = caps.empty() ? 1 : (int)caps.size();
    unsigned long long* counter = sc.get<unsigned long long>(groups);
    CK(cudaMemsetAsync(counter, 0, sizeof(unsigned long long) * groups, st));

    SearchArgs a;
    fill_search_args(idx, a);
    a.rerank_mult = sp.rerank_mult;
    a.Q = dQ;
    a.nq = nq;
    a.kq = dk;
    a.efq = def;
    a.k_uniform = sp.k_uniform;
    a.ef_uniform = sp.ef_uniform;
    a.ef_upper = sp.ef_upper;
    a.descend_all = sp.descend_all;
    a.ef_l1 = sp.ef_l1;
    a.exact_upper = sp.exact_upper;
    a.top_exact = top_exact;
    a.exact_method = has_exact ? sp.exact_method : HENN_EXACT_SORT;
    a.team = team;
    int32_t launches = 0;
    if (has_exact && sp.exact_method == HENN_EXACT_TILES) {
      // batched candidates of the exact layer: queries against all its points
      const henn_index::EntryOps& eo = entry_ops(idx, top_exact, st);
      const int64_t s = eo.size;
      const int32_t dpad = idx->dpad;
      float* qn = sc.get<float>(nq);
      uint64_t* pkeys = sc.get<uint64_t>((size_t)nq * 32);
      int32_t* perr = sc.get<int32_t>(1);
      CK(cudaMemsetAsync(perr, 0, sizeof(int32_t), st));
      if (eo.engine == HENN_TILES_TCGEN05) {
        const int32_t dkk = round_up(dpad, 64);
        void* qh = sc.get<uint16_t>((size_t)nq * dkk);
        void* ql = sc.get<uint16_t>((size_t)nq * dkk);
        // queries read over the host link once: the query preparation also
        // leaves a device copy for the search kernel
        float* qraw = q_in_host ? sc.get<float>((size_t)nq * idx->d) : nullptr;
        launch_entry_queries(dQ, nq, idx->d, dpad, idx->metric, eo.mean, nullptr, qh, ql, dkk, qn, qraw, st);
        if (qraw) a.Q = qraw;
        // a small layer: the distance matrix itself (written and read once,
        // coalesced) and a selection pass at full occupancy; else the
        // running lists inside the tile epilogue
        const int64_t ldo = (s + 63) / 64 * 64;  // 16-bit keys: rows of whole 128-byte lines
        if (s <= kDenseExactMax) {
          int l2 = 0;
          CK(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, idx->device));
          const double chunk_bytes =
              HENN_EXACT_L2_SHARE > 0 ? std::max(8.0 * (1 << 20), (double)l2 / HENN_EXACT_L2_SHARE) : 1.0 * (1 << 30);
          int64_t qc = (int64_t)(chunk_bytes / (2.0 * (double)ldo)) / 128 * 128;
          qc = std::max<int64_t>(128, std::min<int64_t>(qc, nq));
          uint16_t* dm = sc.get<uint16_t>((size_t)qc * ldo);
          // each row's 32-column chunk minima: whole 256-column tiles, 8 per tile
          const int64_t ldc = (s + 255) / 256 * 8;
          float* cmn = sc.get<float>((size_t)qc * ldc);
          for (int64_t q0 = 0; q0 < nq; q0 += qc) {
            const int64_t cn = std::min<int64_t>(qc, nq - q0);
            CK(launch_tile_cross_tc(static_cast<uint16_t*>(qh) + q0 * dkk, static_cast<uint16_t*>(ql) + q0 * dkk,
                                    qn + q0, cn, eo.maps, eo.norms, s, dkk, nullptr, dm, ldo, cmn, ldc, perr,
                                    sp.tile_n, st));
            launch_select_top32(dm, cmn, cn, s, ldo, ldc, pkeys + q0 * 32, true, st);
            launches += q0 > 0 ? 2 : 1;
          }
        } else {
          CK(launch_tile_cross_tc(qh, ql, qn, nq, eo.maps, eo.norms, s, dkk, pkeys, nullptr, 0, nullptr, 0, perr,
                                  sp.tile_n, st));
        }
        a.pre_tile_u = tc_tile_unit_error(dkk);
        launches += 2;
      } else {
        float* qo = sc.get<float>((size_t)nq * dpad);
        float* qraw = q_in_host ? sc.get<float>((size_t)nq * idx->d) : nullptr;
        launch_entry_queries(dQ, nq, idx->d, dpad, idx->metric, eo.mean, qo, nullptr, nullptr, 0, qn, qraw, st);
        if (qraw) a.Q = qraw;
        const int64_t rb = (nq + 63) / 64;
        const int32_t splits =
            (int32_t)std::max<int64_t>(1, std::min<int64_t>((2 * 152 + rb - 1) / rb, (s + 4095) / 4096));
        uint64_t* cand = splits > 1 ? sc.get<uint64_t>((size_t)splits * nq * 32) : pkeys;
        launch_tile_topk_simt(qo, qn, nq, eo.xo, eo.norms, s, dpad, 2, 32, splits, cand, st);
        if (splits > 1) launch_merge_splits(cand, nq, 32, splits, pkeys, st);
        a.pre_tile_u = (dpad + 8.0) * std::ldexp(1.0, -24);
        launches += splits > 1 ? 3 : 2;
      }
      CKL("exact-layer tiles");
      a.pre_keys = pkeys;
      a.pre_qnorm = qn;
      a.pre_nmax = eo.nmax;
      a.pre_err = perr;
    }
    a.ef_cap = ef_cap;
    a.hash_bits = hb;
    a.keys = dkeys;
    a.out_ids = dids;
    a.out_d = dd;
    a.out_stride = out_stride;
    a.stats = dstats;
    a.counter = counter;

    std::unique_lock<std::mutex> tlk(idx->time_mu, std::defer_lock);
    if (sp.time_kernel) {
      tlk.lock();
      for (cudaEvent_t& e : idx->tev)
        if (!e) CK(cudaEventCreate(&e));
      CK(cudaEventRecord(idx->tev[0], st));
    }
    launches += groups;
    if (groups == 1) {
      a.order = d_order;
      size_t smem = search_team_smem(ef_cap, hb, idx->dpad, team) * teams;
      int64_t blocks_needed = (nq + teams - 1) / teams;
      int grid = (int)std::min<int64_t>(persistent_grid(idx->device, warps, smem), blocks_needed);
      CK(launch_search(a, warps, grid, st));
    } else {
      std::lock_guard<std::mutex> lk(idx->side_mu);
      while ((int)idx->side.size() < groups) {
        cudaStream_t t;
        CK(cudaStreamCreateWithFlags(&t, cudaStreamNonBlocking));
        idx->side.push_back(t);
      }
      cudaEvent_t fork;
      CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
      CK(cudaEventRecord(fork, st));
      for (int g = 0; g < groups; ++g) {
        cudaStream_t t = idx->side[g];
        CK(cudaStreamWaitEvent(t, fork, 0));
        SearchArgs ag = a;
        ag.order = d_order + begin[g];
        ag.nq = count[g];
        ag.ef_cap = caps[g];
        ag.hash_bits = pick_hash_bits(caps[g]);
        ag.counter = counter + g;
        size_t smem = search_team_smem(ag.ef_cap, ag.hash_bits, idx->dpad, team) * teams;
        int64_t blocks_needed = (count[g] + teams - 1) / teams;
        int grid = (int)std::min<int64_t>(persistent_grid(idx->device, warps, smem), blocks_needed);
        CK(launch_search(ag, warps, grid, t));
        cudaEvent_t join;
        CK(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        CK(cudaEventRecord(join, t));
        CK(cudaStreamWaitEvent(st, join, 0));
        cudaEventDestroy(join);
      }
      cudaEventDestroy(fork);
    }
    if (sp.time_kernel) {
      CK(cudaEventRecord(idx->tev[1], st));
      idx->t_launches = launches;
      idx->t_valid = true;
      tlk.unlock();
    }
    if (!q_on_device) {
      if (!out_in_place) {
        CK(cudaMemcpyAsync(out_ids, dids, sizeof(int64_t) * nq * out_stride, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(out_dists, dd, sizeof(float) * nq * out_stride, cudaMemcpyDeviceToHost, st));
      }
      if (sp.stats) CK(cudaMemcpyAsync(sp.stats, dstats, sizeof(int32_t) * nq * 4, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    return f.status;
  } catch (const std::exception& e) {
    g_error = e.what();
    return HENN_ERR_CUDA;
  }
}

extern "C" henn_status henn_last_search_ms(const henn_index* idx, float* ms, int32_t* launches) {
  g_error.clear();
  try {
    require(idx != nullptr, "index is NULL");
    std::lock_guard<std::mutex> lk(idx->time_mu);
    require(idx->t_valid, "no search with time_kernel = 1 ran on this index");
    if (ms) {
      CK(cudaEventSynchronize(idx->tev[1]));
      CK(cudaEventElapsedTime(ms, idx->tev[0], idx->tev[1]));
    }
    if (launches) *launches = idx->t_launches;
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    return f.status;
  }
}

// ------------------------------------------------------ greedy probes

extern "C" henn_status henn_greedy_probe(const henn_index* idx, int32_t layer, const float* Q, int64_t nq,
                                         const int32_t* starts, int32_t S, int32_t* out_node, float* out_dist,
                                         int32_t* out_hops, void* stream) {
  g_error.clear();
  try {
    require(idx != nullptr, "index is NULL");
    require(layer >= 0 && layer <= idx->L, "layer out of range");
    require(nq >= 0 && S >= 1, "nq must be >= 0 and S >= 1");
    if (nq == 0) return HENN_OK;
    require(Q && starts && out_node && out_dist, "Q / starts / out_node / out_dist must not be NULL");
    const LayerDev& Ly = idx->layers[layer];
    GreedyProbeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.layer.adj = Ly.adj;
    a.layer.vec = Ly.vec;
    a.layer.scale = Ly.vscale;
    a.layer.down = Ly.down;
    a.layer.size = Ly.size;
    a.dpad = idx->dpad;
    a.d = idx->d;
    a.metric = idx->metric;
    a.Q = Q;
    a.nq = nq;
    a.starts = starts;
    a.S = S;
    a.out_node = out_node;
    a.out_dist = out_dist;
    a.out_hops = out_hops;
    CK(launch_greedy_probe(a, idx->storage, (cudaStream_t)stream));
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    return f.status;
  } catch (const std::exception& e) {
    g_error = e.what();
    return HENN_ERR_CUDA;
  }
}

// ------------------------------------------------------ introspection

extern "C" henn_status henn_index_get_info(const henn_index* idx, henn_index_info* info) {
  g_error.clear();
  if (!idx || !info) {
    g_error = "NULL argument";
    return HENN_ERR_INVALID_ARG;
  }
  std::memset(info, 0, sizeof(*info));
  info->struct_size = sizeof(*info);
  info->n = idx->n;
  info->d = idx->d;
  info->metric = idx->metric;
  info->storage = idx->storage;
  info->graph = idx->graph;
  info->M = idx->M;
  info->Mmax = idx->Mmax;
  info->L = idx->L;
  for (int32_t i = 0; i <= idx->L && i < HENN_MAX_LAYERS; ++i) {
    info->sizes[i] = idx->layers[i].size;
    info->attempts[i] = idx->attempts[i];
    info->ambiguous_rings[i] = idx->ambiguous[i];
  }
  info->device_bytes = idx->bytes;
  info->uncertified_rows = idx->uncertified;
  info->build_seconds = idx->build_seconds;
  info->tile_seconds = idx->tile_seconds;
  info->tile_flops = idx->tile_flops;
  info->tile_engine = idx->tile_engine;
  info->graph_instantiations = idx->graph_instantiations;
  info->graph_updates = idx->graph_updates;
  return HENN_OK;
}

extern "C" henn_status henn_index_get_layer(const henn_index* idx, int32_t layer, int32_t* ids, int32_t* down,
                                            int32_t* adj, int32_t* fwd, float* fwd_d) {
  g_error.clear();
  try {
    require(idx != nullptr, "index is NULL");
    require(layer >= 0 && layer <= idx->L, "layer out of range");
    const LayerDev& Ly = idx->layers[layer];
    const int64_t s = Ly.size;
    CK(cudaDeviceSynchronize());
    if (ids) {
      if (layer == 0) {
        for (int64_t i = 0; i < s; ++i) ids[i] = (int32_t)i;
      } else {
        CK(cudaMemcpy(ids, Ly.ids, sizeof(int32_t) * s, cudaMemcpyDeviceToHost));
      }
    }
    if (down) {
      if (layer == 0) {
        for (int64_t i = 0; i < s; ++i) down[i] = -1;
      } else {
        CK(cudaMemcpy(down, Ly.down, sizeof(int32_t) * s, cudaMemcpyDeviceToHost));
      }
    }
    if (adj) CK(cudaMemcpy(adj, Ly.adj, sizeof(int32_t) * s * kMmax, cudaMemcpyDeviceToHost));
    if (fwd) CK(cudaMemcpy(fwd, Ly.fwd, sizeof(int32_t) * s * idx->M, cudaMemcpyDeviceToHost));
    if (fwd_d) CK(cudaMemcpy(fwd_d, Ly.fwd_d, sizeof(float) * s * idx->M, cudaMemcpyDeviceToHost));
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    return f.status;
  }
}

// ------------------------------------------------- standalone kernels

extern "C" henn_status henn_exact_knn(const float* X, int64_t n, int32_t d, const float* Q, int64_t nq, int32_t k,
                                      int32_t metric, int64_t* out_ids, float* out_dists, void* stream) {
  g_error.clear();
  try {
    require(X && Q && out_ids && out_dists, "NULL pointer");
    require(n >= 1 && n < (1LL << 31) && nq >= 0, "sizes");
    require(d >= 1 && d <= kMaxD, "d must be in [1, 1024]");
    require(k >= 1 && k <= 112, "k must be in [1, 112]");
    require(metric == HENN_L2 || metric == HENN_ANGULAR, "metric");
    if (nq == 0) return HENN_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t dpad = round_up(d, 32);
    Scratch sc(st);
    float* xp = sc.get<float>((size_t)n * dpad);
    float* qp = sc.get<float>((size_t)nq * dpad);
    CK(cudaMemsetAsync(xp, 0, sizeof(float) * n * dpad, st));
    CK(cudaMemsetAsync(qp, 0, sizeof(float) * nq * dpad, st));
    CK(cudaMemcpy2DAsync(xp, sizeof(float) * dpad, X, sizeof(float) * d, sizeof(float) * d, n, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpy2DAsync(qp, sizeof(float) * dpad, Q, sizeof(float) * d, sizeof(float) * d, nq, cudaMemcpyDeviceToDevice, st));
    float* xn = sc.get<float>(n);
    float* qn = sc.get<float>(nq);
    if (metric == HENN_ANGULAR) {
      launch_inv_norms(xp, n, dpad, xn, st);
      launch_normalise(xp, xn, n, dpad, xp, st);
      launch_inv_norms(qp, nq, dpad, qn, st);
      launch_normalise(qp, qn, nq, dpad, qp, st);
    }
    // squared norms of the (possibly normalised) rows
    float* mean0 = sc.get<float>(dpad);
    CK(cudaMemsetAsync(mean0, 0, sizeof(float) * dpad, st));
    int32_t* invx = sc.get<int32_t>(n);
    int32_t* invq = sc.get<int32_t>(nq);
    float* xo = sc.get<float>((size_t)n * dpad);
    float* qo = sc.get<float>((size_t)nq * dpad);
    launch_order_gather(xp, nullptr, n, dpad, 0, 0, HENN_GRAPH_KNN, mean0, invx, xo, xn, st);
    launch_order_gather(qp, nullptr, nq, dpad, 0, 0, HENN_GRAPH_KNN, mean0, invq, qo, qn, st);
    int32_t KP = 32;
    while (KP < k + 16) KP <<= 1;
    int sms = 152;
    int64_t rb = (nq + 63) / 64;
    int32_t splits = (int32_t)std::max<int64_t>(1, std::min<int64_t>((2 * sms + rb - 1) / rb, (n + 4095) / 4096));
    uint64_t* cand = sc.get<uint64_t>((size_t)splits * nq * KP);
    launch_tile_topk_simt(qo, qn, nq, xo, xn, n, dpad, 2, KP, splits, cand, st);
    uint64_t* merged = cand;
    if (splits > 1) {
      merged = sc.get<uint64_t>((size_t)nq * KP);
      launch_merge_splits(cand, nq, KP, splits, merged, st);
    }
    launch_rerank_queries(qo, nq, xo, dpad, metric, merged, KP, k, out_ids, out_dists, st);
    CKL("exact knn");
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    return f.status;
  }
}

extern "C" henn_status henn_quantize_rows(const float* X, int64_t n, int32_t d, int32_t storage, void* out, float* scales,
                                          void* stream) {
  g_error.clear();
  try {
    require(X && out, "NULL pointer");
    require(n >= 0 && d >= 1, "sizes");
    require(storage == HENN_BF16 || (storage == HENN_FP8E4M3 && scales), "storage (FP8 needs scales)");
    if (n == 0) return HENN_OK;
    launch_quantize(X, n, d, d, d, storage, out, scales, (cudaStream_t)stream);
    CKL("quantize");
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    return f.status;
  }
}

// ------------------------------------------------------------- serving

struct henn_server {
  const henn_index* idx = nullptr;
  henn_serve_params p;
  ServeArgs args;
  int warps = kSearchWarps, grid = 0;
  cudaStream_t kst = nullptr, cst = nullptr;
  // device
  float* qring = nullptr;
  ServeDesc* desc = nullptr;
  int64_t* oids = nullptr;
  float* od = nullptr;
  long long* published = nullptr;
  unsigned long long* taken = nullptr;
  unsigned long long* last_active = nullptr;
  int* stop = nullptr;
  // mapped host memory
  int* done_h = nullptr;
  int* done_d = nullptr;
  // host bookkeeping
  struct Req {
    int64_t id = 0, start = 0;
    int32_t nq = 0, k = 0;
    bool active = false, collected = false;
  };
  std::vector<Req> slots;
  std::deque<int32_t> order;  // slots in submission order (ring reclamation)
  std::vector<ServeDesc> hdesc;
  int64_t head = 0, tail = 0, next_id = 1;
  bool launched = false;
  std::mutex mu;

  ~henn_server() {
    if (stop) {
      int one = 1;
      cudaMemcpyAsync(stop, &one, sizeof(int), cudaMemcpyHostToDevice, cst);
      cudaStreamSynchronize(cst);
    }
    if (kst) cudaStreamSynchronize(kst);
    for (void* q : {(void*)qring, (void*)desc, (void*)oids, (void*)od, (void*)published, (void*)taken,
                    (void*)last_active, (void*)stop})
      if (q) cudaFree(q);
    if (done_h) cudaFreeHost(done_h);
    if (kst) cudaStreamDestroy(kst);
    if (cst) cudaStreamDestroy(cst);
  }

  // relaunch the kernel when it has ended and published items are waiting
  void ensure_running() {
    if (launched) {
      cudaError_t q = cudaStreamQuery(kst);
      if (q == cudaErrorNotReady) return;
      CK(q);
      unsigned long long tk = 0;
      CK(cudaMemcpyAsync(&tk, taken, sizeof(tk), cudaMemcpyDeviceToHost, cst));
      CK(cudaStreamSynchronize(cst));
      if ((int64_t)tk >= head) return;
    } else if (head == 0) {
      return;
    }
    // all ones = "no activity yet": the first warp to look starts the
    // kernel's idle clock (see k_serve)
    CK(cudaMemsetAsync(last_active, 0xFF, sizeof(unsigned long long), kst));
    CK(launch_serve(args, warps, grid, kst));
    launched = true;
  }

  void copy_ring(void* ring, const void* src, size_t row_bytes, int64_t start, int32_t n, cudaMemcpyKind kind,
                 bool to_ring) {
    const int64_t cap = p.ring_rows;
    const int64_t s0 = start % cap;
    const int64_t n1 = std::min<int64_t>(n, cap - s0);
    char* r = static_cast<char*>(ring);
    const char* h = static_cast<const char*>(src);
    if (to_ring) {
      CK(cudaMemcpyAsync(r + s0 * row_bytes, h, n1 * row_bytes, kind, cst));
      if (n > n1) CK(cudaMemcpyAsync(r, h + n1 * row_bytes, (n - n1) * row_bytes, kind, cst));
    }
  }
};

extern "C" void henn_serve_params_default(henn_serve_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->struct_size = sizeof(*p);
  p->ring_rows = 65536;
  p->max_requests = 1024;
  p->max_k = 100;
  p->max_ef = 512;
  p->ef_upper = 1;
  p->descend_all = 0;
  p->rerank_mult = 4;
  p->idle_ms = 20;
}

extern "C" henn_status henn_serve_create(const henn_index* idx, const henn_serve_params* pp, henn_server** out) {
  g_error.clear();
  if (out) *out = nullptr;
  henn_server* sv = nullptr;
  try {
    require(idx && out, "NULL argument");
    henn_serve_params p;
    henn_serve_params_default(&p);
    if (pp) {
      require(pp->struct_size == sizeof(henn_serve_params), "henn_serve_params.struct_size mismatch");
      p = *pp;
    }
    require(p.ring_rows >= 1 && p.ring_rows <= (1 << 26), "ring_rows must be in [1, 2^26]");
    require(p.max_requests >= 1 && p.max_requests <= (1 << 20), "max_requests must be in [1, 2^20]");
    require(p.max_k >= 1 && p.max_k <= 1024, "max_k must be in [1, 1024]");
    require(p.max_ef >= 1 && p.max_ef <= 1024, "max_ef must be in [1, 1024]");
    require(p.ef_upper >= 0 && p.ef_upper <= 1024, "ef_upper must be in [0, 1024]");
    require(p.ef_l1 >= 0 && p.ef_l1 <= 1024, "ef_l1 must be in [0, 1024]");
    require(p.exact_upper >= 0, "exact_upper must be >= 0");
    require(p.idle_ms >= 1 && p.idle_ms <= 10000, "idle_ms must be in [1, 10000]");
    if (p.rerank_mult <= 0) p.rerank_mult = 4;
    // the lowest upper layer with at most exact_upper points: its exact set
    // by the in-kernel sort (in the visited table's space), so that no
    // separate launch has to share the GPU with the resident kernel
    int32_t top_exact = idx->L;
    bool has_exact = false;
    for (int32_t li = 1; p.exact_upper > 0 && li <= idx->L; ++li)
      if (idx->layers[li].size <= p.exact_upper) {
        top_exact = li;
        has_exact = true;
        break;
      }
    sv = new henn_server();
    sv->idx = idx;
    sv->p = p;
    CK(cudaStreamCreateWithFlags(&sv->kst, cudaStreamNonBlocking));
    CK(cudaStreamCreateWithFlags(&sv->cst, cudaStreamNonBlocking));
    const int64_t cap = p.ring_rows;
    CK(cudaMalloc(&sv->qring, sizeof(float) * cap * idx->d));
    CK(cudaMalloc(&sv->desc, sizeof(ServeDesc) * cap));
    CK(cudaMalloc(&sv->oids, sizeof(int64_t) * cap * p.max_k));
    CK(cudaMalloc(&sv->od, sizeof(float) * cap * p.max_k));
    CK(cudaMalloc(&sv->published, sizeof(long long)));
    CK(cudaMalloc(&sv->taken, sizeof(unsigned long long)));
    CK(cudaMalloc(&sv->stop, sizeof(int)));
    CK(cudaMalloc(&sv->last_active, sizeof(unsigned long long)));
    CK(cudaMemset(sv->published, 0, sizeof(long long)));
    CK(cudaMemset(sv->taken, 0, sizeof(unsigned long long)));
    CK(cudaMemset(sv->stop, 0, sizeof(int)));
    CK(cudaHostAlloc(&sv->done_h, sizeof(int) * p.max_requests, cudaHostAllocMapped));
    CK(cudaHostGetDevicePointer((void**)&sv->done_d, sv->done_h, 0));
    std::memset(sv->done_h, 0, sizeof(int) * p.max_requests);
    sv->slots.resize(p.max_requests);
    // kernel shape: the shared-memory class of the widest admitted beam
    const int need = std::max(std::max(std::max(p.max_k, p.max_ef), std::max(p.ef_upper, p.ef_l1)),
                              std::min(p.max_ef, p.rerank_mult * p.max_k));
    int ef_cap = 32;
    while (ef_cap < need) ef_cap <<= 1;
    int hb = pick_hash_bits(ef_cap);
    if (has_exact) {
      // the exact layer's keys take the visited table's space
      while (hb < 12 && (1 << (hb - 1)) < idx->layers[top_exact].size) ++hb;
      require(idx->layers[top_exact].size <= (1 << (hb - 1)),
              "exact_upper: the exact layer of a server must have at most 2048 points");
    }
    SearchArgs& a = sv->args.base;
    fill_search_args(idx, a);
    a.rerank_mult = p.rerank_mult;
    a.ef_upper = p.ef_upper;
    a.descend_all = p.descend_all;
    a.ef_l1 = p.ef_l1;
    a.exact_upper = has_exact ? p.exact_upper : 0;
    a.top_exact = top_exact;
    a.exact_method = HENN_EXACT_SORT;
    a.ef_cap = ef_cap;
    a.hash_bits = hb;
    a.out_stride = p.max_k;
    sv->args.qring = sv->qring;
    sv->args.desc = sv->desc;
    sv->args.cap = cap;
    sv->args.out_ids = sv->oids;
    sv->args.out_d = sv->od;
    sv->args.published = sv->published;
    sv->args.taken = sv->taken;
    sv->args.stop = sv->stop;
    sv->args.done = sv->done_d;
    sv->args.last_active = sv->last_active;
    sv->args.idle_ns = (long long)p.idle_ms * 1000000ll;
    sv->grid = persistent_grid(idx->device, sv->warps, search_warp_smem(ef_cap, hb, idx->dpad) * sv->warps);
    CK(cudaDeviceSynchronize());
    *out = sv;
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    delete sv;
    return f.status;
  }
}

extern "C" henn_status henn_serve_submit(henn_server* sv, const float* Q, int32_t nq, int32_t k, int32_t ef,
                                         const uint64_t* keys, int64_t* request_id) {
  g_error.clear();
  try {
    require(sv && Q && request_id, "NULL argument");
    require(nq >= 1 && nq <= sv->p.ring_rows, "nq must be in [1, ring_rows]");
    require(k >= 1 && k <= sv->p.max_k, "k must be in [1, max_k]");
    require(ef >= 1 && ef <= sv->p.max_ef, "ef must be in [1, max_ef]");
    std::lock_guard<std::mutex> lock(sv->mu);
    int32_t slot = -1;
    for (int32_t i = 0; i < (int32_t)sv->slots.size(); ++i)
      if (!sv->slots[i].active) {
        slot = i;
        break;
      }
    if (slot < 0 || sv->head - sv->tail + nq > sv->p.ring_rows) {
      g_error = "serving budget full (request slots or ring rows)";
      return HENN_ERR_BUSY;
    }
    const int64_t id = sv->next_id++;
    const int64_t start = sv->head;
    sv->hdesc.resize(nq);
    for (int32_t i = 0; i < nq; ++i) {
      sv->hdesc[i].slot = slot;
      sv->hdesc[i].k = k;
      sv->hdesc[i].ef = ef;
      sv->hdesc[i].pad = 0;
      sv->hdesc[i].key = keys ? keys[i] : ((uint64_t)id << 20) + (uint64_t)i;
    }
    sv->copy_ring(sv->qring, Q, sizeof(float) * sv->idx->d, start, nq, cudaMemcpyHostToDevice, true);
    sv->copy_ring(sv->desc, sv->hdesc.data(), sizeof(ServeDesc), start, nq, cudaMemcpyHostToDevice, true);
    __atomic_store_n(&sv->done_h[slot], 0, __ATOMIC_RELEASE);
    long long pub = start + nq;
    // same stream as the ring copies: the kernel sees the new count only
    // after the rows and descriptors have landed
    CK(cudaMemcpyAsync(sv->published, &pub, sizeof(pub), cudaMemcpyHostToDevice, sv->cst));
    CK(cudaStreamSynchronize(sv->cst));
    sv->head = pub;
    henn_server::Req& r = sv->slots[slot];
    r.id = id;
    r.start = start;
    r.nq = nq;
    r.k = k;
    r.active = true;
    r.collected = false;
    sv->order.push_back(slot);
    sv->ensure_running();
    *request_id = id;
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    return f.status;
  }
}

extern "C" henn_status henn_serve_poll(henn_server* sv, int64_t request_id, int32_t* done, int64_t* out_ids,
                                       float* out_dists) {
  g_error.clear();
  try {
    require(sv && done && out_ids && out_dists, "NULL argument");
    std::lock_guard<std::mutex> lock(sv->mu);
    int32_t slot = -1;
    for (int32_t i = 0; i < (int32_t)sv->slots.size(); ++i)
      if (sv->slots[i].active && !sv->slots[i].collected && sv->slots[i].id == request_id) {
        slot = i;
        break;
      }
    require(slot >= 0, "unknown or already collected request");
    henn_server::Req& r = sv->slots[slot];
    sv->ensure_running();
    if (__atomic_load_n(&sv->done_h[slot], __ATOMIC_ACQUIRE) < r.nq) {
      *done = 0;
      return HENN_OK;
    }
    const int64_t cap = sv->p.ring_rows;
    const int64_t s0 = r.start % cap;
    const int64_t n1 = std::min<int64_t>(r.nq, cap - s0);
    const size_t spitch_i = sizeof(int64_t) * sv->p.max_k, spitch_f = sizeof(float) * sv->p.max_k;
    CK(cudaMemcpy2DAsync(out_ids, sizeof(int64_t) * r.k, sv->oids + s0 * sv->p.max_k, spitch_i, sizeof(int64_t) * r.k,
                         n1, cudaMemcpyDeviceToHost, sv->cst));
    CK(cudaMemcpy2DAsync(out_dists, sizeof(float) * r.k, sv->od + s0 * sv->p.max_k, spitch_f, sizeof(float) * r.k, n1,
                         cudaMemcpyDeviceToHost, sv->cst));
    if (r.nq > n1) {
      CK(cudaMemcpy2DAsync(out_ids + n1 * r.k, sizeof(int64_t) * r.k, sv->oids, spitch_i, sizeof(int64_t) * r.k,
                           r.nq - n1, cudaMemcpyDeviceToHost, sv->cst));
      CK(cudaMemcpy2DAsync(out_dists + n1 * r.k, sizeof(float) * r.k, sv->od, spitch_f, sizeof(float) * r.k,
                           r.nq - n1, cudaMemcpyDeviceToHost, sv->cst));
    }
    CK(cudaStreamSynchronize(sv->cst));
    r.collected = true;
    // release ring rows in submission order
    while (!sv->order.empty() && sv->slots[sv->order.front()].collected) {
      henn_server::Req& f = sv->slots[sv->order.front()];
      sv->tail = f.start + f.nq;
      f.active = false;
      sv->order.pop_front();
    }
    *done = 1;
    return HENN_OK;
  } catch (const Failure& f) {
    g_error = f.msg;
    return f.status;
  }
}

extern "C" void henn_serve_destroy(henn_server* sv) { delete sv; }

// Internal to the library (C++ linkage, not part of the C ABI): the search
// arguments of an index and the device it lives on, for other translation
// units that launch the search kernel.
namespace henn {
void index_search_args(const henn_index* idx, SearchArgs& a, int* device) {
  fill_search_args(idx, a);
  *device = idx->device;
}
void set_last_error(const std::string& msg) { g_error = msg; }
}  // namespace henn
