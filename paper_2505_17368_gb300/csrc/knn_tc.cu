// knn_tc.cu -- construction distance tiles on the 5th-generation tensor
// cores (tcgen05 + TMA + TMEM), with the running top-KP per row fused into
// the epilogue.  Same contract as the SIMT engine in knn.cu: the tile value
// is |a|^2 + |b|^2 - 2<a,b> of centred vectors and every row keeps its KP
// smallest (distance, column) keys.  Modes 0 and 1 take rows and columns
// from one layer in insertion order, column c valid for row r iff c < r
// (causal, NSW) or c != r (kNN graph); mode 2 takes the rows from one set
// (queries) and every column from another (a layer's points); mode 3 is
// mode 2 writing every tile value (the distance matrix, as 16-bit keys that
// keep the order of the distances) instead of lists.
//
// Precision: each FP32 operand is split into x = hi + lo with hi =
// bf16(x), lo = bf16(x - hi); the tile accumulates hi.hi + lo.hi + hi.lo in
// FP32 (kind::f16, BF16 inputs), a relative error of about 3 * 2^-18 per
// product plus the FP32 accumulation, so the certified candidate pool of
// the exact FP32 rerank stays small.
//
// Layout of one CTA (192 threads): warp 0 issues TMA loads, warp 1 owns
// TMEM and issues the MMAs (one thread), warps 2-5 drain the accumulators
// (TMEM lanes 32*(w%4)..+31 = rows of the 128-row block).  Rows of at most
// 128 values: the A block (128 rows, hi and lo planes) stays in shared
// memory and B tiles (256 columns x 64 values of one plane) stream through
// a 3-stage ring.  Wider rows (up to 1024 values): the A block no longer
// fits, so each 64-wide slice of the tile arrives as three items of a
// 5-stage ring -- the slice of A (hi and lo planes, 16 KB each), then B hi,
// then B lo (32 KB each) -- and the A block is read again for every tile
// (from L2, where one CTA's block stays hot).  Two 256-column FP32
// accumulators in TMEM let the epilogue of tile t overlap the MMAs of tile
// t+1.  Every wait is bounded; a timeout sets an error flag and the CTA
// releases its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <atomic>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace henn {

namespace tc {

constexpr int BM = 128;          // rows per block (TMEM lanes)
constexpr int BN_MAX = 256;      // columns per tile, the wider choice (UMMA N = 128 or 256)
constexpr int BK = 64;           // BF16 values per 128-byte swizzle row
constexpr int NS = 3;            // B pipeline stages (resident A)
constexpr int NS_STR = 5;        // pipeline stages (streamed A)
constexpr int A_CHUNK = BM * BK * 2;  // 16 KB
constexpr int STAGE = 32768;     // bytes of one stage of the streamed pipeline
constexpr int MAX_KC_RES = 2;    // resident A: dpad <= 128, at most 2 chunks of 64 per plane
constexpr int MAX_KC = 16;       // streamed A: dpad <= 1024
constexpr int KP = 32;
constexpr int S_LD = 33;
constexpr long long kSpinLimit = 1ll << 18;  // x 20 us hint: seconds at most

// Resident A (rows of at most 128 values); BN columns per tile.
template <int BN>
struct SmemRes {
  // 1024-byte aligned operand buffers first
  uint8_t a[2 * MAX_KC_RES][A_CHUNK];  // hi chunks then lo chunks
  uint8_t b[NS][BN * BK * 2];
  // running top-KP of each row: a max-heap of keys, 1-based (children of
  // p at 2p and 2p + 1, so a sibling pair is one 16-byte load), root = the
  // KP-th smallest so far; slot KP + 1 holds 0 (no child), slot 0 is unused
  uint64_t heap[BM][KP + 2];
  alignas(16) float ncol[4][BN];   // column norms of the current tile, one copy per epilogue warp
  float s[4][32][S_LD];            // epilogue transposition, one slab per warp
  uint64_t full[NS], empty[NS], tfull[2], tempty[2], afull;
  uint32_t tmem_base;
  int abort;
};

// Streamed A (wider rows): a ring of 32 KB stages, each holding the A slice
// of one 64-wide slice (hi plane, then lo plane) or one plane of a B slice;
// the rest as above.
template <int BN>
struct SmemStr {
  uint8_t ring[NS_STR][STAGE];
  uint64_t heap[BM][KP + 2];
  alignas(16) float ncol[4][BN];
  float s[4][32][S_LD];
  uint64_t full[NS_STR], empty[NS_STR], tfull[2], tempty[2], afull;
  uint32_t tmem_base;
  int abort;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Bounded wait for the phase with the given parity; false on timeout.  Each
// try_wait may suspend the thread for up to 20 us (the suspend-time hint)
// instead of returning at once, so waiting warps do not take issue slots.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          long long limit) {
  const uint32_t addr = smem_u32(bar);
  for (long long i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity), "r"(20000)
        : "memory");
    if (done) return true;
    if ((i & 63) == 63 && *abort_flag) return false;
  }
  return false;
}

// Bulk tensor store of a shared-memory box to global memory (bulk group
// of the issuing thread), and the waits on this thread's bulk groups.
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int x, int y) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
                   reinterpret_cast<uint64_t>(map)),
               "r"(smem_u32(src)), "r"(x), "r"(y)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_le1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// (a, b) <- (c - 2a, d - 2b) as one paired FMA, each element rounded as
// fmaf(-2, a, c) would round it
__device__ __forceinline__ void fma2_m2(float& a, float& b, float c, float d) {
  asm("{\n\t.reg .b64 va, m2, cc;\n\t"
      "mov.b64 va, {%0, %1};\n\t"
      "mov.b64 m2, {%4, %4};\n\t"
      "mov.b64 cc, {%2, %3};\n\t"
      "fma.rn.f32x2 va, va, m2, cc;\n\t"
      "mov.b64 {%0, %1}, va;\n\t}"
      : "+f"(a), "+f"(b)
      : "f"(c), "f"(d), "f"(-2.f));
}

// (a, b) <- (a + x, b + x) as one paired add
__device__ __forceinline__ void add2_s(float& a, float& b, float x) {
  asm("{\n\t.reg .b64 va, xx;\n\t"
      "mov.b64 va, {%0, %1};\n\t"
      "mov.b64 xx, {%2, %2};\n\t"
      "add.rn.f32x2 va, va, xx;\n\t"
      "mov.b64 {%0, %1}, va;\n\t}"
      : "+f"(a), "+f"(b)
      : "f"(x));
}

// max(x, 0) that keeps a NaN (max.NaN)
__device__ __forceinline__ float max_nan0(float x) {
  float r;
  asm("max.NaN.f32 %0, %1, 0f00000000;" : "=f"(r) : "f"(x));
  return r;
}

// Distance keys of the mode-3 matrix: bits 30..15 of a distance that is
// >= 0 (or -0, +inf, NaN), an order-preserving 16-bit code (8 exponent and 8
// mantissa bits; -0 maps to the code of +0, +inf to 0xFF00, NaN above it).
// A key k stands for every distance in [k << 15, (k + 1) << 15) read as
// float bits: the distance rounded down to 8 mantissa bits.  Two keys per
// word, the first column in the low half (the lower address).
__device__ __forceinline__ uint32_t key16x2(float a, float b) {
  return ((__float_as_uint(a) >> 15) & 0xFFFFu) | ((__float_as_uint(b) << 1) & 0xFFFF0000u);
}
// the lower end of a distance's key bucket, as a float
__device__ __forceinline__ float key16_floor(float x) { return __uint_as_float((__float_as_uint(x) >> 15) << 15); }

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle,
// 8-row groups 1024 bytes apart (stride byte offset), version 1.
__device__ __forceinline__ uint64_t smem_desc(const void* p) {
  uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;              // start address
  d |= (uint64_t)(16 >> 4) << 16;            // leading byte offset (unused for SW128 K-major)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset
  d |= 1ull << 46;                           // descriptor version
  d |= 2ull << 61;                           // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N = BN, M = 128.
template <int BN>
__device__ __forceinline__ constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int BN>
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc<BN>()), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// The load split in two, for two chunks behind one wait: the issue, whose
// registers are not read before tmem_ld_wait (which waits for every earlier
// load of the thread) and, for the other chunk's registers, tmem_regs_after.
__device__ __forceinline__ void tmem_ld32_issue(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

#define HENN_R32_INOUT(r)                                                                                     \
  "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), \
      "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]),  \
      "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), \
      "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31])

__device__ __forceinline__ void tmem_ld_wait(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;" : HENN_R32_INOUT(r) : : "memory");
}

// no instruction: r is read only after this point (placed after a wait)
__device__ __forceinline__ void tmem_regs_after(uint32_t (&r)[32]) {
  asm volatile("" : HENN_R32_INOUT(r) : : "memory");
}
#undef HENN_R32_INOUT

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Replaces the root of a row's max-heap (heap[1..KP], heap[KP + 1] = 0) by
// a smaller key and sifts it down.  The heap is 4-ary: the children of node
// p are 4p - 2 .. 4p + 1 (node 8's last child is the sentinel), read as two
// 16-byte loads, three levels below the root where a binary heap has five.
static_assert(KP == 32, "node 8's children end at the sentinel KP + 1");
__device__ __forceinline__ void heap_replace(uint64_t* heap, uint64_t key) {
  int p = 1;
  for (int c = 2; c <= KP; c = 4 * p - 2) {
    const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(heap + c);
    const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(heap + c + 2);
    const bool ra = a.y > a.x, rb = b.y > b.x;
    const uint64_t ma = ra ? a.y : a.x, mb = rb ? b.y : b.x;
    const bool second = mb > ma;
    const uint64_t mv = second ? mb : ma;
    if (mv < key) break;  // keys are distinct
    heap[p] = mv;
    p = c + (second ? 2 + (rb ? 1 : 0) : (ra ? 1 : 0));
  }
  heap[p] = key;
}

}  // namespace tc

using namespace tc;

// EPI: epilogue warps, 4 (one per TMEM sub-partition; the per-row lists of
// modes 0-2 need it) or 8 (mode 3: two per sub-partition, each taking half of
// every tile's chunks); the launch has 64 + 32 * EPI threads
template <bool kStream, int BN, int EPI>
__global__ void __launch_bounds__(64 + 32 * EPI, 1)
    k_tile_topk_tc(const __grid_constant__ CUtensorMap ta_hi, const __grid_constant__ CUtensorMap ta_lo,
                   const __grid_constant__ CUtensorMap tb_hi, const __grid_constant__ CUtensorMap tb_lo,
                   const __grid_constant__ CUtensorMap to_d,
                   const float* __restrict__ norms, const float* __restrict__ norms_c, int64_t s, int64_t sc,
                   int32_t kc, int32_t mode, uint64_t* __restrict__ out, uint16_t* __restrict__ out_d, int64_t ldo,
                   float* __restrict__ out_cmin, int64_t ldc,
                   int32_t nsplit, int32_t* __restrict__ err, long long spin_limit, int32_t hold) {
  using Smem = typename std::conditional<kStream, SmemStr<BN>, SmemRes<BN>>::type;
  constexpr int NST = kStream ? NS_STR : NS;
  constexpr int B_CHUNK = BN * BK * 2;  // one plane of a B slice
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  Smem& sm = *reinterpret_cast<Smem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nrb = (s + BM - 1) / BM;
  // nsplit CTAs per row block (mode 3, which keeps no per-row lists), each
  // taking a contiguous run of the block's tiles
  const int64_t bid = blockIdx.x / nsplit;
  const int sp = (int)(blockIdx.x % nsplit);
  const int64_t rb = (mode == 0) ? (nrb - 1 - bid) : bid;
  const int64_t r0 = rb * BM;
  // s rows; sc columns (== s unless mode 2 or 3)
  const int64_t cend = (mode == 0) ? min(s, r0 + BM) : sc;
  const int nt_all = (int)((cend + BN - 1) / BN);
  const int tps = (nt_all + nsplit - 1) / nsplit;
  const int t0 = min(nt_all, sp * tps);
  const int nt = min(nt_all, t0 + tps) - t0;  // this CTA's tiles: t0 .. t0 + nt - 1
  const int chunks_per_tile = 2 * kc;  // (B_hi, B_lo) per 64-wide slice

  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      tc::mbar_init(&sm.full[i], 1);
      tc::mbar_init(&sm.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&sm.tfull[i], 1);
      tc::mbar_init(&sm.tempty[i], EPI);  // every epilogue warp frees it
    }
    tc::mbar_init(&sm.afull, 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  for (int i = threadIdx.x; i < BM * (KP + 2); i += blockDim.x)
    (&sm.heap[0][0])[i] = (i % (KP + 2) == KP + 1) ? 0ull : kEmpty;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(tc::smem_u32(&sm.tmem_base)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = sm.tmem_base;
  volatile int* abort_flag = &sm.abort;

  if (warp == 0) {
    // ---------------- TMA producer (with `hold` it issues nothing, so the
    // other warps' waits run out with no copy in flight: the host's way to
    // test the timeout path)
    if (lane == 0 && !hold) {
      long long it = 0;
      bool ok = true;
      if constexpr (!kStream) {
        tc::mbar_expect_tx(&sm.afull, (uint32_t)(2 * kc * A_CHUNK));
        for (int c = 0; c < kc; ++c) {
          tc::tma_load_2d(sm.a[c], &ta_hi, &sm.afull, c * BK, (int)r0);
          tc::tma_load_2d(sm.a[MAX_KC_RES + c], &ta_lo, &sm.afull, c * BK, (int)r0);
        }
        for (int lt = 0; lt < nt && ok; ++lt) {
          const int t = t0 + lt;
          for (int j = 0; j < chunks_per_tile && ok; ++j, ++it) {
            const int st = (int)(it % NST);
            const uint32_t ph = (uint32_t)((it / NST) & 1);
            if (!tc::mbar_wait(&sm.empty[st], ph ^ 1u, abort_flag, spin_limit)) {
              ok = false;
              break;
            }
            tc::mbar_expect_tx(&sm.full[st], (uint32_t)B_CHUNK);
            const int slice = j >> 1;
            tc::tma_load_2d(sm.b[st], (j & 1) ? &tb_lo : &tb_hi, &sm.full[st], slice * BK, t * BN);
          }
        }
      } else {
        // per slice: the A slice (hi | lo), B hi, B lo, in this order
        for (int lt = 0; lt < nt && ok; ++lt) {
          const int t = t0 + lt;
          for (int j = 0; j < kc && ok; ++j) {
            for (int part = 0; part < 3; ++part, ++it) {
              const int st = (int)(it % NST);
              const uint32_t ph = (uint32_t)((it / NST) & 1);
              if (!tc::mbar_wait(&sm.empty[st], ph ^ 1u, abort_flag, spin_limit)) {
                ok = false;
                break;
              }
              if (part == 0) {
                tc::mbar_expect_tx(&sm.full[st], (uint32_t)(2 * A_CHUNK));
                tc::tma_load_2d(sm.ring[st], &ta_hi, &sm.full[st], j * BK, (int)r0);
                tc::tma_load_2d(sm.ring[st] + A_CHUNK, &ta_lo, &sm.full[st], j * BK, (int)r0);
              } else {
                tc::mbar_expect_tx(&sm.full[st], (uint32_t)B_CHUNK);
                tc::tma_load_2d(sm.ring[st], part == 1 ? &tb_hi : &tb_lo, &sm.full[st], j * BK, t * BN);
              }
            }
          }
        }
      }
      if (!ok) {
        atomicOr(err, 1);
        sm.abort = 1;
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      bool ok = kStream ? true : tc::mbar_wait(&sm.afull, 0, abort_flag, spin_limit);
      long long it = 0;
      for (int lt = 0; lt < nt && ok; ++lt) {
        const int as = lt & 1;
        const uint32_t aph = (uint32_t)((lt >> 1) & 1);
        if (!tc::mbar_wait(&sm.tempty[as], aph ^ 1u, abort_flag, spin_limit)) {
          ok = false;
          break;
        }
        tc::fence_after();
        const uint32_t dt = tmem + (uint32_t)(as * BN);
        uint32_t acc = 0;
        if constexpr (!kStream) {
          for (int j = 0; j < chunks_per_tile; ++j, ++it) {
            const int st = (int)(it % NST);
            const uint32_t ph = (uint32_t)((it / NST) & 1);
            if (!tc::mbar_wait(&sm.full[st], ph, abort_flag, spin_limit)) {
              ok = false;
              break;
            }
            tc::fence_after();
            const int slice = j >> 1;
            const bool b_is_lo = (j & 1);
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              const uint64_t bd = tc::smem_desc(sm.b[st] + k * 32);
              // B_hi pairs with A_hi and A_lo; B_lo pairs with A_hi
              tc::mma_bf16<BN>(dt, tc::smem_desc(sm.a[slice] + k * 32), bd, acc);
              acc = 1;
              if (!b_is_lo) tc::mma_bf16<BN>(dt, tc::smem_desc(sm.a[MAX_KC_RES + slice] + k * 32), bd, 1);
            }
            tc::mma_commit(&sm.empty[st]);
          }
        } else {
          for (int j = 0; j < kc && ok; ++j, it += 3) {
            const int sa = (int)(it % NST), sh = (int)((it + 1) % NST), sl = (int)((it + 2) % NST);
            if (!tc::mbar_wait(&sm.full[sa], (uint32_t)((it / NST) & 1), abort_flag, spin_limit) ||
                !tc::mbar_wait(&sm.full[sh], (uint32_t)(((it + 1) / NST) & 1), abort_flag, spin_limit)) {
              ok = false;
              break;
            }
            tc::fence_after();
            const uint8_t* a_hi = sm.ring[sa];
            const uint8_t* a_lo = sm.ring[sa] + A_CHUNK;
            // B hi pairs with A hi and A lo; its stage is free after these
#pragma unroll
            for (int k = 0; k < BK / 16; ++k) {
              const uint64_t bd = tc::smem_desc(sm.ring[sh] + k * 32);
              tc::mma_bf16<BN>(dt, tc::smem_desc(a_hi + k * 32), bd, acc);
              acc = 1;
              tc::mma_bf16<BN>(dt, tc::smem_desc(a_lo + k * 32), bd, 1);
            }
            tc::mma_commit(&sm.empty[sh]);
            if (!tc::mbar_wait(&sm.full[sl], (uint32_t)(((it + 2) / NST) & 1), abort_flag, spin_limit)) {
              ok = false;
              break;
            }
            tc::fence_after();
            // B lo pairs with A hi
#pragma unroll
            for (int k = 0; k < BK / 16; ++k)
              tc::mma_bf16<BN>(dt, tc::smem_desc(a_hi + k * 32), tc::smem_desc(sm.ring[sl] + k * 32), 1);
            tc::mma_commit(&sm.empty[sa]);
            tc::mma_commit(&sm.empty[sl]);
          }
        }
        if (!ok) break;
        tc::mma_commit(&sm.tfull[as]);
      }
      if (!ok) {
        atomicOr(err, 2);
        sm.abort = 1;
      }
    }
  } else {
    // ---------------- epilogue: warps 2..5, or 2..9 in mode 3 (two warps
    // per TMEM sub-partition, each taking half of every tile's chunks)
    const int ew = warp - 2;
    const int sub = warp & 3;  // TMEM sub-partition of this warp
    constexpr int halves = EPI / 4;
    const int qlo = (ew >> 2) * (BN / 32) / halves, qhi = qlo + (BN / 32) / halves;  // this warp's chunks
    const int ews = ew & 3;  // per-sub-partition staging, shared by its warps on disjoint chunks
    const int row_l = 32 * sub + lane;
    const int64_t grow = r0 + row_l;
    const float nrow = grow < s ? norms[grow] : 0.f;
    // valid columns of this row: [0, lim), minus the row itself for kNN
    const int32_t lim = grow >= s ? 0 : (int32_t)(mode == 0 ? grow : sc);
    const int32_t self = mode == 1 ? (int32_t)grow : -1;
    const float kInf = __int_as_float(0x7f800000);
    // the row's threshold with its own norm folded in:
    // n_row + n_col - 2v <= thr  <=>  n_col - 2v <= thr - n_row
    float thr_adj = kInf;
    uint64_t* heap = sm.heap[row_l];
    uint64_t root = kEmpty;
    // mode 3 keeps no lists: the heap space holds each warp's 4 KB store
    // box (1024-byte aligned)
    uint32_t* m3_stage = reinterpret_cast<uint32_t*>(&sm.heap[0][0]) + ew * 1024;
    bool ok = true;
    float pn[BN / 32];  // column norms of the next tile, one per lane and chunk
#pragma unroll
    for (int q = 0; q < BN / 32; ++q) {
      const int64_t c = (int64_t)t0 * BN + q * 32 + lane;
      pn[q] = c < sc && q >= qlo && q < qhi ? __ldg(norms_c + c) : 0.f;
    }
    for (int lt = 0; lt < nt; ++lt) {
      const int t = t0 + lt;
      const int as = lt & 1;
      const uint32_t aph = (uint32_t)((lt >> 1) & 1);
      if (!tc::mbar_wait(&sm.tfull[as], aph, abort_flag, spin_limit)) {
        ok = false;
        break;
      }
      tc::fence_after();
      // this tile's column norms, staged once (read back as broadcasts);
      // the next tile's are loaded now and land while this one is drained
      float* ncs = sm.ncol[ews];
#pragma unroll
      for (int q = 0; q < BN / 32; ++q)
        if (q >= qlo && q < qhi) ncs[q * 32 + lane] = pn[q];
#pragma unroll
      for (int q = 0; q < BN / 32; ++q) {
        const int64_t c = (int64_t)(t + 1) * BN + q * 32 + lane;
        pn[q] = c < sc && q >= qlo && q < qhi ? __ldg(norms_c + c) : 0.f;
      }
      if (mode == 3 && out_cmin)
        for (int q = qlo; q < qhi; ++q) sm.s[ews][lane][q] = kInf;
      __syncwarp();
      const uint32_t tacc = tmem + ((uint32_t)(32 * sub) << 16) + (uint32_t)(as * BN);
      // n_col - 2<a,b> for the 32 columns of chunk q, in place, and their
      // minimum
      auto prep = [&](const int q, float (&v)[32]) {
        const float4* n4 = reinterpret_cast<const float4*>(ncs + q * 32);
        float vmin = kInf;
#pragma unroll
        for (int j4 = 0; j4 < 8; ++j4) {
          const float4 nn = n4[j4];
          tc::fma2_m2(v[4 * j4 + 0], v[4 * j4 + 1], nn.x, nn.y);
          tc::fma2_m2(v[4 * j4 + 2], v[4 * j4 + 3], nn.z, nn.w);
          vmin = fminf(vmin, fminf(fminf(v[4 * j4 + 0], v[4 * j4 + 1]), fminf(v[4 * j4 + 2], v[4 * j4 + 3])));
        }
        return vmin;
      };
      // the row lists: the columns of chunk c0 under the row's threshold
      // offered to its heap (rows in parallel, one per lane)
      auto lists = [&](const int64_t c0, float (&v)[32], const float vmin) {
        const bool maybe = vmin <= thr_adj;
        if (!__any_sync(0xffffffffu, maybe)) return;
        unsigned keep = 0;
        if (maybe) {
          // columns c0 + j valid for this row, as a bit mask
          const int32_t rem = lim - (int32_t)c0;
          unsigned vmask = rem >= 32 ? 0xffffffffu : (rem <= 0 ? 0u : ((1u << rem) - 1u));
          const int32_t so = self - (int32_t)c0;
          if (so >= 0 && so < 32) vmask &= ~(1u << so);
#pragma unroll
          for (int j = 0; j < 32; ++j) keep |= (v[j] <= thr_adj) ? (1u << j) : 0u;
          keep &= vmask;
        }
        if (keep) {
          // this lane's row: stage the passing values, then offer them to
          // the row's heap one by one
          float* srow = sm.s[ews][lane];
#pragma unroll
          for (int j = 0; j < 32; ++j) srow[j] = v[j];
          do {
            const int j = __ffs(keep) - 1;
            keep &= keep - 1;
            const float dv = fmaxf(nrow + srow[j], 0.f);
            const uint64_t key = pack(dv, (uint32_t)(c0 + j));
            if (!isinf(dv) && key < root) {
              tc::heap_replace(heap, key);
              root = heap[1];
              const float nthr = root == kEmpty ? kInf : key_dist(root);
              // slightly permissive: rounding of the folded threshold must
              // not drop a column the certified pool counts on
              thr_adj = nthr - nrow + 1e-6f * (fabsf(nthr) + fabsf(nrow));
            }
          } while (keep);
        }
        __syncwarp();
      };
      if (mode != 3) {
        // two chunks at a time: both TMEM loads behind one wait, the two
        // chunks' distance terms interleaved, then their inserts in chunk
        // order (the same lists as one chunk at a time)
#pragma unroll 1
        for (int q = 0; q < BN / 32; q += 2) {
          const int64_t ca = (int64_t)t * BN + q * 32, cb = ca + 32;
          uint32_t ra[32], rb[32];
          tc::tmem_ld32_issue(tacc + (uint32_t)q * 32, ra);
          tc::tmem_ld32_issue(tacc + (uint32_t)(q + 1) * 32, rb);
          tc::tmem_ld_wait(ra);
          tc::tmem_regs_after(rb);
          if (ca >= cend) continue;  // warp-uniform
          float va[32], vb[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            va[i] = __uint_as_float(ra[i]);
            vb[i] = __uint_as_float(rb[i]);
          }
          const float ma = prep(q, va);
          const float mb = prep(q + 1, vb);
          lists(ca, va, ma);
          if (cb < cend) lists(cb, vb, mb);  // warp-uniform
        }
      }
      // mode 3: the distances as 16-bit keys, two 32-column chunks (64
      // columns, one 128-byte row of the box) at a time behind one TMEM wait
#pragma unroll 1
      for (int q = qlo; q < qhi && mode == 3; q += 2) {
        const int64_t c0 = (int64_t)t * BN + q * 32;
        uint32_t ra[32], rb[32];
        tc::tmem_ld32_issue(tacc + (uint32_t)q * 32, ra);
        tc::tmem_ld32_issue(tacc + (uint32_t)(q + 1) * 32, rb);
        tc::tmem_ld_wait(ra);
        tc::tmem_regs_after(rb);
        if (c0 >= cend) continue;  // warp-uniform
        // the row's 64 distances, each formed as in the lists above (+inf
        // past the last column; NaN kept, which no selection takes), as
        // keys staged in this warp's 32 x 64 box in shared memory (128-byte
        // rows, 16-byte pieces swizzled by row, as the tensor map's 128B
        // swizzle expects) and written by one bulk tensor store
        uint32_t* buf = m3_stage;
        if (lane == 0) tc::bulk_wait_read_all();  // this warp's last store has read the box
        __syncwarp();
        uint4* brow = reinterpret_cast<uint4*>(buf + lane * 32);
        float cm[2] = {kInf, kInf};  // each chunk's minimum for this row (fminf passes over a NaN)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          uint32_t(&r)[32] = h == 0 ? ra : rb;
          const float4* n4 = reinterpret_cast<const float4*>(ncs + (q + h) * 32);
          const int64_t ch0 = c0 + 32 * h;
          if (ch0 + 32 <= sc) {  // warp-uniform: every column of the chunk valid
#pragma unroll
            for (int j4 = 0; j4 < 8; j4 += 2) {
              float o[8];
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const float4 nn = n4[j4 + u];
                float t0 = __uint_as_float(r[4 * (j4 + u) + 0]), t1 = __uint_as_float(r[4 * (j4 + u) + 1]);
                float t2 = __uint_as_float(r[4 * (j4 + u) + 2]), t3 = __uint_as_float(r[4 * (j4 + u) + 3]);
                tc::fma2_m2(t0, t1, nn.x, nn.y);
                tc::fma2_m2(t2, t3, nn.z, nn.w);
                tc::add2_s(t0, t1, nrow);
                tc::add2_s(t2, t3, nrow);
                o[4 * u + 0] = max_nan0(t0);
                o[4 * u + 1] = max_nan0(t1);
                o[4 * u + 2] = max_nan0(t2);
                o[4 * u + 3] = max_nan0(t3);
              }
#pragma unroll
              for (int e = 0; e < 8; ++e) cm[h] = fminf(cm[h], o[e]);
              brow[(4 * h + j4 / 2) ^ (lane & 7)] =
                  make_uint4(key16x2(o[0], o[1]), key16x2(o[2], o[3]), key16x2(o[4], o[5]), key16x2(o[6], o[7]));
            }
          } else {
#pragma unroll
            for (int j4 = 0; j4 < 8; j4 += 2) {
              float o[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) {
                const int j = 4 * j4 + e;
                const float nc = ncs[(q + h) * 32 + j];
                o[e] = ch0 + j < sc ? max_nan0(nrow + fmaf(-2.f, __uint_as_float(r[j]), nc)) : kInf;
                cm[h] = fminf(cm[h], o[e]);
              }
              brow[(4 * h + j4 / 2) ^ (lane & 7)] =
                  make_uint4(key16x2(o[0], o[1]), key16x2(o[2], o[3]), key16x2(o[4], o[5]), key16x2(o[6], o[7]));
            }
          }
        }
        if (out_cmin) {
          // the lower ends of the minima's key buckets: the minimum of a
          // chunk's key lower ends
          sm.s[ews][lane][q] = key16_floor(cm[0]);
          sm.s[ews][lane][q + 1] = key16_floor(cm[1]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) tc::tma_store_2d(&to_d, buf, (int)c0, (int)(r0 + 32 * sub));
        __syncwarp();
      }
      if (mode == 3 && out_cmin && grow < s) {
        // this row's chunk minima of this warp's chunks, as 8-byte stores
        float2* dst = reinterpret_cast<float2*>(out_cmin + grow * ldc + (int64_t)t * (BN / 32) + qlo);
        const float* src = sm.s[ews][lane] + qlo;
        for (int j = 0; j < (qhi - qlo) / 2; ++j) dst[j] = make_float2(src[2 * j], src[2 * j + 1]);
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&sm.tempty[as]);
    }
    if (!ok) {
      if (lane == 0) atomicOr(err, 4);
      sm.abort = 1;
    }
    if (mode == 3 && lane == 0) tc::bulk_wait_all();
    // this warp's 32 rows, each heap sorted ascending across the warp
    __syncwarp();
    for (int i = 0; i < 32 && mode != 3; ++i) {
      const int64_t gr = r0 + 32 * sub + i;
      const uint64_t x = warp_sort_asc(sm.heap[32 * sub + i][1 + lane]);
      if (gr < s) out[gr * KP + lane] = x;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (sm.abort) {
    // let any bulk copy still in flight land before the CTA leaves
    __nanosleep(100000);
  }
  if (warp == 1) {
    tc::fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem));
  }
}

// ------------------------------------------------------------- host side

__global__ void k_split_bf16(const float* __restrict__ x, int64_t s, int32_t dpad, int32_t dk,
                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t total = s * dk;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / dk;
    const int32_t k = (int32_t)(i - r * dk);
    const float v = k < dpad ? x[r * dpad + k] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
  }
}

// Wait bound of the pipeline's mbarrier waits and the producer hold, from
// the environment: HENN_TILE_SPIN_LIMIT (iterations of a try_wait that may
// suspend up to 20 us; default and maximum kSpinLimit) and
// HENN_TILE_HOLD_LOADS=1 (the producer issues no copy).  Together they make
// the waits run out on purpose, with nothing in flight, so that tests can
// check that a timeout comes back as an error status and leaves the
// context usable.
static void wait_policy(long long* spin_limit, int32_t* hold) {
  *spin_limit = kSpinLimit;
  *hold = 0;
  if (const char* e = std::getenv("HENN_TILE_SPIN_LIMIT")) {
    const long long v = std::atoll(e);
    if (v >= 1 && v < kSpinLimit) *spin_limit = v;
  }
  if (const char* e = std::getenv("HENN_TILE_HOLD_LOADS")) *hold = std::atoi(e) != 0;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 16-bit key matrix of `rows` x ld, stored by boxes of 32 rows x 64 keys
// (128-byte box rows, 128B swizzle)
static bool make_store_map(CUtensorMap* m, const void* base, int64_t rows, int64_t ld) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {64, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

static bool make_map(CUtensorMap* m, const void* base, int64_t rows, int32_t dk, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)dk, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)dk * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool tc_tiles_supported(int32_t dpad, int32_t KPv) { return dpad <= BK * MAX_KC && KPv == KP; }

static_assert(sizeof(SmemRes<256>) + 1024 <= 227 * 1024, "shared memory of one CTA");
static_assert(sizeof(SmemStr<256>) + 1024 <= 227 * 1024, "shared memory of one CTA");
static_assert(sizeof(((SmemRes<128>*)nullptr)->heap) >= 4 * 8192, "mode 3 store boxes fit in the heap space");
static_assert(offsetof(SmemRes<128>, heap) % 1024 == 0 && offsetof(SmemRes<256>, heap) % 1024 == 0,
              "store boxes 1024-byte aligned");
static_assert(offsetof(SmemStr<128>, heap) % 1024 == 0 && offsetof(SmemStr<256>, heap) % 1024 == 0,
              "store boxes 1024-byte aligned");
static_assert((2 * A_CHUNK) <= STAGE && BN_MAX * BK * 2 <= STAGE && A_CHUNK % 1024 == 0,
              "an A slice (hi | lo) or a plane of a B slice fills one stage");

// The kernel variant for kc slices of 64 values per plane, and its shared
// memory; the dynamic shared-memory attribute is set once per device and
// variant.
struct TileVariant {
  void (*fn)(CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, CUtensorMap, const float*, const float*, int64_t,
             int64_t, int32_t, int32_t, uint64_t*, uint16_t*, int64_t, float*, int64_t, int32_t, int32_t*, long long,
             int32_t);
  size_t smem;
};

static cudaError_t tile_variant(int32_t kc, int32_t bn, bool matrix, TileVariant* v) {
  static std::atomic<bool> attr_set[8][64];
  const int stream = kc > MAX_KC_RES ? 1 : 0;
  const int narrow = bn == 128 ? 1 : 0;
  const int which = 4 * (matrix ? 1 : 0) + 2 * stream + narrow;
  switch (which) {
    case 0: v->fn = k_tile_topk_tc<false, 256, 4>; v->smem = sizeof(SmemRes<256>); break;
    case 1: v->fn = k_tile_topk_tc<false, 128, 4>; v->smem = sizeof(SmemRes<128>); break;
    case 2: v->fn = k_tile_topk_tc<true, 256, 4>; v->smem = sizeof(SmemStr<256>); break;
    case 3: v->fn = k_tile_topk_tc<true, 128, 4>; v->smem = sizeof(SmemStr<128>); break;
    case 4: v->fn = k_tile_topk_tc<false, 256, 8>; v->smem = sizeof(SmemRes<256>); break;
    case 5: v->fn = k_tile_topk_tc<false, 128, 8>; v->smem = sizeof(SmemRes<128>); break;
    case 6: v->fn = k_tile_topk_tc<true, 256, 8>; v->smem = sizeof(SmemStr<256>); break;
    default: v->fn = k_tile_topk_tc<true, 128, 8>; v->smem = sizeof(SmemStr<128>); break;
  }
  v->smem += 1024;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64 || !attr_set[which][dev].load()) {
    e = cudaFuncSetAttribute(v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v->smem);
    if (e != cudaSuccess) return e;
    if (dev < 64) attr_set[which][dev].store(true);
  }
  return cudaSuccess;
}

cudaError_t launch_tile_topk_tc(const float* xo, const float* norms, int64_t s, int32_t dpad, int32_t mode,
                                uint64_t* out, void* scratch_hi, void* scratch_lo, int32_t* err, cudaStream_t st) {
  const int32_t dk = ((dpad + BK - 1) / BK) * BK;
  __nv_bfloat16* hi = static_cast<__nv_bfloat16*>(scratch_hi);
  __nv_bfloat16* lo = static_cast<__nv_bfloat16*>(scratch_lo);
  k_split_bf16<<<152 * 8, 256, 0, st>>>(xo, s, dpad, dk, hi, lo);
  CUtensorMap mah, mal, mbh, mbl;
  if (!make_map(&mah, hi, s, dk, BM) || !make_map(&mal, lo, s, dk, BM) || !make_map(&mbh, hi, s, dk, BN_MAX) ||
      !make_map(&mbl, lo, s, dk, BN_MAX))
    return cudaErrorInvalidValue;
  TileVariant v;
  cudaError_t e = tile_variant(dk / BK, BN_MAX, false, &v);
  if (e != cudaSuccess) return e;
  const int64_t nrb = (s + BM - 1) / BM;
  CUtensorMap none;  // no matrix output in modes 0 and 1
  std::memset(&none, 0, sizeof(none));
  long long spin_limit;
  int32_t hold;
  wait_policy(&spin_limit, &hold);
  v.fn<<<(unsigned)nrb, 192, v.smem, st>>>(mah, mal, mbh, mbl, none, norms, norms, s, s, dk / BK, mode, out, nullptr,
                                           0, nullptr, 0, 1, err, spin_limit, hold);
  return cudaGetLastError();
}

void launch_split_bf16(const float* x, int64_t s, int32_t dpad, int32_t dk, void* hi, void* lo, cudaStream_t st) {
  k_split_bf16<<<152 * 8, 256, 0, st>>>(x, s, dpad, dk, static_cast<__nv_bfloat16*>(hi),
                                        static_cast<__nv_bfloat16*>(lo));
}

bool make_column_maps(const void* b_hi, const void* b_lo, int64_t nb, int32_t dk, void* maps) {
  CUtensorMap* m = static_cast<CUtensorMap*>(maps);
  return dk % BK == 0 && dk / BK <= MAX_KC && nb >= 1 && make_map(&m[0], b_hi, nb, dk, 256) &&
         make_map(&m[1], b_lo, nb, dk, 256) && make_map(&m[2], b_hi, nb, dk, 128) && make_map(&m[3], b_lo, nb, dk, 128);
}

cudaError_t launch_tile_cross_tc(const void* a_hi, const void* a_lo, const float* a_norms, int64_t na,
                                 const void* b_maps, const float* b_norms, int64_t nb, int32_t dk, uint64_t* out,
                                 uint16_t* out_d, int64_t ldo, float* out_cmin, int64_t ldc, int32_t* err,
                                 int32_t tile_n, cudaStream_t st) {
  const int32_t BN = tile_n == 128 ? 128 : 256;
  if (dk % BK != 0 || dk / BK > MAX_KC || na < 1 || nb < 1) return cudaErrorInvalidValue;
  // key rows of whole 128-byte lines, 128-byte aligned (the selection drops them from L2 by line)
  if (out_d && (ldo % 64 != 0 || ldo < nb || (reinterpret_cast<uintptr_t>(out_d) & 127) != 0))
    return cudaErrorInvalidValue;
  // chunk minima: rows of ldc floats covering every tile's BN / 32 chunks, 16-byte aligned
  if (out_cmin && (!out_d || ldc % 8 != 0 || ldc * 32 < (nb + 255) / 256 * 256 ||
                   (reinterpret_cast<uintptr_t>(out_cmin) & 15) != 0))
    return cudaErrorInvalidValue;
  CUtensorMap mah, mal;
  if (!make_map(&mah, a_hi, na, dk, BM) || !make_map(&mal, a_lo, na, dk, BM)) return cudaErrorInvalidValue;
  const CUtensorMap& mbh = static_cast<const CUtensorMap*>(b_maps)[BN == 128 ? 2 : 0];
  const CUtensorMap& mbl = static_cast<const CUtensorMap*>(b_maps)[BN == 128 ? 3 : 1];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  TileVariant v;
  e = tile_variant(dk / BK, BN, out_d != nullptr, &v);
  if (e != cudaSuccess) return e;
  const int64_t nrb = (na + BM - 1) / BM;
  // mode 3: split each row block's tiles over nsplit CTAs (one CTA per SM
  // fits), choosing the split with the fewest tile-times over all waves
  int32_t nsplit = 1;
  if (out_d) {
    int sms = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
    const int64_t nt_all = (nb + BN - 1) / BN;
    double best = 1e300;
    for (int64_t k = 1; k <= nt_all && k <= 16; ++k) {
      const int64_t waves = (nrb * k + sms - 1) / sms;
      const double cost = (double)waves * (double)((nt_all + k - 1) / k + 1);  // +1: a CTA's fixed work
      if (cost < best) {
        best = cost;
        nsplit = (int32_t)k;
      }
    }
  }
  CUtensorMap mo;
  std::memset(&mo, 0, sizeof(mo));
  if (out_d && !make_store_map(&mo, out_d, na, ldo)) return cudaErrorInvalidValue;
  long long spin_limit;
  int32_t hold;
  wait_policy(&spin_limit, &hold);
  // mode 3: eight epilogue warps (two per TMEM sub-partition); mode 2: four
  v.fn<<<(unsigned)(nrb * nsplit), out_d ? 64 + 32 * 8 : 64 + 32 * 4, v.smem, st>>>(mah, mal, mbh, mbl, mo, a_norms, b_norms, na, nb, dk / BK,
                                                     out_d ? 3 : 2, out, out_d, ldo, out_cmin, ldc, nsplit, err,
                                                     spin_limit, hold);
  return cudaGetLastError();
}

}  // namespace henn
