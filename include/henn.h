/*
 * henn.h -- C ABI of libhenn, a GB300 (sm_103a) implementation of the data
 * parallel hot path of HENN, the Hierarchical epsilon-Net Navigation graph
 * for approximate nearest neighbour search (arXiv 2505.17368).
 *
 * The problem (Sec. 2, "Data Model" and "Problem setting"): n points x_i in
 * R^d with a distance (l2, or angular 1 - cos per App. G); for a query q
 * return k points of X with the smallest distance, approximately, with high
 * Recall@k.  The index (Def. 1) is a stack of layers L_0 = X, L_1, ..., L_L,
 * each an eps-net of the one below it for ring ranges (Def. 2, Eq. 1,
 * Alg. 1, Alg. 2), each with its own navigable graph (App. B), linked
 * between layers by the copies of the same point.  A query descends from a
 * random node of the top layer by greedy search (Alg. 4) and runs a beam of
 * width ef on the bottom layer (Sec. 2.2, last paragraph).
 *
 * Conventions shared by every call
 *  - Vectors are float32, row-major, rows of d values, no padding.
 *  - Pointers marked "device" are CUDA device pointers of the current
 *    device; "host" pointers are ordinary (pageable or pinned) memory.
 *    Calls with an `on_device` flag take all their array arguments from
 *    that side.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Device-side
 *    calls are stream ordered: they return after enqueueing, results are
 *    valid once the stream has been synchronised.  Host-side calls
 *    synchronise the stream before returning.
 *  - The caller owns every array it passes; the library copies what it
 *    keeps.  The index owns its device memory until henn_free().
 *  - No call throws.  Each returns a henn_status; on failure nothing is
 *    written to *out handles and henn_last_error() describes the failure.
 *  - A const index may be searched concurrently from several host threads
 *    and streams.
 *
 * Random numbers (ring ranges, samples, insertion order, entry nodes) come
 * from SplitMix64 (Steele, Lea & Flood 2014) used counter-style:
 *   mix64(z)      = SplitMix64 output finaliser
 *   derive(h, w)  = mix64(h + (w + 1) * 0x9E3779B97F4A7C15)
 *   bounded(u, s) = floor(u * s / 2^64)
 * keyed by the tags below; the same seed gives the same index on any GPU.
 */
#ifndef HENN_H
#define HENN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HENN_ABI_VERSION 1

/* RNG stream tags (ASCII words). */
#define HENN_TAG_SAMPLE 0x53414D50ULL  /* "SAMP" Alg. 2 draws with replacement        */
#define HENN_TAG_RCENTRE 0x5243454EULL /* "RCEN" centre of a sampled ring range        */
#define HENN_TAG_RSTART 0x52535441ULL  /* "RSTA" first rank of a sampled ring range    */
#define HENN_TAG_ORDER 0x4F524452ULL   /* "ORDR" NSW insertion order of a layer        */
#define HENN_TAG_ENTRY 0x454E5452ULL   /* "ENTR" random top-layer node of a query      */
#define HENN_TAG_HALVE 0x48414C56ULL   /* "HALV" coin of a matched pair, Alg. 3 halving */
#define HENN_TAG_INSERT 0x494E5352ULL  /* "INSR" layer promotion coin of an inserted point */

typedef enum {
  HENN_OK = 0,
  HENN_ERR_INVALID_ARG = 1,      /* a size, pointer or parameter is out of range      */
  HENN_ERR_OOM = 2,              /* device allocation failed                          */
  HENN_ERR_CUDA = 3,             /* a CUDA runtime call or kernel failed              */
  HENN_ERR_EPSNET_NOT_FOUND = 4, /* Alg. 2 found no eps-net within max_attempts       */
  HENN_ERR_TIMEOUT = 5,          /* a bounded device wait ran out                     */
  HENN_ERR_UNSUPPORTED = 6,      /* valid request this build cannot serve             */
  HENN_ERR_BUSY = 7              /* serving: no request slot or ring space right now  */
} henn_status;

typedef enum { HENN_L2 = 0, HENN_ANGULAR = 1 } henn_metric;

/* Storage of the vectors the search traverses.  BF16 and FP8 keep an FP32
 * copy as well, used for the exact rerank of the final candidates. */
typedef enum { HENN_F32 = 0, HENN_BF16 = 1, HENN_FP8E4M3 = 2 } henn_storage;

/* Navigable graph of each layer (App. B; App. G "Navigation Graphs"). */
typedef enum { HENN_GRAPH_NSW = 0, HENN_GRAPH_KNN = 1 } henn_graph;

/* Layer sampler: SAMPLING = Alg. 2 (draws with replacement, ring-range
 * verification, Las-Vegas retries); HALVING = Alg. 3 BuildEpsNetDiscV2 (m
 * halving steps over a matching of consecutive list entries, one member of
 * each pair kept by a coin, no verification). */
typedef enum { HENN_SAMPLER_SAMPLING = 0, HENN_SAMPLER_HALVING = 1 } henn_sampler;

/* Engine for the construction distance tiles: AUTO = tcgen05 where it
 * applies (M <= 16; rows of up to 128 values keep the row block resident in
 * shared memory, wider rows stream it slice by slice), else SIMT FP32. */
typedef enum { HENN_TILES_AUTO = 0, HENN_TILES_SIMT = 1, HENN_TILES_TCGEN05 = 2 } henn_tiles;

/* ------------------------------------------------------------------ build */

typedef struct {
  uint32_t struct_size;  /* sizeof(henn_build_params), for ABI checks          */
  int32_t metric;        /* henn_metric                                         */
  int32_t storage;       /* henn_storage                                        */
  int32_t graph;         /* henn_graph                                          */
  int32_t m;             /* layer decay 2^m (Alg. 1, Lemma 1); 1..8, default 4  */
  int32_t max_layers;    /* L of Alg. 1; 0 = while |L_{i-1}| >= 2^m (Cor. 3)    */
  double eps_c0;         /* c0 of Eq. 1; default 1.0                            */
  int32_t num_ranges;    /* r, the "range size" of App. G; default 100          */
  int32_t max_attempts;  /* Las-Vegas repeats of Alg. 2 per layer; default 64   */
  int32_t M;             /* forward links per inserted point; default 16        */
  int32_t Mmax;          /* adjacency row width; 32 (only 32 is supported)      */
  int32_t tiles;         /* henn_tiles                                          */
  uint64_t seed;         /* index seed                                          */
  int32_t sampler;       /* henn_sampler; default SAMPLING                      */
  double resample_share; /* App. C, Delete: an upper layer whose live points
                            fall below this share of a fresh sample of the
                            live layer below, ceil(live / 2^m), is resampled
                            and the hierarchy rebuilt above it; default 0.5,
                            <= 0: never (tombstones only)                    */
} henn_build_params;

/* Fills *p with the defaults above (struct_size included). */
void henn_build_params_default(henn_build_params* p);

typedef struct henn_index henn_index; /* opaque, owned by the library */

/*
 * henn_build -- BuildHENN (Alg. 1).
 * X: n x d float32 (device if x_on_device, else host); 1 <= n < 2^31,
 * 1 <= d <= 1024, finite values.  For every layer i >= 1 (while i <=
 * max_layers and |L_{i-1}| >= 2^m): draw ceil(|L_{i-1}|/2^m) samples of
 * L_{i-1} with replacement (Alg. 2, Cor. 2), keep the distinct ones, accept
 * them when every one of num_ranges random ring ranges (Def. 2) holding
 * floor(eps*s)+1 points, eps from Eq. 1, contains one of them (IsEpsNet,
 * App. B practical implementation), else draw again; with
 * sampler = HENN_SAMPLER_HALVING the layer is instead m halving steps of
 * L_{i-1} (Alg. 3, BuildEpsNetDiscV2).  Every layer then gets
 * its navigable graph: each point links to the M nearest points inserted
 * before it (NSW, App. B; or its M nearest overall for HENN_GRAPH_KNN) and
 * each row keeps its nearest predecessor plus the nearest Mmax-1 of its
 * forward and reverse links.
 * On success *out owns device memory for the vectors, layers and graphs.
 * Errors: HENN_ERR_INVALID_ARG, HENN_ERR_OOM, HENN_ERR_CUDA,
 * HENN_ERR_EPSNET_NOT_FOUND.  Synchronises `stream` before returning.
 */
henn_status henn_build(const float* X, int64_t n, int32_t d, int32_t x_on_device,
                       const henn_build_params* p, void* stream, henn_index** out);

/*
 * henn_insert -- Insert (App. C, dynamic setting) of n_new points, appended
 * after the indexed ones: the j-th gets global id n + j.  X: n_new x d
 * float32 (device if x_on_device, else host).  Each point joins layer 0 and
 * then layer i while it is in layer i-1 and its coin
 * bounded(derive(derive(derive(seed, INSR), id), i), 2^m) is 0 (the rate at
 * which the built layers thin out; no layer above L is created).  In every
 * layer it joins it is appended last in the insertion order, so its
 * forward list is its M nearest current members (exact FP32, ties by
 * position), points of one call being inserted one after another; the
 * layer's adjacency is then the edge rule over the updated forward lists
 * (the rows of its forward neighbours gain it as a reverse link).  Device
 * arrays grow by doubling.  NSW graphs only (HENN_ERR_UNSUPPORTED for kNN
 * graphs, where earlier points' own lists would change).  Synchronises
 * `stream` before returning.  Not safe concurrently with searches on idx;
 * servers made from idx before the call still point at the old arrays and
 * must be destroyed first.
 */
henn_status henn_insert(henn_index* idx, const float* X, int64_t n_new, int32_t x_on_device, void* stream);

/*
 * henn_delete -- Delete (App. C).  The points with these global ids (HOST
 * array of n int64, each in [0, number of points)) no longer appear in
 * search results: they stay in their layers and graphs as waypoints
 * (tombstones), and a result is the first k live entries of the final
 * candidate list.  Then, as App. C prescribes when a layer has shrunk too
 * far: the lowest upper layer i whose live points number fewer than
 * resample_share (of the build parameters) times ceil(live(L_{i-1}) / 2^m)
 * is resampled from the live points of layer i - 1 (Alg. 2, or Alg. 3, with
 * the build's seed and layer numbers) and the hierarchy is rebuilt from it
 * to the root (membership, down pointers, graphs, traversal copies); layer
 * 0 keeps every point.  Servers made from idx before the call do not see
 * it and must be destroyed first.  Not safe concurrently with searches on
 * idx.  Synchronises `stream`.  Errors: HENN_ERR_INVALID_ARG for an id out
 * of range; a failed resampling as henn_build (HENN_ERR_EPSNET_NOT_FOUND).
 */
henn_status henn_delete(henn_index* idx, const int64_t* ids, int64_t n, void* stream);

/* Releases the index and its device memory.  NULL is a no-op. */
void henn_free(henn_index* idx);

/* ----------------------------------------------------------------- search */

typedef struct {
  uint32_t struct_size;       /* sizeof(henn_search_params)                         */
  const int32_t* k;           /* per-query k, or NULL to use k_uniform              */
  const int32_t* ef;          /* per-query beam width, or NULL to use ef_uniform    */
  int32_t k_uniform;          /* default 10                                         */
  int32_t ef_uniform;         /* default 64; a beam is never narrower than k        */
  int32_t rerank_mult;        /* BF16/FP8: exact FP32 rerank of the best
                                 rerank_mult * k candidates; 0 = 4                  */
  const uint64_t* query_keys; /* per-query RNG key for the entry node, or NULL to
                                 use the query's row index                          */
  int32_t* stats;             /* optional, 4 int32 per query: distance evaluations,
                                 layer-0 expansions, upper-layer moves, visited-set
                                 evictions                                          */
  int32_t warps_per_block;    /* 0 = autotuned                                      */
  int32_t hash_bits;          /* log2 visited-set slots per query, 0 = autotuned    */
  int32_t ef_upper;           /* beam width on layers >= 1; 0 or 1 = GreedySearch of
                                 Alg. 4 (default 1)                                 */
  int32_t descend_all;        /* with ef_upper > 1: enter each layer at the copies of
                                 all candidates of the layer above instead of the
                                 best one only (default 0)                          */
  int32_t ef_l1;              /* beam width on layer 1 only; 0 = ef_upper          */
  int32_t exact_upper;        /* upper layers of at most this many points give
                                 their exact candidate set (the layer's nearest
                                 max(width, 1) points, by the traversal distance)
                                 instead of a walk; 0 = never (default).  Only the
                                 lowest such layer is computed: its result
                                 replaces those of the layers above it           */
  int32_t exact_method;       /* how that layer's set is found (henn_exact_method):
                                 SORT: per query, every point evaluated and sorted
                                 in the visited table (layer of at most
                                 2^(hash_bits - 1) points; default);
                                 TILES: one batched distance-tile launch
                                 (tcgen05) gives each query 32
                                 candidates, rescored in traversal precision and
                                 kept when a tile-error certificate proves them
                                 to hold the set, else a scan of the layer;
                                 SCAN: every point evaluated, running top 32.
                                 TILES and SCAN: any layer size; with descend_all
                                 the layer's width must be <= 32.  All three give
                                 the same set                                     */
  int32_t time_kernel;        /* 1: record device events around this call's
                                 search launches (henn_last_search_ms)           */
  int32_t team_size;          /* warps answering one query: 1 (default), 2 or 4;
                                 0 = 1.  The team's warps share the distance work
                                 of every beam expansion (shorter latency per
                                 query, fewer queries in flight); results do not
                                 depend on it.  Must divide warps_per_block     */
  int32_t tile_n;             /* columns per tensor-core tile of exact_method
                                 TILES: 128 or 256 (0 = 256); same results      */
} henn_search_params;

/* exact_method values */
typedef enum { HENN_EXACT_SORT = 0, HENN_EXACT_TILES = 1, HENN_EXACT_SCAN = 2 } henn_exact_method;

void henn_search_params_default(henn_search_params* sp);

/*
 * henn_search -- Query of Alg. 4 for a batch: one persistent search launch,
 * preceded with exact_method TILES by the query-preparation, distance-tile
 * and top-32 selection launches of the exact layer.
 * Q: nq x d float32.  Per query: entry = a random node of the top layer
 * (keyed by query_keys[q]), greedy search (Alg. 4 GreedySearch) on layers
 * L..1 (or a beam of width ef_upper, the candidate set of Sec. 2.2 applied
 * on every layer), each entered at the copy of the previous result, then the
 * best-first beam of width max(ef, k) on layer 0; BF16/FP8 indexes then
 * rerank the best rerank_mult*k candidates with exact FP32 distances.
 * out_ids (int64) / out_dists (float32): nq rows of out_stride >= max k;
 * row q holds k[q] results in ascending distance (l2: Euclidean distance,
 * angular: 1 - cos), padded with -1 / +inf.  All arrays (Q, k, ef,
 * query_keys, stats, outputs) are device pointers if q_on_device, else host
 * pointers (the call then copies, runs and synchronises).  Host queries and
 * host outputs in page-locked memory that the device can address
 * (cudaHostAlloc, cudaMallocHost, cudaHostRegister with mapping) are read
 * and written in place by the kernels over the host link instead of being
 * staged through device memory (the outputs only when both are); the
 * caller must not touch them until the call returns.
 * Errors: HENN_ERR_INVALID_ARG (k < 1, k > 1024, ef > 4096, stride < k,
 * NULL pointers), HENN_ERR_OOM, HENN_ERR_CUDA.
 */
henn_status henn_search(const henn_index* idx, const float* Q, int64_t nq, int32_t q_on_device,
                        const henn_search_params* sp, int64_t* out_ids, float* out_dists,
                        int32_t out_stride, void* stream);

/*
 * henn_last_search_ms -- device time of the search-kernel launches of the
 * last henn_search on this index made with time_kernel = 1 (events recorded
 * on its stream, around the launches only: query preparation and the tile
 * launch of exact_method TILES are outside), and the number of kernel
 * launches that call made.  Waits for the end event.  Either output may be
 * NULL.  Errors: HENN_ERR_INVALID_ARG if no timed search ran on the index.
 * One timed search at a time per index.
 */
henn_status henn_last_search_ms(const henn_index* idx, float* ms, int32_t* launches);

/* ------------------------------------------------------ introspection */

#define HENN_MAX_LAYERS 32

typedef struct {
  uint32_t struct_size;
  int64_t n;
  int32_t d, metric, storage, graph, M, Mmax;
  int32_t L;                               /* layers above L_0                */
  int64_t sizes[HENN_MAX_LAYERS];          /* |L_i|, i = 0..L                 */
  int32_t attempts[HENN_MAX_LAYERS];       /* Alg. 2 attempt that succeeded   */
  int32_t ambiguous_rings[HENN_MAX_LAYERS];/* rings re-decided in FP64        */
  int64_t device_bytes;                    /* index memory on the device      */
  int64_t uncertified_rows;                /* rows whose tile candidates had to
                                              be recomputed exactly           */
  double build_seconds;                    /* wall time of henn_build         */
  double tile_seconds;                     /* device time of the distance-tile
                                              launches (CUDA events)          */
  double tile_flops;                       /* their algorithmic flops: 2 d per
                                              valid (row, column) pair        */
  int32_t tile_engine;                     /* henn_tiles used for layer 0     */
  int32_t graph_instantiations;            /* build steps run as CUDA graphs:
                                              executable graphs instantiated  */
  int32_t graph_updates;                   /* ... and steps that relaunched an
                                              instantiated graph updated in
                                              place (same topology)           */
} henn_index_info;

henn_status henn_index_get_info(const henn_index* idx, henn_index_info* info);

/*
 * Copies layer `layer` to HOST arrays (any may be NULL):
 *   ids   [|L_i|]        global point ids, ascending
 *   down  [|L_i|]        position of each point in layer i-1 (layer >= 1)
 *   adj   [|L_i| * Mmax] layer-local neighbour indices, -1 padded
 *   fwd   [|L_i| * M]    forward links (nearest earlier-inserted points)
 *   fwd_d [|L_i| * M]    their distances (squared l2, or 1 - cos)
 * Synchronises the device.
 */
henn_status henn_index_get_layer(const henn_index* idx, int32_t layer, int32_t* ids, int32_t* down,
                                 int32_t* adj, int32_t* fwd, float* fwd_d);

/*
 * henn_greedy_probe -- GreedySearch of Alg. 4 on one layer of the index from
 * given start nodes, one probe per (query, start).  The recall bound
 * rho_delta of Def. 3 is the smallest k such that a probe from a random start
 * ends among the query's k nearest points with probability >= delta; this
 * call gives the end points to rank.
 *   layer     0..L
 *   Q         nq x d float32 query rows, DEVICE memory
 *   starts    nq x S int32 start positions in the layer (0 .. |L_layer|-1),
 *             DEVICE memory; a start outside that range yields -1
 *   out_node  nq x S int32 DEVICE: the local minimum reached (layer position;
 *             layer 0 positions are the global ids)
 *   out_dist  nq x S float32 DEVICE: its distance to the query in the
 *             traversal precision (squared l2, or 2 (1 - cos))
 *   out_hops  nq x S int32 DEVICE, or NULL: moves made
 * Ties go to the smaller index, and the walk moves only to a strictly closer
 * node.  Asynchronous on `stream`.  Errors: HENN_ERR_INVALID_ARG for a bad
 * layer, NULL pointers or S < 1.
 */
henn_status henn_greedy_probe(const henn_index* idx, int32_t layer, const float* Q, int64_t nq, const int32_t* starts,
                              int32_t S, int32_t* out_node, float* out_dist, int32_t* out_hops, void* stream);

/* ------------------------------------------------- standalone kernels */

/*
 * Exact k nearest neighbours of each query among the n base vectors (the
 * k-NN query of Sec. 2): tiled distances plus an exact FP32 rerank.  All
 * pointers device; out rows of k (int64 ids, float distances as in
 * henn_search).  1 <= k <= 112, 1 <= d <= 1024.
 */
henn_status henn_exact_knn(const float* X, int64_t n, int32_t d, const float* Q, int64_t nq, int32_t k,
                           int32_t metric, int64_t* out_ids, float* out_dists, void* stream);

/*
 * Precision copy of rows (device pointers): HENN_BF16 writes n*d uint16
 * (round to nearest even); HENN_FP8E4M3 writes n*d bytes of E4M3 codes of
 * x / scale with scale = max|x_row| / 448 (FP32; 1 for an all-zero row),
 * round to nearest even, saturating, and the n scales.
 */
henn_status henn_quantize_rows(const float* X, int64_t n, int32_t d, int32_t storage, void* out,
                               float* scales, void* stream);

/*
 * henn_search_host_noalloc -- henn_search for callers that cannot allocate
 * device memory.  The paper has no counterpart: this is a deployment
 * variant of the same batched search (same kernel, same results as
 * henn_search with host buffers and uniform k / ef).
 *
 * Who needs it: processes whose device memory belongs to another allocator
 * (a serving framework's arena, a deep-learning framework's caching pool)
 * and code that must not allocate while it runs.  henn_search with host
 * buffers allocates device staging and a work counter on every call; this
 * call allocates nothing.  Its scratch -- the work counter, the device copy
 * of the queries and of the results -- is one file-scope device array of
 * 16 MiB that every GPU loading the library holds until the process exits.
 *
 * Q: nq x d float32 rows (host).  out_ids / out_dists: nq x out_stride
 * (host), filled as henn_search fills them.  k, ef, ef_upper uniform for
 * the batch.  The index's device must be current.  The call copies in,
 * searches, copies out and synchronises `stream` before returning.
 * Limit: 256 + nq*(4 d) + nq*out_stride*12 bytes (each part rounded up to
 * 256) must fit in 16 MiB, about 26,000 queries at d = 128, k = 10;
 * larger batches return HENN_ERR_INVALID_ARG with the byte counts (split
 * the batch).  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array: calls whose work overlaps on the
 * GPU (from several host threads or streams) race and must be serialised
 * by the caller.  Errors as henn_search, message in henn_last_error().
 */
henn_status henn_search_host_noalloc(const henn_index* idx, const float* Q, int64_t nq, int32_t k, int32_t ef,
                                     int32_t ef_upper, int64_t* out_ids, float* out_dists, int32_t out_stride,
                                     void* stream);

/* ---------------------------------------------------------------- serving */

/*
 * Continuous batching (the serving loop).  A server owns one persistent
 * kernel that answers queries from a ring of work items in HBM: requests
 * (a batch of query rows with their own k and beam width) are admitted
 * while their rows fit the ring and a request slot is free, published to
 * the running kernel, and answered as warps free up, overlapping with the
 * requests already on the device.  A query's result depends only on the
 * query, its k, ef and key, so it is the same whatever else is in flight.
 * Each query is answered exactly as henn_search answers it (Alg. 4 + beam).
 *
 * Budgets fixed at creation: ring_rows (HBM: ring_rows * (4 d + 12 max_k)
 * bytes), max_requests slots, max_k, max_ef (the shared-memory class of the
 * kernel: requests with a wider beam are refused).  Host memory passed to
 * submit / poll is read / written during the call only.  Calls are
 * thread-safe.  The kernel leaves after idle_ms without work and is
 * relaunched by the next submit or poll.
 */
typedef struct {
  uint32_t struct_size;
  int32_t ring_rows;     /* queries in flight at most (default 65536)           */
  int32_t max_requests;  /* request slots (default 1024)                        */
  int32_t max_k;         /* largest k, also the result row width (default 100)  */
  int32_t max_ef;        /* largest beam width (default 512)                    */
  int32_t ef_upper;      /* as in henn_search_params (default 1)                */
  int32_t descend_all;   /* as in henn_search_params (default 0)                */
  int32_t rerank_mult;   /* as in henn_search_params (default 4)                */
  int32_t idle_ms;       /* kernel idle exit, milliseconds (default 20)         */
  int32_t ef_l1;         /* as in henn_search_params (default 0)                */
  int32_t exact_upper;   /* as in henn_search_params, by the SORT method: the
                            lowest upper layer of at most exact_upper points
                            (and at most 2048) gives its exact candidate set
                            (default 0 = never)                               */
} henn_serve_params;

typedef struct henn_server henn_server; /* opaque */

void henn_serve_params_default(henn_serve_params* p);

/* Creates a server for `idx` (which must outlive it).  Errors:
 * HENN_ERR_INVALID_ARG, HENN_ERR_OOM, HENN_ERR_CUDA. */
henn_status henn_serve_create(const henn_index* idx, const henn_serve_params* p, henn_server** out);

/* Submits nq query rows (host, nq x d float32) with one k and ef, and
 * optional per-query entry keys (host, NULL = request id * 2^20 + row).
 * On success *request_id identifies the request.  HENN_ERR_BUSY when the
 * ring or the request slots are full (poll and retry); HENN_ERR_INVALID_ARG
 * for nq < 1, nq > ring_rows, k outside [1, max_k], ef outside [1, max_ef]. */
henn_status henn_serve_submit(henn_server* s, const float* Q, int32_t nq, int32_t k, int32_t ef,
                              const uint64_t* keys, int64_t* request_id);

/* Non-blocking: *done = 0 while the request runs; when it has finished,
 * *done = 1 and its results are copied to out_ids / out_dists (host, nq x
 * k, layout as henn_search), and the request's ring rows are released.
 * HENN_ERR_INVALID_ARG for an unknown or already collected request. */
henn_status henn_serve_poll(henn_server* s, int64_t request_id, int32_t* done, int64_t* out_ids,
                            float* out_dists);

/* Stops the kernel (waits for it) and frees the server.  NULL is a no-op. */
void henn_serve_destroy(henn_server* s);

/* Message of the last failure on this host thread ("" if none). */
const char* henn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HENN_H */
