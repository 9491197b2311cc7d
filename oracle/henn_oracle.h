/*
 * henn_oracle.h -- plain FP64 CPU oracle for HENN (Hierarchical epsilon-Net
 * Navigation graph, arXiv 2505.17368).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * statement of what the GPU path computes.  Only the test-suite, the smoke
 * check in __graft_entry__.py and the CPU-baseline leg of bench.py may load
 * it; the product library (libhenn) never links, includes or calls it, and
 * it shares no code, header, table or constant generator with the CUDA path.
 *
 * Conventions
 *  - Points are float32 row-major (n x d), promoted to double on use.
 *  - Squared L2 distances are sum_k (x_k - y_k)^2 summed in index order, one
 *    rounding per operation (compile with -ffp-contract=off).
 *  - Angular distance is 1 - <x,y> / (|x| |y|)  (App. G, angular metric).
 *  - Every argmin / sort is over (distance, index) pairs, a total order.
 *  - Layer 0 is all points 0..n-1; layer i >= 1 is a sorted subset of layer
 *    i-1.  Graph rows hold layer-local indices (positions inside the layer).
 *
 * Random numbers: SplitMix64 (Steele, Lea & Flood 2014), counter style.
 *   mix64(z)      : the SplitMix64 output finaliser
 *   derive(h, w)  : mix64(h + (w + 1) * 0x9E3779B97F4A7C15), i.e. output w of
 *                   a SplitMix64 generator seeded with h
 *   bounded(u, s) : floor(u * s / 2^64)
 * Streams are nested derive() calls; see henn_oracle.c for each stream.
 */
#ifndef HENN_ORACLE_H
#define HENN_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* stream tags (ASCII words) */
#define HO_TAG_SAMPLE 0x53414D50ULL /* "SAMP": with-replacement draws, Alg. 2 */
#define HO_TAG_RCENTRE 0x5243454EULL /* "RCEN": ring centre, App. B practical impl. */
#define HO_TAG_RSTART 0x52535441ULL /* "RSTA": ring start rank */
#define HO_TAG_ORDER 0x4F524452ULL  /* "ORDR": NSW insertion order */
#define HO_TAG_ENTRY 0x454E5452ULL  /* "ENTR": random root node, Alg. 4 */
#define HO_TAG_HALVE 0x48414C56ULL  /* "HALV": coin of each matched pair, Alg. 3 */

#define HO_L2 0
#define HO_ANGULAR 1
#define HO_GRAPH_NSW 0
#define HO_GRAPH_KNN 1

void ho_set_threads(int32_t n);
uint64_t ho_mix64(uint64_t z);
uint64_t ho_derive(uint64_t h, uint64_t w);
uint64_t ho_bounded(uint64_t u, uint64_t s);

/* Insertion rank of layer-local index x in a layer of size s (a keyed
 * pseudo-random permutation of 0..s-1). */
int64_t ho_order_rank(uint64_t seed, int32_t layer, int64_t s, int64_t x);

/* Smallest heavy-ring size w = floor(eps(s) * s) + 1 with eps(s) from Eq. 1
 * (natural log); returns s + 1 when eps >= 1 (no heavy ring exists). */
int64_t ho_ring_window(double c0, int32_t d, int64_t s, int32_t m);

/* distance between two float32 vectors in FP64 (metric HO_L2 -> squared L2) */
double ho_dist(const float* a, const float* b, int32_t d, int32_t metric);

/* Alg. 2, one attempt: t draws with replacement from positions 0..s-1 of
 * the previous layer, deduplicated; writes the sorted distinct positions
 * and returns their count. */
int64_t ho_sample_positions(uint64_t seed, int32_t layer, int32_t attempt, int64_t s, int64_t t,
                            int64_t* out_pos);

/* IsEpsNet with r sampled ring ranges (App. B practical implementation).
 * prev: global ids of layer i-1 (s of them).  net_pos: sorted positions in
 * prev of the candidate layer (nnet of them).  Returns 1 if every sampled
 * ring of >= w points holds a candidate, else 0.  exhaustive=1 checks every
 * (centre in prev, window start) pair instead of r sampled ones.
 * ring_ok (optional, r entries) receives the per-ring verdicts. */
int32_t ho_verify(const float* X, int32_t d, int32_t metric, const int64_t* prev, int64_t s,
                  const int64_t* net_pos, int64_t nnet, uint64_t seed, int32_t layer,
                  int32_t attempt, int32_t r, int64_t w, int32_t exhaustive, uint8_t* ring_ok);

/* Alg. 1 hierarchy (membership only).  Writes per-layer sizes, the
 * concatenated sorted global ids of layers 1.., the concatenated down
 * pointers (position of each layer-i point in layer i-1), and the attempt
 * index that succeeded per layer.  Returns the number of layers above
 * layer 0 (L), or -1 if some layer found no epsilon-net within max_attempts.
 * Buffers must hold n entries (sizes/attempts: 64). */
int32_t ho_build_layers(const float* X, int64_t n, int32_t d, int32_t metric, int32_t m,
                        int32_t max_layers, double c0, int32_t r, int32_t max_attempts,
                        uint64_t seed, int32_t exhaustive, int64_t* sizes, int64_t* ids,
                        int64_t* down, int32_t* attempts);

/* The same layers built from layer `first_layer` on, the layer below being
 * the s0 global ids prev_ids (ascending): layer first_layer is sampled from
 * them, the next from it, and so on.  sizes / attempts are indexed by layer
 * number (entries first_layer.. written); ids / down are concatenated from
 * first_layer on, down holding positions in prev_ids for first_layer.
 * Returns the highest layer built (first_layer - 1 if none), or -1 if some
 * layer found no epsilon-net.  Used by the delete path of App. C to
 * resample a layer from the live points of the layer below. */
int32_t ho_build_layers_from(const float* X, int32_t d, int32_t metric, int32_t m, int32_t max_layers,
                             double c0, int32_t r, int32_t max_attempts, uint64_t seed, int32_t exhaustive,
                             int32_t first_layer, const int64_t* prev_ids, int64_t s0, int64_t* sizes,
                             int64_t* ids, int64_t* down, int32_t* attempts);

/* Alg. 3 BuildEpsNetDiscV2: m halving steps of the positions 0..s-1 of the
 * previous layer.  Each step matches the current list in consecutive pairs
 * (positions 2j, 2j+1 of the list: one arbitrary matching), keeps one
 * member of each pair by a coin, bounded(derive(derive(derive(derive(seed,
 * HALV), layer), step), j), 2), and keeps an unmatched last element.
 * Writes the surviving positions in ascending order; returns their count. */
int64_t ho_halving_positions(uint64_t seed, int32_t layer, int64_t s, int32_t m, int64_t* out_pos);

/* Alg. 1 hierarchy with the halving sampler instead of Alg. 2: layers while
 * |L_{i-1}| >= 2^m (and i <= max_layers when set).  Same outputs as
 * ho_build_layers; no verification, so no attempts. */
int32_t ho_build_layers_halving(int64_t n, int32_t m, int32_t max_layers, uint64_t seed, int64_t* sizes,
                                int64_t* ids, int64_t* down);

/* Forward lists of one layer: for each point p the M nearest by (dist,
 * index) among points of lower insertion rank (graph=NSW) or among all other
 * points (graph=KNN).  ids: global ids of the layer (s).  fwd: s*M local
 * indices (-1 pad); fwd_d: matching distances (+inf pad). */
void ho_forward_lists(const float* X, int32_t d, int32_t metric, const int64_t* ids, int64_t s,
                      uint64_t seed, int32_t layer, int32_t M, int32_t graph, int32_t* fwd,
                      double* fwd_d);

/* Forward list of the single point p (same definition as above). */
void ho_forward_row(const float* X, int32_t d, int32_t metric, const int64_t* ids, int64_t s,
                    uint64_t seed, int32_t layer, int32_t M, int32_t graph, int64_t p, int32_t* fwd,
                    double* fwd_d);

/* Edge rule: N(j) = [pred(j)] ++ the Mmax-1 smallest (dist, index) of
 * (fwd(j) U rev(j)) \ {pred(j)}, -1 padded.  pred(j) = fwd(j)[0] for graph
 * NSW; for graph KNN no slot is reserved. */
void ho_edge_rule(const int32_t* fwd, const double* fwd_d, int64_t s, int32_t M, int32_t Mmax,
                  int32_t graph, int32_t* adj);

/* Query (Alg. 4 + candidate-set beam on layer 0; ef_upper > 1 runs a beam
 * of that width on layers >= 1 too, ef_l1 > 0 overrides it on layer 1,
 * descend_all enters each layer at all candidates of the beam above;
 * upper layers of at most exact_upper points give their exact candidate set
 * of that width instead of a walk, 0 = never).
 * nlayers = L + 1; sizes[0] = n.  ids/down: concatenated for layers 1..L;
 * adj: concatenated per layer 0..L, Mmax per row.  k[q], ef[q] per query.
 * out_ids (int64) / out_d (double) have stride out_stride; distances are
 * true L2 (sqrt) or angular.  stats (optional, 4 per query): distance
 * evaluations, layer-0 expansions, upper-layer moves/expansions, entry
 * local index. */
void ho_search(const float* X, int64_t n, int32_t d, int32_t metric, int32_t nlayers,
               const int64_t* sizes, const int64_t* ids, const int64_t* down, const int32_t* adj,
               int32_t Mmax, const float* Q, int64_t nq, const int32_t* k, const int32_t* ef,
               int32_t ef_upper, int32_t ef_l1, int32_t descend_all, int64_t exact_upper, uint64_t seed,
               const uint64_t* keys, int64_t* out_ids, double* out_d, int32_t out_stride, int64_t* stats);

/* Greedy search on one layer (Alg. 4 GreedySearch); returns the local index
 * reached and writes the number of moves to *hops. */
int64_t ho_greedy_layer(const float* X, int32_t d, int32_t metric, const int64_t* ids,
                        const int32_t* adj, int32_t Mmax, const float* q, int64_t start,
                        int64_t* hops, int64_t* evals);

/* Exact k nearest neighbours by brute force (Sec. 2 problem setting). */
void ho_bruteforce(const float* X, int64_t n, int32_t d, int32_t metric, const float* Q, int64_t nq,
                   int32_t k, int64_t* out_ids, double* out_d);

/* Number formats: round-to-nearest-even float32 -> bfloat16 bits, and
 * float32 -> OCP FP8 E4M3 bits with saturation to +-448. */
uint16_t ho_bf16_bits(float x);
uint8_t ho_e4m3_bits(float x);
double ho_e4m3_value(uint8_t code);

#ifdef __cplusplus
}
#endif
#endif
