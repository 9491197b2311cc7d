/*
 * henn_oracle.c -- plain FP64 CPU oracle for HENN (arXiv 2505.17368).
 *
 * TEST INFRASTRUCTURE ONLY: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py.  The product library never links or calls
 * it.  Everything here is deliberately slow and literal: plain loops,
 * FP64 arithmetic, linear scans, qsort.  Each function names the passage of
 * the paper it restates.
 *
 * Parity status: every function is pinned by tests/test_oracle_pins.py
 * except the constant in the query-time bound of Thm. 1 (the paper gives no
 * constant; only the polylog shape is checked).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared (no
 * -ffast-math).  OpenMP only splits independent rows or queries across
 * threads; every result is the same for any thread count.
 */
#include "henn_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Number of OpenMP threads used by the loops below (results do not depend
 * on it). */
void ho_set_threads(int32_t n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ RNG */

/* SplitMix64 output function (Steele, Lea & Flood 2014). */
uint64_t ho_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Output number w (0-based) of SplitMix64 seeded with h. */
uint64_t ho_derive(uint64_t h, uint64_t w) { return ho_mix64(h + (w + 1ULL) * 0x9E3779B97F4A7C15ULL); }

/* Uniform integer in [0, s): high word of the 128-bit product u * s. */
uint64_t ho_bounded(uint64_t u, uint64_t s) {
  return (uint64_t)(((unsigned __int128)u * (unsigned __int128)s) >> 64);
}

/* ---------------------------------------------------- insertion order */

/* The NSW graph inserts the points of a layer one at a time in random order
 * (App. B, Navigable Graphs; App. G, Methods).  The order is a keyed
 * pseudo-random permutation of 0..s-1: a balanced 4-round Feistel network
 * (Luby & Rackoff 1988) on 2h bits whose round function is SplitMix64,
 * restricted to [0, s) by cycle walking (Black & Rogaway 2002). */
static uint64_t feistel(uint64_t key, int half_bits, uint64_t x) {
  const uint64_t mask = (1ULL << half_bits) - 1ULL;
  uint64_t left = x >> half_bits;
  uint64_t right = x & mask;
  for (uint64_t round = 0; round < 4; ++round) {
    uint64_t f = ho_derive(ho_derive(key, round), right) & mask;
    uint64_t new_right = left ^ f;
    left = right;
    right = new_right;
  }
  return (left << half_bits) | right;
}

int64_t ho_order_rank(uint64_t seed, int32_t layer, int64_t s, int64_t x) {
  if (s <= 1) return 0;
  int bits = 2;
  while ((1LL << bits) < s) ++bits;
  if (bits & 1) ++bits;
  uint64_t key = ho_derive(ho_derive(seed, HO_TAG_ORDER), (uint64_t)layer);
  uint64_t y = feistel(key, bits / 2, (uint64_t)x);
  while (y >= (uint64_t)s) y = feistel(key, bits / 2, y);
  return (int64_t)y;
}

/* ------------------------------------------------------------- metric */

/* Sec. 2 "Data Model": l_p distance with p = 2 (squared; the square root is
 * monotone so every order and ring test is unchanged).  App. G: angular
 * distance 1 - cos. */
double ho_dist(const float* a, const float* b, int32_t d, int32_t metric) {
  if (metric == HO_ANGULAR) {
    double ab = 0.0, aa = 0.0, bb = 0.0;
    for (int32_t k = 0; k < d; ++k) {
      ab += (double)a[k] * (double)b[k];
      aa += (double)a[k] * (double)a[k];
      bb += (double)b[k] * (double)b[k];
    }
    return 1.0 - ab / (sqrt(aa) * sqrt(bb));
  }
  double acc = 0.0;
  for (int32_t k = 0; k < d; ++k) {
    double t = (double)a[k] - (double)b[k];
    acc += t * t;
  }
  return acc;
}

static double reported_dist(double v, int32_t metric) { return metric == HO_ANGULAR ? v : sqrt(v); }

typedef struct {
  double d;
  int64_t i;
} pair_t;

static int pair_less(pair_t a, pair_t b) { return a.d < b.d || (a.d == b.d && a.i < b.i); }

static int pair_cmp(const void* pa, const void* pb) {
  pair_t a = *(const pair_t*)pa, b = *(const pair_t*)pb;
  if (pair_less(a, b)) return -1;
  if (pair_less(b, a)) return 1;
  return 0;
}

/* ---------------------------------------------------------- Eq. 1 window */

/* eps(s) = c0 * d * log(s) / s * 2^m (Eq. 1, natural log).  A ring is heavy
 * when it holds MORE than eps*s points (definition of an eps-net, App. B),
 * so the smallest heavy ring has floor(eps*s) + 1 points.  eps*s is
 * evaluated as ((c0 * d) * log(s)) * 2^m. */
int64_t ho_ring_window(double c0, int32_t d, int64_t s, int32_t m) {
  double es = c0 * (double)d;
  es = es * log((double)s);
  es = es * (double)(1LL << m);
  if (!(es < (double)s)) return s + 1;
  return (int64_t)floor(es) + 1;
}

/* ---------------------------------------------------------- Alg. 2 draw */

/* One Monte-Carlo draw of Alg. 2: t samples with replacement (App. G,
 * Implementation Details; App. D parallel sampling), the layer being the
 * distinct set.  Draw j of attempt a for layer i picks position
 * bounded(derive(derive(derive(derive(seed, SAMP), i), a), j), s). */
int64_t ho_sample_positions(uint64_t seed, int32_t layer, int32_t attempt, int64_t s, int64_t t,
                            int64_t* out_pos) {
  uint8_t* hit = (uint8_t*)calloc((size_t)s, 1);
  uint64_t base = ho_derive(ho_derive(ho_derive(seed, HO_TAG_SAMPLE), (uint64_t)layer), (uint64_t)attempt);
  for (int64_t j = 0; j < t; ++j) hit[ho_bounded(ho_derive(base, (uint64_t)j), (uint64_t)s)] = 1;
  int64_t cnt = 0;
  for (int64_t p = 0; p < s; ++p)
    if (hit[p]) out_pos[cnt++] = p;
  free(hit);
  return cnt;
}

/* Alg. 3 (BuildEpsNetDiscV2): m halving steps, each over an arbitrary
 * matching of the current set (here: consecutive pairs of the list) keeping
 * one member of each pair at random. */
int64_t ho_halving_positions(uint64_t seed, int32_t layer, int64_t s, int32_t m, int64_t* out_pos) {
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s > 0 ? s : 1));
  for (int64_t p = 0; p < s; ++p) cur[p] = p;
  int64_t c = s;
  for (int32_t step = 0; step < m; ++step) {
    uint64_t base = ho_derive(ho_derive(ho_derive(seed, HO_TAG_HALVE), (uint64_t)layer), (uint64_t)step);
    int64_t next = 0;
    for (int64_t j = 0; 2 * j < c; ++j) {
      if (2 * j + 1 < c) {
        uint64_t coin = ho_bounded(ho_derive(base, (uint64_t)j), 2);
        cur[next++] = cur[2 * j + coin];
      } else {
        cur[next++] = cur[2 * j]; /* unmatched last element */
      }
    }
    c = next;
  }
  for (int64_t j = 0; j < c; ++j) out_pos[j] = cur[j];
  free(cur);
  return c;
}

int32_t ho_build_layers_halving(int64_t n, int32_t m, int32_t max_layers, uint64_t seed, int64_t* sizes,
                                int64_t* ids, int64_t* down) {
  int64_t* prev = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) prev[i] = i;
  int64_t s = n, off = 0;
  sizes[0] = n;
  int32_t L = 0;
  for (int32_t layer = 1; layer < 64; ++layer) {
    if (max_layers > 0 && layer > max_layers) break;
    if (s < (1LL << m)) break;
    int64_t cnt = ho_halving_positions(seed, layer, s, m, pos);
    for (int64_t j = 0; j < cnt; ++j) {
      ids[off + j] = prev[pos[j]];
      down[off + j] = pos[j];
    }
    for (int64_t j = 0; j < cnt; ++j) prev[j] = ids[off + j];
    off += cnt;
    s = cnt;
    sizes[layer] = cnt;
    L = layer;
  }
  free(prev);
  free(pos);
  return L;
}

/* ------------------------------------------------------- IsEpsNet check */

/* One ring range (Def. 2) centred at a point of the previous layer: the
 * points whose rank in the (dist, index) order around the centre lies in
 * [a0, a0 + w - 1].  As a ring it is the closed distance interval
 * [D(a0), D(a0 + w - 1)].  Returns 1 if a candidate lies in it. */
static int ring_hit(const double* dist, const pair_t* sorted, int64_t a0, int64_t w,
                    const int64_t* net_pos, int64_t nnet) {
  double lo = sorted[a0].d, hi = sorted[a0 + w - 1].d;
  for (int64_t j = 0; j < nnet; ++j) {
    double v = dist[net_pos[j]];
    if (lo <= v && v <= hi) return 1;
  }
  return 0;
}

static void centre_order(const float* X, int32_t d, int32_t metric, const int64_t* prev, int64_t s,
                         int64_t centre_pos, double* dist, pair_t* sorted) {
  const float* c = X + (size_t)prev[centre_pos] * d;
  for (int64_t x = 0; x < s; ++x) {
    dist[x] = ho_dist(c, X + (size_t)prev[x] * d, d, metric);
    sorted[x].d = dist[x];
    sorted[x].i = x;
  }
  qsort(sorted, (size_t)s, sizeof(pair_t), pair_cmp);
}

/* App. B "Practical Implementation" / App. G: instead of every range, r
 * ranges are drawn uniformly at random and the candidate must hit each.
 * Ring rho of attempt a at layer i: centre position
 * bounded(derive(derive(derive(derive(seed, RCEN), i), a), rho), s), start
 * rank bounded(derive(derive(derive(derive(seed, RSTA), i), a), rho), s-w+1),
 * w points.  w > s means eps >= 1: no heavy ring, the check passes. */
int32_t ho_verify(const float* X, int32_t d, int32_t metric, const int64_t* prev, int64_t s,
                  const int64_t* net_pos, int64_t nnet, uint64_t seed, int32_t layer,
                  int32_t attempt, int32_t r, int64_t w, int32_t exhaustive, uint8_t* ring_ok) {
  if (w > s) {
    if (ring_ok)
      for (int32_t q = 0; q < r; ++q) ring_ok[q] = 1;
    return 1;
  }
  double* dist = (double*)malloc(sizeof(double) * (size_t)s);
  pair_t* sorted = (pair_t*)malloc(sizeof(pair_t) * (size_t)s);
  int32_t all = 1;
  if (exhaustive) {
    for (int64_t c = 0; c < s && all; ++c) {
      centre_order(X, d, metric, prev, s, c, dist, sorted);
      for (int64_t a0 = 0; a0 + w <= s; ++a0)
        if (!ring_hit(dist, sorted, a0, w, net_pos, nnet)) {
          all = 0;
          break;
        }
    }
  } else {
    uint64_t bc = ho_derive(ho_derive(ho_derive(seed, HO_TAG_RCENTRE), (uint64_t)layer), (uint64_t)attempt);
    uint64_t bs = ho_derive(ho_derive(ho_derive(seed, HO_TAG_RSTART), (uint64_t)layer), (uint64_t)attempt);
#pragma omp parallel reduction(& : all)
    {
      double* tdist = (double*)malloc(sizeof(double) * (size_t)s);
      pair_t* tsorted = (pair_t*)malloc(sizeof(pair_t) * (size_t)s);
#pragma omp for schedule(dynamic, 1)
      for (int32_t q = 0; q < r; ++q) {
        int64_t c = (int64_t)ho_bounded(ho_derive(bc, (uint64_t)q), (uint64_t)s);
        int64_t a0 = (int64_t)ho_bounded(ho_derive(bs, (uint64_t)q), (uint64_t)(s - w + 1));
        centre_order(X, d, metric, prev, s, c, tdist, tsorted);
        int ok = ring_hit(tdist, tsorted, a0, w, net_pos, nnet);
        if (ring_ok) ring_ok[q] = (uint8_t)ok;
        if (!ok) all = 0;
      }
      free(tdist);
      free(tsorted);
    }
  }
  free(dist);
  free(sorted);
  return all;
}

/* ------------------------------------------------------------- Alg. 1 */

/* BuildHENN (Alg. 1) membership part: layer i is an eps(|L_{i-1}|)-net of
 * layer i-1 found by the Las-Vegas loop of Alg. 2, with |L_i| drawn as
 * ceil(|L_{i-1}| / 2^m) samples (Cor. 2).  Layers are built while i <=
 * max_layers (0: no limit) and |L_{i-1}| >= 2^m. */
int32_t ho_build_layers_from(const float* X, int32_t d, int32_t metric, int32_t m, int32_t max_layers,
                             double c0, int32_t r, int32_t max_attempts, uint64_t seed, int32_t exhaustive,
                             int32_t first_layer, const int64_t* prev_ids, int64_t s0, int64_t* sizes,
                             int64_t* ids, int64_t* down, int32_t* attempts) {
  int64_t* prev = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s0 > 0 ? s0 : 1));
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s0 > 0 ? s0 : 1));
  for (int64_t i = 0; i < s0; ++i) prev[i] = prev_ids[i];
  int64_t s = s0;
  int64_t off = 0;
  int32_t L = first_layer - 1;
  const int64_t decay = 1LL << m;
  for (int32_t layer = first_layer; layer < 64; ++layer) {
    if (max_layers > 0 && layer > max_layers) break;
    if (s < decay) break;
    int64_t t = (s + decay - 1) / decay;
    int64_t w = ho_ring_window(c0, d, s, m);
    int32_t found = -1;
    int64_t cnt = 0;
    for (int32_t a = 0; a < max_attempts; ++a) {
      cnt = ho_sample_positions(seed, layer, a, s, t, pos);
      if (ho_verify(X, d, metric, prev, s, pos, cnt, seed, layer, a, r, w, exhaustive, NULL)) {
        found = a;
        break;
      }
    }
    if (found < 0) {
      free(prev);
      free(pos);
      return -1;
    }
    for (int64_t j = 0; j < cnt; ++j) {
      ids[off + j] = prev[pos[j]];
      down[off + j] = pos[j];
    }
    for (int64_t j = 0; j < cnt; ++j) prev[j] = ids[off + j];
    off += cnt;
    s = cnt;
    sizes[layer] = cnt;
    attempts[layer] = found;
    L = layer;
  }
  free(prev);
  free(pos);
  return L;
}

int32_t ho_build_layers(const float* X, int64_t n, int32_t d, int32_t metric, int32_t m,
                        int32_t max_layers, double c0, int32_t r, int32_t max_attempts,
                        uint64_t seed, int32_t exhaustive, int64_t* sizes, int64_t* ids,
                        int64_t* down, int32_t* attempts) {
  int64_t* all = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) all[i] = i;
  sizes[0] = n;
  attempts[0] = 0;
  const int32_t L = ho_build_layers_from(X, d, metric, m, max_layers, c0, r, max_attempts, seed, exhaustive, 1,
                                         all, n, sizes, ids, down, attempts);
  free(all);
  return L;
}

/* -------------------------------------------------- navigable graphs */

/* Insert (dv, v) into the ascending list best[0..*cnt) capped at cap. */
static void keep_best(pair_t* best, int32_t* cnt, int32_t cap, double dv, int64_t v) {
  pair_t e = {dv, v};
  if (*cnt == cap && !pair_less(e, best[cap - 1])) return;
  int32_t j = (*cnt < cap) ? (*cnt)++ : cap - 1;
  while (j > 0 && pair_less(e, best[j - 1])) {
    best[j] = best[j - 1];
    --j;
  }
  best[j] = e;
}

/* NSW (App. B, Navigable Graphs; App. G): each point, when inserted, is
 * linked to its nearest already-inserted points.  Written here as the exact
 * definition that incremental greedy insertion approximates: the M nearest
 * by (dist, index) among points of lower insertion rank.  graph=KNN: the M
 * nearest among all other points (App. G, knn graph). */
void ho_forward_lists(const float* X, int32_t d, int32_t metric, const int64_t* ids, int64_t s,
                      uint64_t seed, int32_t layer, int32_t M, int32_t graph, int32_t* fwd,
                      double* fwd_d) {
  int64_t* rank = (int64_t*)malloc(sizeof(int64_t) * (size_t)(s > 0 ? s : 1));
  for (int64_t x = 0; x < s; ++x) rank[x] = ho_order_rank(seed, layer, s, x);
#pragma omp parallel
  {
  pair_t* best = (pair_t*)malloc(sizeof(pair_t) * (size_t)M);
#pragma omp for schedule(dynamic, 16)
  for (int64_t p = 0; p < s; ++p) {
    int32_t cnt = 0;
    const float* xp = X + (size_t)ids[p] * d;
    for (int64_t q = 0; q < s; ++q) {
      if (q == p) continue;
      if (graph == HO_GRAPH_NSW && rank[q] >= rank[p]) continue;
      keep_best(best, &cnt, M, ho_dist(xp, X + (size_t)ids[q] * d, d, metric), q);
    }
    for (int32_t j = 0; j < M; ++j) {
      fwd[p * M + j] = j < cnt ? (int32_t)best[j].i : -1;
      fwd_d[p * M + j] = j < cnt ? best[j].d : INFINITY;
    }
  }
  free(best);
  }
  free(rank);
}

/* The forward list of one point p, same definition as ho_forward_lists
 * (for sampled checks of large layers). */
void ho_forward_row(const float* X, int32_t d, int32_t metric, const int64_t* ids, int64_t s,
                    uint64_t seed, int32_t layer, int32_t M, int32_t graph, int64_t p, int32_t* fwd,
                    double* fwd_d) {
  pair_t* best = (pair_t*)malloc(sizeof(pair_t) * (size_t)M);
  int64_t rp = ho_order_rank(seed, layer, s, p);
  int32_t cnt = 0;
  const float* xp = X + (size_t)ids[p] * d;
  for (int64_t q = 0; q < s; ++q) {
    if (q == p) continue;
    if (graph == HO_GRAPH_NSW && ho_order_rank(seed, layer, s, q) >= rp) continue;
    keep_best(best, &cnt, M, ho_dist(xp, X + (size_t)ids[q] * d, d, metric), q);
  }
  for (int32_t j = 0; j < M; ++j) {
    fwd[j] = j < cnt ? (int32_t)best[j].i : -1;
    fwd_d[j] = j < cnt ? best[j].d : INFINITY;
  }
  free(best);
}

/* Edge rule (reading of App. B NSW): links are undirected at insertion, so
 * a node sees its forward list and every later node that linked to it; the
 * list is capped at Mmax, always keeping the nearest predecessor pred(j) =
 * fwd(j)[0] so that the graph stays connected. */
void ho_edge_rule(const int32_t* fwd, const double* fwd_d, int64_t s, int32_t M, int32_t Mmax,
                  int32_t graph, int32_t* adj) {
  /* candidate lists: fwd(j) then rev(j) */
  int64_t* deg = (int64_t*)calloc((size_t)s + 1, sizeof(int64_t));
  for (int64_t p = 0; p < s; ++p)
    for (int32_t j = 0; j < M; ++j)
      if (fwd[p * M + j] >= 0) deg[fwd[p * M + j]]++;
  int64_t* start = (int64_t*)calloc((size_t)s + 1, sizeof(int64_t));
  for (int64_t v = 0; v < s; ++v) start[v + 1] = start[v] + deg[v];
  pair_t* rev = (pair_t*)malloc(sizeof(pair_t) * (size_t)(start[s] > 0 ? start[s] : 1));
  int64_t* fill = (int64_t*)calloc((size_t)s + 1, sizeof(int64_t));
  for (int64_t p = 0; p < s; ++p)
    for (int32_t j = 0; j < M; ++j) {
      int32_t v = fwd[p * M + j];
      if (v < 0) continue;
      rev[start[v] + fill[v]].d = fwd_d[p * M + j];
      rev[start[v] + fill[v]].i = p;
      fill[v]++;
    }
  pair_t* cand = (pair_t*)malloc(sizeof(pair_t) * (size_t)(M + start[s] + 1));
  for (int64_t v = 0; v < s; ++v) {
    int64_t c = 0;
    for (int32_t j = 0; j < M; ++j)
      if (fwd[v * M + j] >= 0) {
        cand[c].d = fwd_d[v * M + j];
        cand[c].i = fwd[v * M + j];
        ++c;
      }
    for (int64_t e = start[v]; e < start[v + 1]; ++e) cand[c++] = rev[e];
    qsort(cand, (size_t)c, sizeof(pair_t), pair_cmp);
    int32_t reserve = (graph == HO_GRAPH_NSW && fwd[v * M] >= 0);
    int32_t pred = reserve ? fwd[v * M] : -1;
    int32_t out = 0;
    if (reserve) adj[v * Mmax + out++] = pred;
    int64_t last = -1;
    for (int64_t e = 0; e < c && out < Mmax; ++e) {
      if (cand[e].i == pred || cand[e].i == last) continue; /* sorted: duplicates adjacent */
      adj[v * Mmax + out++] = (int32_t)cand[e].i;
      last = cand[e].i;
    }
    while (out < Mmax) adj[v * Mmax + out++] = -1;
  }
  free(cand);
  free(fill);
  free(rev);
  free(start);
  free(deg);
}

/* --------------------------------------------------------------- query */

static const float* layer_point(const float* X, int32_t d, const int64_t* ids, int64_t local) {
  return X + (size_t)(ids ? ids[local] : local) * d;
}

/* GreedySearch of Alg. 4: move to the closest neighbour (ties by index)
 * while it is strictly closer than the current node. */
int64_t ho_greedy_layer(const float* X, int32_t d, int32_t metric, const int64_t* ids,
                        const int32_t* adj, int32_t Mmax, const float* q, int64_t start,
                        int64_t* hops, int64_t* evals) {
  int64_t curr = start;
  double dcurr = ho_dist(q, layer_point(X, d, ids, curr), d, metric);
  int64_t moves = 0, ev = 1;
  for (;;) {
    int64_t next = -1;
    double dnext = INFINITY;
    for (int32_t j = 0; j < Mmax; ++j) {
      int32_t u = adj[curr * Mmax + j];
      if (u < 0) continue;
      double du = ho_dist(q, layer_point(X, d, ids, u), d, metric);
      ++ev;
      if (next < 0 || du < dnext || (du == dnext && u < next)) {
        next = u;
        dnext = du;
      }
    }
    if (next < 0 || dnext >= dcurr) break;
    curr = next;
    dcurr = dnext;
    ++moves;
  }
  if (hops) *hops = moves;
  if (evals) *evals = ev;
  return curr;
}

/* Best-first beam of width ef on one layer (the candidate set of Sec. 2.2
 * for k > 1), written with the two explicit lists of the usual
 * formulation: C = candidates to expand, W = the ef best seen.  Pop the
 * nearest c of C; stop if it is farther than the worst of W while W is
 * full; otherwise evaluate every unvisited neighbour u of c and keep it in
 * C and W if W is not full or u beats the worst of W.  On return W[0..*nw)
 * is sorted ascending.  ids maps layer-local indices to points (NULL for
 * layer 0).  visited has one byte per local index. */
static void beam_layer(const float* X, int32_t d, int32_t metric, const int64_t* ids, const int32_t* adj,
                       int32_t Mmax, const float* q, const int64_t* entries, int64_t nentries, int32_t ef,
                       uint8_t* visited, int64_t size, pair_t* C, pair_t* W, int64_t* nw_out, int64_t* evals,
                       int64_t* expansions) {
  memset(visited, 0, (size_t)size);
  int64_t nc = 0, nw = 0;
  /* entries: one node, or the copies of the candidates of the layer above
   * (best first, at most ef of them) */
  for (int64_t t = 0; t < nentries && t < ef; ++t) {
    int64_t entry = entries[t];
    double de = ho_dist(q, layer_point(X, d, ids, entry), d, metric);
    ++*evals;
    visited[entry] = 1;
    C[nc].d = de;
    C[nc++].i = entry;
    W[nw].d = de;
    W[nw++].i = entry;
  }
  while (nc > 0) {
    int64_t bi = 0;
    for (int64_t j = 1; j < nc; ++j)
      if (pair_less(C[j], C[bi])) bi = j;
    pair_t c = C[bi];
    C[bi] = C[--nc];
    int64_t wi = 0;
    for (int64_t j = 1; j < nw; ++j)
      if (pair_less(W[wi], W[j])) wi = j;
    if (nw == ef && pair_less(W[wi], c)) break;
    ++*expansions;
    for (int32_t j = 0; j < Mmax; ++j) {
      int32_t u = adj[c.i * Mmax + j];
      if (u < 0 || visited[u]) continue;
      visited[u] = 1;
      double du = ho_dist(q, layer_point(X, d, ids, u), d, metric);
      ++*evals;
      pair_t pu = {du, u};
      int64_t mi = 0;
      for (int64_t t = 1; t < nw; ++t)
        if (pair_less(W[mi], W[t])) mi = t;
      if (nw < ef || pair_less(pu, W[mi])) {
        C[nc++] = pu;
        W[nw++] = pu;
        if (nw > ef) {
          mi = 0;
          for (int64_t t = 1; t < nw; ++t)
            if (pair_less(W[mi], W[t])) mi = t;
          W[mi] = W[--nw];
        }
      }
    }
  }
  qsort(W, (size_t)nw, sizeof(pair_t), pair_cmp);
  *nw_out = nw;
}

/* Query (Sec. 2.2 and Alg. 4): random node of the top layer L_L (Alg. 4
 * prints "root (L_0)"; the text of Sec. 2.2 says the root is L_L), a search
 * per layer, each layer entered at the copy of the previous result.  On
 * layers L..1 the search is Alg. 4's GreedySearch when the layer's width
 * is <= 1, else the beam of that width (reading of Sec. 2.2: a set of
 * candidates at each step) whose best node is taken down; the width is
 * ef_upper, or ef_l1 on layer 1 when ef_l1 > 0.  Layer 0 runs the beam of width
 * max(ef, k) and returns its first k entries. */
/* The exact candidate set of one layer: the `width` points of the layer
 * nearest to q in (distance, index) order, written to W; returns their
 * number.  Used for upper layers of at most exact_upper points. */
static int64_t exact_layer(const float* X, int32_t d, int32_t metric, const int64_t* ids, int64_t s,
                           const float* q, int32_t width, pair_t* C, pair_t* W) {
  for (int64_t j = 0; j < s; ++j) {
    C[j].d = ho_dist(q, layer_point(X, d, ids, j), d, metric);
    C[j].i = j;
  }
  qsort(C, (size_t)s, sizeof(pair_t), pair_cmp);
  int64_t nw = width < s ? width : s;
  for (int64_t j = 0; j < nw; ++j) W[j] = C[j];
  return nw;
}

void ho_search(const float* X, int64_t n, int32_t d, int32_t metric, int32_t nlayers,
               const int64_t* sizes, const int64_t* ids, const int64_t* down, const int32_t* adj,
               int32_t Mmax, const float* Q, int64_t nq, const int32_t* k, const int32_t* ef,
               int32_t ef_upper, int32_t ef_l1, int32_t descend_all, int64_t exact_upper, uint64_t seed,
               const uint64_t* keys, int64_t* out_ids, double* out_d, int32_t out_stride, int64_t* stats) {
  int32_t L = nlayers - 1;
  /* offsets of each layer inside the concatenated arrays */
  int64_t id_off[66], adj_off[66];
  id_off[0] = 0;
  id_off[1] = 0;
  adj_off[0] = 0;
  for (int32_t i = 1; i <= L; ++i) id_off[i + 1] = id_off[i] + sizes[i];
  for (int32_t i = 0; i < L; ++i) adj_off[i + 1] = adj_off[i] + sizes[i] * Mmax;
  int32_t ef_max = ef_upper > 1 ? ef_upper : 1;
  if (ef_l1 > ef_max) ef_max = ef_l1;
  for (int64_t qi = 0; qi < nq; ++qi) {
    int32_t e = ef[qi] > k[qi] ? ef[qi] : k[qi];
    if (e > ef_max) ef_max = e;
  }
  uint64_t entry_key = ho_derive(seed, HO_TAG_ENTRY);
#pragma omp parallel
  {
  uint8_t* visited = (uint8_t*)malloc((size_t)n);
  pair_t* C = (pair_t*)malloc(sizeof(pair_t) * (size_t)(n + 1));
  pair_t* W = (pair_t*)malloc(sizeof(pair_t) * (size_t)(ef_max + 1));
  int64_t* seeds = (int64_t*)malloc(sizeof(int64_t) * (size_t)(ef_max + 1));
#pragma omp for schedule(dynamic, 1)
  for (int64_t qi = 0; qi < nq; ++qi) {
    const float* q = Q + (size_t)qi * d;
    uint64_t key = keys ? keys[qi] : (uint64_t)qi;
    int64_t evals = 0, hops_upper = 0, expansions = 0, nw = 0;
    /* S1: random node of the top layer */
    int64_t e = (int64_t)ho_bounded(ho_derive(entry_key, key), (uint64_t)sizes[L]);
    int64_t entry = e;
    /* S2: layers L..1, then down to the copy in the layer below; with
     * descend_all the layer below is entered at the copies of all the
     * candidates of a beam, else at the best one */
    int64_t nseeds = 1;
    seeds[0] = e;
    for (int32_t i = L; i >= 1; --i) {
      int64_t c;
      const int32_t width = (i == 1 && ef_l1 > 0) ? ef_l1 : ef_upper;
      if (sizes[i] <= exact_upper) {
        /* a small layer: its exact candidate set instead of the walk */
        nw = exact_layer(X, d, metric, ids + id_off[i], sizes[i], q, width > 1 ? width : 1, C, W);
        evals += sizes[i];
        if (descend_all && width > 1) {
          for (int64_t t = 0; t < nw; ++t) seeds[t] = down[id_off[i] + W[t].i];
          nseeds = nw;
        } else {
          seeds[0] = down[id_off[i] + W[0].i];
          nseeds = 1;
        }
      } else if (width <= 1) {
        int64_t h = 0, ev = 0;
        c = ho_greedy_layer(X, d, metric, ids + id_off[i], adj + adj_off[i], Mmax, q, seeds[0], &h, &ev);
        hops_upper += h;
        evals += ev;
        seeds[0] = down[id_off[i] + c];
        nseeds = 1;
      } else {
        int64_t ex = 0;
        beam_layer(X, d, metric, ids + id_off[i], adj + adj_off[i], Mmax, q, seeds, nseeds, width, visited,
                   sizes[i], C, W, &nw, &evals, &ex);
        hops_upper += ex;
        if (descend_all) {
          for (int64_t t = 0; t < nw; ++t) seeds[t] = down[id_off[i] + W[t].i];
          nseeds = nw;
        } else {
          seeds[0] = down[id_off[i] + W[0].i];
          nseeds = 1;
        }
      }
    }
    /* S3: beam of width ef' = max(ef, k) on layer 0 */
    int32_t efq = ef[qi] > k[qi] ? ef[qi] : k[qi];
    beam_layer(X, d, metric, NULL, adj, Mmax, q, seeds, nseeds, efq, visited, n, C, W, &nw, &evals, &expansions);
    for (int32_t j = 0; j < out_stride; ++j) {
      int in = j < k[qi] && j < nw;
      out_ids[qi * out_stride + j] = in ? W[j].i : -1;
      out_d[qi * out_stride + j] = in ? reported_dist(W[j].d, metric) : INFINITY;
    }
    if (stats) {
      stats[qi * 4 + 0] = evals;
      stats[qi * 4 + 1] = expansions;
      stats[qi * 4 + 2] = hops_upper;
      stats[qi * 4 + 3] = entry;
    }
  }
  free(seeds);
  free(W);
  free(C);
  free(visited);
  }
}

/* ------------------------------------------------------- ground truth */

/* k-NN query (Sec. 2, Problem setting): the k smallest (dist, index). */
void ho_bruteforce(const float* X, int64_t n, int32_t d, int32_t metric, const float* Q, int64_t nq,
                   int32_t k, int64_t* out_ids, double* out_d) {
#pragma omp parallel
  {
  pair_t* best = (pair_t*)malloc(sizeof(pair_t) * (size_t)k);
#pragma omp for schedule(dynamic, 4)
  for (int64_t qi = 0; qi < nq; ++qi) {
    int32_t cnt = 0;
    for (int64_t x = 0; x < n; ++x)
      keep_best(best, &cnt, k, ho_dist(Q + (size_t)qi * d, X + (size_t)x * d, d, metric), x);
    for (int32_t j = 0; j < k; ++j) {
      out_ids[qi * k + j] = j < cnt ? best[j].i : -1;
      out_d[qi * k + j] = j < cnt ? reported_dist(best[j].d, metric) : INFINITY;
    }
  }
  free(best);
  }
}

/* ------------------------------------------------------ number formats */

static float bf16_value(uint16_t b) {
  uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

/* bfloat16 = the top 16 bits of a float32 (1 sign, 8 exponent, 7 fraction
 * bits).  Round to nearest: of the two bfloat16 values around x (the
 * truncation and the next one away from zero) take the nearer, on a tie the
 * one with an even last fraction bit. */
uint16_t ho_bf16_bits(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  if (isnan(x)) return (uint16_t)((u >> 16) | 0x0040);
  uint16_t lo = (uint16_t)(u >> 16);
  float vlo = bf16_value(lo);
  if (vlo == x) return lo;
  uint16_t hi = (uint16_t)(lo + 1);
  /* above the largest finite value the next neighbour is 2^128 as if the
   * exponent were unbounded (IEEE 754 overflow rule); choosing it gives
   * infinity */
  double vhi = ((hi & 0x7FFF) == 0x7F80) ? ldexp(signbit(x) ? -1.0 : 1.0, 128) : (double)bf16_value(hi);
  double dlo = fabs((double)x - (double)vlo);
  double dhi = fabs(vhi - (double)x);
  if (dlo < dhi) return lo;
  if (dhi < dlo) return hi;
  return (lo & 1) ? hi : lo;
}

/* OCP 8-bit floating point E4M3: 1 sign, 4 exponent (bias 7), 3 fraction
 * bits; exponent field 0 is subnormal (f * 2^-9); S.1111.111 is NaN; no
 * infinities; largest finite value 1.75 * 2^8 = 448. */
double ho_e4m3_value(uint8_t code) {
  int sign = code >> 7;
  int e = (code >> 3) & 15;
  int f = code & 7;
  double v;
  if (e == 15 && f == 7) return NAN;
  if (e == 0)
    v = ldexp((double)f, -9);
  else
    v = ldexp(1.0 + f / 8.0, e - 7);
  return sign ? -v : v;
}

/* Round to nearest, ties to an even code, magnitudes above 448 (and
 * infinities) saturate to 448, NaN stays NaN. */
uint8_t ho_e4m3_bits(float x) {
  uint8_t sign = signbit(x) ? 0x80 : 0x00;
  if (isnan(x)) return (uint8_t)(sign | 0x7F);
  double a = fabs((double)x);
  if (a >= 448.0) return (uint8_t)(sign | 0x7E);
  /* largest code c with value(c) <= a; codes 0..0x7E are increasing */
  uint8_t c = 0;
  while (c < 0x7E && ho_e4m3_value((uint8_t)(c + 1)) <= a) ++c;
  if (ho_e4m3_value(c) == a) return (uint8_t)(sign | c);
  double dlo = a - ho_e4m3_value(c);
  double dhi = ho_e4m3_value((uint8_t)(c + 1)) - a;
  uint8_t pick = dlo < dhi ? c : (dhi < dlo ? (uint8_t)(c + 1) : ((c & 1) ? (uint8_t)(c + 1) : c));
  return (uint8_t)(sign | pick);
}
