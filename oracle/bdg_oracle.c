/*
 * bdg_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously-correct CPU statement of what the Binary Distributed
 * Graph hot path computes (Zhao et al., "Large-Scale Visual Search with Binary
 * Distributed Graph at Alibaba"). Only tests/, the smoke check and the bench's
 * CPU-baseline leg may load it. It shares no code, header or table with the
 * CUDA library; the product path never calls it.
 *
 * Conventions used throughout:
 *   - codes: row-major uint64 [n][W], bit j of a code in word j/64 at bit j%64;
 *   - a neighbour key is the pair (distance, id) compared lexicographically;
 *     it is stored as one uint64 (d << 32 | id), valid because d <= 64*W < 2^31
 *     and 0 <= id < 2^31, so integer order of the word is the pair order;
 *   - rows with fewer than k candidates are padded with (d = bits + 1, id = -1).
 *
 * Parity status per function (pins live in tests/test_oracle_*.py):
 *   or_hamming, or_knn_exact, or_bkmeans, or_route, or_routes_coarse, or_routes_gap,
 *   or_knn_partitioned, or_search, or_rerank_f32/_f64, or_propagate, or_prune
 *   -- pinned (brute force,
 *   invariants, closed forms, hand-worked fixtures).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define KEY(d, id) ((((uint64_t)(uint32_t)(d)) << 32) | (uint64_t)(uint32_t)(id))
#define KEY_D(k) ((int32_t)((k) >> 32))
#define KEY_ID(k) ((int32_t)((k) & 0xffffffffu))

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

/* Hamming distance l_h of Section 3: number of differing bits,
 * sum over words of popcount(a XOR b). */
int32_t or_hamming(const uint64_t* a, const uint64_t* b, int32_t W) {
  int32_t d = 0;
  for (int32_t w = 0; w < W; ++w) d += __builtin_popcountll(a[w] ^ b[w]);
  return d;
}

/* Write the first k of a sorted key array, padding to k. */
static void emit_topk(const uint64_t* keys, int64_t n, int32_t k, int32_t bits,
                      int32_t* ids, int32_t* dist) {
  for (int32_t r = 0; r < k; ++r) {
    if (r < n) { ids[r] = KEY_ID(keys[r]); dist[r] = KEY_D(keys[r]); }
    else { ids[r] = -1; dist[r] = bits + 1; }
  }
}

/* Exact k-NN lists of the query points qidx[0..nq) over all n points
 * (the ideal k-NN graph B(l_i) of Section 3 under d = l_h):
 *   G*(i) = first k of sort over (d(i, j), j) for all j != i.
 * Outputs are [nq][k]. */
void or_knn_exact(const uint64_t* codes, int64_t n, int32_t W, int32_t k,
                  const int64_t* qidx, int64_t nq, int32_t* out_ids, int32_t* out_dist) {
  const int32_t bits = 64 * W;
#pragma omp parallel
  {
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t q = 0; q < nq; ++q) {
      const int64_t i = qidx[q];
      int64_t c = 0;
      for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        keys[c++] = KEY(or_hamming(codes + i * W, codes + j * W, W), j);
      }
      qsort(keys, (size_t)c, sizeof(uint64_t), cmp_u64);
      emit_topk(keys, c, k, bits, out_ids + q * k, out_dist + q * k);
    }
    free(keys);
  }
}

/* Bk-means of Section 3.2 (Eq. 1 objective, Eq. 2 update) on a down-sample.
 *   init: c_j = code of sample[j], j < m (requires S >= m);
 *   each of `iters` iterations:
 *     assign: r(i) = argmin over (d(y_i, c_j), j)        (exhaustive, Section 3.2)
 *     update: c_j bit b = majority of the members' bit b; a tie (2*n1 == p)
 *             keeps the previous bit; an empty cluster keeps its centre.
 *   loss[it] = sum_i d(y_i, c_{r(i)}) right after the assign step of iteration
 *   `it` (Eq. 1: for 0/1 vectors the squared L2 norm equals the Hamming
 *   distance), and loss[iters] = the objective of the final centres after one
 *   more assign. Non-increasing by construction. */
void or_bkmeans(const uint64_t* codes, int32_t W, const int64_t* sample, int64_t S,
                int32_t m, int32_t iters, uint64_t* centroids, int64_t* loss,
                int32_t* assign) {
  const int32_t bits = 64 * W;
  for (int32_t j = 0; j < m; ++j)
    memcpy(centroids + (int64_t)j * W, codes + sample[j] * W, sizeof(uint64_t) * W);
  int64_t* ones = (int64_t*)calloc((size_t)m * bits, sizeof(int64_t));
  int64_t* count = (int64_t*)calloc((size_t)m, sizeof(int64_t));
  for (int32_t it = 0; it <= iters; ++it) {
    int64_t J = 0;
#pragma omp parallel for reduction(+ : J) schedule(static)
    for (int64_t s = 0; s < S; ++s) {
      const uint64_t* y = codes + sample[s] * W;
      int32_t best_d = bits + 1, best_j = -1;
      for (int32_t j = 0; j < m; ++j) {
        int32_t d = or_hamming(y, centroids + (int64_t)j * W, W);
        if (d < best_d) { best_d = d; best_j = j; }  /* strict: lower j wins ties */
      }
      assign[s] = best_j;
      J += best_d;
    }
    if (loss) loss[it] = J;
    if (it == iters) break;
    memset(ones, 0, sizeof(int64_t) * (size_t)m * bits);
    memset(count, 0, sizeof(int64_t) * (size_t)m);
    for (int64_t s = 0; s < S; ++s) {
      const uint64_t* y = codes + sample[s] * W;
      const int32_t j = assign[s];
      count[j] += 1;
      for (int32_t b = 0; b < bits; ++b)
        ones[(int64_t)j * bits + b] += (int64_t)((y[b / 64] >> (b % 64)) & 1u);
    }
    for (int32_t j = 0; j < m; ++j) {
      if (count[j] == 0) continue;
      uint64_t* c = centroids + (int64_t)j * W;
      for (int32_t b = 0; b < bits; ++b) {
        const int64_t twice = 2 * ones[(int64_t)j * bits + b];
        const uint64_t mask = (uint64_t)1 << (b % 64);
        if (twice > count[j]) c[b / 64] |= mask;
        else if (twice < count[j]) c[b / 64] &= ~mask;
        /* equal: keep the previous bit */
      }
    }
  }
  free(ones);
  free(count);
}

/* Map step of Section 3.2: the t nearest centres of each point, ordered by
 * (d(y_i, c_c), c). Slot 0 is the nearest ("home", the flagged record). */
void or_route(const uint64_t* codes, int64_t n, int32_t W, const uint64_t* centroids,
              int32_t m, int32_t t, int32_t* routes, int32_t* rdist) {
#pragma omp parallel
  {
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)m);
#pragma omp for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      for (int32_t c = 0; c < m; ++c)
        keys[c] = KEY(or_hamming(codes + i * W, centroids + (int64_t)c * W, W), c);
      qsort(keys, (size_t)m, sizeof(uint64_t), cmp_u64);
      for (int32_t s = 0; s < t; ++s) {
        routes[i * t + s] = KEY_ID(keys[s]);
        if (rdist) rdist[i * t + s] = KEY_D(keys[s]);
      }
    }
    free(keys);
  }
}

/* The coarse_num rule of Section 3.2: the number of nearest centres a point is
 * mapped to varies so that the points held by its centres add up to a fixed
 * total. Given each point's t nearest centres in order (routes [n][t], slot 0
 * the home) and the home counts |H_p| = #{ j : routes[j][0] = p }, point i keeps
 * slot 0 and keeps slot s >= 1 while the centres before it hold fewer than
 * coarse_num points:
 *   keep(i, s)  <=>  s = 0  or  sum_{s' < s} |H_{routes[i][s']}| < coarse_num,
 * i.e. the shortest prefix holding at least coarse_num points (all t slots
 * when even they hold fewer). Dropped slots become -1. home_count receives
 * |H_p| for p in [0, m). */
void or_routes_coarse(const int32_t* routes, int64_t n, int32_t t, int32_t m,
                      int64_t coarse_num, int32_t* out, int32_t* home_count) {
  for (int32_t p = 0; p < m; ++p) home_count[p] = 0;
  for (int64_t j = 0; j < n; ++j) {
    const int32_t h = routes[j * t];
    if (h >= 0 && h < m) home_count[h] += 1;
  }
  for (int64_t i = 0; i < n; ++i) {
    int64_t held = 0;  /* points in the centres kept so far */
    for (int32_t s = 0; s < t; ++s) {
      const int32_t p = routes[i * t + s];
      const int keep = (s == 0) || (held < coarse_num);
      out[i * t + s] = keep ? p : -1;
      if (keep && p >= 0 && p < m) held += home_count[p];
    }
  }
}

/* Distance-gap rule (not in the paper; a non-learned variable number of probes
 * next to coarse_num): keep the home (slot 0) and every further slot s whose
 * centre is at most delta farther from the point than the home's centre,
 * rdist[s] - rdist[0] <= delta; the other slots become -1. routes, rdist:
 * [n][t] t-nearest-centre routes and their distances. */
void or_routes_gap(const int32_t* routes, const int32_t* rdist, int64_t n, int32_t t,
                   int32_t delta, int32_t* out) {
  for (int64_t i = 0; i < n; ++i)
    for (int32_t s = 0; s < t; ++s) {
      const int keep = (s == 0) || (rdist[i * t + s] - rdist[i * t] <= delta);
      out[i * t + s] = keep ? routes[i * t + s] : -1;
    }
}

/* Single-pass divide-and-conquer graph of Section 3.2, as a plain definition:
 *   home(j) = routes[j][0],   C(i) = { j != i : home(j) in T(i) },
 *   G(i)    = first k of sort over (d(i, j), j) for j in C(i).
 * This is what Map -> Shuffle -> Reduce1 (each routed record searched against
 * the home records of its centre) -> Shuffle -> Reduce2 (merge-sort per label)
 * produces, because the home sets are disjoint. Enumerated directly over all j
 * (no partition-major structure), for the query points qidx. */
void or_knn_partitioned(const uint64_t* codes, int64_t n, int32_t W, const int32_t* routes,
                        int32_t t, int32_t k, const int64_t* qidx, int64_t nq,
                        int32_t* out_ids, int32_t* out_dist) {
  const int32_t bits = 64 * W;
#pragma omp parallel
  {
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 4)
    for (int64_t q = 0; q < nq; ++q) {
      const int64_t i = qidx[q];
      int64_t c = 0;
      for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const int32_t hj = routes[j * t];
        int in_t = 0;
        for (int32_t s = 0; s < t; ++s) in_t |= (hj >= 0 && routes[i * t + s] == hj);
        if (!in_t) continue;
        keys[c++] = KEY(or_hamming(codes + i * W, codes + j * W, W), j);
      }
      qsort(keys, (size_t)c, sizeof(uint64_t), cmp_u64);
      emit_topk(keys, c, k, bits, out_ids + q * k, out_dist + q * k);
    }
    free(keys);
  }
}

/* Graph pruning of Section 3.4, after the occlusion rule of FANNG (Harwood and
 * Drummond, CVPR 2016). The candidates of point x are the ids listed in its row
 * (ids outside [0, n), x itself and repeats dropped), taken in order of
 * (d(x, y), y). A candidate y is kept unless a neighbour z kept before it lies
 * closer to y than x does:
 *   keep(y)  <=>  no kept z with d(z, y) < d(x, y),
 * and at most L are kept (the walk stops there). The row is written in kept
 * order (which is (d, id) order), padded to L with (-1, bits + 1). */
void or_prune(const uint64_t* codes, int64_t n, int32_t W, const int32_t* ids_in, int32_t k,
              int32_t L, int32_t* out_ids, int32_t* out_dist) {
  const int32_t bits = 64 * W;
#pragma omp parallel
  {
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(k + 1));
    int32_t* kept = (int32_t*)malloc(sizeof(int32_t) * (size_t)(L + 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t x = 0; x < n; ++x) {
      int64_t c = 0;
      for (int32_t a = 0; a < k; ++a) {
        const int32_t y = ids_in[x * k + a];
        if (y < 0 || y >= n || y == x) continue;
        int seen = 0;
        for (int64_t b = 0; b < c; ++b) seen |= (KEY_ID(keys[b]) == y);
        if (!seen) keys[c++] = KEY(or_hamming(codes + x * W, codes + (int64_t)y * W, W), y);
      }
      qsort(keys, (size_t)c, sizeof(uint64_t), cmp_u64);
      int32_t nk = 0;
      for (int64_t b = 0; b < c && nk < L; ++b) {
        const int32_t y = KEY_ID(keys[b]), dxy = KEY_D(keys[b]);
        int occluded = 0;
        for (int32_t e = 0; e < nk && !occluded; ++e)
          occluded = or_hamming(codes + (int64_t)kept[e] * W, codes + (int64_t)y * W, W) < dxy;
        if (!occluded) {
          kept[nk] = y;
          out_ids[x * L + nk] = y;
          out_dist[x * L + nk] = dxy;
          ++nk;
        }
      }
      for (int32_t r = nk; r < L; ++r) { out_ids[x * L + r] = -1; out_dist[x * L + r] = bits + 1; }
    }
    free(keys);
    free(kept);
  }
}

/* One round of neighbourhood propagation (Section 3.3): every point x is
 * compared with the neighbours of its neighbours (the "second floor"), and its
 * new list is the first k of sort over (d, id) of its current list together
 * with those candidates:
 *   G'(x) = first k of sort_{(d, id)} ( G(x) u { y in G(z) : z in G(x), y != x } ),
 * every id counted once; ids -1 (padding) are ignored. All rows read the input
 * graph G (ids [n][k], distances recomputed from the codes), none reads G'.
 * The propagation filter of Section 3.6 (3) only drops candidates that cannot
 * enter the first k, so it is not applied here. */
void or_propagate(const uint64_t* codes, int64_t n, int32_t W, const int32_t* ids_in, int32_t k,
                  int32_t* out_ids, int32_t* out_dist) {
  const int32_t bits = 64 * W;
#pragma omp parallel
  {
    uint64_t* keys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(k + (int64_t)k * k + 1));
#pragma omp for schedule(dynamic, 16)
    for (int64_t x = 0; x < n; ++x) {
      int64_t c = 0;
      for (int32_t a = 0; a < k; ++a) {
        const int32_t z = ids_in[x * k + a];
        if (z < 0 || z >= n) continue;
        if (z != x) keys[c++] = KEY(or_hamming(codes + x * W, codes + (int64_t)z * W, W), z);
        for (int32_t b2 = 0; b2 < k; ++b2) {
          const int32_t y = ids_in[(int64_t)z * k + b2];
          if (y < 0 || y >= n || y == x) continue;
          keys[c++] = KEY(or_hamming(codes + x * W, codes + (int64_t)y * W, W), y);
        }
      }
      qsort(keys, (size_t)c, sizeof(uint64_t), cmp_u64);
      int64_t u = 0;  /* every id once */
      for (int64_t i = 0; i < c; ++i)
        if (u == 0 || keys[i] != keys[u - 1]) keys[u++] = keys[i];
      emit_topk(keys, u, k, bits, out_ids + x * k, out_dist + x * k);
    }
    free(keys);
  }
}

/* ---- binary heaps over keys (min-heap; a max-heap stores ~key) ---- */
typedef struct { uint64_t* a; int64_t n; } heap_t;
static void heap_push(heap_t* h, uint64_t v) {
  int64_t i = h->n++;
  h->a[i] = v;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h->a[p] <= h->a[i]) break;
    uint64_t tmp = h->a[p]; h->a[p] = h->a[i]; h->a[i] = tmp;
    i = p;
  }
}
static uint64_t heap_pop(heap_t* h) {
  uint64_t top = h->a[0];
  h->a[0] = h->a[--h->n];
  int64_t i = 0;
  for (;;) {
    int64_t l = 2 * i + 1, r = l + 1, s = i;
    if (l < h->n && h->a[l] < h->a[s]) s = l;
    if (r < h->n && h->a[r] < h->a[s]) s = r;
    if (s == i) break;
    uint64_t tmp = h->a[s]; h->a[s] = h->a[i]; h->a[i] = tmp;
    i = s;
  }
  return top;
}

/* Search procedure of Section 3.5 (long-link entry + hill climbing), best-first:
 *   keys kappa(j) = (d(q, j), j);
 *   entry e = argmin over the sampled points E of kappa;
 *   visited = {e}; Cand = min-heap {kappa(e)}; Pool = max-heap {kappa(e)}, |Pool| <= ef;
 *   while Cand non-empty:
 *     c = pop-min(Cand);
 *     if |Pool| == ef and kappa(c) > max(Pool): stop;
 *     for n in G(c) in list order, n != -1, n not visited:
 *       mark n visited;
 *       if |Pool| < ef or kappa(n) < max(Pool):
 *         push n into Cand and Pool; if |Pool| > ef: drop max(Pool).
 *   result = Pool ascending, first R' = min(ef, R) keys, padded to R.
 * counters[q] = {expansions (nodes whose lists were scanned), distance evaluations}. */
void or_search(const uint64_t* codes, int64_t n, int32_t W, const int32_t* graph, int32_t deg,
               const int32_t* entry, int32_t S, const uint64_t* queries, int64_t nq,
               const int32_t* ef, int32_t R, int32_t* out_ids, int32_t* out_dist,
               int64_t* counters) {
  const int32_t bits = 64 * W;
#pragma omp parallel
  {
    uint8_t* visited = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint64_t* cand_buf = NULL;
    uint64_t* pool_buf = NULL;
    int64_t cap = 0;
#pragma omp for schedule(dynamic, 8)
    for (int64_t q = 0; q < nq; ++q) {
      const uint64_t* y = queries + q * W;
      const int32_t efq = ef[q];
      int64_t need = (int64_t)efq + (int64_t)deg + 2;
      if (n + 2 > need) need = n + 2;
      if (need > cap) {
        free(cand_buf); free(pool_buf);
        cap = need;
        cand_buf = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)cap);
        pool_buf = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)cap);
      }
      heap_t cand = {cand_buf, 0}, pool = {pool_buf, 0}; /* pool holds ~key */
      int64_t n_touched = 0, expansions = 0, dist_evals = 0;
      uint64_t best = ~(uint64_t)0;
      for (int32_t s = 0; s < S; ++s) {
        uint64_t kk = KEY(or_hamming(y, codes + (int64_t)entry[s] * W, W), entry[s]);
        ++dist_evals;
        if (kk < best) best = kk;
      }
      const int32_t e = KEY_ID(best);
      visited[e] = 1; touched[n_touched++] = e;
      heap_push(&cand, best);
      heap_push(&pool, ~best);
      while (cand.n > 0) {
        const uint64_t c = heap_pop(&cand);
        if (pool.n == efq && c > ~pool.a[0]) break;
        ++expansions;
        const int32_t* nb = graph + (int64_t)KEY_ID(c) * deg;
        for (int32_t s = 0; s < deg; ++s) {
          const int32_t v = nb[s];
          if (v < 0 || visited[v]) continue;
          visited[v] = 1; touched[n_touched++] = v;
          const uint64_t kv = KEY(or_hamming(y, codes + (int64_t)v * W, W), v);
          ++dist_evals;
          if (pool.n < efq || kv < ~pool.a[0]) {
            heap_push(&cand, kv);
            heap_push(&pool, ~kv);
            if (pool.n > efq) heap_pop(&pool);
          }
        }
      }
      /* pool as ascending keys */
      const int64_t np = pool.n;
      for (int64_t r = 0; r < np; ++r) pool_buf[r] = ~pool_buf[r];
      qsort(pool_buf, (size_t)np, sizeof(uint64_t), cmp_u64);
      const int64_t keep = np < R ? np : R;
      for (int32_t r = 0; r < R; ++r) {
        if (r < keep) {
          out_ids[q * R + r] = KEY_ID(pool_buf[r]);
          out_dist[q * R + r] = KEY_D(pool_buf[r]);
        } else {
          out_ids[q * R + r] = -1;
          out_dist[q * R + r] = bits + 1;
        }
      }
      if (counters) { counters[2 * q] = expansions; counters[2 * q + 1] = dist_evals; }
      for (int64_t r = 0; r < n_touched; ++r) visited[touched[r]] = 0;
    }
    free(visited); free(touched); free(cand_buf); free(pool_buf);
  }
}

/* Real-valued re-rank of Section 3.5 with d = l2 of Section 3:
 * s(j) = sum_u (q_u - x_{j,u})^2 accumulated in order u = 0..D-1 in single
 * precision, then the first k of sort over (s, j); entries j = -1 are skipped;
 * rows with fewer than k valid candidates pad with (inf, -1). */
typedef struct { float s; int32_t id; } fkey_t;
static int cmp_fkey(const void* a, const void* b) {
  const fkey_t* x = (const fkey_t*)a; const fkey_t* y = (const fkey_t*)b;
  if (x->s < y->s) return -1;
  if (x->s > y->s) return 1;
  return (x->id > y->id) - (x->id < y->id);
}
typedef struct { double s; int32_t id; } dkey_t;
static int cmp_dkey(const void* a, const void* b) {
  const dkey_t* x = (const dkey_t*)a; const dkey_t* y = (const dkey_t*)b;
  if (x->s < y->s) return -1;
  if (x->s > y->s) return 1;
  return (x->id > y->id) - (x->id < y->id);
}

void or_rerank_f32(const float* feats, int32_t D, const float* qfeats, const int32_t* cand,
                   int64_t nq, int32_t R, int32_t k, int32_t* out_ids, float* out_d) {
#pragma omp parallel
  {
    fkey_t* keys = (fkey_t*)malloc(sizeof(fkey_t) * (size_t)(R > 0 ? R : 1));
#pragma omp for schedule(static)
    for (int64_t q = 0; q < nq; ++q) {
      int32_t c = 0;
      for (int32_t r = 0; r < R; ++r) {
        const int32_t j = cand[q * R + r];
        if (j < 0) continue;
        float s = 0.0f;
        for (int32_t u = 0; u < D; ++u) {
          const float diff = qfeats[q * D + u] - feats[(int64_t)j * D + u];
          s = s + diff * diff;
        }
        keys[c].s = s; keys[c].id = j; ++c;
      }
      qsort(keys, (size_t)c, sizeof(fkey_t), cmp_fkey);
      for (int32_t r = 0; r < k; ++r) {
        out_ids[q * k + r] = r < c ? keys[r].id : -1;
        out_d[q * k + r] = r < c ? keys[r].s : INFINITY;
      }
    }
    free(keys);
  }
}

/* Same definition in double precision (the tolerance reference). */
void or_rerank_f64(const float* feats, int32_t D, const float* qfeats, const int32_t* cand,
                   int64_t nq, int32_t R, int32_t k, int32_t* out_ids, double* out_d) {
#pragma omp parallel
  {
    dkey_t* keys = (dkey_t*)malloc(sizeof(dkey_t) * (size_t)(R > 0 ? R : 1));
#pragma omp for schedule(static)
    for (int64_t q = 0; q < nq; ++q) {
      int32_t c = 0;
      for (int32_t r = 0; r < R; ++r) {
        const int32_t j = cand[q * R + r];
        if (j < 0) continue;
        double s = 0.0;
        for (int32_t u = 0; u < D; ++u) {
          const double diff = (double)qfeats[q * D + u] - (double)feats[(int64_t)j * D + u];
          s += diff * diff;
        }
        keys[c].s = s; keys[c].id = j; ++c;
      }
      qsort(keys, (size_t)c, sizeof(dkey_t), cmp_dkey);
      for (int32_t r = 0; r < k; ++r) {
        out_ids[q * k + r] = r < c ? keys[r].id : -1;
        out_d[q * k + r] = r < c ? keys[r].s : INFINITY;
      }
    }
    free(keys);
  }
}
