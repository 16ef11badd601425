/*
 * bdg.h -- C ABI of the B300 (sm_103a) Binary Distributed Graph library.
 *
 * The library builds a k-nearest-neighbour graph over packed binary codes under
 * Hamming distance and searches it, following Zhao et al., "Large-Scale Visual
 * Search with Binary Distributed Graph at Alibaba": Hamming distance and the
 * k-NN label sets B(l_i) of Section 3, binary codes of Section 3.1, Bk-means
 * (Eq. 1-2) and the single-pass divide-and-conquer build of Section 3.2, and the
 * search procedure with real-valued re-rank of Section 3.5.
 *
 * Conventions for every call:
 *   - Array arguments are DEVICE pointers unless a comment says "host". The
 *     caller owns every array it passes in or out; the library owns only what a
 *     handle (bdg_graph, bdg_router) holds and frees it in the matching _free.
 *   - Codes: uint64 [n][W] row-major, W = bits / 64, bit j of a code in word
 *     j / 64 at bit position j % 64 (least-significant bit first). bits is a
 *     multiple of 64 with W in {1, 2, 4, 8, 16}.
 *   - Neighbour lists order candidates by (distance, id) ascending. Rows with
 *     fewer valid entries than requested are padded with id = -1 and
 *     distance = bits + 1.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). Calls enqueue
 *     work and return without synchronising unless documented otherwise.
 *   - Every call returns a bdg_status; arguments are checked before any work is
 *     enqueued. On failure bdg_last_error() gives a message for the calling
 *     thread. No call aborts or throws.
 */
#ifndef BDG_H_
#define BDG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  BDG_OK = 0,
  BDG_EINVAL = -1,        /* an argument is out of range or inconsistent */
  BDG_ENOMEM = -2,        /* a device allocation failed or the budget is exceeded */
  BDG_ECUDA = -3,         /* a CUDA runtime call failed (message has the CUDA error) */
  BDG_ETIMEOUT = -4,      /* a bounded device wait gave up */
  BDG_EUNSUPPORTED = -5   /* the configuration is valid but not built (e.g. W = 3) */
} bdg_status;

/* Message of the last failed call on this host thread ("" if none). */
const char* bdg_last_error(void);

/* Library version as an integer (major * 10000 + minor * 100 + patch). */
int32_t bdg_version(void);

/* Device memory budget of the library in bytes (0 = unlimited). Allocations
 * that would take the library's live total above it fail with BDG_ENOMEM. */
bdg_status bdg_set_memory_budget(uint64_t bytes);
uint64_t bdg_memory_in_use(void);

/* Number of kernels this library has launched in the process so far. */
int64_t bdg_launch_count(void);

/* Event timing of the library's main kernels on their launch streams (off by
 * default). bdg_profile_read synchronises on the recorded events and returns
 * the summed device time and launch count of the kernel `name` ("knn",
 * "merge", "route", "search", "rerank"); bdg_profile_reset drops all records. */
void bdg_profile_enable(int32_t on);
bdg_status bdg_profile_read(const char* name, double* total_ms, int64_t* launches);
void bdg_profile_reset(void);

/* ------------------------------------------------------------------ pieces */

/* Hamming k-NN of Section 3 / the nearest-centre map step of Section 3.2:
 * for each of the n points, the t nearest of m centres ordered by
 * (d(y_i, c_c), c). routes/rdist: [n][t] int32. 1 <= t <= min(m, 16). */
bdg_status bdg_route(const uint64_t* codes, int64_t n, int32_t bits, const uint64_t* centroids,
                     int32_t m, int32_t t, int32_t* routes, int32_t* rdist, void* stream);

/* The coarse_num rule of Section 3.2: the number of nearest centres a point is
 * mapped to varies so that the points held by its centres add up to a fixed
 * total. routes: [n][t] int32, in place, each row the point's t nearest
 * centres in order (slot 0 = home, as bdg_route writes them). home_count:
 * out [m] int32, |H_p| = #{ j : routes[j][0] = p } (caller-owned device
 * memory). Point i keeps slot 0 and keeps slot s >= 1 while the centres before
 * it hold fewer than coarse_num points (sum of home_count over slots < s);
 * later slots become -1 (the build then probes nothing there). So each point
 * keeps the shortest prefix of its centres holding at least coarse_num
 * points, or all t. Slots outside [0, m) hold no points. Requires
 * 1 <= t <= 16, m >= 1, coarse_num >= 0; BDG_EINVAL otherwise. */
bdg_status bdg_routes_coarse(int32_t* routes, int64_t n, int32_t t, int32_t m, int64_t coarse_num,
                             int32_t* home_count, void* stream);

/* A distance-gap number of probes (not in the paper: the non-learned baseline
 * of the learned router's variable number of probes, next to coarse_num). In
 * place on t-nearest-centre routes [n][t] (device) and their distances rdist
 * [n][t] (from bdg_route): slot s >= 1 becomes -1 when rdist[s] - rdist[0] >
 * delta, i.e. every centre at most delta farther than the home's stays probed.
 * Requires 1 <= t <= 16; BDG_EINVAL otherwise. */
bdg_status bdg_routes_gap(int32_t* routes, const int32_t* rdist, int64_t n, int32_t t,
                          int32_t delta, void* stream);

/* Bk-means of Section 3.2 (objective Eq. 1, update Eq. 2) on the down-sample
 * codes[sample[0..S)]: centres start as the codes of sample[0..m); each of
 * `iters` iterations assigns every sample point to its nearest centre by
 * (distance, centre index) and sets each centre bit to the majority of its
 * members' bits, keeping the previous bit on a tie and the previous centre
 * when the cluster is empty. centroids: out [m][W]. loss: optional out int64
 * [iters + 1], the objective after each assign step (NULL to skip).
 * Requires m <= S. Sample ids must lie in [0, n); the kernels cannot check
 * device-side ids before launch, so an id outside that range is read as the
 * all-zero code (never outside `codes`) and the result is then unspecified. */
bdg_status bdg_bkmeans(const uint64_t* codes, int64_t n, int32_t bits, const int64_t* sample,
                       int64_t S, int32_t m, int32_t iters, uint64_t* centroids, int64_t* loss,
                       void* stream);

/* Exact k-NN rows of Section 3 (the ideal B(l_i) under d = l_h) for selected
 * points: row r is the first k of sort over (d(rows[r], j), j) for all
 * j != rows[r] in [0, N). The brute-force judge of a graph's recall.
 * rows: [nrows] int32; out_ids/out_dist: [nrows][k]. 1 <= k <= 128, k < N. */
bdg_status bdg_knn_rows(const uint64_t* codes, int64_t N, int32_t bits, const int32_t* rows,
                        int64_t nrows, int32_t k, int32_t* out_ids, int32_t* out_dist,
                        void* stream);

/* bdg_bkmeans without any device allocation (the paper has no counterpart).
 * It is for callers that must not allocate device memory: processes whose
 * device memory belongs to an outside manager (a framework's pool, a fixed
 * arena set up at start-up), and loops that must never reach the allocator
 * because an allocation there can synchronise the device or fail under memory
 * pressure. Same arguments and results as bdg_bkmeans. Its scratch is one fixed
 * 16 MiB array inside the library, reserved on every GPU that loads the
 * library until the process exits; calls needing more
 * (bdg_bkmeans_scratch_bytes > 16 MiB; S = 16384, m = 256, 512 bits needs about
 * 1.8 MiB) fail with BDG_EINVAL before any work. The first call on a device
 * looks up the array's device address (once per device, with that device
 * current) and caches it for the life of the process; do not use the entry
 * point after cudaDeviceReset (the cached address then no longer names the
 * array). All
 * calls share the one array, which keeps the last call's contents: calls that
 * may overlap on the GPU (different streams, or different host threads) race
 * and must be ordered by the caller. No cudaMalloc/cudaFree or allocating
 * library routine is called. */
bdg_status bdg_bkmeans_noalloc(const uint64_t* codes, int64_t n, int32_t bits,
                               const int64_t* sample, int64_t S, int32_t m, int32_t iters,
                               uint64_t* centroids, int64_t* loss, void* stream);

/* ------------------------------------------------------------------ build */

/* The `partitions` argument of the build (Section 3.2). */
typedef struct bdg_partitions {
  int32_t m;                  /* number of partitions (1 = exact brute force) */
  int32_t t;                  /* partitions probed per point, home included; 1 <= t <= m, t <= 16 */
  const uint64_t* centroids;  /* [m][W] binary centres, or NULL: run Bk-means first */
  const int64_t* bk_sample;   /* [bk_sample_size] point ids in [0, N) of the Bk-means down-sample */
  int64_t bk_sample_size;     /* >= m when centroids == NULL */
  int32_t bk_iters;           /* Bk-means iterations (the paper uses fewer than 10) */
  const int32_t* routes;      /* [N][t] precomputed routes (slot 0 = home), or NULL; a row
                                 must hold distinct partitions; values outside [0, m) are
                                 ignored (that slot contributes no neighbours) */
  const int32_t* entry;       /* [n_entry] long-link sample ids kept with the graph (Section 3.5) */
  int32_t n_entry;            /* 1 <= n_entry */
  int32_t tile_visitors;      /* work-item size in visitors: 0 (= 128) or 128 */
  int32_t kernel;             /* Reduce-1 kernel: 0 = auto (tensor cores for 256/512-bit
                                 codes and k <= 64, else popcount), 1 = popcount, 2 = tensor */
  int64_t coarse_num;         /* 0: every point probes its t nearest centres. > 0: the
                                 library's routes are cut by the coarse_num rule of
                                 Section 3.2 (see bdg_routes_coarse), t being the most a
                                 point may probe; needs routes == NULL */
  int32_t class_kernel[3];    /* Reduce-1 variant per partition size class (class 0:
                                 |H_p| >= 4096, class 1: 512 <= |H_p| < 4096, class 2:
                                 |H_p| < 512): 0 = follow `kernel`, 1 = popcount (64-visitor
                                 sub-tiles), 2 = tensor (128 x 128 tiles), 3 = popcount with
                                 32-visitor sub-tiles. Results are identical for any choice */
} bdg_partitions;

typedef struct bdg_graph bdg_graph; /* opaque; owns ids/dists/entry, borrows codes */

/* Single-pass divide-and-conquer k-NN graph of Section 3.2 on one GPU:
 *   route every point to its t nearest centres (slot 0 = home, the flagged
 *   record of the Map step), group points by home and by routed partition
 *   (Shuffle 1), compute for every routed point the exact k nearest home
 *   records of each of its partitions with a fused Hamming + top-k kernel
 *   (Reduce 1), and merge the t partial lists per point (Shuffle 2 + Reduce 2).
 * The result equals G(i) = first k of sort over (d(i, j), j) for j != i whose
 * home is one of i's t partitions; with m = 1 it is the exact k-NN graph.
 * codes: [N][W] borrowed (must outlive the graph). 1 <= k <= 128, k < N,
 * N < 2^31. *out receives a new graph handle; free with bdg_graph_free. */
bdg_status bdg_build_graph(const uint64_t* codes, int64_t N, int32_t bits, int32_t k,
                           const bdg_partitions* partitions, void* stream, bdg_graph** out);

/* A build plan: the whole build of bdg_build_graph (Bk-means, routing,
 * bucketing, the Reduce-1 kernel, the merge) captured once into a CUDA graph
 * over scratch and graph storage allocated once, then replayed by
 * bdg_build_plan_run (one graph launch per build). With partitions->kernel = 0
 * and no class_kernel set, an autotuner runs every Reduce-1 variant (popcount
 * with 64- and with 32-visitor sub-tiles, tensor cores with 128 x 128 tiles) on
 * this very workload, times each partition size class (the persistent kernels
 * take one class's work items per launch), and keeps the fastest variant per
 * class; the choice is cached per (device, bits, k, N, m, t) in the file named
 * by $BDG_AUTOTUNE_CACHE (default
 * ~/.cache/bdg_autotune.txt; an unwritable cache is ignored). Every array the
 * partitions reference and the codes must stay alive and are re-read at each
 * run (their contents may change between runs; their sizes may not). Creating
 * a plan synchronises `stream`. */
typedef struct bdg_build_plan bdg_build_plan;
bdg_status bdg_build_plan_create(const uint64_t* codes, int64_t N, int32_t bits, int32_t k,
                                 const bdg_partitions* partitions, void* stream,
                                 bdg_build_plan** out);
bdg_status bdg_build_plan_run(bdg_build_plan* plan, void* stream);
/* Device time in ms of the Reduce-1 step (the fused Hamming + top-k kernel and
 * its fix-up) of the most recent run, from events recorded inside the graph.
 * Synchronises on that run. */
bdg_status bdg_build_plan_kernel_ms(bdg_build_plan* plan, float* ms);
/* The plan's graph (rows rewritten by every run), the chosen kernel (1 popcount,
 * 2 tensor) and, when the autotuner ran, both measured build times in ms (-1 if
 * not measured). */
/* One build from host memory: copies host_codes ([N][W], the plan's codes
 * size) into the device codes the plan was created with, replays the build and
 * copies the graph rows back into host_ids (and host_dists unless NULL), each
 * [N][k] int32, all enqueued on `stream` (asynchronous: synchronise the stream
 * before reading the rows or reusing host_codes; page-locked host buffers let
 * the copies run asynchronously). Plans on different streams overlap one
 * build's copies with another's kernels. The paper's records arrive from and
 * leave for disk; this is the host-memory boundary of one build. */
bdg_status bdg_build_plan_run_host(bdg_build_plan* plan, const uint64_t* host_codes,
                                   int32_t* host_ids, int32_t* host_dists, void* stream);
bdg_status bdg_build_plan_info(const bdg_build_plan* plan, const bdg_graph** graph,
                               int32_t* kernel, float* ms_popc, float* ms_tc);
/* The plan's Reduce-1 variant per partition size class (variant[3]: 1 popcount,
 * 2 tensor, 3 popcount with 32-visitor sub-tiles), the classes' size bounds
 * (size_lo[3] <= |H_p| < size_hi[3]) and, when the autotuner ran, the measured
 * Reduce-1 ms of every variant on every class (ms[3 variants][3 classes],
 * variant v at row v - 1; -1 = not measured). Any output pointer may be NULL. */
bdg_status bdg_build_plan_classes(const bdg_build_plan* plan, int32_t* variant, int32_t* size_lo,
                                  int32_t* size_hi, float* ms);
void bdg_build_plan_free(bdg_build_plan* plan);

/* Device pointers to the graph rows: ids/dists [N][k] int32, row i sorted by
 * (distance, id). Any output pointer may be NULL. Host scalars n/k/bits. */
bdg_status bdg_graph_info(const bdg_graph* g, const int32_t** ids, const int32_t** dists,
                          int64_t* n, int32_t* k, int32_t* bits);

/* Neighbourhood propagation (Section 3.3, with the propagation filter of
 * Section 3.6 (3)): `rounds` synchronous rounds, each replacing every row by
 *   G'(x) = first k of sort_{(d, id)} ( G(x) u { y in G(z) : z in G(x), y != x } ),
 * every id once (the neighbours of the neighbours are the "second floor"). Reads
 * g's rows, which must be sorted by (distance, id) with padding last (every
 * graph this library builds or loads is), and writes a new graph *out (same k,
 * entry sample and borrowed codes; free it with bdg_graph_free). k <= 128.
 * Asynchronous on `stream`; BDG_EINVAL for rounds < 1, BDG_EUNSUPPORTED for
 * k > 128, BDG_ENOMEM if the rows (and, for rounds > 1, one scratch pair) do
 * not fit the memory budget. */
bdg_status bdg_graph_propagate(const bdg_graph* g, int32_t rounds, void* stream, bdg_graph** out);

/* Graph pruning of Section 3.4, after FANNG's occlusion rule (Harwood and
 * Drummond, CVPR 2016): the neighbours y of x listed in g's row (ids outside
 * [0, N), x itself and repeats dropped) are taken in (d(x, y), y) order, with
 * distances recomputed from the codes; y is kept unless a neighbour z kept
 * before it has d(z, y) < d(x, y) (an equal distance does not occlude), and at
 * most L are kept. Writes a new graph *out with k = L (rows in kept order,
 * padded with id -1, distance bits + 1; same entry sample and borrowed codes;
 * free it with bdg_graph_free). Asynchronous on `stream`. BDG_EINVAL unless
 * 1 <= L <= min(g's k, 64); BDG_EUNSUPPORTED for g's k > 128; BDG_ENOMEM if the
 * new rows do not fit the memory budget. */
bdg_status bdg_graph_prune(const bdg_graph* g, int32_t L, void* stream, bdg_graph** out);

/* Multi-shard build of Section 3.4: the points are split into S contiguous
 * shards, shard s holding points [off[s], off[s+1]) with off[s] = floor(s N / S),
 * and each shard gets its own divide-and-conquer graph over its points only
 * (local ids 0 .. n_s - 1), as bdg_build_graph builds it. The binary centres do
 * not depend on the shard, so Bk-means runs once, on the whole data (with
 * partitions->bk_sample, global ids), unless partitions->centroids is given;
 * every shard is routed with the same centres. partitions->entry holds S
 * consecutive samples of n_entry LOCAL ids, one per shard; partitions->routes,
 * when given, is the [N][t] array for all points (shard s reads its rows).
 * out: host array of S handles, each a graph that borrows codes + off[s] * W;
 * free each with bdg_graph_free (on failure none is returned). 1 <= S <= 32;
 * every shard needs k < n_s. */
bdg_status bdg_build_sharded(const uint64_t* codes, int64_t N, int32_t bits, int32_t k,
                             const bdg_partitions* partitions, int32_t S, void* stream,
                             bdg_graph** out);

/* Search over a multi-shard index (Sections 3.4 and 4): each of the S shard
 * graphs (shards[s] holding global ids off[s] .. off[s] + n_s - 1, off[s] the
 * sum of the earlier shards' sizes) answers every query as bdg_search does; the
 * answers are merged into the first min(ef[q], R) pairs by (distance, global
 * id), padded to R with (-1, bits + 1). All shards must have the queries' bits.
 * out_ids/out_dist: [nq][R] global ids and distances. Scratch of S * nq * R * 8
 * bytes is taken from the memory budget. 1 <= S <= 32, S * R <= 6144. */
bdg_status bdg_search_sharded(const bdg_graph* const* shards, int32_t S, const uint64_t* queries,
                              int64_t nq, const int32_t* ef, int32_t ef_max, int32_t R,
                              int32_t* out_ids, int32_t* out_dist, void* stream);

/* Merge of partial k-lists (Shuffle 2 + Reduce 2 of Section 3.2 across GPUs):
 * for each of n points, S sorted rows of k (id, distance) pairs from disjoint
 * candidate sets (e.g. the rows that S ranks built over disjoint sets of
 * partitions) become the first k pairs of their union by (distance, id).
 * ids/dists: [S][n][k] int32 (device; id -1 = padding, skipped); out_ids /
 * out_dists: [n][k], padded with (-1, bits + 1). 1 <= S <= 32, S k <= 6144.
 * Asynchronous on `stream`. */
bdg_status bdg_merge_lists(const int32_t* ids, const int32_t* dists, int32_t S, int64_t n,
                           int32_t k, int32_t bits, int32_t* out_ids, int32_t* out_dists,
                           void* stream);

/* (Not in the paper) a search layout that trades device memory for latency:
 * stores, next to the graph's rows, the codes of every row's neighbours
 * ([N][k][W] words, N * k * bits / 8 bytes: 10 GB for 10M points, k = 32,
 * 256-bit codes), so that bdg_search reads a node's neighbour codes as one
 * contiguous block whose address is known as soon as the node is chosen,
 * instead of one random code per neighbour after its id has arrived. Results
 * are unchanged. The copy reflects the graph and the codes at the time of the
 * call; a second call does nothing, so after changing the codes build a new
 * graph. The copy is owned by the graph and freed with it. Asynchronous
 * on `stream`; BDG_ENOMEM if the copy does not fit the memory budget. */
bdg_status bdg_graph_pack_codes(bdg_graph* g, void* stream);

/* Save to / load from a file: header {magic "BDG1", version, N, bits, k, n_entry}
 * followed by ids, dists and entry ids (little-endian int32). Synchronous.
 * load borrows `codes` ([N][W], device) for later searches. */
bdg_status bdg_graph_save(const bdg_graph* g, const char* path);
bdg_status bdg_graph_load(const char* path, const uint64_t* codes, bdg_graph** out);
void bdg_graph_free(bdg_graph* g);

/* ------------------------------------------------------------------ search */

/* Search procedure of Section 3.5, per query q (keys kappa(j) = (d(q, j), j)):
 * the entry is the nearest long-link sample point; then best-first hill
 * climbing on the graph with a pool of the ef best keys seen, expanding the
 * best unexpanded pool entry until none is left. Writes the first
 * min(ef[q], R) pool keys ascending, padded to R.
 * queries: [nq][W]. ef: [nq] int32 (a per-query pool size; batches may mix
 * sizes). ef_max (host): an upper bound of ef over the batch, 1 <= ef_max <=
 * 2048; it sizes the per-query pool (shared memory per query in flight:
 * 26.3 KB above 1536, 14.8 KB up to 1536, 10.3 KB up to 1024, less below).
 * A query whose ef is outside [1, ef_max]
 * gets a row of padding and expansions = -1. out_ids/out_dist: [nq][R].
 * expansions: optional out [nq] int32 (nodes whose lists were scanned). */
bdg_status bdg_search(const bdg_graph* g, const uint64_t* queries, int64_t nq, const int32_t* ef,
                      int32_t ef_max, int32_t R, int32_t* out_ids, int32_t* out_dist,
                      int32_t* expansions, void* stream);

/* Real-valued re-rank of Section 3.5 (d = l2 of Section 3): for each query the
 * squared L2 distance between qfeats[q] and feats[j] for every candidate j of
 * cand[q] (entries -1 skipped), computed in FP32, and the first k by
 * (distance, id). feats: [N][D] f32, qfeats: [nq][D] f32, cand: [nq][R] int32.
 * out_ids: [nq][k] int32, out_d2: [nq][k] f32 (padded with -1 / +inf).
 * D in {128, 256, 512, 1024}; feats/qfeats 16-byte aligned; 1 <= k <= 32;
 * 1 <= R <= 2048. Candidate ids outside [0, N) are skipped like -1. */
bdg_status bdg_rerank(const float* feats, int64_t N, int32_t D, const float* qfeats,
                      const int32_t* cand, int64_t nq, int32_t R, int32_t k, int32_t* out_ids,
                      float* out_d2, void* stream);

/* bdg_search followed by bdg_rerank of its R binary candidates with the query
 * features: the full online path of Section 3.5. cand_ids/cand_dist: [nq][R]
 * int32 caller-owned buffers that receive the binary candidates. */
bdg_status bdg_search_rerank(const bdg_graph* g, const uint64_t* queries, const float* qfeats,
                             const float* feats, int32_t D, int64_t nq, const int32_t* ef,
                             int32_t ef_max, int32_t R, int32_t k, int32_t* cand_ids,
                             int32_t* cand_dist, int32_t* out_ids, float* out_d2, void* stream);

/* ------------------------------------------------------------------ serving */
/* Continuous-batching request loop around bdg_search_rerank (the online path of
 * Section 3.5). A scheduler thread keeps up to n_streams batches in flight;
 * whenever a stream is free it packs the oldest queued requests into a batch
 * of at most max_batch queries, admitting a request only while the device
 * memory of all in-flight batches stays within memory_budget bytes (0 = no
 * limit; a query needs 8W + 4D + 4 + 8R + 8k bytes). Requests that arrive
 * while batches run are admitted as streams and memory free up, so their work
 * overlaps with the running batches. Each query's result depends only on the
 * query and its ef. The graph and feats are borrowed and must outlive the
 * server. 1 <= k <= 32, k <= R <= 2048, 1 <= ef_max <= 2048, 1 <= n_streams
 * <= 16. */
typedef struct bdg_server bdg_server;
bdg_status bdg_server_create(const bdg_graph* g, const float* feats, int32_t D, int32_t R,
                             int32_t k, int32_t ef_max, int32_t max_batch, int32_t n_streams,
                             uint64_t memory_budget, bdg_server** out);
/* queries [nq][W], qfeats [nq][D], ef [nq]: HOST arrays, copied before return.
 * 1 <= nq <= max_batch. *request_id identifies the request for bdg_server_wait. */
bdg_status bdg_server_submit(bdg_server* s, const uint64_t* queries, const float* qfeats,
                             const int32_t* ef, int32_t nq, int64_t* request_id);
/* Waits up to timeout_ms for the request; copies its [nq][k] ids and squared
 * distances to HOST outputs (either may be NULL) and its latency from submit to
 * completion; BDG_ETIMEOUT if not done in time (the request stays queued). */
bdg_status bdg_server_wait(bdg_server* s, int64_t request_id, int32_t* out_ids, float* out_d2,
                           double* latency_ms, int32_t timeout_ms);
bdg_status bdg_server_stats(bdg_server* s, int64_t* batches, int64_t* queries, int64_t* pending,
                            uint64_t* in_flight_bytes);
void bdg_server_free(bdg_server* s);

/* ------------------------------------------------------------------ learned router */
/* The paper routes each point to its t nearest binary centres (Section 3.2).
 * The router keeps the nearest centre as the home (slot 0) and picks the other
 * P - 1 probed partitions with a small BF16 MLP trained on where a point's exact
 * neighbours live:
 *   h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2),
 *   z = [h2 | s] W3^T + b3 (FP32 accumulate), s in {-1, +1}^code_bits the
 *   point's code (bit set = +1; code_bits = 0: z = h2 W3^T + b3)
 *   loss = -(1/B) sum_i sum_p q_ip log softmax(z_i)_p,
 *   q_ip = #{j in labels[i] : j == p} / #{valid labels of i}
 *   (labels: partitions where i's neighbours live, -1 = none; a row without a
 *   valid label contributes neither loss nor gradient)
 * Adam (beta 0.9 / 0.999, eps 1e-8) on FP32 master weights with BF16 copies.
 * With W3 = [0 | (2 c_p - 1) / 2] and b3 = 0 the logits are bits / 2 - d(y, c_p):
 * the router then routes exactly like the nearest-centre rule, and training
 * starts from the method's own routing. */
typedef struct bdg_router bdg_router;

/* init_params: device FP32, packed W1[h1][d_in] b1[h1] W2[h2][h1] b2[h2]
 * W3[m][h2 + code_bits] b3[m] (copied). d_in, h1, h2, m and max_batch multiples
 * of 8; code_bits 0 or a multiple of 64 up to 1024. Synchronous. */
bdg_status bdg_router_create(int32_t d_in, int32_t h1, int32_t h2, int32_t m, int32_t code_bits,
                             const float* init_params, int32_t max_batch, bdg_router** out);
void bdg_router_free(bdg_router* r);
/* Device pointers to the packed FP32 parameters, the gradients of the last
 * training step (same layout), the last loss (scalar) and an error word. */
bdg_status bdg_router_info(const bdg_router* r, float** params, float** grads, int64_t* n_params,
                           float** loss, int32_t** err);
/* x: [B][d_in] BF16 (device); codes: [B][code_bits / 64] packed codes (device;
 * required when code_bits > 0, else ignored). logits: [B][m] FP32. B <= max_batch. */
bdg_status bdg_router_forward(bdg_router* r, const void* x, const uint64_t* codes, int32_t B,
                              float* logits, void* stream);
/* One training step on a batch: forward, loss, backward into the gradient
 * buffer, and (apply_update != 0) an Adam update with learning rate lr.
 * labels: [B][kt] int32 partition ids (-1 entries ignored). exclude: [B] int32
 * or NULL: partition exclude[i] (the home, which is always probed) is left out
 * of row i's softmax and targets. B % 8 == 0. */
bdg_status bdg_router_train_step(bdg_router* r, const void* x, const uint64_t* codes,
                                 const int32_t* labels, int32_t kt, const int32_t* exclude,
                                 int32_t B, float lr, int32_t apply_update, void* stream);
/* routes[i] = {home[i], then the P - 1 other partitions of largest logit,
 * ties by partition index}. x: [N][d_in] BF16, codes: [N][code_bits / 64]
 * (when code_bits > 0), home: [N], routes: [N][P], P <= 17. */
bdg_status bdg_router_route(bdg_router* r, const void* x, const uint64_t* codes, int64_t N,
                            const int32_t* home, int32_t P, int32_t* routes, void* stream);

/* Shortlist head. The last layer evaluated only on a shortlist of Q candidate
 * partitions per point, cand[i][0..Q) (device int32; in this library the Q
 * nearest centres of the Map step of Section 3.2 from bdg_route, so cand[i][0]
 * is the home; -1 = no candidate, never the home slot):
 *   z_ij = [h2_i | s_i] . W3[cand_ij] + b3[cand_ij]   (-inf where cand_ij < 0)
 *   loss = -(1/B) sum_i sum_j q_ij log softmax(z_i)_j,
 *   q_ij = #{labels of i equal to cand_ij} / #{labels of i found in cand_i}
 * (a row none of whose labels is shortlisted contributes neither loss nor
 * gradient). The probe choice keeps the home and adds, by (-z, partition), the
 * other shortlisted partitions whose logit is at least (largest shortlisted
 * logit - theta), computed in FP32, at most pmax - 1 of them: a variable number
 * of probed partitions per point, the learned counterpart of the coarse_num
 * rule of Section 3.2. With the prior weights a (c_p - 1/2) in W3's code
 * columns (zero elsewhere, b3 = 0) the logits are a (bits/2 - d(y, c_p)) and the
 * rule keeps exactly the centres within theta / a of the nearest one.
 * Q <= 16; h2 + code_bits <= 2048. */
/* logits: [B][Q] FP32 (device). B <= max_batch. */
bdg_status bdg_router_forward_shortlist(bdg_router* r, const void* x, const uint64_t* codes,
                                        const int32_t* cand, int32_t Q, int32_t B,
                                        float* logits, void* stream);
/* One training step of the shortlist head (forward, loss, backward through all
 * layers, Adam when apply_update != 0). labels: [B][kt] int32 partition ids
 * (the homes of the point's exact neighbours; -1 ignored). B % 8 == 0. */
bdg_status bdg_router_train_step_shortlist(bdg_router* r, const void* x, const uint64_t* codes,
                                           const int32_t* cand, int32_t Q, const int32_t* labels,
                                           int32_t kt, int32_t B, float lr, int32_t apply_update,
                                           void* stream);
/* routes: [N][pmax] int32 (device): the probe choice above, -1 after the last
 * kept partition; logits: [N][Q] FP32 or NULL. 1 <= pmax <= Q, theta >= 0.
 * order: NULL, or a permutation of 0..N-1 (device int32 [N]) in which the
 * points are processed (results land in their own rows either way): points
 * sharing a home share most of their shortlist, so the home order lets
 * consecutive points reuse the same rows of W3 from cache. Runs in chunks of
 * 2^18 points with a stream-ordered workspace of chunk x (h1 + h2 +
 * code_bits) BF16 values (plus the chunk's gathered inputs with an order);
 * BDG_ENOMEM if it cannot be had. */
bdg_status bdg_router_route_shortlist(bdg_router* r, const void* x, const uint64_t* codes,
                                      const int32_t* cand, int32_t Q, int64_t N, float theta,
                                      int32_t pmax, const int32_t* order, int32_t* routes,
                                      float* logits, void* stream);

/* The router's tensor-core GEMM (tcgen05, BF16 operands, FP32 accumulation):
 *   C[M][N] = epilogue(A[M][K] * B[N][K]^T), A and B row-major with K contiguous;
 * epilogue: + bias[N] (if given), relu (if relu != 0), times [mask[M][N] > 0] (if
 * mask given, BF16), written as FP32 (out_f32) and/or BF16 (out_bf16);
 * colsum[N] += column sums of the result (if given). K % 8 == 0. err: device
 * int32 set non-zero if a bounded wait gave up. The paper has no counterpart:
 * it is the building block of the router above. */
bdg_status bdg_gemm_bf16(const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                         const float* bias, const void* mask, int32_t relu, float* out_f32,
                         void* out_bf16, float* colsum, int32_t* err, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* BDG_H_ */
