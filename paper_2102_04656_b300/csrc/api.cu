// api.cu -- the C ABI of include/bdg.h: argument checks, the memory budget,
// graph handles, and the order of launches of a build or a search. No compute
// happens here; every step of the path runs in the kernels of the other files.
#include <sys/stat.h>

#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"


struct bdg_graph {
  int64_t n;
  int32_t k, bits, W, n_entry;
  const uint64_t* codes;  // borrowed
  int32_t* ids;           // [n][k]
  int32_t* dists;         // [n][k]
  int32_t* entry;         // [n_entry]
  uint64_t* entry_codes;  // [n_entry][W] contiguous copy of the entry sample's codes
  uint64_t* nbr_codes = nullptr;  // [n][k][W] neighbours' codes (bdg_graph_pack_codes), or null
};

namespace {

thread_local char g_err[512] = "";
std::atomic<uint64_t> g_in_use{0};
std::atomic<uint64_t> g_budget{0};

bool valid_w(int W) { return W == 1 || W == 2 || W == 4 || W == 8 || W == 16; }

bdg_status check_bits(int32_t bits) {
  if (bits <= 0 || bits % 64 != 0 || !valid_w(bits / 64))
    return bdg_set_error(BDG_EINVAL, "bits = %d: must be 64 * W with W in {1,2,4,8,16}", bits);
  return BDG_OK;
}

bdg_status reserve(size_t bytes) {
  const uint64_t b = g_budget.load();
  const uint64_t now = g_in_use.fetch_add(bytes) + bytes;
  if (b != 0 && now > b) {
    g_in_use.fetch_sub(bytes);
    return bdg_set_error(BDG_ENOMEM, "memory budget exceeded: %llu + %zu > %llu bytes",
                         (unsigned long long)(now - bytes), bytes, (unsigned long long)b);
  }
  return BDG_OK;
}
void release(size_t bytes) { g_in_use.fetch_sub(bytes); }

// Device allocation (synchronous) counted against the budget.
bdg_status dalloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return BDG_OK;
  BDG_TRY(reserve(bytes));
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    release(bytes);
    *p = nullptr;
    return bdg_set_error(BDG_ENOMEM, "cudaMalloc of %zu bytes failed", bytes);
  }
  return BDG_OK;
}
void dfree(void* p, size_t bytes) {
  if (p) { cudaFree(p); release(bytes); }
}

// Stream-ordered scratch, counted against the budget while it lives.
struct Scratch {
  void* p = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  bdg_status alloc(size_t b, cudaStream_t s) {
    st = s;
    if (b == 0) return BDG_OK;
    BDG_TRY(reserve(b));
    if (cudaMallocAsync(&p, b, s) != cudaSuccess) {
      cudaGetLastError();
      release(b);
      p = nullptr;
      return bdg_set_error(BDG_ENOMEM, "cudaMallocAsync of %zu bytes failed", b);
    }
    bytes = b;
    return BDG_OK;
  }
  ~Scratch() {
    if (p) { cudaFreeAsync(p, st); release(bytes); }
  }
};

inline size_t al(size_t b) { return (b + 255) & ~size_t(255); }

// ---- launch accounting and per-kernel event timing ----
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_prof_on{false};
std::mutex g_prof_mu;
struct ProfSlot {
  std::string name;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev;
};
std::vector<ProfSlot> g_prof;

// Keep freed stream-ordered scratch cached in the device's pool between calls
// (the default pool returns memory to the driver at every synchronisation).
void keep_pool_cached() {
  static bool done[64] = {false};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  done[dev] = true;
}

}  // namespace

void bdg_note_launch(int n) { g_launches.fetch_add(n); }

bdg_prof_scope::bdg_prof_scope(const char* name, cudaStream_t s) : slot(-1), st(s) {
  if (!g_prof_on.load()) return;
  // events recorded into a stream capture would become graph nodes whose
  // timings are never valid: a capturing stream is not profiled
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (size_t i = 0; i < g_prof.size(); ++i)
    if (g_prof[i].name == name) slot = (int)i;
  if (slot < 0) {
    g_prof.push_back(ProfSlot{name, {}});
    slot = (int)g_prof.size() - 1;
  }
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, st);
  g_prof[slot].ev.push_back({a, b});
}

bdg_prof_scope::~bdg_prof_scope() {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEventRecord(g_prof[slot].ev.back().second, st);
}

bdg_status bdg_set_error(bdg_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return s;
}

// Whether "auto" picks the tensor-core Reduce-1 kernel where it applies
// (BDG_KNN_KERNEL=popc|tc overrides; the default is the tensor path).
bool bdg_tc_default() {
  const char* e = getenv("BDG_KNN_KERNEL");
  if (e && strcmp(e, "popc") == 0) return false;
  return true;
}

int bdg_num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cache[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

extern "C" {

const char* bdg_last_error(void) { return g_err; }
int32_t bdg_version(void) { return 100; }

int64_t bdg_launch_count(void) { return g_launches.load(); }

void bdg_profile_enable(int32_t on) { g_prof_on.store(on != 0); }

bdg_status bdg_profile_read(const char* name, double* total_ms, int64_t* launches) {
  if (!name || !total_ms || !launches) return bdg_set_error(BDG_EINVAL, "profile: null argument");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  *total_ms = 0.0;
  *launches = 0;
  for (auto& sl : g_prof) {
    if (sl.name != name) continue;
    for (auto& e : sl.ev) {
      float ms = 0.f;
      BDG_CUDA_TRY(cudaEventSynchronize(e.second));
      BDG_CUDA_TRY(cudaEventElapsedTime(&ms, e.first, e.second));
      *total_ms += ms;
      *launches += 1;
    }
  }
  return BDG_OK;
}

void bdg_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (auto& sl : g_prof)
    for (auto& e : sl.ev) {
      cudaEventSynchronize(e.second);
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
  g_prof.clear();
}

bdg_status bdg_set_memory_budget(uint64_t bytes) {
  g_budget.store(bytes);
  return BDG_OK;
}
uint64_t bdg_memory_in_use(void) { return g_in_use.load(); }

bdg_status bdg_route(const uint64_t* codes, int64_t n, int32_t bits, const uint64_t* centroids,
                     int32_t m, int32_t t, int32_t* routes, int32_t* rdist, void* stream) {
  BDG_TRY(check_bits(bits));
  if (n < 0 || m < 1 || t < 1 || t > m || t > 16)
    return bdg_set_error(BDG_EINVAL, "route: n=%lld m=%d t=%d", (long long)n, m, t);
  if (n > 0 && (!codes || !centroids || !routes))
    return bdg_set_error(BDG_EINVAL, "route: null pointer");
  const int W = bits / 64;
  cudaStream_t st = (cudaStream_t)stream;
  if (n > 0 && bdg_route_small_ok(W, m, t) && bdg_tc_default()) {  // few centres
    keep_pool_cached();
    Scratch sc;
    const size_t b = bdg_route_small_bytes(m, W);
    BDG_TRY(sc.alloc(b, st));
    return bdg_launch_route_small(codes, n, W, centroids, m, t, routes, rdist, sc.p, b, st);
  }
  if (n > 0 && bdg_route_tc_ok(W, n, m, t) && bdg_tc_default()) {
    keep_pool_cached();
    Scratch sc;
    const size_t b = bdg_route_tc_bytes(n, m, W, t);
    BDG_TRY(sc.alloc(b, st));
    return bdg_launch_route_tc(codes, n, W, centroids, m, t, routes, rdist, sc.p, b, st);
  }
  return bdg_launch_route(codes, n, W, centroids, m, t, routes, rdist, st);
}

bdg_status bdg_routes_coarse(int32_t* routes, int64_t n, int32_t t, int32_t m, int64_t coarse_num,
                             int32_t* home_count, void* stream) {
  if (n < 0 || m < 1 || t < 1 || t > 16 || coarse_num < 0)
    return bdg_set_error(BDG_EINVAL, "routes_coarse: n=%lld m=%d t=%d coarse_num=%lld",
                         (long long)n, m, t, (long long)coarse_num);
  if (!home_count || (n > 0 && !routes))
    return bdg_set_error(BDG_EINVAL, "routes_coarse: null pointer");
  return bdg_launch_routes_coarse(routes, n, t, m, coarse_num, home_count, (cudaStream_t)stream);
}

bdg_status bdg_routes_gap(int32_t* routes, const int32_t* rdist, int64_t n, int32_t t,
                         int32_t delta, void* stream) {
  if (n < 0 || t < 1 || t > 16)
    return bdg_set_error(BDG_EINVAL, "routes_gap: n=%lld t=%d", (long long)n, t);
  if (n > 0 && (!routes || !rdist)) return bdg_set_error(BDG_EINVAL, "routes_gap: null pointer");
  return bdg_launch_routes_gap(routes, rdist, n, t, delta, (cudaStream_t)stream);
}

bdg_status bdg_bkmeans(const uint64_t* codes, int64_t n, int32_t bits, const int64_t* sample,
                       int64_t S, int32_t m, int32_t iters, uint64_t* centroids, int64_t* loss,
                       void* stream) {
  BDG_TRY(check_bits(bits));
  if (m < 1 || S < m || iters < 0 || !codes || !sample || !centroids || n < 1)
    return bdg_set_error(BDG_EINVAL, "bkmeans: n=%lld S=%lld m=%d iters=%d", (long long)n,
                         (long long)S, m, iters);
  cudaStream_t st = (cudaStream_t)stream;
  const int W = bits / 64;
  keep_pool_cached();
  Scratch sc;
  const size_t sb = bdg_bkmeans_scratch_bytes(S, m, W);
  BDG_TRY(sc.alloc(sb, st));
  return bdg_launch_bkmeans(codes, n, W, sample, S, m, iters, centroids, loss, sc.p, sb, st);
}

}  // extern "C"

namespace {

// Everything a build needs besides the data: validated settings and the
// scratch layout (routes, centres, Bk-means, CSR, partial lists, expanded
// homes, fix-up flags), so that a build can be enqueued into caller-provided
// scratch (bdg_build_graph) or captured once into a CUDA graph (build plans).
constexpr int kLocPivots = 16;      // pivot homes per partition of the locality order
constexpr int64_t kLocMinHomes = 2048;  // mean |H_p| from which the order is built

struct BuildCfg {
  int W, m, t, tile_v;
  int pivots;  // locality order of H_p over this many pivot homes (0: id order)
  bool need_routes, need_bk, use_tc, tc_ok, route_tc, route_small;
  int kmap[BDG_SIZE_CLASSES];  // Reduce-1 variant (BDG_KV_*) per partition size class
  int64_t coarse;
  size_t b_routes, b_cent, b_bk, b_csr, b_part, b_hexp, b_fix, b_cnt, b_rtc, total;
};

bdg_status build_validate(const uint64_t* codes, int64_t N, int32_t bits, int32_t k,
                          const bdg_partitions* P, BuildCfg* c) {
  BDG_TRY(check_bits(bits));
  if (!codes || !P) return bdg_set_error(BDG_EINVAL, "build: null codes or partitions");
  if (N < 2 || N >= (int64_t(1) << 31))
    return bdg_set_error(BDG_EINVAL, "build: N = %lld out of [2, 2^31)", (long long)N);
  if (k < 1 || k > 128 || k >= N)
    return bdg_set_error(BDG_EINVAL, "build: k = %d must be in [1, min(128, N-1)]", k);
  const int m = P->m, t = P->t;
  if (m < 1 || t < 1 || t > m || t > 16)
    return bdg_set_error(BDG_EINVAL, "build: m = %d, t = %d (need 1 <= t <= min(m, 16))", m, t);
  if (!P->entry || P->n_entry < 1)
    return bdg_set_error(BDG_EINVAL, "build: an entry sample (n_entry >= 1) is required");
  c->W = bits / 64; c->m = m; c->t = t;
  c->need_routes = (P->routes == nullptr) && m > 1;
  c->need_bk = c->need_routes && P->centroids == nullptr;
  if (P->coarse_num < 0 || (P->coarse_num > 0 && P->routes != nullptr))
    return bdg_set_error(BDG_EINVAL, "build: coarse_num = %lld needs library routing "
                         "(routes == NULL; cut given routes with bdg_routes_coarse)",
                         (long long)P->coarse_num);
  c->coarse = c->need_routes ? P->coarse_num : 0;
  if (c->need_bk && (!P->bk_sample || P->bk_sample_size < m || P->bk_iters < 0))
    return bdg_set_error(BDG_EINVAL, "build: Bk-means needs bk_sample with >= m ids");
  if (P->tile_visitors != 0 && P->tile_visitors != bdg_knn_tile_visitors(c->W))
    return bdg_set_error(BDG_EUNSUPPORTED, "build: tile_visitors %d not built for %d bits",
                         P->tile_visitors, bits);
  if (P->kernel < 0 || P->kernel > 2)
    return bdg_set_error(BDG_EINVAL, "build: kernel = %d (0 auto, 1 popcount, 2 tensor)",
                         P->kernel);
  c->tc_ok = bdg_knn_tc_supported(c->W, k) && (m > 1 || N < (1 << 21));
  if (P->kernel == 2 && !c->tc_ok)
    return bdg_set_error(BDG_EUNSUPPORTED,
                         "build: the tensor path needs 256/512-bit codes, k <= 64 and, with "
                         "m = 1, N < 2^21");
  for (int i = 0; i < BDG_SIZE_CLASSES; ++i) {
    const int v = P->class_kernel[i];
    if (v < 0 || v > 3)
      return bdg_set_error(BDG_EINVAL, "build: class_kernel[%d] = %d (0 follow kernel, 1 popcount, "
                           "2 tensor, 3 popcount with 32-visitor sub-tiles)", i, v);
    if (v == BDG_KV_TC && !c->tc_ok)
      return bdg_set_error(BDG_EUNSUPPORTED, "build: class_kernel[%d] = 2 but the tensor path "
                           "does not apply", i);
  }
  if (P->kernel == 3)
    return bdg_set_error(BDG_EINVAL, "build: kernel = 3 is a per-class choice (class_kernel)");
  const int kdef = P->kernel == 2 || (P->kernel == 0 && c->tc_ok && bdg_tc_default())
                       ? BDG_KV_TC : BDG_KV_POPC;
  c->use_tc = false;
  for (int i = 0; i < BDG_SIZE_CLASSES; ++i) {
    c->kmap[i] = P->class_kernel[i] ? P->class_kernel[i] : kdef;
    c->use_tc = c->use_tc || c->kmap[i] == BDG_KV_TC;
  }
  c->tile_v = bdg_knn_tile_visitors(c->W);
  const int W = c->W;
  c->b_routes = c->need_routes || m == 1 ? al((size_t)N * t * 4) : 0;
  c->b_cent = c->need_bk ? al((size_t)m * W * 8) : 0;
  c->b_bk = c->need_bk ? al(bdg_bkmeans_scratch_bytes(P->bk_sample_size, m, W)) : 0;
  // homes in locality order for the tensor path where partitions span many
  // tiles (own tile first in round A; candidate words keep (d, id) order); with
  // 512-bit codes only: with 256-bit codes (k = 32, ~10,000 homes per
  // partition) it measured slower
  c->pivots = c->tc_ok && W == 8 && m > 1 && N / m >= kLocMinHomes ? kLocPivots : 0;
  c->b_csr = al(bdg_csr_bytes(N, m, t, W, c->tile_v, c->pivots));
  c->b_part = t > 1 ? al((size_t)N * k * 8) : 0;  // running k-lists
  c->b_hexp = c->tc_ok ? al(bdg_knn_tc_hexp_bytes(N, m, W)) : 0;
  c->b_fix = c->tc_ok ? al((size_t)N * t) + al(64) : 0;
  c->b_cnt = c->coarse > 0 ? al((size_t)m * 4) : 0;
  // library routing on the tensor cores where the codes allow it
  // (all centres in shared memory when they are few)
  c->route_small = c->need_routes && bdg_route_small_ok(W, m, t) && bdg_tc_default();
  c->route_tc = c->need_routes && !c->route_small && bdg_route_tc_ok(W, N, m, t) &&
                bdg_tc_default();
  c->b_rtc = c->route_small ? al(bdg_route_small_bytes(m, W))
             : c->route_tc  ? al(bdg_route_tc_bytes(N, m, W, t))
                            : 0;
  c->total = c->b_routes + c->b_cent + c->b_bk + c->b_csr + c->b_part + c->b_hexp + c->b_fix +
             c->b_cnt + c->b_rtc;
  return BDG_OK;
}

bdg_status graph_alloc(const BuildCfg& c, const uint64_t* codes, int64_t N, int32_t bits,
                       int32_t k, const bdg_partitions* P, bdg_graph** out) {
  bdg_graph* g = new bdg_graph();
  g->n = N; g->k = k; g->bits = bits; g->W = c.W; g->n_entry = P->n_entry; g->codes = codes;
  bdg_status s = dalloc((void**)&g->ids, (size_t)N * k * 4);
  if (s == BDG_OK) s = dalloc((void**)&g->dists, (size_t)N * k * 4);
  if (s == BDG_OK) s = dalloc((void**)&g->entry, (size_t)P->n_entry * 4);
  if (s == BDG_OK) s = dalloc((void**)&g->entry_codes, (size_t)P->n_entry * c.W * 8);
  if (s != BDG_OK) { bdg_graph_free(g); return s; }
  *out = g;
  return BDG_OK;
}

// Enqueue every step of the build into g using `scratch` (c.total bytes).
// kmap: the Reduce-1 variant of each size class. cls_ev (optional, t x
// BDG_SIZE_CLASSES x 2 events): each class's Reduce-1 launches of each round are
// recorded between a pair of events, and every class gets its own launch.
bdg_status build_enqueue(const BuildCfg& c, const int* kmap, bdg_graph* g, const uint64_t* codes,
                         int64_t N, int32_t bits, int32_t k, const bdg_partitions* P,
                         void* scratch, cudaStream_t st, cudaEvent_t ev0 = nullptr,
                         cudaEvent_t ev1 = nullptr, cudaEvent_t* cls_ev = nullptr) {
  bool use_tc = false, uniform = true;
  for (int i = 0; i < BDG_SIZE_CLASSES; ++i) {
    use_tc = use_tc || kmap[i] == BDG_KV_TC;
    uniform = uniform && kmap[i] == kmap[0];
  }
  const bool split = !uniform || cls_ev != nullptr;
  const int W = c.W, m = c.m, t = c.t;
  char* p = (char*)scratch;
  int32_t* routes = (int32_t*)P->routes;
  if (c.b_routes) { routes = (int32_t*)p; p += c.b_routes; }
  uint64_t* cent = (uint64_t*)P->centroids;
  if (c.b_cent) { cent = (uint64_t*)p; p += c.b_cent; }
  void* bk = p; p += c.b_bk;
  void* csr_mem = p; p += c.b_csr;
  uint64_t* partial = c.b_part ? (uint64_t*)p : nullptr;
  p += c.b_part;
  uint8_t* hexp = c.b_hexp ? (uint8_t*)p : nullptr;
  p += c.b_hexp;
  int8_t* fixflag = c.b_fix ? (int8_t*)p : nullptr;
  int32_t* tc_err = c.b_fix ? (int32_t*)(p + al((size_t)N * t)) : nullptr;
  p += c.b_fix;
  int32_t* home_count = c.b_cnt ? (int32_t*)p : nullptr;
  p += c.b_cnt;
  void* rtc = c.b_rtc ? (void*)p : nullptr;

  BDG_CUDA_TRY(cudaMemcpyAsync(g->entry, P->entry, (size_t)P->n_entry * 4,
                               cudaMemcpyDeviceToDevice, st));
  BDG_TRY(bdg_launch_gather_codes(codes, N, g->entry, P->n_entry, W, g->entry_codes, st));
  if (m == 1) {
    BDG_CUDA_TRY(cudaMemsetAsync(routes, 0, (size_t)N * 4, st));
  } else if (c.need_routes) {
    if (c.need_bk)
      BDG_TRY(bdg_launch_bkmeans(codes, N, W, P->bk_sample, P->bk_sample_size, m, P->bk_iters,
                                 cent, nullptr, bk, c.b_bk, st));
    if (c.route_small)
      BDG_TRY(bdg_launch_route_small(codes, N, W, cent, m, t, routes, nullptr, rtc, c.b_rtc, st));
    else if (c.route_tc)
      BDG_TRY(bdg_launch_route_tc(codes, N, W, cent, m, t, routes, nullptr, rtc, c.b_rtc, st));
    else
      BDG_TRY(bdg_launch_route(codes, N, W, cent, m, t, routes, nullptr, st));
    if (c.coarse > 0)
      BDG_TRY(bdg_launch_routes_coarse(routes, N, t, m, c.coarse, home_count, st));
  }
  if (t > 1) {  // running lists start empty (a point without a valid home keeps none)
    BDG_CUDA_TRY(cudaMemsetAsync(partial, 0xff, (size_t)N * k * 8, st));
  } else if (P->routes != nullptr) {  // rows of points without a valid home read as padding
    BDG_TRY(bdg_launch_fill_pad(g->ids, g->dists, N * (int64_t)k, bits, st));
  }
  bdg_csr csr;
  BDG_TRY(bdg_build_csr(codes, N, W, routes, m, t, c.tile_v, c.pivots, csr_mem, &csr, st));
  // Reduce 1: round A = every point against its home partition (it starts the
  // point's running k-list); then one sub-round per further route slot, each
  // point visiting one partition, its threshold starting at the k-th key of its
  // running list and its row merged into that list (no two rows of a sub-round
  // belong to the same point)
  bdg_knn_args a;
  a.codes = codes; a.N = N; a.m = m; a.t = t; a.k = k; a.bits = bits;
  a.tile_v = c.tile_v; a.partial = partial; a.out_ids = g->ids; a.out_dist = g->dists;
  a.out_by_pos = 0;
  a.fixflag = nullptr;
  // optional timing of the Reduce-1 step (recorded also inside a captured graph)
  if (ev0) BDG_CUDA_TRY(cudaEventRecordWithFlags(ev0, st, cudaEventRecordExternal));
  if (use_tc) BDG_CUDA_TRY(cudaMemsetAsync(fixflag, 0, al((size_t)N * t) + al(64), st));
  bool expanded = false;
  for (int round = 0; round < t; ++round) {
    a.csr = round == 0 ? bdg_csr_round_a(csr) : bdg_csr_subround(csr, round);
    a.home_kth = round == 0 ? nullptr : partial;
    a.merge_running = round == 0 ? 0 : 1;
    for (int cl = 0; cl < (split ? BDG_SIZE_CLASSES : 1); ++cl) {
      a.size_lo = split ? kBdgClassLo[cl] : 0;
      a.size_hi = split ? kBdgClassHi[cl] : 0x7fffffff;
      a.item_counter = csr.counters + (size_t)t * m + (size_t)round * BDG_SIZE_CLASSES + cl;
      cudaEvent_t* ce = cls_ev ? cls_ev + 2 * ((size_t)round * BDG_SIZE_CLASSES + cl) : nullptr;
      if (ce) BDG_CUDA_TRY(cudaEventRecord(ce[0], st));
      if (kmap[cl] == BDG_KV_TC) {
        bdg_knn_tc_args ta;
        ta.base = a; ta.hexp = hexp; ta.err = tc_err;
        ta.fixflag = fixflag + (round == 0 ? 0 : N);  // sub-round positions are absolute
        BDG_TRY(bdg_launch_knn_tc(ta, W, !expanded, st));
        expanded = true;
      } else {
        BDG_TRY(bdg_launch_knn_popc(a, W, st, kmap[cl] == BDG_KV_POPC32));
      }
      if (ce) BDG_CUDA_TRY(cudaEventRecord(ce[1], st));
    }
  }
  if (ev1) BDG_CUDA_TRY(cudaEventRecordWithFlags(ev1, st, cudaEventRecordExternal));
  if (t > 1) BDG_TRY(bdg_launch_finalize(partial, N, k, bits, g->ids, g->dists, st));
  return BDG_OK;
}

}  // namespace

extern "C" {

bdg_status bdg_build_graph(const uint64_t* codes, int64_t N, int32_t bits, int32_t k,
                           const bdg_partitions* P, void* stream, bdg_graph** out) {
  if (!out) return bdg_set_error(BDG_EINVAL, "build: out is NULL");
  *out = nullptr;
  BuildCfg c;
  BDG_TRY(build_validate(codes, N, bits, k, P, &c));
  if (!c.use_tc) {  // no expanded operand or fix-up flags needed
    c.total -= c.b_hexp + c.b_fix;
    c.b_hexp = c.b_fix = 0;
  }
  cudaStream_t st = (cudaStream_t)stream;
  keep_pool_cached();
  bdg_graph* g = nullptr;
  BDG_TRY(graph_alloc(c, codes, N, bits, k, P, &g));
  Scratch sc;
  bdg_status s = sc.alloc(c.total, st);
  if (s == BDG_OK) s = build_enqueue(c, c.kmap, g, codes, N, bits, k, P, sc.p, st);
  if (s != BDG_OK) { bdg_graph_free(g); return s; }
  *out = g;
  return BDG_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- build plans
struct bdg_build_plan {
  bdg_graph* g = nullptr;
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernel = 0;          // 1 popcount, 2 tensor (2 when any size class uses it)
  float ms_popc = -1.f, ms_tc = -1.f;
  int kmap[BDG_SIZE_CLASSES] = {0, 0, 0};  // variant per size class
  // measured Reduce-1 ms per (variant - 1, class), -1 = not measured
  float cls_ms[3][BDG_SIZE_CLASSES] = {{-1.f, -1.f, -1.f}, {-1.f, -1.f, -1.f},
                                       {-1.f, -1.f, -1.f}};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the Reduce-1 step of each replay
  int64_t launches = 0;    // kernels in the captured graph
};

namespace {

std::string tune_key(int64_t N, int32_t bits, int32_t k, const bdg_partitions* P) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  char buf[512];
  std::string name(prop.name);
  for (auto& ch : name) if (ch == ' ') ch = '_';
  snprintf(buf, sizeof(buf), "classes2|%s|bits=%d|k=%d|N=%lld|m=%d|t=%d|coarse=%lld",
           name.c_str(), bits, k, (long long)N, P->m, P->t, (long long)P->coarse_num);
  return buf;
}

std::string tune_path() {
  const char* e = getenv("BDG_AUTOTUNE_CACHE");
  if (e && *e) return e;
  const char* h = getenv("HOME");
  return std::string(h ? h : "/tmp") + "/.cache/bdg_autotune.txt";
}

// The cache holds one line per key: the variant of each size class, then the
// measured Reduce-1 ms of every (variant, class). Returns true when found.
bool tune_lookup(const std::string& key, int* kmap) {
  FILE* f = fopen(tune_path().c_str(), "r");
  if (!f) return false;
  char line[1024];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    char k2[512];
    int v[BDG_SIZE_CLASSES];
    if (sscanf(line, "%511s %d %d %d", k2, &v[0], &v[1], &v[2]) == 4 && key == k2) {
      bool ok = true;
      for (int i = 0; i < BDG_SIZE_CLASSES; ++i) ok = ok && v[i] >= 1 && v[i] <= 3;
      if (ok) {
        for (int i = 0; i < BDG_SIZE_CLASSES; ++i) kmap[i] = v[i];
        found = true;
      }
    }
  }
  fclose(f);
  return found;
}

void tune_store(const std::string& key, const int* kmap, const float (*ms)[BDG_SIZE_CLASSES]) {
  const std::string path = tune_path();
  const size_t slash = path.rfind('/');
  if (slash != std::string::npos) {
    const std::string dir = path.substr(0, slash);
    mkdir(dir.c_str(), 0755);  // the cache directory may not exist yet
  }
  FILE* f = fopen(path.c_str(), "a");
  if (!f) return;  // the cache is an optimisation only
  fprintf(f, "%s %d %d %d", key.c_str(), kmap[0], kmap[1], kmap[2]);
  for (int v = 0; v < 3; ++v)
    for (int c = 0; c < BDG_SIZE_CLASSES; ++c) fprintf(f, " %.3f", ms[v][c]);
  fprintf(f, "\n");
  fclose(f);
}

// One warm build, then one build with every size class launched on its own
// between events: per-class Reduce-1 ms (summed over rounds) into cls_ms[c],
// the whole Reduce-1 step's ms returned (-1 on failure).
float time_build(const BuildCfg& c, const int* kmap, bdg_graph* g, const uint64_t* codes,
                 int64_t N, int32_t bits, int32_t k, const bdg_partitions* P, void* scratch,
                 cudaStream_t st, float* cls_ms) {
  const int t = c.t;
  std::vector<cudaEvent_t> ev((size_t)t * BDG_SIZE_CLASSES * 2);
  for (auto& e : ev) cudaEventCreate(&e);
  float total = -1.f;
  if (build_enqueue(c, kmap, g, codes, N, bits, k, P, scratch, st) == BDG_OK &&
      build_enqueue(c, kmap, g, codes, N, bits, k, P, scratch, st, nullptr, nullptr,
                    ev.data()) == BDG_OK &&
      cudaEventSynchronize(ev.back()) == cudaSuccess) {
    total = 0.f;
    for (int cl = 0; cl < BDG_SIZE_CLASSES; ++cl) {
      float sum = 0.f;
      for (int r = 0; r < t; ++r) {
        float ms = 0.f;
        const size_t x = 2 * ((size_t)r * BDG_SIZE_CLASSES + cl);
        cudaEventElapsedTime(&ms, ev[x], ev[x + 1]);
        sum += ms;
      }
      cls_ms[cl] = sum;
      total += sum;
    }
  }
  cudaGetLastError();
  for (auto& e : ev) cudaEventDestroy(e);
  return total;
}

}  // namespace

extern "C" {

bdg_status bdg_build_plan_create(const uint64_t* codes, int64_t N, int32_t bits, int32_t k,
                                 const bdg_partitions* P, void* stream, bdg_build_plan** out) {
  if (!out) return bdg_set_error(BDG_EINVAL, "plan: out is NULL");
  *out = nullptr;
  BuildCfg c;
  BDG_TRY(build_validate(codes, N, bits, k, P, &c));
  cudaStream_t st = (cudaStream_t)stream;
  bdg_build_plan* plan = new bdg_build_plan();
  auto fail = [&](bdg_status e) { bdg_build_plan_free(plan); return e; };
  bdg_status s = graph_alloc(c, codes, N, bits, k, P, &plan->g);
  if (s != BDG_OK) return fail(s);
  plan->scratch_bytes = c.total;
  s = dalloc(&plan->scratch, c.total);
  if (s != BDG_OK) return fail(s);
  // Reduce-1 variant per partition size class: fixed by the caller (kernel or
  // class_kernel), else measured once per device and shape: every variant runs
  // every class, and each class keeps its fastest variant
  bool fixed = P->kernel != 0;
  for (int i = 0; i < BDG_SIZE_CLASSES; ++i) fixed = fixed || P->class_kernel[i] != 0;
  for (int i = 0; i < BDG_SIZE_CLASSES; ++i) plan->kmap[i] = c.kmap[i];
  if (!fixed) {
    const std::string key = tune_key(N, bits, k, P);
    if (!tune_lookup(key, plan->kmap)) {
      const int variants[3] = {BDG_KV_POPC, BDG_KV_TC, BDG_KV_POPC32};
      for (int vi = 0; vi < 3; ++vi) {
        const int v = variants[vi];
        // the plan's scratch holds the tensor path's buffers whenever it applies
        if (v == BDG_KV_TC && !(c.tc_ok && bdg_tc_default())) continue;
        int km[BDG_SIZE_CLASSES] = {v, v, v};
        const float ms = time_build(c, km, plan->g, codes, N, bits, k, P, plan->scratch, st,
                                    plan->cls_ms[v - 1]);
        if (v == BDG_KV_POPC) plan->ms_popc = ms;
        if (v == BDG_KV_TC) plan->ms_tc = ms;
      }
      for (int cl = 0; cl < BDG_SIZE_CLASSES; ++cl) {
        int best = 0;
        for (int vi = 0; vi < 3; ++vi) {
          const float ms = plan->cls_ms[variants[vi] - 1][cl];
          if (ms < 0.f) continue;
          if (best == 0 || ms < plan->cls_ms[best - 1][cl]) best = variants[vi];
        }
        plan->kmap[cl] = best ? best : c.kmap[cl];
      }
      tune_store(key, plan->kmap, plan->cls_ms);
    }
  }
  plan->kernel = BDG_KV_POPC;
  for (int i = 0; i < BDG_SIZE_CLASSES; ++i)
    if (plan->kmap[i] == BDG_KV_TC) plan->kernel = BDG_KV_TC;
  // warm once outside capture (lazy module loading, function attributes), then capture
  s = build_enqueue(c, plan->kmap, plan->g, codes, N, bits, k, P, plan->scratch, st);
  if (s != BDG_OK) return fail(s);
  if (cudaStreamSynchronize(st) != cudaSuccess)
    return fail(bdg_set_error(BDG_ECUDA, "plan: warm-up build failed"));
  cudaStream_t cap;
  if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&plan->ev0) != cudaSuccess || cudaEventCreate(&plan->ev1) != cudaSuccess)
    return fail(bdg_set_error(BDG_ECUDA, "plan: stream or event creation failed"));
  const int64_t l0 = g_launches.load();
  bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) == cudaSuccess;
  const bdg_status se =
      ok ? build_enqueue(c, plan->kmap, plan->g, codes, N, bits, k, P, plan->scratch, cap,
                         plan->ev0, plan->ev1)
         : BDG_OK;
  plan->launches = g_launches.load() - l0;
  ok = (cudaStreamEndCapture(cap, &plan->graph) == cudaSuccess) && ok && se == BDG_OK;
  ok = ok && cudaGraphInstantiate(&plan->exec, plan->graph, 0) == cudaSuccess;
  cudaStreamDestroy(cap);
  if (!ok) {
    cudaGetLastError();
    return fail(se != BDG_OK ? se : bdg_set_error(BDG_ECUDA, "plan: graph capture failed"));
  }
  *out = plan;
  return BDG_OK;
}

bdg_status bdg_build_plan_run(bdg_build_plan* plan, void* stream) {
  if (!plan || !plan->exec) return bdg_set_error(BDG_EINVAL, "plan: not instantiated");
  BDG_CUDA_TRY(cudaGraphLaunch(plan->exec, (cudaStream_t)stream));
  bdg_note_launch((int)plan->launches);
  return BDG_OK;
}

bdg_status bdg_build_plan_run_host(bdg_build_plan* plan, const uint64_t* host_codes,
                                   int32_t* host_ids, int32_t* host_dists, void* stream) {
  if (!plan || !plan->exec) return bdg_set_error(BDG_EINVAL, "plan: not instantiated");
  if (!host_codes || !host_ids)
    return bdg_set_error(BDG_EINVAL, "plan_run_host: host codes and ids are required");
  cudaStream_t st = (cudaStream_t)stream;
  const bdg_graph* g = plan->g;
  const size_t code_bytes = (size_t)g->n * g->W * 8, row_bytes = (size_t)g->n * g->k * 4;
  BDG_CUDA_TRY(cudaMemcpyAsync(const_cast<uint64_t*>(g->codes), host_codes, code_bytes,
                               cudaMemcpyHostToDevice, st));
  BDG_CUDA_TRY(cudaGraphLaunch(plan->exec, st));
  bdg_note_launch((int)plan->launches);
  BDG_CUDA_TRY(cudaMemcpyAsync(host_ids, g->ids, row_bytes, cudaMemcpyDeviceToHost, st));
  if (host_dists)
    BDG_CUDA_TRY(cudaMemcpyAsync(host_dists, g->dists, row_bytes, cudaMemcpyDeviceToHost, st));
  return BDG_OK;
}

bdg_status bdg_build_plan_kernel_ms(bdg_build_plan* plan, float* ms) {
  if (!plan || !ms) return bdg_set_error(BDG_EINVAL, "plan: null argument");
  BDG_CUDA_TRY(cudaEventSynchronize(plan->ev1));
  BDG_CUDA_TRY(cudaEventElapsedTime(ms, plan->ev0, plan->ev1));
  return BDG_OK;
}

bdg_status bdg_build_plan_info(const bdg_build_plan* plan, const bdg_graph** graph,
                               int32_t* kernel, float* ms_popc, float* ms_tc) {
  if (!plan) return bdg_set_error(BDG_EINVAL, "plan is NULL");
  if (graph) *graph = plan->g;
  if (kernel) *kernel = plan->kernel;
  if (ms_popc) *ms_popc = plan->ms_popc;
  if (ms_tc) *ms_tc = plan->ms_tc;
  return BDG_OK;
}

bdg_status bdg_build_plan_classes(const bdg_build_plan* plan, int32_t* variant, int32_t* size_lo,
                                  int32_t* size_hi, float* ms) {
  if (!plan) return bdg_set_error(BDG_EINVAL, "plan is NULL");
  for (int c = 0; c < BDG_SIZE_CLASSES; ++c) {
    if (variant) variant[c] = plan->kmap[c];
    if (size_lo) size_lo[c] = kBdgClassLo[c];
    if (size_hi) size_hi[c] = kBdgClassHi[c];
    for (int v = 0; v < 3; ++v)
      if (ms) ms[v * BDG_SIZE_CLASSES + c] = plan->cls_ms[v][c];
  }
  return BDG_OK;
}

void bdg_build_plan_free(bdg_build_plan* plan) {
  if (!plan) return;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->ev0) cudaEventDestroy(plan->ev0);
  if (plan->ev1) cudaEventDestroy(plan->ev1);
  dfree(plan->scratch, plan->scratch_bytes);
  bdg_graph_free(plan->g);
  delete plan;
}

bdg_status bdg_knn_rows(const uint64_t* codes, int64_t N, int32_t bits, const int32_t* rows,
                        int64_t nrows, int32_t k, int32_t* out_ids, int32_t* out_dist,
                        void* stream) {
  BDG_TRY(check_bits(bits));
  if (N < 2 || N >= (int64_t(1) << 31) || k < 1 || k > 128 || k >= N || nrows < 0 ||
      nrows >= (int64_t(1) << 31))
    return bdg_set_error(BDG_EINVAL, "knn_rows: N=%lld nrows=%lld k=%d", (long long)N,
                         (long long)nrows, k);
  if (nrows == 0) return BDG_OK;
  if (!codes || !rows || !out_ids || !out_dist)
    return bdg_set_error(BDG_EINVAL, "knn_rows: null pointer");
  cudaStream_t st = (cudaStream_t)stream;
  const int W = bits / 64;
  const int tile_v = bdg_knn_tile_visitors(W);
  keep_pool_cached();
  const bool use_tc = bdg_knn_tc_supported(W, k) && N < (1 << 21) && bdg_tc_default();
  Scratch sc;
  const size_t b = al(bdg_csr_rows_bytes(N, nrows, tile_v));
  const size_t b_hexp = use_tc ? al(bdg_knn_tc_hexp_bytes(N, 1, W)) : 0;
  const size_t b_fix = use_tc ? al((size_t)nrows) + al(64) : 0;
  BDG_TRY(sc.alloc(b + b_hexp + b_fix, st));
  bdg_csr csr;
  BDG_TRY(bdg_build_csr_rows(codes, N, rows, nrows, tile_v, sc.p, &csr, st));
  bdg_knn_args a;
  a.codes = codes; a.csr = csr; a.N = N; a.m = 1; a.t = 1; a.k = k; a.bits = bits;
  a.tile_v = tile_v; a.partial = nullptr; a.out_ids = out_ids; a.out_dist = out_dist;
  a.item_counter = csr.counters + 2;
  a.out_by_pos = 1;
  a.fixflag = nullptr;
  a.home_kth = nullptr;
  a.merge_running = 0;
  if (!use_tc) return bdg_launch_knn_popc(a, W, st);
  char* q = (char*)sc.p + b;
  bdg_knn_tc_args ta;
  ta.base = a;
  ta.hexp = (uint8_t*)q;
  ta.fixflag = (int8_t*)(q + b_hexp);
  ta.err = (int32_t*)(q + b_hexp + al((size_t)nrows));
  BDG_CUDA_TRY(cudaMemsetAsync(ta.fixflag, 0, b_fix, st));
  return bdg_launch_knn_tc(ta, W, true, st);
}

bdg_status bdg_graph_info(const bdg_graph* g, const int32_t** ids, const int32_t** dists,
                          int64_t* n, int32_t* k, int32_t* bits) {
  if (!g) return bdg_set_error(BDG_EINVAL, "graph is NULL");
  if (ids) *ids = g->ids;
  if (dists) *dists = g->dists;
  if (n) *n = g->n;
  if (k) *k = g->k;
  if (bits) *bits = g->bits;
  return BDG_OK;
}

void bdg_graph_free(bdg_graph* g) {
  if (!g) return;
  dfree(g->ids, (size_t)g->n * g->k * 4);
  dfree(g->dists, (size_t)g->n * g->k * 4);
  dfree(g->entry, (size_t)g->n_entry * 4);
  dfree(g->entry_codes, (size_t)g->n_entry * g->W * 8);
  if (g->nbr_codes) dfree(g->nbr_codes, (size_t)g->n * g->k * g->W * 8);
  delete g;
}

bdg_status bdg_graph_save(const bdg_graph* g, const char* path) {
  if (!g || !path) return bdg_set_error(BDG_EINVAL, "save: null argument");
  BDG_CUDA_TRY(cudaDeviceSynchronize());
  std::vector<int32_t> ids((size_t)g->n * g->k), dists((size_t)g->n * g->k), entry(g->n_entry);
  BDG_CUDA_TRY(cudaMemcpy(ids.data(), g->ids, ids.size() * 4, cudaMemcpyDeviceToHost));
  BDG_CUDA_TRY(cudaMemcpy(dists.data(), g->dists, dists.size() * 4, cudaMemcpyDeviceToHost));
  BDG_CUDA_TRY(cudaMemcpy(entry.data(), g->entry, entry.size() * 4, cudaMemcpyDeviceToHost));
  FILE* f = fopen(path, "wb");
  if (!f) return bdg_set_error(BDG_EINVAL, "save: cannot open %s", path);
  const int32_t hdr[6] = {0x31474442 /* "BDG1" */, 1, (int32_t)(g->n & 0x7fffffff), g->bits, g->k,
                          g->n_entry};
  bool ok = fwrite(hdr, 4, 6, f) == 6 && fwrite(ids.data(), 4, ids.size(), f) == ids.size() &&
            fwrite(dists.data(), 4, dists.size(), f) == dists.size() &&
            fwrite(entry.data(), 4, entry.size(), f) == entry.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? BDG_OK : bdg_set_error(BDG_EINVAL, "save: write to %s failed", path);
}

bdg_status bdg_graph_propagate(const bdg_graph* g, int32_t rounds, void* stream,
                               bdg_graph** out) {
  if (!out) return bdg_set_error(BDG_EINVAL, "propagate: out is NULL");
  *out = nullptr;
  if (!g || rounds < 1)
    return bdg_set_error(BDG_EINVAL, "propagate: graph %p, rounds = %d (>= 1)", (const void*)g,
                         rounds);
  if (g->k > bdg_propagate_max_k())
    return bdg_set_error(BDG_EUNSUPPORTED, "propagate: k = %d (at most %d)", g->k,
                         bdg_propagate_max_k());
  cudaStream_t st = (cudaStream_t)stream;
  keep_pool_cached();
  bdg_graph* h = new bdg_graph();
  h->n = g->n; h->k = g->k; h->bits = g->bits; h->W = g->W; h->n_entry = g->n_entry;
  h->codes = g->codes;
  const size_t rows = (size_t)g->n * g->k * 4;
  bdg_status s = dalloc((void**)&h->ids, rows);
  if (s == BDG_OK) s = dalloc((void**)&h->dists, rows);
  if (s == BDG_OK) s = dalloc((void**)&h->entry, (size_t)g->n_entry * 4);
  if (s == BDG_OK) s = dalloc((void**)&h->entry_codes, (size_t)g->n_entry * g->W * 8);
  if (s != BDG_OK) { bdg_graph_free(h); return s; }
  // rounds alternate between the output rows and one scratch pair, ending in the output
  Scratch sc;
  if (rounds > 1) s = sc.alloc(2 * rows, st);
  if (s != BDG_OK) { bdg_graph_free(h); return s; }
  int32_t* ping_ids = rounds > 1 ? (int32_t*)sc.p : nullptr;
  int32_t* ping_d = rounds > 1 ? (int32_t*)((char*)sc.p + rows) : nullptr;
  Scratch so;  // processing order of the points
  int32_t* perm = nullptr;
  s = so.alloc(bdg_propagate_order_bytes(g->n), st);
  if (s == BDG_OK) s = bdg_launch_propagate_order(g->codes, g->n, g->W, so.p, &perm, st);
  if (s != BDG_OK) { bdg_graph_free(h); return s; }
  const int32_t* in_ids = g->ids;
  const int32_t* in_d = g->dists;
  for (int r = 0; r < rounds; ++r) {
    // the last round writes the output, the one before it the scratch pair, and so on
    const bool to_out = ((rounds - 1 - r) & 1) == 0;
    int32_t* o_ids = to_out ? h->ids : ping_ids;
    int32_t* o_d = to_out ? h->dists : ping_d;
    s = bdg_launch_propagate(g->codes, g->n, g->W, g->k, perm, in_ids, in_d, o_ids, o_d, st);
    if (s != BDG_OK) { bdg_graph_free(h); return s; }
    in_ids = o_ids;
    in_d = o_d;
  }
  if (cudaMemcpyAsync(h->entry, g->entry, (size_t)g->n_entry * 4, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(h->entry_codes, g->entry_codes, (size_t)g->n_entry * g->W * 8,
                      cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    bdg_graph_free(h);
    return bdg_set_error(BDG_ECUDA, "propagate: entry copy failed");
  }
  *out = h;
  return BDG_OK;
}

bdg_status bdg_graph_prune(const bdg_graph* g, int32_t L, void* stream, bdg_graph** out) {
  if (!out) return bdg_set_error(BDG_EINVAL, "prune: out is NULL");
  *out = nullptr;
  if (!g) return bdg_set_error(BDG_EINVAL, "prune: graph is NULL");
  if (g->k > bdg_prune_max_k())
    return bdg_set_error(BDG_EUNSUPPORTED, "prune: k = %d (at most %d)", g->k,
                         bdg_prune_max_k());
  if (L < 1 || L > g->k || L > bdg_prune_max_l())
    return bdg_set_error(BDG_EINVAL, "prune: L = %d (need 1 <= L <= min(k = %d, %d))", L, g->k,
                         bdg_prune_max_l());
  cudaStream_t st = (cudaStream_t)stream;
  keep_pool_cached();
  bdg_graph* h = new bdg_graph();
  h->n = g->n; h->k = L; h->bits = g->bits; h->W = g->W; h->n_entry = g->n_entry;
  h->codes = g->codes;
  const size_t rows = (size_t)g->n * L * 4;
  bdg_status s = dalloc((void**)&h->ids, rows);
  if (s == BDG_OK) s = dalloc((void**)&h->dists, rows);
  if (s == BDG_OK) s = dalloc((void**)&h->entry, (size_t)g->n_entry * 4);
  if (s == BDG_OK) s = dalloc((void**)&h->entry_codes, (size_t)g->n_entry * g->W * 8);
  if (s == BDG_OK)
    s = bdg_launch_prune(g->codes, g->n, g->W, g->k, L, g->ids, h->ids, h->dists, st);
  if (s != BDG_OK) { bdg_graph_free(h); return s; }
  if (cudaMemcpyAsync(h->entry, g->entry, (size_t)g->n_entry * 4, cudaMemcpyDeviceToDevice, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(h->entry_codes, g->entry_codes, (size_t)g->n_entry * g->W * 8,
                      cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    bdg_graph_free(h);
    return bdg_set_error(BDG_ECUDA, "prune: entry copy failed");
  }
  *out = h;
  return BDG_OK;
}

bdg_status bdg_graph_pack_codes(bdg_graph* g, void* stream) {
  if (!g) return bdg_set_error(BDG_EINVAL, "pack_codes: graph is NULL");
  if (g->nbr_codes) return BDG_OK;  // already packed
  const size_t bytes = (size_t)g->n * g->k * g->W * 8;
  BDG_TRY(dalloc((void**)&g->nbr_codes, bytes));
  const bdg_status s = bdg_launch_gather_codes(g->codes, g->n, g->ids, g->n * (int64_t)g->k, g->W,
                                               g->nbr_codes, (cudaStream_t)stream);
  if (s != BDG_OK) {
    dfree(g->nbr_codes, bytes);
    g->nbr_codes = nullptr;
  }
  return s;
}

bdg_status bdg_graph_load(const char* path, const uint64_t* codes, bdg_graph** out) {
  if (!path || !codes || !out) return bdg_set_error(BDG_EINVAL, "load: null argument");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return bdg_set_error(BDG_EINVAL, "load: cannot open %s", path);
  int32_t hdr[6];
  if (fread(hdr, 4, 6, f) != 6 || hdr[0] != 0x31474442 || hdr[1] != 1 || hdr[2] < 2 ||
      hdr[4] < 1 || hdr[5] < 1 || check_bits(hdr[3]) != BDG_OK) {
    fclose(f);
    return bdg_set_error(BDG_EINVAL, "load: %s is not a BDG1 graph file", path);
  }
  bdg_graph* g = new bdg_graph();
  g->n = hdr[2]; g->bits = hdr[3]; g->W = hdr[3] / 64; g->k = hdr[4]; g->n_entry = hdr[5];
  g->codes = codes;
  std::vector<int32_t> ids((size_t)g->n * g->k), dists((size_t)g->n * g->k), entry(g->n_entry);
  const bool ok = fread(ids.data(), 4, ids.size(), f) == ids.size() &&
                  fread(dists.data(), 4, dists.size(), f) == dists.size() &&
                  fread(entry.data(), 4, entry.size(), f) == entry.size();
  fclose(f);
  if (!ok) { delete g; return bdg_set_error(BDG_EINVAL, "load: %s is truncated", path); }
  bdg_status s = dalloc((void**)&g->ids, ids.size() * 4);
  if (s == BDG_OK) s = dalloc((void**)&g->dists, dists.size() * 4);
  if (s == BDG_OK) s = dalloc((void**)&g->entry, entry.size() * 4);
  if (s == BDG_OK) s = dalloc((void**)&g->entry_codes, entry.size() * g->W * 8);
  if (s != BDG_OK) { bdg_graph_free(g); return s; }
  if (cudaMemcpy(g->ids, ids.data(), ids.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(g->dists, dists.data(), dists.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(g->entry, entry.data(), entry.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    bdg_graph_free(g);
    return bdg_set_error(BDG_ECUDA, "load: copy to device failed");
  }
  s = bdg_launch_gather_codes(codes, g->n, g->entry, g->n_entry, g->W, g->entry_codes, nullptr);
  if (s == BDG_OK && cudaDeviceSynchronize() != cudaSuccess)
    s = bdg_set_error(BDG_ECUDA, "load: gathering the entry codes failed");
  if (s != BDG_OK) { bdg_graph_free(g); return s; }
  *out = g;
  return BDG_OK;
}

bdg_status bdg_search(const bdg_graph* g, const uint64_t* queries, int64_t nq, const int32_t* ef,
                      int32_t ef_max, int32_t R, int32_t* out_ids, int32_t* out_dist,
                      int32_t* expansions, void* stream) {
  if (!g) return bdg_set_error(BDG_EINVAL, "search: graph is NULL");
  if (nq < 0 || R < 1 || ef_max < 1 || ef_max > 2048)
    return bdg_set_error(BDG_EINVAL, "search: nq=%lld R=%d ef_max=%d", (long long)nq, R, ef_max);
  if (nq > 0 && (!queries || !ef || !out_ids || !out_dist))
    return bdg_set_error(BDG_EINVAL, "search: null pointer");
  bdg_graph_view v{g->codes, g->ids, g->entry, g->entry_codes, g->n, g->k, g->bits, g->n_entry};
  v.nbr_codes = g->nbr_codes;
  return bdg_launch_search(v, queries, nq, ef, ef_max, R, out_ids, out_dist, expansions,
                           (cudaStream_t)stream);
}

bdg_status bdg_build_sharded(const uint64_t* codes, int64_t N, int32_t bits, int32_t k,
                             const bdg_partitions* P, int32_t S, void* stream, bdg_graph** out) {
  if (!out || !P || !codes) return bdg_set_error(BDG_EINVAL, "build_sharded: null argument");
  if (S < 1 || S > BDG_MAX_SHARDS)
    return bdg_set_error(BDG_EINVAL, "build_sharded: S = %d (1 .. %d)", S, BDG_MAX_SHARDS);
  for (int s = 0; s < S; ++s) out[s] = nullptr;
  BDG_TRY(check_bits(bits));
  if (N < 2 || N >= (int64_t(1) << 31))
    return bdg_set_error(BDG_EINVAL, "build_sharded: N = %lld", (long long)N);
  if (!P->entry || P->n_entry < 1)
    return bdg_set_error(BDG_EINVAL, "build_sharded: an entry sample per shard is required");
  const int W = bits / 64;
  for (int s = 0; s < S; ++s) {
    const int64_t ns = (int64_t)(s + 1) * N / S - (int64_t)s * N / S;
    if (k >= ns)
      return bdg_set_error(BDG_EINVAL, "build_sharded: shard %d holds %lld points (k = %d)", s,
                           (long long)ns, k);
  }
  cudaStream_t st = (cudaStream_t)stream;
  keep_pool_cached();
  // the centres, once, over the whole data
  Scratch sc;
  const uint64_t* cent = P->centroids;
  if (P->m > 1 && !cent && !P->routes) {
    if (!P->bk_sample || P->bk_sample_size < P->m || P->bk_iters < 0)
      return bdg_set_error(BDG_EINVAL, "build_sharded: Bk-means needs bk_sample with >= m ids");
    BDG_TRY(sc.alloc(al((size_t)P->m * W * 8), st));
    BDG_TRY(bdg_bkmeans(codes, N, bits, P->bk_sample, P->bk_sample_size, P->m, P->bk_iters,
                        (uint64_t*)sc.p, nullptr, stream));
    cent = (const uint64_t*)sc.p;
  }
  for (int s = 0; s < S; ++s) {
    const int64_t o = (int64_t)s * N / S, ns = (int64_t)(s + 1) * N / S - o;
    bdg_partitions Ps = *P;
    Ps.centroids = cent;
    Ps.entry = P->entry + (size_t)s * P->n_entry;
    Ps.routes = P->routes ? P->routes + (size_t)o * P->t : nullptr;
    const bdg_status r = bdg_build_graph(codes + (size_t)o * W, ns, bits, k, &Ps, stream, &out[s]);
    if (r != BDG_OK) {
      for (int u = 0; u <= s; ++u) {
        if (out[u]) bdg_graph_free(out[u]);
        out[u] = nullptr;
      }
      return r;
    }
  }
  return BDG_OK;
}

bdg_status bdg_search_sharded(const bdg_graph* const* shards, int32_t S, const uint64_t* queries,
                              int64_t nq, const int32_t* ef, int32_t ef_max, int32_t R,
                              int32_t* out_ids, int32_t* out_dist, void* stream) {
  if (!shards || S < 1 || S > BDG_MAX_SHARDS || R < 1 || S * R > 6144)
    return bdg_set_error(BDG_EINVAL, "search_sharded: S = %d, R = %d (1 <= S <= %d, S R <= 6144)",
                         S, R, BDG_MAX_SHARDS);
  if (nq < 0 || ef_max < 1 || ef_max > 1024)
    return bdg_set_error(BDG_EINVAL, "search_sharded: nq=%lld ef_max=%d", (long long)nq, ef_max);
  if (nq > 0 && (!queries || !ef || !out_ids || !out_dist))
    return bdg_set_error(BDG_EINVAL, "search_sharded: null pointer");
  bdg_shard_offsets off{};
  int64_t o = 0;
  for (int s = 0; s < S; ++s) {
    if (!shards[s]) return bdg_set_error(BDG_EINVAL, "search_sharded: shard %d is NULL", s);
    if (shards[s]->bits != shards[0]->bits)
      return bdg_set_error(BDG_EINVAL, "search_sharded: shards of different code widths");
    off.off[s] = o;
    o += shards[s]->n;
  }
  if (o >= (int64_t(1) << 31))
    return bdg_set_error(BDG_EINVAL, "search_sharded: %lld points in all (< 2^31)", (long long)o);
  if (nq == 0) return BDG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  keep_pool_cached();
  const size_t part = (size_t)nq * R * 4;
  Scratch sc;
  BDG_TRY(sc.alloc(2 * al(part * S), st));
  int32_t* ids = (int32_t*)sc.p;
  int32_t* dist = (int32_t*)((char*)sc.p + al(part * S));
  for (int s = 0; s < S; ++s) {
    const bdg_graph* g = shards[s];
    bdg_graph_view v{g->codes, g->ids, g->entry, g->entry_codes, g->n, g->k, g->bits, g->n_entry};
    v.nbr_codes = g->nbr_codes;
    BDG_TRY(bdg_launch_search(v, queries, nq, ef, ef_max, R, ids + (size_t)s * nq * R,
                              dist + (size_t)s * nq * R, nullptr, st));
  }
  return bdg_launch_shard_merge(ids, dist, S, nq, R, off, ef, ef_max, shards[0]->bits, out_ids,
                                out_dist, st);
}

bdg_status bdg_merge_lists(const int32_t* ids, const int32_t* dists, int32_t S, int64_t n,
                           int32_t k, int32_t bits, int32_t* out_ids, int32_t* out_dists,
                           void* stream) {
  if (S < 1 || S > BDG_MAX_SHARDS || k < 1 || S * k > 6144 || n < 0 || bits < 64 || bits > 1024)
    return bdg_set_error(BDG_EINVAL, "merge_lists: S = %d, k = %d, n = %lld, bits = %d "
                         "(1 <= S <= %d, S k <= 6144)", S, k, (long long)n, bits,
                         BDG_MAX_SHARDS);
  if (n > 0 && (!ids || !dists || !out_ids || !out_dists))
    return bdg_set_error(BDG_EINVAL, "merge_lists: null pointer");
  bdg_shard_offsets off{};
  return bdg_launch_shard_merge(ids, dists, S, n, k, off, nullptr, 0, bits, out_ids, out_dists,
                                (cudaStream_t)stream);
}

bdg_status bdg_rerank(const float* feats, int64_t N, int32_t D, const float* qfeats,
                      const int32_t* cand, int64_t nq, int32_t R, int32_t k, int32_t* out_ids,
                      float* out_d2, void* stream) {
  if (nq < 0 || N < 1 || R < 1 || R > 2048 || k < 1 || k > 32)
    return bdg_set_error(BDG_EINVAL, "rerank: N=%lld nq=%lld R=%d k=%d", (long long)N,
                         (long long)nq, R, k);
  if (D != 128 && D != 256 && D != 512 && D != 1024)
    return bdg_set_error(BDG_EUNSUPPORTED, "rerank: D = %d not in {128,256,512,1024}", D);
  if (nq > 0 && (!feats || !qfeats || !cand || !out_ids || !out_d2))
    return bdg_set_error(BDG_EINVAL, "rerank: null pointer");
  if (((uintptr_t)feats | (uintptr_t)qfeats) & 15)
    return bdg_set_error(BDG_EINVAL, "rerank: feature arrays must be 16-byte aligned");
  return bdg_launch_rerank(feats, N, D, qfeats, cand, nq, R, k, out_ids, out_d2,
                           (cudaStream_t)stream);
}

bdg_status bdg_search_rerank(const bdg_graph* g, const uint64_t* queries, const float* qfeats,
                             const float* feats, int32_t D, int64_t nq, const int32_t* ef,
                             int32_t ef_max, int32_t R, int32_t k, int32_t* cand_ids,
                             int32_t* cand_dist, int32_t* out_ids, float* out_d2, void* stream) {
  BDG_TRY(bdg_search(g, queries, nq, ef, ef_max, R, cand_ids, cand_dist, nullptr, stream));
  return bdg_rerank(feats, g->n, D, qfeats, cand_ids, nq, R, k, out_ids, out_d2, stream);
}

}  // extern "C"
