// route.cu -- nearest-centre routing (Map step, Section 3.2) and Bk-means
// (Section 3.2, Eq. 1-2) on packed binary codes.
//
// Routing on the ALU (the tensor-core paths for 256/512-bit codes are in
// route_small.cu, up to 256 centres, and below, from 1,024 centres): one thread
// per point keeps its t best (distance, centre) keys in registers while centre
// codes stream through shared memory in chunks (every thread of the block reads
// the same centre word, a broadcast). The work is n * m * W XOR+POPC word pairs,
// ALU (POPC) bound.
//
// Bk-means: assign = routing with t = 1 over the down-sample (route_small.cu
// where it applies); update = per-bit
// member counts by integer atomics (order-independent, so deterministic) and a
// per-word majority with "tie keeps the previous bit" (the reading of Eq. 2's
// sgn at zero); the objective of Eq. 1 (Hamming = squared L2 for 0/1 vectors)
// is summed after each assign.
#include "common.cuh"

namespace {

constexpr int kRouteThreads = 256;

template <int W, int MAXT>
__global__ void __launch_bounds__(kRouteThreads)
route_kernel(const uint64_t* __restrict__ codes, int64_t n, const uint64_t* __restrict__ cent,
             int m, int t, int32_t* __restrict__ routes, int32_t* __restrict__ rdist,
             unsigned long long* __restrict__ loss_sum) {
  constexpr int kChunk = (W <= 4) ? 1024 : 4096 / W;  // centres per smem chunk
  __shared__ uint64_t sc[kChunk * W];
  const int64_t i = (int64_t)blockIdx.x * kRouteThreads + threadIdx.x;
  const bool live = i < n;
  uint64_t y[W];
#pragma unroll
  for (int w = 0; w < W; ++w) y[w] = live ? codes[i * W + w] : 0ull;
  uint64_t best[MAXT];
#pragma unroll
  for (int s = 0; s < MAXT; ++s) best[s] = BDG_KEY_INF;
  uint64_t worst = BDG_KEY_INF;  // == best[t - 1]

  for (int c0 = 0; c0 < m; c0 += kChunk) {
    const int cn = min(kChunk, m - c0);
    __syncthreads();
    for (int x = threadIdx.x; x < cn * W; x += kRouteThreads) sc[x] = cent[(int64_t)c0 * W + x];
    __syncthreads();
    for (int c = 0; c < cn; ++c) {
      uint32_t d = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) d += __popcll(y[w] ^ sc[c * W + w]);
      const uint64_t key = bdg_key(d, (uint32_t)(c0 + c));
      if (key < worst) {
        // sorted insertion from the back: slot s takes its predecessor if the
        // key goes further forward, else the key itself; slots >= t are unused
#pragma unroll
        for (int s = MAXT - 1; s >= 0; --s) {
          if (s < t && key < best[s]) {
            const uint64_t prev = (s > 0) ? best[s - 1] : 0ull;
            best[s] = (s > 0 && key < prev) ? prev : key;
          }
        }
#pragma unroll
        for (int s = 0; s < MAXT; ++s)
          if (s == t - 1) worst = best[s];
      }
    }
  }
  if (loss_sum) {
    // objective of Eq. 1 for the nearest centre, one atomic per warp
    unsigned long long v = live ? (unsigned long long)bdg_key_d(best[0]) : 0ull;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss_sum, v);
  }
  if (!live) return;
#pragma unroll
  for (int s = 0; s < MAXT; ++s) {
    if (s < t) {
      routes[i * t + s] = bdg_key_id(best[s]);
      if (rdist) rdist[i * t + s] = bdg_key_d(best[s]);
    }
  }
}

template <int W>
bdg_status route_w(const uint64_t* codes, int64_t n, const uint64_t* cent, int m, int t,
                   int32_t* routes, int32_t* rdist, unsigned long long* loss, cudaStream_t st,
                   const char* prof_name = "route") {
  if (n == 0) return BDG_OK;
  const int grid = bdg_cdiv(n, kRouteThreads);
  bdg_prof_scope prof(prof_name, st);
  if (t == 1)
    route_kernel<W, 1><<<grid, kRouteThreads, 0, st>>>(codes, n, cent, m, t, routes, rdist, loss);
  else if (t <= 4)
    route_kernel<W, 4><<<grid, kRouteThreads, 0, st>>>(codes, n, cent, m, t, routes, rdist, loss);
  else if (t <= 8)
    route_kernel<W, 8><<<grid, kRouteThreads, 0, st>>>(codes, n, cent, m, t, routes, rdist, loss);
  else
    route_kernel<W, 16><<<grid, kRouteThreads, 0, st>>>(codes, n, cent, m, t, routes, rdist, loss);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

// Sample codes codes[ids[s]]; an id outside [0, N) reads as the all-zero code
// (the argument check cannot see device-side ids, so the kernel never reads
// outside the codes).
__global__ void gather_rows(const uint64_t* __restrict__ codes, int64_t N,
                            const int64_t* __restrict__ ids, int64_t S, int W,
                            uint64_t* __restrict__ out) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= S * W) return;
  const int64_t s = x / W;
  const int64_t id = ids[s];
  out[x] = (id >= 0 && id < N) ? codes[id * W + (x - s * W)] : 0ull;
}

// Per-bit member counts: one warp per sample point, lanes over bits.
__global__ void bk_count(const uint64_t* __restrict__ scodes, int64_t S, int W,
                         const int32_t* __restrict__ assign, int32_t* __restrict__ ones,
                         int32_t* __restrict__ count) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= S) return;
  const int c = assign[s];
  const int bits = 64 * W;
  for (int b = lane; b < bits; b += 32) {
    if ((scodes[s * W + (b >> 6)] >> (b & 63)) & 1ull) atomicAdd(&ones[(int64_t)c * bits + b], 1);
  }
  if (lane == 0) atomicAdd(&count[c], 1);
}

// Majority per centre word; a tie keeps the previous bit, an empty cluster keeps its centre.
__global__ void bk_update(uint64_t* __restrict__ cent, int m, int W,
                          const int32_t* __restrict__ ones, const int32_t* __restrict__ count) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (int64_t)m * W) return;
  const int c = (int)(x / W), w = (int)(x - (int64_t)c * W);
  const int p = count[c];
  if (p == 0) return;
  const int bits = 64 * W;
  uint64_t v = cent[x];
  for (int j = 0; j < 64; ++j) {
    const int twice = 2 * ones[(int64_t)c * bits + w * 64 + j];
    const uint64_t mask = 1ull << j;
    if (twice > p) v |= mask;
    else if (twice < p) v &= ~mask;
  }
  cent[x] = v;
}

// ---- coarse_num (Section 3.2): a point keeps its home and further nearest
// centres only while the centres kept so far hold fewer than coarse_num points.
// Pass 1 counts the homes |H_p| (block-local shared-memory histogram when m
// fits, flushed with one global atomic per non-empty bin); pass 2 trims each
// row in place, one thread per point (the row is read whole before any write).
constexpr int kHistThreads = 512;
constexpr int kHistSmemBins = 12288;  // 48 KB of int32 bins

__global__ void __launch_bounds__(kHistThreads)
home_hist_kernel(const int32_t* __restrict__ routes, int64_t n, int t, int m,
                 int32_t* __restrict__ cnt) {
  extern __shared__ int32_t hb[];
  const bool local = m <= kHistSmemBins;
  if (local)
    for (int p = threadIdx.x; p < m; p += kHistThreads) hb[p] = 0;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * kHistThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kHistThreads) {
    const int32_t h = routes[i * t];
    if (h >= 0 && h < m) atomicAdd(local ? &hb[h] : &cnt[h], 1);
  }
  if (!local) return;
  __syncthreads();
  for (int p = threadIdx.x; p < m; p += kHistThreads)
    if (hb[p] != 0) atomicAdd(&cnt[p], hb[p]);
}

template <int MAXT>
__global__ void coarse_trim_kernel(int32_t* __restrict__ routes, int64_t n, int t, int m,
                                   int64_t coarse, const int32_t* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t r[MAXT];
#pragma unroll
  for (int s = 0; s < MAXT; ++s) r[s] = s < t ? routes[i * t + s] : -1;
  int64_t held = 0;
#pragma unroll
  for (int s = 0; s < MAXT; ++s) {
    if (s >= t) break;
    const bool keep = s == 0 || held < coarse;
    if (keep && r[s] >= 0 && r[s] < m) held += cnt[r[s]];
    if (!keep) routes[i * t + s] = -1;
  }
}

// Distance-gap rule: slot s >= 1 stays only if its centre is at most delta
// farther from the point than the home's centre.
__global__ void gap_trim_kernel(int32_t* __restrict__ routes, const int32_t* __restrict__ rdist,
                                int64_t n, int t, int delta) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n * t) return;
  const int64_t i = x / t;
  const int s = (int)(x - i * t);
  if (s > 0 && rdist[x] - rdist[i * t] > delta) routes[x] = -1;
}

}  // namespace

bdg_status bdg_launch_routes_gap(int32_t* routes, const int32_t* rdist, int64_t n, int t,
                                 int delta, cudaStream_t st) {
  if (n == 0) return BDG_OK;
  gap_trim_kernel<<<bdg_cdiv(n * t, 256), 256, 0, st>>>(routes, rdist, n, t, delta);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

bdg_status bdg_launch_route(const uint64_t* codes, int64_t n, int W, const uint64_t* cent, int m,
                            int t, int32_t* routes, int32_t* rdist, cudaStream_t st) {
  BDG_DISPATCH_W(W, route_w, codes, n, cent, m, t, routes, rdist, nullptr, st);
}

// ---- routing on the tensor cores. The t nearest centres of a point are its t
// nearest "homes" in one partition whose homes are the m centres: the Reduce-1
// tile of knn_tc.cu (FP8 +-1 MMA, fused (d, id) top-k) with the points as
// visitors, k = t and no self pair. Centre index order is the home position
// order, so ties fall by (d, c) exactly as in route_kernel; results are
// identical. Work: n * m * bits MMA ops, against n * m * W XOR + POPC word pairs
// on the ALU path.
// Each 128-point item loads its visitors' codes into tensor memory once and
// then runs m / 128 tiles, so this path pays off only with many centres
// (measured on B300: 10M points x 10,000 centres, 256-bit: 94-119 ms against
// 169-212 ms on the ALU; 2M x 256 centres, 512-bit: 4.0 against 1.8 ms, where
// route_small.cu's resident centres take 0.55 ms).
constexpr int kRouteTcMinCentres = 1024;
bool bdg_route_tc_ok(int W, int64_t n, int m, int t) {
  return bdg_knn_tc_supported(W, t) && n < (int64_t(1) << 31) && m >= kRouteTcMinCentres &&
         m < (1 << 21);
}

size_t bdg_route_tc_bytes(int64_t n, int m, int W, int t) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const int tile_v = bdg_knn_tile_visitors(W);
  return al(bdg_csr_centres_bytes(n, m, tile_v)) + al(bdg_knn_tc_hexp_bytes(m, 1, W)) +
         al((size_t)n) + al(64) + al((size_t)n * t * 4);
}

bdg_status bdg_launch_route_tc(const uint64_t* codes, int64_t n, int W, const uint64_t* cent,
                               int m, int t, int32_t* routes, int32_t* rdist, void* scratch,
                               size_t scratch_bytes, cudaStream_t st) {
  if (n == 0) return BDG_OK;
  if (scratch_bytes < bdg_route_tc_bytes(n, m, W, t))
    return bdg_set_error(BDG_EINVAL, "route: tensor-path scratch too small");
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const int tile_v = bdg_knn_tile_visitors(W);
  char* p = (char*)scratch;
  bdg_csr csr;
  BDG_TRY(bdg_build_csr_centres(cent, m, n, tile_v, p, &csr, st));
  p += al(bdg_csr_centres_bytes(n, m, tile_v));
  uint8_t* hexp = (uint8_t*)p;   p += al(bdg_knn_tc_hexp_bytes(m, 1, W));
  int8_t* fixflag = (int8_t*)p;  p += al((size_t)n);
  int32_t* err = (int32_t*)p;    p += al(64);
  if (!rdist) rdist = (int32_t*)p;
  BDG_CUDA_TRY(cudaMemsetAsync(fixflag, 0, al((size_t)n) + al(64), st));
  bdg_knn_args a;
  a.codes = codes; a.csr = csr; a.N = m; a.m = 1; a.t = 1; a.k = t; a.bits = 64 * W;
  a.tile_v = tile_v; a.partial = nullptr; a.out_ids = routes; a.out_dist = rdist;
  a.item_counter = csr.counters + 2;
  a.out_by_pos = 1;
  a.fixflag = nullptr;
  a.home_kth = nullptr;
  a.merge_running = 0;
  a.prof = "route";
  bdg_knn_tc_args ta;
  ta.base = a;
  ta.hexp = hexp;
  ta.fixflag = fixflag;
  ta.err = err;
  return bdg_launch_knn_tc(ta, W, true, st);
}

bdg_status bdg_launch_routes_coarse(int32_t* routes, int64_t n, int t, int m, int64_t coarse,
                                    int32_t* home_count, cudaStream_t st) {
  BDG_CUDA_TRY(cudaMemsetAsync(home_count, 0, (size_t)m * 4, st));
  if (n == 0) return BDG_OK;
  const size_t smem = m <= kHistSmemBins ? (size_t)m * 4 : 0;
  if (smem > 48 * 1024)
    BDG_CUDA_TRY(cudaFuncSetAttribute(home_hist_kernel,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t need = bdg_cdiv(n, kHistThreads);
  const int64_t cap = (int64_t)bdg_num_sms() * 2;
  const int grid = (int)(need < cap ? need : cap);
  bdg_prof_scope prof("routes_coarse", st);
  home_hist_kernel<<<grid, kHistThreads, smem, st>>>(routes, n, t, m, home_count);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  coarse_trim_kernel<16><<<(int)bdg_cdiv(n, 256), 256, 0, st>>>(routes, n, t, m, coarse,
                                                                home_count);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

size_t bdg_bkmeans_scratch_bytes(int64_t S, int m, int W) {
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  // + the expanded centres when the assignment runs on the tensor cores
  return al(S * W * 8) + al(S * 4) + al(S * 4) + al((size_t)m * 64 * W * 4) + al((size_t)m * 4) +
         al(8 * 64) + (bdg_route_small_ok(W, m, 1) ? al(bdg_route_small_bytes(m, W)) : 0);
}

namespace {
template <int W>
bdg_status bk_assign_w(const uint64_t* scodes, int64_t S, const uint64_t* cent, int m,
                       int32_t* assign, int32_t* adist, unsigned long long* loss, cudaStream_t st) {
  return route_w<W>(scodes, S, cent, m, 1, assign, adist, loss, st, "bkmeans_assign");
}
}  // namespace

bdg_status bdg_launch_bkmeans(const uint64_t* codes, int64_t N, int W, const int64_t* sample,
                              int64_t S, int m, int iters, uint64_t* cent, int64_t* loss,
                              void* scratch, size_t scratch_bytes, cudaStream_t st) {
  if (scratch_bytes < bdg_bkmeans_scratch_bytes(S, m, W))
    return bdg_set_error(BDG_EINVAL, "bkmeans scratch too small");
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  char* p = (char*)scratch;
  uint64_t* scodes = (uint64_t*)p; p += al(S * W * 8);
  int32_t* assign = (int32_t*)p;   p += al(S * 4);
  int32_t* adist = (int32_t*)p;    p += al(S * 4);
  int32_t* ones = (int32_t*)p;     p += al((size_t)m * 64 * W * 4);
  int32_t* count = (int32_t*)p;    p += al((size_t)m * 4) + al(8 * 64);
  // the assignment on the tensor cores (all centres in shared memory) where it applies
  const bool small = bdg_route_small_ok(W, m, 1) && bdg_tc_default();
  void* rs_scratch = small ? (void*)p : nullptr;
  const size_t rs_bytes = small ? bdg_route_small_bytes(m, W) : 0;
  gather_rows<<<bdg_cdiv(S * W, 256), 256, 0, st>>>(codes, N, sample, S, W, scodes);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  // init: c_j = code of sample[j]
  BDG_CUDA_TRY(cudaMemcpyAsync(cent, scodes, (size_t)m * W * 8, cudaMemcpyDeviceToDevice, st));
  if (loss) BDG_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(int64_t) * (iters + 1), st));
  for (int it = 0; it <= iters; ++it) {
    unsigned long long* lptr = loss ? (unsigned long long*)(loss + it) : nullptr;
    bdg_status s;
    auto run = [&]() -> bdg_status {
      if (small)
        return bdg_launch_route_small(scodes, S, W, cent, m, 1, assign, adist, rs_scratch, rs_bytes,
                                      st, lptr, "bkmeans_assign");
      BDG_DISPATCH_W(W, bk_assign_w, scodes, S, cent, m, assign, adist, lptr, st);
    };
    s = run();
    if (s != BDG_OK) return s;
    if (it == iters) break;
    BDG_CUDA_TRY(cudaMemsetAsync(ones, 0, (size_t)m * 64 * W * 4, st));
    BDG_CUDA_TRY(cudaMemsetAsync(count, 0, (size_t)m * 4, st));
    bk_count<<<bdg_cdiv(S * 32, 256), 256, 0, st>>>(scodes, S, W, assign, ones, count);
    BDG_CUDA_TRY(cudaGetLastError());
    bk_update<<<bdg_cdiv((int64_t)m * W, 256), 256, 0, st>>>(cent, m, W, ones, count);
    BDG_CUDA_TRY(cudaGetLastError());
    bdg_note_launch(2);
  }
  return BDG_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free Bk-means. Some callers cannot call cudaMalloc at all:
// processes whose device memory is owned by an external manager, or
// latency-critical loops that must never reach the allocator (an allocation
// can synchronise the device or fail under memory pressure). For them the
// Bk-means scratch lives in one file-scope device array of fixed size,
// reserved on every GPU that loads this library for as long as the process
// lives.
#define BDG_BK_NOALLOC_BYTES (16u << 20)
static __device__ __align__(256) unsigned char g_bk_noalloc_scratch[BDG_BK_NOALLOC_BYTES];

#include <mutex>

namespace {
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {nullptr};

// Device address of the static scratch for the current device. In host code
// the array's name is only a host-side handle, never a device address, so it
// is looked up once per device (with that device current) and cached for the
// life of the process; after cudaDeviceReset the cached address is stale, which
// the header states.
bdg_status noalloc_scratch(void** out) {
  int dev = 0;
  BDG_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return bdg_set_error(BDG_EUNSUPPORTED, "device %d >= 64", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_ptr[dev] == nullptr) {
    void* p = nullptr;
    BDG_CUDA_TRY(cudaGetSymbolAddress(&p, g_bk_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return BDG_OK;
}
}  // namespace

extern "C" bdg_status bdg_bkmeans_noalloc(const uint64_t* codes, int64_t n, int32_t bits,
                                          const int64_t* sample, int64_t S, int32_t m,
                                          int32_t iters, uint64_t* centroids, int64_t* loss,
                                          void* stream) {
  if (bits <= 0 || bits % 64 != 0)
    return bdg_set_error(BDG_EINVAL, "bkmeans_noalloc: bits = %d", bits);
  const int W = bits / 64;
  if (!(W == 1 || W == 2 || W == 4 || W == 8 || W == 16))
    return bdg_set_error(BDG_EINVAL, "bkmeans_noalloc: bits = %d not built", bits);
  if (m < 1 || S < m || iters < 0 || !codes || !sample || !centroids || n < 1)
    return bdg_set_error(BDG_EINVAL, "bkmeans_noalloc: n=%lld S=%lld m=%d iters=%d",
                         (long long)n, (long long)S, m, iters);
  const size_t need = bdg_bkmeans_scratch_bytes(S, m, W);
  if (need > BDG_BK_NOALLOC_BYTES)
    return bdg_set_error(BDG_EINVAL,
                         "bkmeans_noalloc: S=%lld, m=%d, bits=%d need %zu scratch bytes; the "
                         "fixed scratch holds %u",
                         (long long)S, m, bits, need, (unsigned)BDG_BK_NOALLOC_BYTES);
  void* scratch = nullptr;
  BDG_TRY(noalloc_scratch(&scratch));
  // every scratch region is rewritten or cleared by the launches themselves:
  // sample codes (gather), assignments (assign), per-bit counts (memset each
  // iteration), so nothing from an earlier call leaks into this one
  return bdg_launch_bkmeans(codes, n, W, sample, S, m, iters, centroids, loss, scratch,
                            BDG_BK_NOALLOC_BYTES, (cudaStream_t)stream);
}
