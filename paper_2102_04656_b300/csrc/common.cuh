// common.cuh -- shared device/host helpers of the BDG CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bdg.h"

// A neighbour key packs (distance, id) into one 64-bit word, distance in the
// high half, so that unsigned integer order is the lexicographic (d, id) order
// that breaks ties everywhere in the method. d <= 1025 and 0 <= id < 2^31.
__host__ __device__ __forceinline__ uint64_t bdg_key(uint32_t d, uint32_t id) {
  return (static_cast<uint64_t>(d) << 32) | id;
}
__host__ __device__ __forceinline__ int32_t bdg_key_d(uint64_t k) { return (int32_t)(k >> 32); }
__host__ __device__ __forceinline__ int32_t bdg_key_id(uint64_t k) {
  return (int32_t)(uint32_t)(k & 0xffffffffu);
}
// Padding key for rows with fewer than k candidates: (bits + 1, id = -1).
__host__ __device__ __forceinline__ uint64_t bdg_pad_key(int32_t bits) {
  return bdg_key((uint32_t)(bits + 1), 0xffffffffu);
}
#define BDG_KEY_INF (~0ull)

// partition size classes of the Reduce-1 launches (see kBdgClassLo/Hi below)
constexpr int BDG_SIZE_CLASSES = 3;

// Host-side error plumbing (api.cu owns the thread-local message).
bdg_status bdg_set_error(bdg_status s, const char* fmt, ...);
#define BDG_CUDA_TRY(expr)                                                              \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess)                                                             \
      return bdg_set_error(BDG_ECUDA, "%s failed: %s (%s:%d)", #expr,                 \
                           cudaGetErrorString(_e), __FILE__, __LINE__);                \
  } while (0)
#define BDG_TRY(expr)                 \
  do {                               \
    bdg_status _s = (expr);          \
    if (_s != BDG_OK) return _s;     \
  } while (0)

static inline int bdg_cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Number of SMs of the current device (cached per process for device 0..63).
int bdg_num_sms();

// Kernel launch accounting (every launcher calls bdg_note_launch once per launch)
// and optional CUDA-event timing of named kernels on their launch stream.
void bdg_note_launch(int n = 1);
struct bdg_prof_scope {
  int slot;
  cudaStream_t st;
  bdg_prof_scope(const char* name, cudaStream_t s);
  ~bdg_prof_scope();
};

// Dispatch a templated launcher on the word count W = bits / 64.
#define BDG_DISPATCH_W(W, FN, ...)                                   \
  switch (W) {                                                       \
    case 1: return FN<1>(__VA_ARGS__);                               \
    case 2: return FN<2>(__VA_ARGS__);                               \
    case 4: return FN<4>(__VA_ARGS__);                               \
    case 8: return FN<8>(__VA_ARGS__);                               \
    case 16: return FN<16>(__VA_ARGS__);                             \
    default:                                                         \
      return bdg_set_error(BDG_EUNSUPPORTED,                         \
                           "code width %d words is not built (1,2,4,8,16)", (int)(W)); \
  }

// ---- internal launchers shared between translation units (all async on `st`) ----
// route.cu
bdg_status bdg_launch_route(const uint64_t* codes, int64_t n, int W, const uint64_t* cent,
                            int m, int t, int32_t* routes, int32_t* rdist, cudaStream_t st);
bdg_status bdg_launch_routes_coarse(int32_t* routes, int64_t n, int t, int m, int64_t coarse,
                                    int32_t* home_count, cudaStream_t st);
bdg_status bdg_launch_routes_gap(int32_t* routes, const int32_t* rdist, int64_t n, int t,
                                 int delta, cudaStream_t st);
bdg_status bdg_launch_bkmeans(const uint64_t* codes, int64_t N, int W, const int64_t* sample,
                              int64_t S, int m, int iters, uint64_t* cent, int64_t* loss,
                              void* scratch, size_t scratch_bytes, cudaStream_t st);
size_t bdg_bkmeans_scratch_bytes(int64_t S, int m, int W);
// routing on the tensor cores (route.cu): the t nearest centres of each point
// as its t nearest homes in one partition whose homes are the centres
// api.cu: whether "auto" takes the tensor-core paths (BDG_KNN_KERNEL=popc turns them off)
bool bdg_tc_default();
// route_small.cu: routing on the tensor cores with all centres in shared memory
bool bdg_route_small_ok(int W, int m, int t);
size_t bdg_route_small_bytes(int m, int W);
// loss: optional, the sum over points of the distance to the nearest centre
bdg_status bdg_launch_route_small(const uint64_t* codes, int64_t n, int W, const uint64_t* cent,
                                  int m, int t, int32_t* routes, int32_t* rdist, void* scratch,
                                  size_t scratch_bytes, cudaStream_t st,
                                  unsigned long long* loss = nullptr,
                                  const char* prof_name = "route");
bool bdg_route_tc_ok(int W, int64_t n, int m, int t);
size_t bdg_route_tc_bytes(int64_t n, int m, int W, int t);
bdg_status bdg_launch_route_tc(const uint64_t* codes, int64_t n, int W, const uint64_t* cent,
                               int m, int t, int32_t* routes, int32_t* rdist, void* scratch,
                               size_t scratch_bytes, cudaStream_t st);
// bucket.cu
struct bdg_csr {
  int32_t* home_off;   // [m + 1]
  int32_t* home_ids;   // [N]      point ids grouped by home partition
  uint64_t* home_codes;// [N][W]   codes in home_ids order (contiguous tiles)
  int32_t* visit_off;  // [m + 1]
  int32_t* visit_ids;  // [N * t]  visitor point ids grouped by routed partition
  int8_t* visit_slot;  // [N * t]  slot s of that partition in the visitor's route list
  int32_t* part_order; // [m]      partitions by decreasing |H_p| (then p)
  int32_t* item_off;   // [m + 1]  work items per partition in part_order order
  int32_t* eoff;       // [m + 1]  row offsets of H_p in the 128-row-padded expanded operand
  int32_t* counters;   // [2 * m + 4] scratch counters
  // round A of a partitioned build visits every point in its home partition
  // (its visitors are H_p itself); the visit_* fields above then hold only the
  // other probed partitions (slots >= 1, round B)
  int32_t* item_off_a; // [m + 1]  work items of round A in part_order order
  int8_t* slot_zero;   // [N]      zeros: the route slot of every round-A visit
  int32_t* home_blocks;// [blocks][m] scratch of the stable home placement
  // item -> its partition's rank in part_order (the r with item_off[r] <= item <
  // item_off[r + 1]): round A at item_lo_a, sub-round s at item_lo + (s - 1) * item_stride
  int32_t* item_lo_a;
  int32_t* item_lo;
  int64_t item_stride;
  int m, t;
  // Locality order of each H_p for the tensor path (both null: id order). The
  // homes of p sorted by (nearest of a few pivot homes of p, id): home_loc holds
  // their ids (round A visits the homes in this order), loc_idr, per row of the
  // 128-row-padded expanded operand, the id rank of the home in that row (its
  // position in home_ids; 0 in padding rows).
  int32_t* home_loc;   // [N]
  int32_t* loc_idr;    // [eoff[m]]
};
// items of one round are at most ceil(visits / tile_v) + m <= N / tile_v + m + 1
inline int64_t bdg_csr_item_stride(int64_t N, int m, int tile_v) {
  return (N + tile_v - 1) / tile_v + m + 1;
}
int bdg_home_block(int64_t N, int m);
// The visits of slot s >= 1 form sub-round s: visit_off / item_off hold t - 1
// consecutive [m + 1] arrays (positions are absolute in visit_ids).
// words: per-partition cursors (t * m), one item counter per (round, size
// class), spares
inline size_t bdg_csr_counter_words(int m, int t) {
  return (size_t)t * m + (size_t)t * BDG_SIZE_CLASSES + 8;
}
inline bdg_csr bdg_csr_subround(const bdg_csr& c, int s) {
  bdg_csr v = c;
  v.visit_off = c.visit_off + (size_t)(s - 1) * (c.m + 1);
  v.item_off = c.item_off + (size_t)(s - 1) * (c.m + 1);
  v.item_lo = c.item_lo + (size_t)(s - 1) * c.item_stride;
  return v;
}
// The CSR view of round A (visitors = homes).
inline bdg_csr bdg_csr_round_a(const bdg_csr& c) {
  bdg_csr a = c;
  a.visit_off = c.home_off;
  a.visit_ids = c.home_loc ? c.home_loc : c.home_ids;
  a.visit_slot = c.slot_zero;
  a.item_off = c.item_off_a;
  a.item_lo = c.item_lo_a;
  return a;
}
// pivots > 1: also the locality order of every H_p over `pivots` pivot homes
size_t bdg_csr_bytes(int64_t N, int m, int t, int W, int tile_v, int pivots);
bdg_status bdg_build_csr(const uint64_t* codes, int64_t N, int W, const int32_t* routes, int m,
                         int t, int tile_v, int pivots, void* mem, bdg_csr* csr,
                         cudaStream_t st);
constexpr int BDG_MAX_PIVOTS = 32;
// one partition: every point is a home (identity order, codes used in place);
// the visitors are the given rows
size_t bdg_csr_rows_bytes(int64_t N, int64_t nrows, int tile_v);
bdg_status bdg_build_csr_rows(const uint64_t* codes, int64_t N, const int32_t* rows,
                              int64_t nrows, int tile_v, void* mem, bdg_csr* csr, cudaStream_t st);
// one partition whose homes are the m centres (ids 0..m-1, codes `cent`) and
// whose visitors are all n points in id order, each marked as a visit of a
// partition that is not its home (slot 1: no self pair)
size_t bdg_csr_centres_bytes(int64_t n, int m, int tile_v);
bdg_status bdg_build_csr_centres(const uint64_t* cent, int m, int64_t n, int tile_v, void* mem,
                                 bdg_csr* csr, cudaStream_t st);
// knn_popc.cu
struct bdg_knn_args {
  const uint64_t* codes;  // [N][W]
  bdg_csr csr;
  int64_t N;
  int m, t, k, bits;
  int tile_v;             // visitors per work item
  uint64_t* partial;      // [N][t][k] keys (t > 1) or NULL
  int32_t* out_ids;       // [N][k] final ids when t == 1
  int32_t* out_dist;      // [N][k]
  int32_t* item_counter;  // zeroed before launch
  int out_by_pos;         // t == 1: write row i of the output for the i-th visitor (not its id)
  const int8_t* fixflag;  // [N * t] or NULL: only visit positions flagged 1 are computed
  // sub-rounds: a visitor's threshold starts at the k-th key of its running list
  // (nothing beyond it can enter the final top-k). NULL = none.
  const uint64_t* home_kth;
  // t > 1: `partial` is the running list [N][k]; round A writes it, the
  // sub-rounds merge their rows into it
  int merge_running;
  // name the launches are timed under (bdg_profile_*); null = the kernel's own
  const char* prof = nullptr;
  // fix-up launch (fixflag set): a device word the flagging kernel sets non-zero
  // when it flags any row; zero means there is nothing to recompute. NULL = always run
  const int32_t* fix_any = nullptr;
  // size class: the launch takes only the items of partitions with
  // size_lo <= |H_p| < size_hi (a contiguous range of part_order, which is
  // sorted by decreasing |H_p|)
  int32_t size_lo = 0;
  int32_t size_hi = 0x7fffffff;
};

// The item range [*ib, *ie) of the partitions with size_lo <= |H_p| < size_hi.
__device__ __forceinline__ void bdg_item_range(const bdg_csr& c, int m, int32_t size_lo,
                                               int32_t size_hi, int32_t* ib, int32_t* ie) {
  auto first_below = [&](int32_t s) {  // first rank whose partition holds fewer than s homes
    int lo = 0, hi = m;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      const int p = c.part_order[mid];
      if (c.home_off[p + 1] - c.home_off[p] >= s) lo = mid + 1; else hi = mid;
    }
    return lo;
  };
  *ib = c.item_off[first_below(size_hi)];
  *ie = c.item_off[first_below(size_lo)];
}

// Reduce-1 kernel variants (work items of 128 visitors each): the tensor-core
// kernel (128 x 128 tiles) and the popcount kernel walking an item in sub-tiles
// of 64 or 32 visitors. Partition size classes (by |H_p|) each get one variant.
enum { BDG_KV_POPC = 1, BDG_KV_TC = 2, BDG_KV_POPC32 = 3 };
// class c holds the partitions with kBdgClassLo[c] <= |H_p| < kBdgClassHi[c]
constexpr int32_t kBdgClassLo[BDG_SIZE_CLASSES] = {4096, 512, 0};
constexpr int32_t kBdgClassHi[BDG_SIZE_CLASSES] = {0x7fffffff, 4096, 512};

// Merge a warp's sorted row L (len keys, then anything >= pad) into the sorted
// running list R[0..k) of the same point (global memory): R becomes the k
// smallest keys of both. The valid keys of R and L are distinct (they come from
// disjoint home sets), so every key's rank is its index plus the number of
// smaller keys in the other list. Keys of L at or above `bound` (the caller's
// copy of R[k - 1], or pad) cannot enter; a row without any key below it leaves
// R untouched, without reading it. k <= 128.
__device__ __forceinline__ void bdg_warp_merge_running(uint64_t* R, const uint64_t* L, int len,
                                                       int k, uint64_t pad, uint64_t bound,
                                                       int lane) {
  const uint64_t lim = bound < pad ? bound : pad;
  if (!(len > 0 && L[0] < lim)) return;  // L is sorted: nothing can enter
  uint64_t rv[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = lane + 32 * q;
    rv[q] = j < k ? R[j] : pad;
  }
  int rc[4] = {0, 0, 0, 0};  // new keys below each running key
  for (int i = 0; i < len; ++i) {
    const uint64_t x = L[i];  // the same for every lane
    if (x >= lim) break;
    int below = 0;            // running keys below x
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      rc[q] += (x < rv[q]);
      below += __popc(__ballot_sync(0xffffffffu, rv[q] < x));
    }
    if (lane == (i & 31) && i + below < k) R[i + below] = x;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = lane + 32 * q;
    if (j < k && rc[q] > 0 && j + rc[q] < k) R[j + rc[q]] = rv[q];
  }
  __syncwarp();
}
// knn_tc.cu: tensor-core (tcgen05, FP8 +-1) Reduce 1 for 256/512-bit codes and k <= 64.
// homes per tensor-core tile: each partition's expanded home operand is padded
// to a multiple of this many rows
constexpr int BDG_TC_TILE = 128;
struct bdg_knn_tc_args {
  bdg_knn_args base;
  uint8_t* hexp;          // expanded home operand, eoff[m] rows x bits bytes
  int8_t* fixflag;        // [N * t] zeroed before launch; rows that overflow are set to 1
  int32_t* err;           // device error words: err[0] bounded waits that gave up,
                          // err[1] set when any row is flagged for the fix-up
};
bool bdg_knn_tc_supported(int W, int k);
size_t bdg_knn_tc_hexp_bytes(int64_t N, int m, int W);
bdg_status bdg_launch_knn_tc(const bdg_knn_tc_args& a, int W, bool expand, cudaStream_t st);
bdg_status bdg_launch_knn_popc(const bdg_knn_args& a, int W, cudaStream_t st,
                               bool narrow = false);
// merge.cu
bdg_status bdg_launch_finalize(const uint64_t* running, int64_t N, int k, int bits, int32_t* ids,
                               int32_t* dist, cudaStream_t st);
bdg_status bdg_launch_fill_pad(int32_t* ids, int32_t* dist, int64_t count, int bits,
                               cudaStream_t st);
bdg_status bdg_launch_gather_codes(const uint64_t* codes, int64_t N, const int32_t* ids, int64_t n,
                                   int W, uint64_t* rows, cudaStream_t st);
// search.cu / rerank.cu
struct bdg_graph_view {
  const uint64_t* codes;
  const int32_t* ids;
  const int32_t* entry;
  const uint64_t* entry_codes;  // [n_entry][W] codes of the entry sample, contiguous
  int64_t n;
  int32_t deg, bits, n_entry;
  const uint64_t* nbr_codes = nullptr;  // [n][deg][W] neighbours' codes next to the rows, or null
};
bdg_status bdg_launch_search(const bdg_graph_view& g, const uint64_t* queries, int64_t nq,
                             const int32_t* ef, int ef_max, int R, int32_t* out_ids,
                             int32_t* out_dist, int32_t* expansions, cudaStream_t st);
// shard.cu: merge of per-shard search answers into one (global ids)
#define BDG_MAX_SHARDS 32
struct bdg_shard_offsets {
  int64_t off[BDG_MAX_SHARDS];  // global id of each shard's local id 0
};
size_t bdg_shard_merge_smem(int S, int R);
bdg_status bdg_launch_shard_merge(const int32_t* ids, const int32_t* dist, int S, int64_t nq,
                                  int R, const bdg_shard_offsets& off, const int32_t* ef,
                                  int ef_max, int bits, int32_t* out_ids, int32_t* out_dist,
                                  cudaStream_t st);
// propagate.cu: one round of neighbourhood propagation, ids/dists [n][k] -> new rows
int bdg_propagate_max_k();
// processing order of the points (perm [n], in scratch of bdg_propagate_order_bytes)
size_t bdg_propagate_order_bytes(int64_t n);
bdg_status bdg_launch_propagate_order(const uint64_t* codes, int64_t n, int W, void* scratch,
                                      int32_t** perm, cudaStream_t st);
bdg_status bdg_launch_propagate(const uint64_t* codes, int64_t n, int W, int k,
                                const int32_t* perm, const int32_t* ids_in,
                                const int32_t* dist_in, int32_t* ids_out, int32_t* dist_out,
                                cudaStream_t st);
// prune.cu: occlusion pruning, ids [n][k] -> ids/dists [n][L]
int bdg_prune_max_k();
int bdg_prune_max_l();
bdg_status bdg_launch_prune(const uint64_t* codes, int64_t n, int W, int k, int L,
                            const int32_t* ids_in, int32_t* ids_out, int32_t* dist_out,
                            cudaStream_t st);
bdg_status bdg_launch_rerank(const float* feats, int64_t N, int D, const float* qfeats,
                             const int32_t* cand, int64_t nq, int R, int k, int32_t* out_ids,
                             float* out_d2, cudaStream_t st);
int bdg_knn_tile_visitors(int W);
// BF16 tcgen05 GEMM with row strides for the mask and the output (gemm_tc.cu)
bdg_status bdg_gemm_bf16_ld(const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                            const float* bias, const void* mask, int32_t ldm, int32_t relu,
                            float* out_f32, void* out_bf16, int32_t ldo, float* colsum,
                            int32_t* err, cudaStream_t st);
