// knn_popc.cu -- Reduce 1 of Section 3.2 on one GPU: for every partition p and
// every point v routed to p, the exact k nearest home points h of p (h != v)
// under Hamming distance, ties broken by id, as a persistent kernel over
// (partition, visitor tile) work items.
//
// Distances: 128-bit-wide XOR + POPC on codes held in registers (visitors) and
// streamed through shared memory (homes, stored word-major so a warp reads 16
// consecutive home words per load without bank conflicts).
//
// Top-k: every visitor row keeps a sorted list of its best k keys
// (d << 32 | id) in shared memory and a threshold = its k-th key. A pair whose
// key is below the threshold is appended to the row's candidate buffer; after
// each home chunk one warp per non-empty row merges the buffer into the list by
// ranks (keys are unique because ids are, so every rank is unique and the merge
// is exact). Only ~k * ln(|H_p| / k) keys per row ever pass the threshold, so
// the merge cost is small next to the distance work.
//
// Scheduling: one CTA pair per SM loops over work items handed out by a device
// counter in LPT order (see bucket.cu); no CTA ever waits on another.
#include "common.cuh"

namespace {

constexpr int kThreads = 256;  // 8 warps
constexpr int kTH = 64;        // homes per shared-memory chunk (== candidate buffer capacity)
constexpr int kHLanes = 16;    // threads across homes; 16 thread rows across visitors

// visitors per thread: 4 (64-visitor sub-tiles) up to 512-bit codes, else 2;
// the narrow variant halves it (32- or 16-visitor sub-tiles)
template <int W, bool NARROW>
struct Cfg {
  static constexpr int RV = ((W <= 8) ? 4 : 2) / (NARROW ? 2 : 1);
  static constexpr int TV = 16 * RV;           // visitors per sub-tile
};

struct Smem {
  uint64_t* topk;  // [TV][k]
  uint64_t* buf;   // [TV][kTH]
  uint64_t* hs;    // [W][kTH] word-major home codes
  uint64_t* thr;   // [TV]
  int32_t* cur;    // [TV] list length
  int32_t* cnt;    // [TV] buffer fill
  int32_t* hid;    // [kTH]
  int32_t* vid;    // [TV]
  int32_t* vslot;  // [TV]
  int32_t* item;   // [1]
};

template <int W, bool NARROW>
__host__ __device__ size_t smem_bytes(int k) {
  constexpr int TV = Cfg<W, NARROW>::TV;
  return (size_t)TV * k * 8 + (size_t)TV * kTH * 8 + (size_t)W * kTH * 8 + TV * 8 + TV * 4 * 4 +
         kTH * 4 + 16;
}

template <int W, bool NARROW>
__device__ Smem carve(char* base, int k) {
  constexpr int TV = Cfg<W, NARROW>::TV;
  Smem s;
  s.topk = (uint64_t*)base;  base += (size_t)TV * k * 8;
  s.buf = (uint64_t*)base;   base += (size_t)TV * kTH * 8;
  s.hs = (uint64_t*)base;    base += (size_t)W * kTH * 8;
  s.thr = (uint64_t*)base;   base += TV * 8;
  s.cur = (int32_t*)base;    base += TV * 4;
  s.cnt = (int32_t*)base;    base += TV * 4;
  s.vid = (int32_t*)base;    base += TV * 4;
  s.vslot = (int32_t*)base;  base += TV * 4;
  s.hid = (int32_t*)base;    base += kTH * 4;
  s.item = (int32_t*)base;
  return s;
}

// Merge the candidate buffer of row v into its sorted list (one warp).
__device__ __forceinline__ void merge_row(const Smem& s, int v, int k, int lane) {
  const int n = s.cnt[v];
  if (n == 0) return;
  uint64_t* L = s.topk + (size_t)v * k;
  const uint64_t* B = s.buf + (size_t)v * kTH;
  const int len = s.cur[v];
  // buffer entries: rank among the buffer + rank in the list
  uint64_t bv[2];
  int bpos[2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int x = lane + 32 * r;
    bv[r] = x < n ? B[x] : BDG_KEY_INF;
    int rb = 0;
    for (int y = 0; y < n; ++y) rb += (B[y] < bv[r]);
    int lo = 0, hi = len;  // lower_bound in L
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (L[mid] < bv[r]) lo = mid + 1; else hi = mid;
    }
    bpos[r] = x < n ? rb + lo : k;
  }
  // list entries shift right by the number of smaller buffer entries
  uint64_t lv[4];
  int lpos[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int x = lane + 32 * r;
    lv[r] = x < len ? L[x] : BDG_KEY_INF;
    int sh = 0;
    if (x < len)
      for (int y = 0; y < n; ++y) sh += (B[y] < lv[r]);
    lpos[r] = x < len ? x + sh : k;
  }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < 4; ++r)
    if (lpos[r] < k) L[lpos[r]] = lv[r];
#pragma unroll
  for (int r = 0; r < 2; ++r)
    if (bpos[r] < k) L[bpos[r]] = bv[r];
  __syncwarp();
  if (lane == 0) {
    const int nl = min(k, len + n);
    s.cur[v] = nl;
    s.thr[v] = (nl == k) ? L[k - 1] : BDG_KEY_INF;
    s.cnt[v] = 0;
  }
}

template <int W, bool NARROW>
__global__ void __launch_bounds__(kThreads, 2)
knn_popc_kernel(bdg_knn_args a) {
  constexpr int RV = Cfg<W, NARROW>::RV;
  constexpr int TV = Cfg<W, NARROW>::TV;
  extern __shared__ __align__(16) char smem_raw[];
  const int k = a.k;
  Smem s = carve<W, NARROW>(smem_raw, k);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int th = tid % kHLanes;         // home lane
  const int tvg = tid / kHLanes;        // visitor row group: rows tvg*RV .. +RV
  const int m = a.m;
  const bdg_csr& c = a.csr;
  int32_t item_begin, item_end;
  bdg_item_range(c, m, a.size_lo, a.size_hi, &item_begin, &item_end);
  const uint64_t pad = bdg_pad_key(a.bits);
  // a fix-up launch with nothing flagged has no work
  if (a.fix_any != nullptr && *reinterpret_cast<const volatile int32_t*>(a.fix_any) == 0) return;

  for (;;) {
    __syncthreads();
    if (tid == 0) *s.item = item_begin + atomicAdd(a.item_counter, 1);
    __syncthreads();
    const int item = *s.item;
    if (item >= item_end) break;
    const int lo = c.item_lo[item];  // rank of the item's partition in part_order
    const int p = c.part_order[lo];
    const int tile = item - c.item_off[lo];
    const int h0 = c.home_off[p];
    const int nh = c.home_off[p + 1] - h0;
    // an item holds a.tile_v visitors, walked in sub-tiles of TV
    for (int sub = 0; sub < a.tile_v / TV; ++sub) {
    const int v0 = c.visit_off[p] + tile * a.tile_v + sub * TV;
    const int nv = min(TV, c.visit_off[p + 1] - v0);
    if (nv <= 0) break;

    for (int r = tid; r < TV; r += kThreads) {
      // fixup mode: only flagged visit positions are computed
      const bool on = r < nv && (a.fixflag == nullptr || a.fixflag[v0 + r] != 0);
      s.vid[r] = on ? c.visit_ids[v0 + r] : -1;
      s.vslot[r] = r < nv ? (int)c.visit_slot[v0 + r] : 0;
      s.cur[r] = 0;
      s.cnt[r] = 0;
      // idle rows and rows of invalid visitor ids accept nothing; in round B a
      // row starts from the k-th key of the visitor's home list
      uint64_t th0 = (r < nv && s.vid[r] >= 0) ? BDG_KEY_INF : 0ull;
      if (a.home_kth != nullptr && th0 != 0ull) th0 = a.home_kth[(int64_t)s.vid[r] * k + (k - 1)];
      s.thr[r] = th0;
    }
    if (a.fixflag != nullptr) {  // skip items without a flagged row
      const int any = __syncthreads_or(tid < TV && s.vid[tid < TV ? tid : 0] >= 0);
      if (!any) continue;
    }
    __syncthreads();
    uint64_t vc[RV][W];
    int32_t myvid[RV];
    int32_t selfid[RV];  // the id that is the row's own point (-2: none to exclude)
    uint64_t thr[RV];
#pragma unroll
    for (int r = 0; r < RV; ++r) {
      const int row = tvg * RV + r;
      myvid[r] = s.vid[row];
      // only a visitor of its own home set (slot 0) can meet itself among the homes
      selfid[r] = s.vslot[row] == 0 ? myvid[r] : -2;
      thr[r] = s.thr[row];
#pragma unroll
      for (int w = 0; w < W; ++w)
        vc[r][w] = myvid[r] >= 0 ? a.codes[(int64_t)myvid[r] * W + w] : 0ull;
    }

    for (int c0 = 0; c0 < nh; c0 += kTH) {
      const int nc = min(kTH, nh - c0);
      // stage the home chunk word-major
      for (int x = tid; x < kTH * W; x += kThreads) {
        const int h = x / W, w = x - h * W;
        s.hs[w * kTH + h] = h < nc ? c.home_codes[(int64_t)(h0 + c0 + h) * W + w] : 0ull;
      }
      for (int h = tid; h < kTH; h += kThreads) s.hid[h] = h < nc ? c.home_ids[h0 + c0 + h] : -1;
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kTH / kHLanes; ++j) {
        const int h = th + kHLanes * j;
        const int32_t hidv = s.hid[h];
        uint64_t hw[W];
#pragma unroll
        for (int w = 0; w < W; ++w) hw[w] = s.hs[w * kTH + h];
#pragma unroll
        for (int r = 0; r < RV; ++r) {
          uint32_t d = 0;
#pragma unroll
          for (int w = 0; w < W; ++w) d += __popcll(vc[r][w] ^ hw[w]);
          const uint64_t key = bdg_key(d, (uint32_t)hidv);
          if (hidv >= 0 && key < thr[r] && hidv != selfid[r]) {
            const int row = tvg * RV + r;
            const int pos = atomicAdd(&s.cnt[row], 1);
            s.buf[(size_t)row * kTH + pos] = key;
          }
        }
      }
      __syncthreads();
      for (int v = warp; v < TV; v += kThreads / 32) merge_row(s, v, k, lane);
      __syncthreads();
#pragma unroll
      for (int r = 0; r < RV; ++r) thr[r] = s.thr[tvg * RV + r];
    }

    // write the rows: final graph rows when t == 1, else the partial list of this slot
    for (int v = warp; v < nv; v += kThreads / 32) {
      const int32_t id = s.vid[v];
      const int len = s.cur[v];
      const uint64_t* L = s.topk + (size_t)v * k;
      if (id < 0 && (!a.out_by_pos || a.fixflag != nullptr)) continue;
      if (a.t == 1) {
        const int64_t row = a.out_by_pos ? (int64_t)(v0 - c.visit_off[p] + v) : (int64_t)id;
        for (int j = lane; j < k; j += 32) {
          const uint64_t key = j < len ? L[j] : pad;
          a.out_ids[row * k + j] = j < len ? bdg_key_id(key) : -1;
          a.out_dist[row * k + j] = bdg_key_d(key);
        }
      } else if (!a.merge_running) {  // round A: the running list starts as this row
        uint64_t* out = a.partial + (int64_t)id * k;
        for (int j = lane; j < k; j += 32) out[j] = j < len ? L[j] : pad;
      } else {
        bdg_warp_merge_running(a.partial + (int64_t)id * k, L, len, k, pad, pad, lane);
      }
    }
    __syncthreads();
    }  // sub-tiles
  }
}

template <int W, bool NARROW>
bdg_status launch_v(const bdg_knn_args& a, cudaStream_t st) {
  const size_t smem = smem_bytes<W, NARROW>(a.k);
  BDG_CUDA_TRY(cudaFuncSetAttribute(knn_popc_kernel<W, NARROW>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  BDG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, knn_popc_kernel<W, NARROW>,
                                                             kThreads, smem));
  if (per_sm < 1) return bdg_set_error(BDG_EUNSUPPORTED, "knn kernel does not fit (k=%d)", a.k);
  const int grid = bdg_num_sms() * per_sm;
  bdg_prof_scope prof(a.prof ? a.prof : (a.fixflag ? "knn_fixup" : "knn"), st);
  knn_popc_kernel<W, NARROW><<<grid, kThreads, smem, st>>>(a);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

template <int W>
bdg_status launch_w(const bdg_knn_args& a, cudaStream_t st, bool narrow) {
  return narrow ? launch_v<W, true>(a, st) : launch_v<W, false>(a, st);
}

}  // namespace

// Work items hold 128 visitors for every code width (the tensor-core kernel's
// tile); the popcount kernel walks an item in sub-tiles of its own size.
int bdg_knn_tile_visitors(int W) { (void)W; return 128; }

bdg_status bdg_launch_knn_popc(const bdg_knn_args& a, int W, cudaStream_t st, bool narrow) {
  if (a.k > 128) return bdg_set_error(BDG_EUNSUPPORTED, "k = %d > 128", a.k);
  BDG_DISPATCH_W(W, launch_w, a, st, narrow);
}
