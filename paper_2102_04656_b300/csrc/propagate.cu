// propagate.cu -- neighbourhood propagation (Section 3.3) with the propagation
// filter of Section 3.6 (3), one round per launch.
//
// For every point x, its new list is the first k by (d, id) of its current list
// and the neighbours of its neighbours (the "second floor"), every id once; all
// rows read the input graph and write a new one. One warp per point:
//   * the current list is kept sorted in shared memory (its k-th key is the
//     filter: a candidate whose key is not below it cannot enter and is
//     dropped as soon as its distance is known);
//   * each first-floor neighbour's list is read whole (up to four ids per
//     lane) while the next one's is loading; a per-warp hash of the ids already
//     seen skips repeats (the second floor overlaps heavily) before the
//     candidates' codes are gathered, all at once;
//   * the keys that pass the filter are ranked across the warp and merged into
//     the list by ranks.
// The result does not depend on the order candidates are met in: the filter
// bound only tightens and is never below the final k-th key. Nor does it depend
// on the order points are processed in, so points go grouped by 16 bits of
// their code (a counting sort): points processed at the same time then tend to
// be neighbours, their second floors overlap and the code gathers hit L2.
#include "common.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kMaxK = 128;
constexpr int kHash = 1024;  // seen-id slots per warp
constexpr int kProbe = 8;
constexpr int kNew = 0, kSeen = 1, kFull = 2;

struct WarpSmem {
  uint64_t list[kMaxK];  // current list, sorted, `size` valid keys
  uint64_t nk[32];       // accepted keys of one batch, sorted
  int32_t hash[kHash];
};

__device__ __forceinline__ int hash_visit(int32_t* h, int32_t id) {
  const uint32_t slot = ((uint32_t)id * 2654435761u) >> (32 - 10);  // kHash = 1024
  for (int p = 0; p < kProbe; ++p) {
    const uint32_t s = (slot + p) & (kHash - 1);
    const int32_t old = atomicCAS(&h[s], -1, id);
    if (old == -1) return kNew;
    if (old == id) return kSeen;
  }
  return kFull;  // window full: not recorded (checked against the list instead)
}

// Is key in the sorted list[0, size)?
__device__ __forceinline__ bool in_list(const uint64_t* list, int size, uint64_t key) {
  int lo = 0, hi = size;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (list[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo < size && list[lo] == key;
}

// ---- processing order: counting sort of the points by 16 code bits
constexpr int kOrderBins = 1 << 16;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ uint32_t order_key(const uint64_t* codes, int64_t x, int W) {
  return (uint32_t)(codes[x * W] & (kOrderBins - 1));
}

__global__ void order_hist(const uint64_t* __restrict__ codes, int64_t n, int W,
                           int32_t* __restrict__ cnt) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[order_key(codes, x, W)], 1);
}

// exclusive prefix sums of the kOrderBins counts, in place (one block)
__global__ void __launch_bounds__(kScanThreads) order_scan(int32_t* __restrict__ cnt) {
  constexpr int kPer = kOrderBins / kScanThreads;
  __shared__ int32_t wsum[kScanThreads / 32];
  const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
  int32_t s = 0;
  for (int i = 0; i < kPer; ++i) s += cnt[t * kPer + i];
  int32_t incl = s;  // inclusive scan over the warp
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[wp] = incl;
  __syncthreads();
  if (wp == 0) {
    int32_t w = wsum[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    wsum[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  int32_t run = incl - s + (wp > 0 ? wsum[wp - 1] : 0);
  for (int i = 0; i < kPer; ++i) {
    const int32_t c = cnt[t * kPer + i];
    cnt[t * kPer + i] = run;
    run += c;
  }
}

__global__ void order_scatter(const uint64_t* __restrict__ codes, int64_t n, int W,
                              int32_t* __restrict__ cur, int32_t* __restrict__ perm) {
  for (int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n;
       x += (int64_t)gridDim.x * blockDim.x)
    perm[atomicAdd(&cur[order_key(codes, x, W)], 1)] = (int32_t)x;
}

template <int W>
__global__ void __launch_bounds__(kWarps * 32)
propagate_kernel(const uint64_t* __restrict__ codes, int64_t n, int k, int bits,
                 const int32_t* __restrict__ perm, const int32_t* __restrict__ ids_in,
                 const int32_t* __restrict__ dist_in, int32_t* __restrict__ ids_out,
                 int32_t* __restrict__ dist_out) {
  extern __shared__ __align__(16) char prop_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  WarpSmem& sm = reinterpret_cast<WarpSmem*>(prop_smem)[warp];
  const uint64_t pad = bdg_pad_key(bits);
  for (int64_t i = (int64_t)blockIdx.x * kWarps + warp; i < n; i += (int64_t)gridDim.x * kWarps) {
    const int64_t x = perm[i];
    uint64_t cx[W];
#pragma unroll
    for (int w = 0; w < W; ++w) cx[w] = codes[x * W + w];
    for (int i = lane; i < kHash; i += 32) sm.hash[i] = -1;
    __syncwarp();
    // the current list: the input row (sorted by (d, id), padding last)
    int size = 0;
    for (int a0 = 0; a0 < k; a0 += 32) {
      const int a = a0 + lane;
      uint64_t key = BDG_KEY_INF;
      if (a < k) {
        const int32_t z = ids_in[x * k + a];
        if (z >= 0 && z < n && z != x) {
          key = bdg_key((uint32_t)dist_in[x * k + a], (uint32_t)z);
          hash_visit(sm.hash, z);
        }
      }
      const unsigned ok = __ballot_sync(0xffffffffu, key != BDG_KEY_INF);
      if (key != BDG_KEY_INF) sm.list[size + __popc(ok & ((1u << lane) - 1))] = key;
      size += __popc(ok);
    }
    __syncwarp();
    uint64_t kth = size == k ? sm.list[k - 1] : BDG_KEY_INF;
    // the second floor: a neighbour's whole list is read at once (up to four ids
    // per lane) while the next neighbour's list is already on its way, and all
    // of its new candidates' codes are gathered before any of them is merged
    constexpr int kB = kMaxK / 32;
    const int nb = (k + 31) >> 5;
    int32_t ynext[kB];
    {
      const int32_t z0 = ids_in[x * k];
#pragma unroll
      for (int q = 0; q < kB; ++q)
        ynext[q] = (z0 >= 0 && z0 < n && q < nb && q * 32 + lane < k)
                       ? ids_in[(int64_t)z0 * k + q * 32 + lane] : -1;
    }
    for (int a = 0; a < k; ++a) {
      int32_t y[kB];
#pragma unroll
      for (int q = 0; q < kB; ++q) y[q] = ynext[q];
      if (a + 1 < k) {  // the next neighbour's list
        const int32_t zn = ids_in[x * k + a + 1];
#pragma unroll
        for (int q = 0; q < kB; ++q)
          ynext[q] = (zn >= 0 && zn < n && q < nb && q * 32 + lane < k)
                         ? ids_in[(int64_t)zn * k + q * 32 + lane] : -1;
      }
      uint64_t key[kB];
      int hv[kB];
#pragma unroll
      for (int q = 0; q < kB; ++q) {
        key[q] = BDG_KEY_INF;
        hv[q] = kSeen;
        if (y[q] >= 0 && y[q] < n && y[q] != x) hv[q] = hash_visit(sm.hash, y[q]);
      }
#pragma unroll
      for (int q = 0; q < kB; ++q) {
        if (hv[q] != kSeen) {
          uint32_t d = 0;
#pragma unroll
          for (int w = 0; w < W; ++w) d += __popcll(cx[w] ^ codes[(int64_t)y[q] * W + w]);
          key[q] = bdg_key(d, (uint32_t)y[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < kB; ++q) {
        if (q >= nb) break;
        bool acc = key[q] < kth;  // the propagation filter
        if (acc && hv[q] == kFull) acc = !in_list(sm.list, size, key[q]);
        const unsigned am = __ballot_sync(0xffffffffu, acc);
        if (am == 0) continue;
        const int na = __popc(am);
        // rank the accepted keys (ids of one row are distinct) and store them sorted
        int rank = 0;
        for (unsigned mm = am; mm; mm &= mm - 1) {
          const uint64_t o = __shfl_sync(0xffffffffu, key[q], __ffs(mm) - 1);
          rank += (o < key[q]);
        }
        if (acc) sm.nk[rank] = key[q];
        __syncwarp();
        // merge by ranks into the list, keeping the first k
        uint64_t lv[kB];
        int lp[kB];
#pragma unroll
        for (int r = 0; r < kB; ++r) {
          const int j = lane + 32 * r;
          lp[r] = kMaxK;
          lv[r] = 0;
          if (j < size) {
            lv[r] = sm.list[j];
            int c = 0;
            for (int i = 0; i < na; ++i) c += (sm.nk[i] < lv[r]);
            lp[r] = j + c;
          }
        }
        uint64_t nv = 0;
        int np = kMaxK;
        if (lane < na) {
          nv = sm.nk[lane];
          int lo = 0, hi = size;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sm.list[mid] < nv) lo = mid + 1; else hi = mid;
          }
          np = lane + lo;
        }
        __syncwarp();
#pragma unroll
        for (int r = 0; r < kB; ++r)
          if (lp[r] < k) sm.list[lp[r]] = lv[r];
        if (np < k) sm.list[np] = nv;
        size = min(k, size + na);
        __syncwarp();
        kth = size == k ? sm.list[k - 1] : BDG_KEY_INF;
      }
    }
    // write the new row
    for (int j = lane; j < k; j += 32) {
      const uint64_t key = j < size ? sm.list[j] : pad;
      ids_out[x * k + j] = j < size ? bdg_key_id(key) : -1;
      dist_out[x * k + j] = bdg_key_d(key);
    }
    __syncwarp();
  }
}

template <int W>
bdg_status launch_w(const uint64_t* codes, int64_t n, int k, int bits, const int32_t* perm,
                    const int32_t* ids_in, const int32_t* dist_in, int32_t* ids_out,
                    int32_t* dist_out, cudaStream_t st) {
  const size_t smem = sizeof(WarpSmem) * kWarps;
  BDG_CUDA_TRY(cudaFuncSetAttribute(propagate_kernel<W>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  BDG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, propagate_kernel<W>,
                                                             kWarps * 32, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (n + kWarps - 1) / kWarps;
  const int64_t cap = (int64_t)bdg_num_sms() * per_sm;
  const int grid = (int)(need < cap ? need : cap);
  bdg_prof_scope prof("propagate", st);
  propagate_kernel<W><<<grid, kWarps * 32, smem, st>>>(codes, n, k, bits, perm, ids_in,
                                                        dist_in, ids_out, dist_out);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

}  // namespace

int bdg_propagate_max_k() { return kMaxK; }

size_t bdg_propagate_order_bytes(int64_t n) { return (size_t)kOrderBins * 4 + (size_t)n * 4; }

bdg_status bdg_launch_propagate_order(const uint64_t* codes, int64_t n, int W, void* scratch,
                                      int32_t** perm, cudaStream_t st) {
  int32_t* cnt = (int32_t*)scratch;
  *perm = cnt + kOrderBins;
  BDG_CUDA_TRY(cudaMemsetAsync(cnt, 0, (size_t)kOrderBins * 4, st));
  if (n == 0) return BDG_OK;
  const int64_t blocks = bdg_cdiv(n, 256), cap = (int64_t)bdg_num_sms() * 8;
  const int grid = (int)(blocks < cap ? blocks : cap);
  order_hist<<<grid, 256, 0, st>>>(codes, n, W, cnt);
  BDG_CUDA_TRY(cudaGetLastError());
  order_scan<<<1, kScanThreads, 0, st>>>(cnt);
  BDG_CUDA_TRY(cudaGetLastError());
  order_scatter<<<grid, 256, 0, st>>>(codes, n, W, cnt, *perm);
  BDG_CUDA_TRY(cudaGetLastError());
  for (int i = 0; i < 3; ++i) bdg_note_launch();
  return BDG_OK;
}

bdg_status bdg_launch_propagate(const uint64_t* codes, int64_t n, int W, int k,
                                const int32_t* perm, const int32_t* ids_in,
                                const int32_t* dist_in, int32_t* ids_out, int32_t* dist_out,
                                cudaStream_t st) {
  if (n == 0) return BDG_OK;
  BDG_DISPATCH_W(W, launch_w, codes, n, k, 64 * W, perm, ids_in, dist_in, ids_out, dist_out,
                 st);
}
