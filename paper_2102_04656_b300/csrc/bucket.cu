// bucket.cu -- the Shuffle of Section 3.2 done in HBM: group points by home
// partition (H_p, whose codes are also copied contiguously so the k-NN kernel
// streams them as dense tiles) and by every routed partition (V_p, with the
// route slot), then lay out the persistent kernel's work items.
//
// Work items are (partition, tile of `tile_v` visitors). Partitions are ordered
// by decreasing |H_p| (every item of p costs tile_v * |H_p| pairs), so the
// dynamic item counter of the persistent kernel hands out the longest items
// first -- the greedy longest-processing-time rule, which is this design's
// stand-in for the paper's data-skew balancing across Reduce nodes
// (Section 3.6 (1)).
#include "common.cuh"

namespace {

constexpr int kScanThreads = 1024;
constexpr int kMaxSortM = 16384;  // partitions sortable by the single-block bitonic sort

// ---- stable placement of the homes: H_p lists point ids in ascending order
// (so a home's position within its partition orders like its id). Points are
// cut into blocks of `bp` consecutive ids: each block counts its homes per
// partition, a column scan turns the counts into each block's start within
// every H_p, and one warp per block then walks its points in order.
__global__ void home_block_count(const int32_t* __restrict__ routes, int64_t N, int t, int m,
                                 int bp, int32_t* __restrict__ bcnt) {
  extern __shared__ int32_t sc[];  // [m]
  for (int p = threadIdx.x; p < m; p += blockDim.x) sc[p] = 0;
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * bp, i1 = min(N, i0 + bp);
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const int32_t h = routes[i * t];
    if (h >= 0 && h < m) atomicAdd(&sc[h], 1);
  }
  __syncthreads();
  for (int p = threadIdx.x; p < m; p += blockDim.x) bcnt[(int64_t)blockIdx.x * m + p] = sc[p];
}

// hcnt[p] = total homes of p; bcnt[b][p] becomes the block's start within H_p
__global__ void home_block_scan(int m, int nblk, int32_t* __restrict__ bcnt,
                                int32_t* __restrict__ hcnt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  int32_t run = 0;
  for (int b = 0; b < nblk; ++b) {
    const int32_t c = bcnt[(int64_t)b * m + p];
    bcnt[(int64_t)b * m + p] = run;
    run += c;
  }
  hcnt[p] = run;
}

__global__ void __launch_bounds__(32)
home_place(const int32_t* __restrict__ routes, int64_t N, int t, int m, int bp,
           const int32_t* __restrict__ bcnt, const int32_t* __restrict__ home_off,
           int32_t* __restrict__ home_ids) {
  extern __shared__ int32_t cur[];  // [m] next position of this block in each H_p
  const int lane = threadIdx.x;
  for (int p = lane; p < m; p += 32)
    cur[p] = home_off[p] + bcnt[(int64_t)blockIdx.x * m + p];
  __syncwarp();
  const int64_t i0 = (int64_t)blockIdx.x * bp, i1 = min(N, i0 + bp);
  for (int64_t c0 = i0; c0 < i1; c0 += 32) {
    const int64_t i = c0 + lane;
    int32_t h = (i < i1) ? routes[i * t] : -1;
    if (h < 0 || h >= m) h = -1;
    const unsigned peers = __match_any_sync(0xffffffffu, h);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const int32_t base = (h >= 0) ? cur[h] : 0;
    __syncwarp();
    if (h >= 0) {
      home_ids[base + rank] = (int32_t)i;
      if (rank == 0) cur[h] = base + __popc(peers);  // the group's first lane advances it
    }
    __syncwarp();
  }
}

__global__ void count_kernel(const int32_t* __restrict__ routes, int64_t N, int t, int m,
                             int32_t* __restrict__ vcnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  // homes are counted and placed in id order by the stable pass below; route
  // values outside [0, m) are ignored
  for (int s = 1; s < t; ++s) {  // slot 0 (the home) is visited in round A from H_p
    const int32_t p = routes[i * t + s];
    if (p >= 0 && p < m) atomicAdd(&vcnt[(s - 1) * m + p], 1);
  }
}

// Block-wide exclusive scan of per-thread totals (1024 threads).
__device__ int32_t block_exclusive_scan(int32_t v, int32_t* warp_tot, int32_t* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int32_t w = warp_tot[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_tot[lane] = w;  // inclusive
  }
  __syncthreads();
  const int32_t base = wid > 0 ? warp_tot[wid - 1] : 0;
  if (total) *total = warp_tot[31];
  const int32_t r = base + x - v;
  __syncthreads();
  return r;
}

// Single block: offsets of H_p and of the visits of every slot s >= 1 (each
// slot's visits form one sub-round, laid out one after the other), partition
// order by decreasing |H_p|, work-item offsets of round A and of every
// sub-round in that order, and scatter cursors.
__global__ void __launch_bounds__(kScanThreads)
plan_kernel(int m, int t, int tile_v, int32_t* __restrict__ hcnt, int32_t* __restrict__ vcnt,
            int32_t* __restrict__ home_off, int32_t* __restrict__ visit_off,
            int32_t* __restrict__ part_order, int32_t* __restrict__ item_off,
            int32_t* __restrict__ eoff, int32_t* __restrict__ item_off_a) {
  extern __shared__ uint64_t skey[];  // [pow2 >= m]
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t total;
  const int per = (m + kScanThreads - 1) / kScanThreads;
  const int b = threadIdx.x * per, e = min(m, b + per);
  // --- homes
  {
    int32_t s = 0;
    for (int p = b; p < e; ++p) s += hcnt[p];
    int32_t run = block_exclusive_scan(s, warp_tot, &total);
    for (int p = b; p < e; ++p) { home_off[p] = run; run += hcnt[p]; }
    if (threadIdx.x == 0) home_off[m] = total;
    __syncthreads();
  }
  // --- visits of slots 1 .. t-1, one block of positions per slot
  int32_t base = 0;
  for (int sl = 1; sl < t; ++sl) {
    const int32_t* cnt = vcnt + (sl - 1) * m;
    int32_t* off = visit_off + (sl - 1) * (m + 1);
    int32_t s = 0;
    for (int p = b; p < e; ++p) s += cnt[p];
    int32_t run = block_exclusive_scan(s, warp_tot, &total);
    run += base;
    for (int p = b; p < e; ++p) { off[p] = run; run += cnt[p]; }
    const int32_t tot = total;
    if (threadIdx.x == 0) off[m] = base + tot;
    base += tot;
    __syncthreads();
  }
  // --- offsets of the 64-row-padded expanded home operand (tensor path)
  {
    int32_t s = 0;
    for (int p = b; p < e; ++p) s += (hcnt[p] + BDG_TC_TILE - 1) & ~(BDG_TC_TILE - 1);
    int32_t run = block_exclusive_scan(s, warp_tot, &total);
    for (int p = b; p < e; ++p) {
      eoff[p] = run;
      run += (hcnt[p] + BDG_TC_TILE - 1) & ~(BDG_TC_TILE - 1);
    }
    if (threadIdx.x == 0) eoff[m] = total;
    __syncthreads();
  }
  // --- sort partitions by (decreasing |H_p|, p)
  int np2 = 1;
  while (np2 < m) np2 <<= 1;
  for (int p = threadIdx.x; p < np2; p += kScanThreads)
    skey[p] = p < m ? ((uint64_t)(0x7fffffff - hcnt[p]) << 32) | (uint32_t)p : ~0ull;
  __syncthreads();
  for (int size = 2; size <= np2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int x = threadIdx.x; x < np2; x += kScanThreads) {
        const int y = x ^ stride;
        if (y > x) {
          const bool up = (x & size) == 0;
          const uint64_t a = skey[x], c = skey[y];
          if ((a > c) == up) { skey[x] = c; skey[y] = a; }
        }
      }
      __syncthreads();
    }
  }
  for (int r = threadIdx.x; r < m; r += kScanThreads) part_order[r] = (int32_t)(skey[r] & 0xffffffffu);
  __syncthreads();
  // --- work items in partition order: round A (homes), then each sub-round
  for (int sl = 0; sl < t; ++sl) {
    const int32_t* cnt = sl == 0 ? hcnt : vcnt + (sl - 1) * m;
    int32_t* io = sl == 0 ? item_off_a : item_off + (sl - 1) * (m + 1);
    int32_t s = 0;
    for (int r = b; r < e; ++r) s += (cnt[part_order[r]] + tile_v - 1) / tile_v;
    int32_t run = block_exclusive_scan(s, warp_tot, &total);
    for (int r = b; r < e; ++r) {
      io[r] = run;
      run += (cnt[part_order[r]] + tile_v - 1) / tile_v;  // an empty H_p still pads its visitors
    }
    if (threadIdx.x == 0) io[m] = total;
    __syncthreads();
  }
  // --- scatter cursors start at the offsets
  for (int p = threadIdx.x; p < m; p += kScanThreads) {
    hcnt[p] = home_off[p];
    for (int sl = 1; sl < t; ++sl) vcnt[(sl - 1) * m + p] = visit_off[(sl - 1) * (m + 1) + p];
  }
}

__global__ void scatter_kernel(const int32_t* __restrict__ routes, int64_t N, int t, int m,
                               int32_t* __restrict__ vcur, int32_t* __restrict__ visit_ids,
                               int8_t* __restrict__ visit_slot) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  for (int s = 1; s < t; ++s) {
    const int32_t p = routes[i * t + s];
    if (p < 0 || p >= m) continue;
    const int32_t pos = atomicAdd(&vcur[(s - 1) * m + p], 1);
    visit_ids[pos] = (int32_t)i;
    visit_slot[pos] = (int8_t)s;
  }
}

// The same two passes with per-block aggregation, while the (t - 1) * m bins
// fit in shared memory: a block takes `pts` points, counts its (slot,
// partition) pairs there and touches each global counter once; the placement
// pass also ranks each pair within its block and bin, reserves the block's
// range of every bin with one global atomic and writes each pair at range start
// + rank. (Few bins with many points per bin made the one-atomic-per-pair
// passes contend.)
constexpr int kAggThreads = 256;
constexpr int kAggBins = 4096;      // (t - 1) * m at most
constexpr int kAggEntries = 8192;   // pts * (t - 1) at most

__global__ void __launch_bounds__(kAggThreads)
count_agg_kernel(const int32_t* __restrict__ routes, int64_t N, int t, int m, int pts,
                 int32_t* __restrict__ vcnt) {
  __shared__ int32_t sh[kAggBins];
  const int nb = (t - 1) * m, ns = t - 1;
  for (int b = threadIdx.x; b < nb; b += kAggThreads) sh[b] = 0;
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * pts;
  for (int e = threadIdx.x; e < pts * ns; e += kAggThreads) {
    const int64_t i = i0 + e / ns;
    if (i >= N) break;
    const int s = 1 + e % ns;
    const int32_t p = routes[i * t + s];
    if (p >= 0 && p < m) atomicAdd(&sh[(s - 1) * m + p], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += kAggThreads)
    if (sh[b] != 0) atomicAdd(&vcnt[b], sh[b]);
}

__global__ void __launch_bounds__(kAggThreads)
scatter_agg_kernel(const int32_t* __restrict__ routes, int64_t N, int t, int m, int pts,
                   int32_t* __restrict__ vcur, int32_t* __restrict__ visit_ids,
                   int8_t* __restrict__ visit_slot) {
  __shared__ int32_t sh[kAggBins];      // counts, then the block's first position per bin
  __shared__ int32_t rank[kAggEntries];  // a pair's rank in its bin within the block (-1: none)
  const int nb = (t - 1) * m, ns = t - 1;
  for (int b = threadIdx.x; b < nb; b += kAggThreads) sh[b] = 0;
  __syncthreads();
  const int64_t i0 = (int64_t)blockIdx.x * pts;
  for (int e = threadIdx.x; e < pts * ns; e += kAggThreads) {
    const int64_t i = i0 + e / ns;
    const int s = 1 + e % ns;
    const int32_t p = i < N ? routes[i * t + s] : -1;
    rank[e] = (p >= 0 && p < m) ? atomicAdd(&sh[(s - 1) * m + p], 1) : -1;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < nb; b += kAggThreads) {
    const int32_t c = sh[b];
    sh[b] = c != 0 ? atomicAdd(&vcur[b], c) : 0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < pts * ns; e += kAggThreads) {
    const int32_t r = rank[e];
    if (r < 0) continue;
    const int64_t i = i0 + e / ns;
    const int s = 1 + e % ns;
    const int32_t pos = sh[(s - 1) * m + routes[i * t + s]] + r;
    visit_ids[pos] = (int32_t)i;
    visit_slot[pos] = (int8_t)s;
  }
}

__global__ void gather_home_codes(const uint64_t* __restrict__ codes,
                                  const int32_t* __restrict__ home_ids,
                                  const int32_t* __restrict__ home_off, int m, int64_t N, int W,
                                  uint64_t* __restrict__ out) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= N * W) return;
  const int64_t r = x / W;
  if (r >= home_off[m]) return;  // points without a valid home are in no H_p
  out[x] = codes[(int64_t)home_ids[r] * W + (x - r * W)];
}

inline size_t al(size_t b) { return (b + 255) & ~size_t(255); }

__global__ void rows_plan_kernel(int64_t N, const int32_t* __restrict__ rows, int64_t nrows,
                                 int tile_v, int32_t* __restrict__ home_off,
                                 int32_t* __restrict__ home_ids, int32_t* __restrict__ visit_off,
                                 int32_t* __restrict__ visit_ids, int8_t* __restrict__ visit_slot,
                                 int32_t* __restrict__ part_order, int32_t* __restrict__ item_off,
                                 int32_t* __restrict__ eoff) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < N) home_ids[x] = (int32_t)x;
  if (x < nrows) {  // ids outside [0, N) become empty rows
    const int32_t r = rows[x];
    visit_ids[x] = (r >= 0 && r < N) ? r : -1;
    visit_slot[x] = 0;
  }
  if (x == 0) {
    home_off[0] = 0; home_off[1] = (int32_t)N;
    visit_off[0] = 0; visit_off[1] = (int32_t)nrows;
    part_order[0] = 0;
    item_off[0] = 0; item_off[1] = (int32_t)((nrows + tile_v - 1) / tile_v);
    eoff[0] = 0; eoff[1] = (int32_t)((N + BDG_TC_TILE - 1) & ~(int64_t)(BDG_TC_TILE - 1));
  }
}

// Routing as one partition: homes = the m centres (ids 0..m-1), visitors = all
// n points in id order, each a visit of slot 1 (not its home set: no self pair).
__global__ void centres_plan_kernel(int64_t n, int m, int tile_v, int32_t* __restrict__ home_off,
                                    int32_t* __restrict__ home_ids,
                                    int32_t* __restrict__ visit_off,
                                    int32_t* __restrict__ visit_ids,
                                    int8_t* __restrict__ visit_slot,
                                    int32_t* __restrict__ part_order,
                                    int32_t* __restrict__ item_off, int32_t* __restrict__ eoff) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < m) home_ids[x] = (int32_t)x;
  if (x < n) {
    visit_ids[x] = (int32_t)x;
    visit_slot[x] = 1;
  }
  if (x == 0) {
    home_off[0] = 0; home_off[1] = m;
    visit_off[0] = 0; visit_off[1] = (int32_t)n;
    part_order[0] = 0;
    item_off[0] = 0; item_off[1] = (int32_t)((n + tile_v - 1) / tile_v);
    eoff[0] = 0; eoff[1] = (m + BDG_TC_TILE - 1) & ~(BDG_TC_TILE - 1);
  }
}

// ---- locality order of H_p (tensor path): the homes of p sorted by (nearest of
// P pivot homes, id). The pivots are the homes at positions (2i + 1) |H_p| / (2P)
// of H_p in id order, and a home's nearest pivot is the first one at the least
// Hamming distance. The order changes no result: candidate words carry the id
// rank (loc_idr), so they still order by (d, id).
//
// Keys: block (p, y) takes the chunks y, y + gridDim.y, ... of 256 homes of p,
// with p's pivots in shared memory; one thread per home.
template <int W>
__global__ void __launch_bounds__(256)
pivot_key_kernel(const uint64_t* __restrict__ home_codes, const int32_t* __restrict__ home_off,
                 int m, int P, int8_t* __restrict__ key) {
  __shared__ uint64_t piv[BDG_MAX_PIVOTS * W];
  const int p = blockIdx.x;
  const int h0 = home_off[p], nh = home_off[p + 1] - h0;
  const int np = min(P, nh);
  if (np <= 1) {  // one pivot or none: every key is 0
    for (int x = blockIdx.y * 256 + threadIdx.x; x < nh; x += gridDim.y * 256) key[h0 + x] = 0;
    return;
  }
  for (int x = threadIdx.x; x < np * W; x += 256) {
    const int i = x / W, w = x % W;
    const int pos = (int)(((2LL * i + 1) * nh) / (2LL * np));
    piv[x] = home_codes[(int64_t)(h0 + pos) * W + w];
  }
  __syncthreads();
  for (int x = blockIdx.y * 256 + threadIdx.x; x < nh; x += gridDim.y * 256) {
    uint64_t hc[W];
#pragma unroll
    for (int w = 0; w < W; ++w) hc[w] = home_codes[(int64_t)(h0 + x) * W + w];
    int best = 0, bd = INT_MAX;
    for (int i = 0; i < np; ++i) {
      int d = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) d += __popcll(hc[w] ^ piv[i * W + w]);
      if (d < bd) { bd = d; best = i; }
    }
    key[h0 + x] = (int8_t)best;
  }
}

// Stable counting sort of each H_p by key, one block of 32 warps per partition:
// warp w owns the w-th of 32 consecutive segments of H_p; the warps count their
// keys, an exclusive scan over (key, warp) gives each warp's cursors, and every
// warp then places its segment in order (ranks among equal keys by lane).
__global__ void __launch_bounds__(1024)
pivot_sort_kernel(const int8_t* __restrict__ key, const int32_t* __restrict__ home_ids,
                  const int32_t* __restrict__ home_off, const int32_t* __restrict__ eoff,
                  int32_t* __restrict__ home_loc, int32_t* __restrict__ loc_idr) {
  __shared__ int32_t wcnt[32][BDG_MAX_PIVOTS];
  const int p = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int h0 = home_off[p], nh = home_off[p + 1] - h0;
  const int64_t e0 = eoff[p];
  const int npad = (nh + BDG_TC_TILE - 1) & ~(BDG_TC_TILE - 1);
  const int seg = (nh + 31) / 32;
  const int s0 = min(nh, warp * seg), s1 = min(nh, s0 + seg);
  if (lane < BDG_MAX_PIVOTS) wcnt[warp][lane] = 0;
  __syncwarp();
  for (int x0 = s0; x0 < s1; x0 += 32) {
    const int x = x0 + lane;
    const int kx = x < s1 ? (int)key[h0 + x] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, kx);
    if (kx >= 0 && __popc(same & ((1u << lane) - 1u)) == 0) wcnt[warp][kx] += __popc(same);
    __syncwarp();
  }
  __syncthreads();
  if (threadIdx.x == 0) {  // cursors: keys in order, warps in order within a key
    int run = 0;
    for (int kk = 0; kk < BDG_MAX_PIVOTS; ++kk)
      for (int w = 0; w < 32; ++w) {
        const int cv = wcnt[w][kk];
        wcnt[w][kk] = run;
        run += cv;
      }
  }
  __syncthreads();
  for (int x0 = s0; x0 < s1; x0 += 32) {
    const int x = x0 + lane;
    const int kx = x < s1 ? (int)key[h0 + x] : -1;
    const unsigned same = __match_any_sync(0xffffffffu, kx);
    const int rank = __popc(same & ((1u << lane) - 1u));
    const int pos = kx >= 0 ? wcnt[warp][kx] + rank : 0;
    __syncwarp();
    if (kx >= 0 && rank == 0) wcnt[warp][kx] += __popc(same);  // the group's first lane advances it
    __syncwarp();
    if (kx >= 0) {
      loc_idr[e0 + pos] = x;
      home_loc[h0 + pos] = home_ids[h0 + x];
    }
  }
  for (int q = nh + (int)threadIdx.x; q < npad; q += 1024) loc_idr[e0 + q] = 0;
}

}  // namespace

size_t bdg_csr_centres_bytes(int64_t n, int m, int tile_v) {
  return al(2 * 4) * 4 + al((size_t)m * 4) + al(n * 4) + al(n) + al(4) + al(8 * 4) +
         al((size_t)((n + tile_v - 1) / tile_v + 1) * 4);
}

bdg_status bdg_build_csr_centres(const uint64_t* cent, int m, int64_t n, int tile_v, void* mem,
                                 bdg_csr* c, cudaStream_t st) {
  char* p = (char*)mem;
  c->home_off = (int32_t*)p;   p += al(2 * 4);
  c->visit_off = (int32_t*)p;  p += al(2 * 4);
  c->item_off = (int32_t*)p;   p += al(2 * 4);
  c->eoff = (int32_t*)p;       p += al(2 * 4);
  c->home_ids = (int32_t*)p;   p += al((size_t)m * 4);
  c->visit_ids = (int32_t*)p;  p += al(n * 4);
  c->visit_slot = (int8_t*)p;  p += al(n);
  c->part_order = (int32_t*)p; p += al(4);
  c->counters = (int32_t*)p;   p += al(8 * 4);
  c->item_lo_a = (int32_t*)p;  // one partition: every item's rank is 0
  c->item_lo = c->item_lo_a;
  c->item_stride = 0;
  c->home_codes = const_cast<uint64_t*>(cent);
  c->item_off_a = c->item_off;
  c->slot_zero = c->visit_slot;
  c->home_blocks = nullptr;
  c->home_loc = c->loc_idr = nullptr;
  c->m = 1;
  c->t = 1;
  BDG_CUDA_TRY(cudaMemsetAsync(c->counters, 0, 8 * 4, st));
  BDG_CUDA_TRY(cudaMemsetAsync(c->item_lo_a, 0, ((n + tile_v - 1) / tile_v + 1) * 4, st));
  const int64_t x = n > m ? n : m;
  centres_plan_kernel<<<bdg_cdiv(x, 256), 256, 0, st>>>(n, m, tile_v, c->home_off, c->home_ids,
                                                        c->visit_off, c->visit_ids, c->visit_slot,
                                                        c->part_order, c->item_off, c->eoff);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

size_t bdg_csr_rows_bytes(int64_t N, int64_t nrows, int tile_v) {
  return al(2 * 4) * 4 + al(N * 4) + al(nrows * 4) + al(nrows) + al(4) + al(8 * 4) +
         al((size_t)((nrows + tile_v - 1) / tile_v + 1) * 4);
}

bdg_status bdg_build_csr_rows(const uint64_t* codes, int64_t N, const int32_t* rows,
                              int64_t nrows, int tile_v, void* mem, bdg_csr* c, cudaStream_t st) {
  char* p = (char*)mem;
  c->home_off = (int32_t*)p;   p += al(2 * 4);
  c->visit_off = (int32_t*)p;  p += al(2 * 4);
  c->item_off = (int32_t*)p;   p += al(2 * 4);
  c->eoff = (int32_t*)p;       p += al(2 * 4);
  c->home_ids = (int32_t*)p;   p += al(N * 4);
  c->visit_ids = (int32_t*)p;  p += al(nrows * 4);
  c->visit_slot = (int8_t*)p;  p += al(nrows);
  c->part_order = (int32_t*)p; p += al(4);
  c->counters = (int32_t*)p;   p += al(8 * 4);
  c->item_lo_a = (int32_t*)p;  // one partition: every item's rank is 0
  c->item_lo = c->item_lo_a;
  c->item_stride = 0;
  c->home_codes = const_cast<uint64_t*>(codes);  // identity order: read the codes in place
  c->item_off_a = c->item_off;
  c->slot_zero = c->visit_slot;
  c->home_blocks = nullptr;
  c->home_loc = c->loc_idr = nullptr;
  c->m = 1;
  c->t = 1;
  BDG_CUDA_TRY(cudaMemsetAsync(c->counters, 0, 8 * 4, st));
  BDG_CUDA_TRY(cudaMemsetAsync(c->item_lo_a, 0, ((nrows + tile_v - 1) / tile_v + 1) * 4, st));
  const int64_t n = N > nrows ? N : nrows;
  rows_plan_kernel<<<bdg_cdiv(n, 256), 256, 0, st>>>(N, rows, nrows, tile_v, c->home_off,
                                                     c->home_ids, c->visit_off, c->visit_ids,
                                                     c->visit_slot, c->part_order, c->item_off,
                                                     c->eoff);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

// points per block of the stable home placement (block counts stay <= 64M words)
int bdg_home_block(int64_t N, int m) {
  int64_t bp = 4096;
  while ((N + bp - 1) / bp * (int64_t)m > (64LL << 20)) bp *= 2;
  return (int)bp;
}

// item_lo[item] = r for r's items: one thread per (round, partition rank r)
__global__ void item_table_kernel(int m, int rounds, const int32_t* __restrict__ item_off_a,
                                  const int32_t* __restrict__ item_off, int64_t stride,
                                  int32_t* __restrict__ item_lo_a, int32_t* __restrict__ item_lo) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (int64_t)rounds * m) return;
  const int round = (int)(x / m), r = (int)(x - (int64_t)round * m);
  const int32_t* io = round == 0 ? item_off_a : item_off + (size_t)(round - 1) * (m + 1);
  int32_t* out = round == 0 ? item_lo_a : item_lo + (size_t)(round - 1) * stride;
  for (int32_t it = io[r]; it < io[r + 1]; ++it) out[it] = r;
}

size_t bdg_csr_bytes(int64_t N, int m, int t, int W, int tile_v, int pivots) {
  const size_t ts = t > 1 ? (size_t)(t - 1) : 1;
  const size_t blk = (size_t)((N + bdg_home_block(N, m) - 1) / bdg_home_block(N, m)) * m * 4;
  const size_t stride = (size_t)bdg_csr_item_stride(N, m, tile_v);
  return al((m + 1) * 4) * 3 + al(ts * (m + 1) * 4) * 2 + al(N * 4) + al(N * W * 8) +
         al(N * t * 4) + al(N * t) + al(m * 4) + al(bdg_csr_counter_words(m, t) * 4) + al(N) +
         al(blk) + al(stride * 4) + al(ts * stride * 4) +
         (pivots > 1 ? al(N * 4) + al((N + (int64_t)BDG_TC_TILE * m) * 4) + al(N) : 0);
}

bdg_status bdg_build_csr(const uint64_t* codes, int64_t N, int W, const int32_t* routes, int m,
                         int t, int tile_v, int pivots, void* mem, bdg_csr* c,
                         cudaStream_t st) {
  if (m > kMaxSortM)
    return bdg_set_error(BDG_EUNSUPPORTED, "m = %d partitions exceeds %d", m, kMaxSortM);
  bdg_prof_scope prof("bucket", st);
  char* p = (char*)mem;
  const size_t ts = t > 1 ? (size_t)(t - 1) : 1;
  c->home_off = (int32_t*)p;   p += al((m + 1) * 4);
  c->visit_off = (int32_t*)p;  p += al(ts * (m + 1) * 4);
  c->item_off = (int32_t*)p;   p += al(ts * (m + 1) * 4);
  c->eoff = (int32_t*)p;       p += al((m + 1) * 4);
  c->home_ids = (int32_t*)p;   p += al(N * 4);
  c->home_codes = (uint64_t*)p; p += al(N * W * 8);
  c->visit_ids = (int32_t*)p;  p += al(N * t * 4);
  c->visit_slot = (int8_t*)p;  p += al(N * t);
  c->part_order = (int32_t*)p; p += al(m * 4);
  c->item_off_a = (int32_t*)p; p += al((m + 1) * 4);
  c->slot_zero = (int8_t*)p;   p += al(N);
  c->home_blocks = (int32_t*)p;
  p += al((size_t)((N + bdg_home_block(N, m) - 1) / bdg_home_block(N, m)) * m * 4);
  c->item_stride = bdg_csr_item_stride(N, m, tile_v);
  c->item_lo_a = (int32_t*)p;  p += al((size_t)c->item_stride * 4);
  c->item_lo = (int32_t*)p;    p += al(ts * (size_t)c->item_stride * 4);
  c->home_loc = c->loc_idr = nullptr;
  if (pivots > 1) {
    if (pivots > BDG_MAX_PIVOTS || (W != 4 && W != 8))
      return bdg_set_error(BDG_EINVAL, "locality order: %d pivots at %d-bit codes", pivots, 64 * W);
    c->home_loc = (int32_t*)p;   p += al(N * 4);
    c->loc_idr = (int32_t*)p;    p += al((N + (int64_t)BDG_TC_TILE * m) * 4);
  }
  int8_t* loc_key = pivots > 1 ? (int8_t*)p : nullptr;  // nearest pivot per home position
  if (pivots > 1) p += al(N);
  c->counters = (int32_t*)p;
  int32_t* hcnt = c->counters;
  int32_t* vcnt = c->counters + m;
  c->m = m;
  c->t = t;
  BDG_CUDA_TRY(cudaMemsetAsync(c->counters, 0, bdg_csr_counter_words(m, t) * 4, st));
  if (t == 1) {  // no sub-rounds: empty visit lists
    BDG_CUDA_TRY(cudaMemsetAsync(c->visit_off, 0, (m + 1) * 4, st));
    BDG_CUDA_TRY(cudaMemsetAsync(c->item_off, 0, (m + 1) * 4, st));
  }
  BDG_CUDA_TRY(cudaMemsetAsync(c->slot_zero, 0, N, st));
  const int g = bdg_cdiv(N, 256);
  // homes: stable, in id order
  const int bp = bdg_home_block(N, m);
  const int nblk = bdg_cdiv(N, bp);
  int32_t* bcnt = c->home_blocks;
  const size_t sm_m = (size_t)m * 4;
  BDG_CUDA_TRY(cudaFuncSetAttribute(home_block_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sm_m));
  BDG_CUDA_TRY(cudaFuncSetAttribute(home_place, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sm_m));
  home_block_count<<<nblk, 256, sm_m, st>>>(routes, N, t, m, bp, bcnt);
  BDG_CUDA_TRY(cudaGetLastError());
  home_block_scan<<<bdg_cdiv(m, 128), 128, 0, st>>>(m, nblk, bcnt, hcnt);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch(2);
  // visits of slots >= 1 (their order within a list does not matter)
  // points per aggregated block: a multiple of the block size, pts * (t - 1)
  // pairs at most kAggEntries
  const bool agg = t >= 2 && (int64_t)(t - 1) * m <= kAggBins;
  const int pts = agg ? std::max(kAggThreads, kAggEntries / (t - 1) / kAggThreads * kAggThreads) : 0;
  const int gagg = agg ? (int)bdg_cdiv(N, pts) : 0;
  if (agg)
    count_agg_kernel<<<gagg, kAggThreads, 0, st>>>(routes, N, t, m, pts, vcnt);
  else
    count_kernel<<<g, 256, 0, st>>>(routes, N, t, m, vcnt);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  int np2 = 1;
  while (np2 < m) np2 <<= 1;
  const size_t smem = (size_t)np2 * 8;
  BDG_CUDA_TRY(cudaFuncSetAttribute(plan_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  plan_kernel<<<1, kScanThreads, smem, st>>>(m, t, tile_v, hcnt, vcnt, c->home_off, c->visit_off,
                                             c->part_order, c->item_off, c->eoff,
                                             c->item_off_a);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  item_table_kernel<<<bdg_cdiv((int64_t)t * m, 128), 128, 0, st>>>(
      m, t, c->item_off_a, c->item_off, c->item_stride, c->item_lo_a, c->item_lo);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  home_place<<<nblk, 32, sm_m, st>>>(routes, N, t, m, bp, bcnt, c->home_off, c->home_ids);
  BDG_CUDA_TRY(cudaGetLastError());
  if (agg)
    scatter_agg_kernel<<<gagg, kAggThreads, 0, st>>>(routes, N, t, m, pts, vcnt, c->visit_ids,
                                                     c->visit_slot);
  else
    scatter_kernel<<<g, 256, 0, st>>>(routes, N, t, m, vcnt, c->visit_ids, c->visit_slot);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch(2);
  gather_home_codes<<<bdg_cdiv(N * W, 256), 256, 0, st>>>(codes, c->home_ids, c->home_off, m, N,
                                                          W, c->home_codes);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  if (pivots > 1) {
    const dim3 kgrid(m, 32);
    if (W == 4)
      pivot_key_kernel<4><<<kgrid, 256, 0, st>>>(c->home_codes, c->home_off, m, pivots, loc_key);
    else
      pivot_key_kernel<8><<<kgrid, 256, 0, st>>>(c->home_codes, c->home_off, m, pivots, loc_key);
    BDG_CUDA_TRY(cudaGetLastError());
    pivot_sort_kernel<<<m, 1024, 0, st>>>(loc_key, c->home_ids, c->home_off, c->eoff,
                                          c->home_loc, c->loc_idr);
    BDG_CUDA_TRY(cudaGetLastError());
    bdg_note_launch(2);
  }
  return BDG_OK;
}
