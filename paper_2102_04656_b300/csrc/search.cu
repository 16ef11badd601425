// search.cu -- the search procedure of Section 3.5 on the GPU: long-link entry
// (nearest of a fixed random sample) followed by best-first hill climbing on
// the k-NN graph with a pool of the ef best keys (d(q, j), j), one warp per query.
//
// The pool is a sorted array in shared memory with an "expanded" flag per slot.
// Each step expands the best unexpanded pool entry: the warp loads its
// neighbour list (32 ids per coalesced load), each lane gathers one neighbour
// code and scores it, the accepted keys are sorted across the warp (bitonic)
// and merged into the pool by ranks.
//
// This reaches exactly the pool of the sequential procedure (candidate min-heap
// + bounded max-heap + visited set):
//  * the best unexpanded pool entry is the candidate heap's minimum whenever
//    the sequential loop would not stop, and no unexpanded entry is left exactly
//    when it stops (evicted candidates are worse than every pool entry, and the
//    pool's worst key only decreases once the pool is full);
//  * adding a whole neighbour list at once gives the best ef of (pool + list),
//    which is what adding the neighbours one by one gives;
//  * a node already seen is either still in the pool (found by binary search and
//    skipped) or worse than the pool's worst key for good (rejected again), so a
//    visited set is only a saving, not a condition of correctness. A small
//    per-warp hash of seen ids avoids most re-gathers; when it is full, ids are
//    simply re-scored.
#include "common.cuh"


namespace {

constexpr int kWarps = 4;
// visited-id hash slots per warp (2^bits): a small table (256) leaves room for
// more warps per SM, which hides more gather latency than the re-scores it
// causes cost; pools above 1,024 keys (~2,000 expansions x 32 neighbours per
// query) take 2,048 slots: with 256 nearly every neighbour was re-scored
template <int CAPW>
struct HashOf { static constexpr int bits = CAPW >= 64 ? 11 : 8; };
constexpr int kProbe = 8;
constexpr int kSmallBatch = 8;  // accepted keys ranked by counting instead of a sort

template <int CAPW>
struct PoolSmem {
  static constexpr int HASH = 1 << HashOf<CAPW>::bits;
  uint64_t key[CAPW * 32];
  uint8_t expd[CAPW * 32];
  uint64_t nk[32];
  int32_t hash[HASH];
};

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a < b ? b : a; }

// Records id in the per-warp visited hash. Returns kNew if it was not there
// (recorded now), kSeen if it was, kFull if its probe window is full (not
// recorded: the id is re-scored and checked against the pool).
constexpr int kNew = 0, kSeen = 1, kFull = 2;
template <int HBITS>
__device__ __forceinline__ int hash_visit(int32_t* h, int32_t id) {
  constexpr int kH = 1 << HBITS;
  uint32_t x = (uint32_t)id * 2654435761u;
  uint32_t slot = x >> (32 - HBITS);
  for (int p = 0; p < kProbe; ++p) {
    const uint32_t sidx = (slot + p) & (kH - 1);
    const int32_t old = atomicCAS(&h[sidx], -1, id);
    if (old == -1) return kNew;
    if (old == id) return kSeen;
  }
  return kFull;
}

// PACKED: the neighbours' codes are read from g.nbr_codes (compiled apart so that
// each layout gets its own register allocation)
template <int W, int CAPW, bool PACKED>
__global__ void __launch_bounds__(kWarps * 32)
search_kernel(bdg_graph_view g, const uint64_t* __restrict__ queries, int64_t nq,
              const int32_t* __restrict__ efs, int R, int32_t* __restrict__ out_ids,
              int32_t* __restrict__ out_dist, int32_t* __restrict__ expansions) {
  constexpr int CAP = CAPW * 32;
  extern __shared__ __align__(16) char search_smem[];
  PoolSmem<CAPW>* sm_all = reinterpret_cast<PoolSmem<CAPW>*>(search_smem);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  PoolSmem<CAPW>& sm = sm_all[warp];
  const uint64_t pad = bdg_pad_key(g.bits);

  for (int64_t q = (int64_t)blockIdx.x * kWarps + warp; q < nq; q += (int64_t)gridDim.x * kWarps) {
    const int ef = efs[q];
    if (ef < 1 || ef > CAP) {
      for (int r = lane; r < R; r += 32) {
        out_ids[q * R + r] = -1;
        out_dist[q * R + r] = g.bits + 1;
      }
      if (expansions && lane == 0) expansions[q] = -1;
      continue;
    }
    uint64_t y[W];
#pragma unroll
    for (int w = 0; w < W; ++w) y[w] = queries[q * W + w];
    for (int x = lane; x < PoolSmem<CAPW>::HASH; x += 32) sm.hash[x] = -1;

    // long-link entry: nearest sampled point by (d, id)
    uint64_t best = BDG_KEY_INF;
    for (int s = lane; s < g.n_entry; s += 32) {
      const int32_t e = g.entry[s];
      if (e < 0 || e >= g.n) continue;  // ids outside the graph are ignored
      uint32_t d = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) d += __popcll(y[w] ^ g.entry_codes[(int64_t)s * W + w]);
      best = umin64(best, bdg_key(d, (uint32_t)e));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = umin64(best, __shfl_xor_sync(0xffffffffu, best, o));
    __syncwarp();
    if (best == BDG_KEY_INF) {  // no valid entry point: an empty result
      for (int r = lane; r < R; r += 32) {
        out_ids[q * R + r] = -1;
        out_dist[q * R + r] = g.bits + 1;
      }
      if (expansions && lane == 0) expansions[q] = 0;
      continue;
    }
    if (lane == 0) {
      sm.key[0] = best;
      sm.expd[0] = 0;
      hash_visit<HashOf<CAPW>::bits>(sm.hash, bdg_key_id(best));
    }
    int size = 1, hint = 0, nexp = 0;
    // speculation: while a node is expanded, the neighbour list of the next
    // unexpanded pool entry is loaded (and its codes prefetched); it is used if
    // that entry is still the one expanded next
    int32_t spec_node = -1, spec_nb = -1;
    __syncwarp();

    for (;;) {
      // first unexpanded slot at or after `hint`, and the one after it
      int slot = -1, slot2 = -1;
      for (int b = hint & ~31; b < size; b += 32) {
        const int j = b + lane;
        unsigned m = __ballot_sync(0xffffffffu, j < size && !sm.expd[j]);
        if (slot < 0 && m) {
          slot = b + __ffs(m) - 1;
          m &= m - 1;
        }
        if (slot >= 0 && m) { slot2 = b + __ffs(m) - 1; break; }
      }
      if (slot < 0) break;
      hint = slot + 1;
      const uint64_t ck = sm.key[slot];
      const int32_t node2 = slot2 >= 0 ? bdg_key_id(sm.key[slot2]) : -1;
      __syncwarp();
      if (lane == 0) sm.expd[slot] = 1;
      ++nexp;
      const int32_t node = bdg_key_id(ck);
      const bool use_spec = node == spec_node;
      const int32_t cur_spec_nb = spec_nb;
      if (g.deg <= 32) {  // load the next candidate's list now; its codes are prefetched below
        spec_node = node2;
        spec_nb = (node2 >= 0 && lane < g.deg) ? g.ids[(int64_t)node2 * g.deg + lane] : -1;
      }
      for (int b0 = 0; b0 < g.deg; b0 += 32) {
        const int32_t nb = use_spec ? cur_spec_nb
                         : (b0 + lane < g.deg) ? g.ids[(int64_t)node * g.deg + b0 + lane] : -1;
        // with the packed layout the neighbour's code sits next to the row: its
        // address depends on the node only, so it is loaded together with the id
        uint64_t pc[W];
        if (PACKED && b0 + lane < g.deg) {
          const uint64_t* src = g.nbr_codes + ((int64_t)node * g.deg + b0 + lane) * W;
          if constexpr (W % 2 == 0) {
#pragma unroll
            for (int w = 0; w < W / 2; ++w) {
              const ulonglong2 u = reinterpret_cast<const ulonglong2*>(src)[w];
              pc[2 * w] = u.x;
              pc[2 * w + 1] = u.y;
            }
          } else {
#pragma unroll
            for (int w = 0; w < W; ++w) pc[w] = src[w];
          }
        }
        uint64_t key = BDG_KEY_INF;
        bool acc = false;
        const int hv = (nb >= 0 && nb < g.n) ? hash_visit<HashOf<CAPW>::bits>(sm.hash, nb) : kSeen;
        if (hv != kSeen) {
          uint32_t d = 0;
          if constexpr (PACKED) {
#pragma unroll
            for (int w = 0; w < W; ++w) d += __popcll(y[w] ^ pc[w]);
          } else {
#pragma unroll
            for (int w = 0; w < W; ++w) d += __popcll(y[w] ^ g.codes[(int64_t)nb * W + w]);
          }
          key = bdg_key(d, (uint32_t)nb);
          const uint64_t worst = sm.key[size - 1];
          acc = (size < ef) || (key < worst);
          // every pool entry was recorded in the hash when it entered, unless its
          // window was full: only an id the hash could not record may be a duplicate
          if (acc && hv == kFull) {  // already in the pool?
            int lo = 0, hi = size;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (sm.key[mid] < key) lo = mid + 1; else hi = mid;
            }
            acc = !(lo < size && sm.key[lo] == key);
          }
        }
        const unsigned am = __ballot_sync(0xffffffffu, acc);
        if (am == 0) continue;
        const int na = __popc(am);
        uint64_t v;
        if (na <= kSmallBatch) {
          // few accepted keys: each finds its rank by comparing with the others
          int rank = 0;
          for (unsigned mm = am; mm; mm &= mm - 1) {
            const int src = __ffs(mm) - 1;
            const uint64_t o = __shfl_sync(0xffffffffu, key, src);
            rank += (o < key) || (o == key && src < lane);  // an id listed twice
          }
          if (acc) sm.nk[rank] = key;
          __syncwarp();
          v = lane < na ? sm.nk[lane] : BDG_KEY_INF;
        } else {
          // sort accepted keys ascending across the warp (rejected = +inf)
          v = acc ? key : BDG_KEY_INF;
#pragma unroll
          for (int k2 = 2; k2 <= 32; k2 <<= 1) {
#pragma unroll
            for (int j = k2 >> 1; j > 0; j >>= 1) {
              const uint64_t o = __shfl_xor_sync(0xffffffffu, v, j);
              const bool up = (lane & k2) == 0;
              const bool low = (lane & j) == 0;
              v = (low == up) ? umin64(v, o) : umax64(v, o);
            }
          }
          sm.nk[lane] = v;
          __syncwarp();
        }
        // new key positions: own rank + rank in the pool
        int newpos = CAP;
        if (lane < na) {
          int lo = 0, hi = size;
          while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sm.key[mid] < v) lo = mid + 1; else hi = mid;
          }
          newpos = lane + lo;
        }
        // pool entries at or after the first new position shift right by the
        // number of smaller new keys; entries before it stay in place. Chunks of
        // 32 slots move top-down, so no entry is overwritten before it is read
        // (an entry only moves up, and the final positions are all distinct).
        const int minpos = (int)__reduce_min_sync(0xffffffffu, (unsigned)newpos);
        for (int base = (size - 1) & ~31; base >= (minpos & ~31); base -= 32) {
          const int j = base + lane;
          uint64_t pk = 0;
          uint8_t pf = 0;
          int pp = CAP;
          if (j >= minpos && j < size) {
            pk = sm.key[j];
            pf = sm.expd[j];
            int lo = 0;
            if (na <= kSmallBatch) {
              for (int i = 0; i < na; ++i) lo += (sm.nk[i] < pk);
            } else {
              int hi = na;
              while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (sm.nk[mid] < pk) lo = mid + 1; else hi = mid;
              }
            }
            pp = j + lo;
          }
          __syncwarp();
          if (pp < ef) { sm.key[pp] = pk; sm.expd[pp] = pf; }
          __syncwarp();
        }
        if (newpos < ef) { sm.key[newpos] = v; sm.expd[newpos] = 0; }
        size = min(ef, size + na);
        hint = min(hint, minpos);
        __syncwarp();
      }
      // codes of the speculated next list: into L2 while the pool is scanned
      if constexpr (PACKED) {
        if (spec_node >= 0 && lane < g.deg)
          asm volatile("prefetch.L2 [%0];" ::"l"(g.nbr_codes +
                                                 ((int64_t)spec_node * g.deg + lane) * W));
      } else {
        if (spec_nb >= 0 && spec_nb < g.n)
          asm volatile("prefetch.L2 [%0];" ::"l"(g.codes + (int64_t)spec_nb * W));
      }
    }
    const int keep = min(size, R);
    for (int r = lane; r < R; r += 32) {
      const uint64_t kk = r < keep ? sm.key[r] : pad;
      out_ids[q * R + r] = r < keep ? bdg_key_id(kk) : -1;
      out_dist[q * R + r] = bdg_key_d(kk);
    }
    if (expansions && lane == 0) expansions[q] = nexp;
    __syncwarp();
  }
}

template <int W, int CAPW, bool PACKED>
bdg_status launch_packed(const bdg_graph_view& g, const uint64_t* queries, int64_t nq,
                      const int32_t* ef, int R, int32_t* out_ids, int32_t* out_dist,
                      int32_t* expansions, cudaStream_t st) {
  const size_t smem = sizeof(PoolSmem<CAPW>) * kWarps;
  BDG_CUDA_TRY(cudaFuncSetAttribute(search_kernel<W, CAPW, PACKED>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  BDG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_kernel<W, CAPW, PACKED>,
                                                             kWarps * 32, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (nq + kWarps - 1) / kWarps;
  const int64_t cap = (int64_t)bdg_num_sms() * per_sm;
  const int grid = (int)(need < cap ? need : cap);
  bdg_prof_scope prof("search", st);
  search_kernel<W, CAPW, PACKED><<<grid, kWarps * 32, smem, st>>>(g, queries, nq, ef, R, out_ids, out_dist,
                                                       expansions);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

template <int W, int CAPW>
bdg_status launch_cap(const bdg_graph_view& g, const uint64_t* queries, int64_t nq,
                      const int32_t* ef, int R, int32_t* out_ids, int32_t* out_dist,
                      int32_t* expansions, cudaStream_t st) {
  if (g.nbr_codes != nullptr)
    return launch_packed<W, CAPW, true>(g, queries, nq, ef, R, out_ids, out_dist, expansions, st);
  return launch_packed<W, CAPW, false>(g, queries, nq, ef, R, out_ids, out_dist, expansions, st);
}

template <int W>
bdg_status launch_w(const bdg_graph_view& g, const uint64_t* queries, int64_t nq,
                    const int32_t* ef, int ef_max, int R, int32_t* out_ids, int32_t* out_dist,
                    int32_t* expansions, cudaStream_t st) {
  if (ef_max <= 64) return launch_cap<W, 2>(g, queries, nq, ef, R, out_ids, out_dist, expansions, st);
  if (ef_max <= 128) return launch_cap<W, 4>(g, queries, nq, ef, R, out_ids, out_dist, expansions, st);
  if (ef_max <= 256) return launch_cap<W, 8>(g, queries, nq, ef, R, out_ids, out_dist, expansions, st);
  if (ef_max <= 512) return launch_cap<W, 16>(g, queries, nq, ef, R, out_ids, out_dist, expansions, st);
  if (ef_max <= 1024) return launch_cap<W, 32>(g, queries, nq, ef, R, out_ids, out_dist, expansions, st);
  if (ef_max <= 1536) return launch_cap<W, 48>(g, queries, nq, ef, R, out_ids, out_dist, expansions, st);
  return launch_cap<W, 64>(g, queries, nq, ef, R, out_ids, out_dist, expansions, st);
}

}  // namespace

bdg_status bdg_launch_search(const bdg_graph_view& g, const uint64_t* queries, int64_t nq,
                             const int32_t* ef, int ef_max, int R, int32_t* out_ids,
                             int32_t* out_dist, int32_t* expansions, cudaStream_t st) {
  if (nq == 0) return BDG_OK;
  const int W = g.bits / 64;
  BDG_DISPATCH_W(W, launch_w, g, queries, nq, ef, ef_max, R, out_ids, out_dist, expansions, st);
}
