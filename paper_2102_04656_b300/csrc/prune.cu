// prune.cu -- graph pruning of Section 3.4 after FANNG's occlusion rule
// (Harwood and Drummond, CVPR 2016).
//
// The candidates of x are the ids of its row (invalid ids, x itself and repeats
// dropped) in (d(x, y), y) order; y is kept unless a neighbour z kept before it
// is strictly closer to y than x is, and at most L are kept.
//
// A group of G lanes handles one point (32 / G points per warp; G grows with the
// code width so that the per-point shared memory stays small):
//   * the group loads the row, the candidates' codes (16-byte loads) into
//     shared memory (rows padded by one word against bank conflicts) and their
//     keys (d(x, y), y);
//   * a row already in strict (d, id) order (every row this library builds) is
//     walked as it is; any other row is ranked by counting (repeats of an id
//     share the key and only the first is placed);
//   * the walk takes the candidates in order, all groups of the warp in step;
//     each lane of a group tests every G-th kept neighbour (d(z, y) against
//     d(x, y)) and one ballot decides. Only kept neighbours are tested, so a row
//     costs at most k * L distances.
// Bytes: the row (4 k), the candidates' codes (8 W k, random rows), the own
// code and the pruned row out (8 L): bound by the code gathers.
#include "common.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kMaxK = 128;
constexpr int kMaxL = 64;

template <int W>
struct PruneCfg {
  // lanes per point, measured: 16 up to 512-bit codes (10M x 256-bit, k = 32: 4, 8, 16,
  // 32 lanes took 26.7, 21.2, 19.8, 34.1 ms; 2M x 512-bit, k = 64: 8, 16, 32 took 22.6,
  // 17.8, 19.3 ms), 32 above
  static constexpr int G = W <= 8 ? 16 : 32;
  static constexpr int kPts = 32 / G;                           // points per warp
  static constexpr int kRow = W + 1;                            // padded code row (words)
};

// Shared memory of one point, in 8-byte words: codes [kc][W + 1], keys [kc],
// then walk order [kc] and kept slots [L] as int16 (kc = k rounded up to even).
__host__ __device__ inline size_t point_words(int k, int W, int L) {
  const int kc = (k + 1) & ~1;
  return (size_t)kc * (W + 1) + kc + (kc + L + 3) / 4;
}

template <int W>
__global__ void __launch_bounds__(kWarps * 32)
prune_kernel(const uint64_t* __restrict__ codes, int64_t n, int k, int L, int bits,
             const int32_t* __restrict__ ids_in, int32_t* __restrict__ ids_out,
             int32_t* __restrict__ dist_out) {
  using C = PruneCfg<W>;
  constexpr int G = C::G, kPts = C::kPts, kRow = C::kRow;
  extern __shared__ __align__(16) uint64_t prune_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / G, lg = lane % G;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
  const int kc = (k + 1) & ~1;
  uint64_t* pcodes = prune_smem + ((size_t)warp * kPts + grp) * point_words(k, W, L);
  uint64_t* pkeys = pcodes + (size_t)kc * kRow;
  int16_t* porder = reinterpret_cast<int16_t*>(pkeys + kc);
  int16_t* pkept = porder + kc;
  const int64_t stride = (int64_t)gridDim.x * kWarps * kPts;
  for (int64_t x0 = ((int64_t)blockIdx.x * kWarps + warp) * kPts; x0 < n; x0 += stride) {
    const int64_t x = x0 + grp;
    const bool live = x < n;
    uint64_t cx[W];
#pragma unroll
    for (int w = 0; w < W; ++w) cx[w] = live ? codes[x * W + w] : 0;
    // candidates: codes into shared memory, keys (d, id)
    for (int a = lg; a < k; a += G) {
      uint64_t key = BDG_KEY_INF;
      const int32_t y = live ? ids_in[x * k + a] : -1;
      if (y >= 0 && y < n && y != x) {
        uint64_t v[W];
        if constexpr (W % 2 == 0) {  // 16-byte loads of the code row
          const ulonglong2* src = reinterpret_cast<const ulonglong2*>(codes + (int64_t)y * W);
#pragma unroll
          for (int w = 0; w < W / 2; ++w) {
            const ulonglong2 u = src[w];
            v[2 * w] = u.x;
            v[2 * w + 1] = u.y;
          }
        } else {
#pragma unroll
          for (int w = 0; w < W; ++w) v[w] = codes[(int64_t)y * W + w];
        }
        uint32_t d = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          pcodes[a * kRow + w] = v[w];
          d += __popcll(v[w] ^ cx[w]);
        }
        key = bdg_key(d, (uint32_t)y);
      }
      pkeys[a] = key;
    }
    __syncwarp();
    // is the row already in strict (d, id) order, padding last?
    bool in_order = true;
    for (int a = lg; a < k; a += G) {
      const uint64_t key = pkeys[a];
      in_order &= key == BDG_KEY_INF || a == 0 || pkeys[a - 1] < key;
      porder[a] = -1;
    }
    for (int e = lg; e < L; e += G) pkept[e] = 0;  // every slot index below stays in range
    const bool sorted = (__ballot_sync(0xffffffffu, !in_order) & gmask) == 0;
    __syncwarp();
    // walk order: the row itself, or positions by counting (a repeat of an
    // earlier key is not placed)
    for (int a = lg; a < k; a += G) {
      const uint64_t key = pkeys[a];
      if (key == BDG_KEY_INF) continue;
      if (sorted) {
        porder[a] = (int16_t)a;
        continue;
      }
      int rank = 0;
      bool dup = false;
      for (int b = 0; b < k; ++b) {
        const uint64_t o = pkeys[b];
        rank += o < key;
        dup |= (o == key) & (b < a);
      }
      if (!dup) porder[rank] = (int16_t)a;
    }
    __syncwarp();
    // the walk, every group of the warp in step
    int nk = 0;
    for (int r = 0; r < k; ++r) {
      const int a = porder[r];
      const bool act = a >= 0 && nk < L;
      const int as = a < 0 ? 0 : a;  // an in-range slot even where it is not used
      bool occ = false;
      if (act) {
        const uint32_t dxy = bdg_key_d(pkeys[as]);
        uint64_t yv[W];
#pragma unroll
        for (int w = 0; w < W; ++w) yv[w] = pcodes[as * kRow + w];
        for (int e = lg; e < nk; e += G) {
          const int z = pkept[e];
          uint32_t d = 0;
#pragma unroll
          for (int w = 0; w < W; ++w) d += __popcll(pcodes[z * kRow + w] ^ yv[w]);
          occ |= d < dxy;
        }
      }
      // every lane takes part in the ballot, whatever its group is doing
      const unsigned bal = __ballot_sync(0xffffffffu, occ);
      const bool keep = act && (bal & gmask) == 0;
      if (keep) {
        if (lg == 0) pkept[nk] = (int16_t)a;
        ++nk;
      }
      __syncwarp();
    }
    if (live) {
      for (int e = lg; e < L; e += G) {
        const uint64_t kk = pkeys[e < nk ? pkept[e] : 0];
        ids_out[x * L + e] = e < nk ? (int32_t)bdg_key_id(kk) : -1;
        dist_out[x * L + e] = e < nk ? (int32_t)bdg_key_d(kk) : bits + 1;
      }
    }
    __syncwarp();
  }
}

template <int W>
bdg_status launch_w(const uint64_t* codes, int64_t n, int k, int L, int bits,
                    const int32_t* ids_in, int32_t* ids_out, int32_t* dist_out,
                    cudaStream_t st) {
  const size_t smem = point_words(k, W, L) * 8 * PruneCfg<W>::kPts * kWarps;
  BDG_CUDA_TRY(cudaFuncSetAttribute(prune_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int per_sm = 0;
  BDG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, prune_kernel<W>,
                                                             kWarps * 32, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t per_block = (int64_t)kWarps * PruneCfg<W>::kPts;
  const int64_t need = (n + per_block - 1) / per_block;
  const int64_t cap = (int64_t)bdg_num_sms() * per_sm;
  const int grid = (int)(need < cap ? need : cap);
  bdg_prof_scope prof("prune", st);
  prune_kernel<W><<<grid, kWarps * 32, smem, st>>>(codes, n, k, L, bits, ids_in, ids_out,
                                                    dist_out);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

}  // namespace

int bdg_prune_max_k() { return kMaxK; }
int bdg_prune_max_l() { return kMaxL; }

bdg_status bdg_launch_prune(const uint64_t* codes, int64_t n, int W, int k, int L,
                            const int32_t* ids_in, int32_t* ids_out, int32_t* dist_out,
                            cudaStream_t st) {
  if (n == 0) return BDG_OK;
  BDG_DISPATCH_W(W, launch_w, codes, n, k, L, 64 * W, ids_in, ids_out, dist_out, st);
}
