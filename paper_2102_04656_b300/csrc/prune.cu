// prune.cu -- graph pruning of Section 3.4 after FANNG's occlusion rule
// (Harwood and Drummond, CVPR 2016), one warp per point.
//
// The candidates of x are the ids of its row (invalid ids, x itself and repeats
// dropped) in (d(x, y), y) order; y is kept unless a neighbour z kept before it
// is strictly closer to y than x is, and at most L are kept. Per warp:
//   * every lane loads the codes of up to four candidates (16-byte loads) into
//     shared memory (rows padded by one word against bank conflicts) and forms
//     its key (d(x, y), y);
//   * ranks by counting give each first occurrence of a key its position in
//     (d, id) order (repeats of an id share the key and only the first is
//     placed; positions left empty by them are skipped);
//   * a warp-uniform walk takes the candidates in that order; each lane tests
//     one or two of the kept neighbours (d(z, y) against d(x, y)) and one ballot
//     decides. Only kept neighbours are tested, so a row costs at most
//     k * L distances, not k^2 / 2.
// Bytes: the row (4 k), the candidates' codes (8 W k, random rows), the own
// code and the pruned row out (8 L): bound by the code gathers.
#include "common.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kMaxK = 128;
constexpr int kMaxL = 64;

template <int W>
struct PruneSmem {
  static constexpr int kRow = W + 1;  // padded code row (u64 words)
  uint64_t codes[kMaxK * kRow];
  uint64_t keys[kMaxK];
  int16_t order[kMaxK];
  int16_t kept[kMaxL];
};

template <int W>
__global__ void __launch_bounds__(kWarps * 32)
prune_kernel(const uint64_t* __restrict__ codes, int64_t n, int k, int L, int bits,
             const int32_t* __restrict__ ids_in, int32_t* __restrict__ ids_out,
             int32_t* __restrict__ dist_out) {
  using Sm = PruneSmem<W>;
  constexpr int kRow = Sm::kRow;
  extern __shared__ __align__(16) char prune_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  Sm& sm = reinterpret_cast<Sm*>(prune_smem)[warp];
  constexpr int kB = kMaxK / 32;
  const int nb = (k + 31) >> 5;
  for (int64_t x = (int64_t)blockIdx.x * kWarps + warp; x < n; x += (int64_t)gridDim.x * kWarps) {
    uint64_t cx[W];
#pragma unroll
    for (int w = 0; w < W; ++w) cx[w] = codes[x * W + w];
    // candidates: codes into shared memory, keys (d, id)
    uint64_t key[kB];
#pragma unroll
    for (int q = 0; q < kB; ++q) {
      key[q] = BDG_KEY_INF;
      const int a = q * 32 + lane;
      if (q < nb && a < k) {
        const int32_t y = ids_in[x * k + a];
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
            sm.codes[a * kRow + w] = v[w];
            d += __popcll(v[w] ^ cx[w]);
          }
          key[q] = bdg_key(d, (uint32_t)y);
        }
        sm.keys[a] = key[q];
        sm.order[a] = -1;
      }
    }
    __syncwarp();
    // position in (d, id) order = number of smaller keys; a repeat of an earlier
    // key is not placed
#pragma unroll
    for (int q = 0; q < kB; ++q) {
      const int a = q * 32 + lane;
      if (q < nb && a < k && key[q] != BDG_KEY_INF) {
        int rank = 0;
        bool dup = false;
        for (int b = 0; b < k; ++b) {
          const uint64_t o = sm.keys[b];
          rank += o < key[q];
          dup |= (o == key[q]) & (b < a);
        }
        if (!dup) sm.order[rank] = (int16_t)a;
      }
    }
    __syncwarp();
    // the walk
    int nk = 0;
    for (int r = 0; r < k && nk < L; ++r) {
      const int a = sm.order[r];
      if (a < 0) continue;
      const uint32_t dxy = bdg_key_d(sm.keys[a]);
      bool occ = false;
      for (int e = lane; e < nk; e += 32) {
        const int z = sm.kept[e];
        uint32_t d = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) d += __popcll(sm.codes[z * kRow + w] ^ sm.codes[a * kRow + w]);
        occ |= d < dxy;
      }
      if (__ballot_sync(0xffffffffu, occ) == 0) {
        if (lane == 0) sm.kept[nk] = (int16_t)a;
        ++nk;
        __syncwarp();
      }
    }
    __syncwarp();
    for (int e = lane; e < L; e += 32) {
      const uint64_t kk = e < nk ? sm.keys[sm.kept[e]] : 0;
      ids_out[x * L + e] = e < nk ? (int32_t)bdg_key_id(kk) : -1;
      dist_out[x * L + e] = e < nk ? (int32_t)bdg_key_d(kk) : bits + 1;
    }
    __syncwarp();
  }
}

template <int W>
bdg_status launch_w(const uint64_t* codes, int64_t n, int k, int L, int bits,
                    const int32_t* ids_in, int32_t* ids_out, int32_t* dist_out,
                    cudaStream_t st) {
  const size_t smem = sizeof(PruneSmem<W>) * kWarps;
  BDG_CUDA_TRY(cudaFuncSetAttribute(prune_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  int per_sm = 0;
  BDG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, prune_kernel<W>,
                                                             kWarps * 32, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (n + kWarps - 1) / kWarps;
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
