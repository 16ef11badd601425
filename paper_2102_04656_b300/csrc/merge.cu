// merge.cu -- (plus two small fill/gather utilities at the end)
// Shuffle 2 + Reduce 2 of Section 3.2: every point's t partial
// k-NN lists (one per routed partition, each sorted by (d, id), padded with
// the pad key) become its final k-NN row.
//
// The home sets are disjoint, so the valid keys of the t lists are distinct and
// every key's final rank is its index in its own list plus the number of
// smaller keys in the other lists (binary searches); ranks below k are written.
// One warp per point; the lists are staged in shared memory.
#include "common.cuh"

namespace {

constexpr int kWarps = 8;

__global__ void __launch_bounds__(kWarps * 32)
merge_kernel(const uint64_t* __restrict__ partial, int64_t N, int t, int k, int bits,
             int32_t* __restrict__ ids, int32_t* __restrict__ dist) {
  extern __shared__ uint64_t sl[];  // [kWarps][t * k]
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kWarps + warp;
  if (i >= N) return;
  uint64_t* L = sl + (size_t)warp * t * k;
  const uint64_t pad = bdg_pad_key(bits);
  const uint64_t* src = partial + i * t * k;
  for (int x = lane; x < t * k; x += 32) L[x] = src[x];
  __syncwarp();
  int valid = 0;  // total valid keys over the lists
  for (int s = 0; s < t; ++s) {
    int lo = 0, hi = k;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (L[s * k + mid] < pad) lo = mid + 1; else hi = mid;
    }
    valid += lo;
  }
  for (int x = lane; x < t * k; x += 32) {
    const uint64_t key = L[x];
    if (key >= pad) continue;
    const int s = x / k;
    int rank = x - s * k;
    for (int o = 0; o < t; ++o) {
      if (o == s) continue;
      const uint64_t* Lo = L + o * k;
      int lo = 0, hi = k;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (Lo[mid] < key) lo = mid + 1; else hi = mid;
      }
      rank += lo;
      if (rank >= k) break;
    }
    if (rank < k) {
      ids[i * k + rank] = bdg_key_id(key);
      dist[i * k + rank] = bdg_key_d(key);
    }
  }
  for (int r = valid + lane; r < k; r += 32) {
    ids[i * k + r] = -1;
    dist[i * k + r] = bits + 1;
  }
}

__global__ void fill_pad_kernel(int32_t* __restrict__ ids, int32_t* __restrict__ dist,
                                int64_t count, int bits) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= count) return;
  ids[x] = -1;
  dist[x] = bits + 1;
}

// rows[i] = codes[ids[i]]; ids outside [0, N) give a zero row
__global__ void gather_codes_kernel(const uint64_t* __restrict__ codes, int64_t N,
                                    const int32_t* __restrict__ ids, int64_t n, int W,
                                    uint64_t* __restrict__ rows) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n * W) return;
  const int64_t r = x / W;
  const int32_t id = ids[r];
  rows[x] = (id >= 0 && id < N) ? codes[(int64_t)id * W + (x - r * W)] : 0ull;
}

}  // namespace

bdg_status bdg_launch_gather_codes(const uint64_t* codes, int64_t N, const int32_t* ids, int64_t n,
                                   int W, uint64_t* rows, cudaStream_t st) {
  if (n == 0) return BDG_OK;
  gather_codes_kernel<<<bdg_cdiv(n * W, 256), 256, 0, st>>>(codes, N, ids, n, W, rows);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

bdg_status bdg_launch_fill_pad(int32_t* ids, int32_t* dist, int64_t count, int bits,
                               cudaStream_t st) {
  if (count == 0) return BDG_OK;
  fill_pad_kernel<<<bdg_cdiv(count, 256), 256, 0, st>>>(ids, dist, count, bits);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

bdg_status bdg_launch_merge(const uint64_t* partial, int64_t N, int t, int k, int bits,
                            int32_t* ids, int32_t* dist, cudaStream_t st) {
  if (N == 0) return BDG_OK;
  const size_t smem = (size_t)kWarps * t * k * 8;
  BDG_CUDA_TRY(cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  bdg_prof_scope prof("merge", st);
  merge_kernel<<<bdg_cdiv(N, kWarps), kWarps * 32, smem, st>>>(partial, N, t, k, bits, ids, dist);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}
