// shard.cu -- the merge step of a multi-shard search (Sections 3.4 and 4): every
// shard answered the query with its own sorted list of R (distance, local id)
// pairs; the answer is the first min(ef, R) of all shards' pairs by
// (distance, global id), global id = shard offset + local id. The same kernel
// merges the partial k-lists of a partition-sharded build (Shuffle 2 and
// Reduce 2 of Section 3.2): S lists of k keys per point, all offsets zero, the
// first k kept (ef == NULL).
//
// One warp per query. The S lists are staged in shared memory as keys
// (d << 32 | global id), padding as +inf; each valid key's place in the answer
// is its position in its own list plus, for every other list, the number of
// keys below it there (a binary search). Global ids differ between shards, so
// no two valid keys are equal and the places are distinct. No sequential merge
// chain: every lane places its keys independently.
#include "common.cuh"

namespace {

constexpr int kWarps = 4;

__device__ __forceinline__ int count_below(const uint64_t* list, int R, uint64_t key) {
  int lo = 0, hi = R;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (list[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kWarps * 32)
shard_merge_kernel(const int32_t* __restrict__ ids, const int32_t* __restrict__ dist, int S,
                   int64_t nq, int R, const __grid_constant__ bdg_shard_offsets off,
                   const int32_t* __restrict__ ef,
                   int ef_max, int bits, int fixed_r, int32_t* __restrict__ out_ids,
                   int32_t* __restrict__ out_dist) {
  extern __shared__ __align__(16) uint64_t merge_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t* keys = merge_smem + (size_t)warp * S * R;
  const int total = S * R;
  for (int64_t q = (int64_t)blockIdx.x * kWarps + warp; q < nq; q += (int64_t)gridDim.x * kWarps) {
    int valid = 0;
    for (int i0 = 0; i0 < total; i0 += 32) {  // warp-uniform trip count (ballot below)
      const int i = i0 + lane;
      bool ok = false;
      if (i < total) {
        const int s = i / R, r = i - s * R;
        const int64_t src = ((int64_t)s * nq + q) * R + r;
        const int32_t id = ids[src];
        ok = id >= 0;
        keys[i] = ok ? bdg_key((uint32_t)dist[src], (uint32_t)(off.off[s] + id)) : BDG_KEY_INF;
      }
      valid += __popc(__ballot_sync(0xffffffffu, ok));
    }
    __syncwarp();
    int rq;
    if (fixed_r > 0) {  // every row keeps its first fixed_r keys
      rq = min(fixed_r, valid);
    } else {
      const int e = ef[q];
      rq = (e >= 1 && e <= ef_max) ? min(min(e, R), valid) : 0;
    }
    for (int i = lane; i < total; i += 32) {
      const uint64_t key = keys[i];
      if (key == BDG_KEY_INF) continue;
      const int s = i / R;
      int place = i - s * R;
      for (int o = 0; o < S; ++o)
        if (o != s) place += count_below(keys + o * R, R, key);
      if (place < rq) {
        out_ids[q * R + place] = (int32_t)bdg_key_id(key);
        out_dist[q * R + place] = (int32_t)bdg_key_d(key);
      }
    }
    for (int p = rq + lane; p < R; p += 32) {
      out_ids[q * R + p] = -1;
      out_dist[q * R + p] = bits + 1;
    }
    __syncwarp();
  }
}

}  // namespace

size_t bdg_shard_merge_smem(int S, int R) { return (size_t)kWarps * S * R * 8; }

bdg_status bdg_launch_shard_merge(const int32_t* ids, const int32_t* dist, int S, int64_t nq,
                                  int R, const bdg_shard_offsets& off, const int32_t* ef,
                                  int ef_max, int bits, int32_t* out_ids, int32_t* out_dist,
                                  cudaStream_t st) {
  if (nq == 0) return BDG_OK;
  const size_t smem = bdg_shard_merge_smem(S, R);
  BDG_CUDA_TRY(cudaFuncSetAttribute(shard_merge_kernel,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  BDG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, shard_merge_kernel,
                                                             kWarps * 32, smem));
  if (per_sm < 1) per_sm = 1;
  const int64_t need = (nq + kWarps - 1) / kWarps;
  const int64_t cap = (int64_t)bdg_num_sms() * per_sm;
  const int grid = (int)(need < cap ? need : cap);
  bdg_prof_scope prof("shard_merge", st);
  shard_merge_kernel<<<grid, kWarps * 32, smem, st>>>(ids, dist, S, nq, R, off, ef, ef_max,
                                                       bits, ef ? 0 : R, out_ids, out_dist);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}
