// merge.cu -- the end of Shuffle 2 + Reduce 2 of Section 3.2, plus two small
// utilities. The Reduce-1 kernels already merge every sub-round's rows into a
// running k-list per point as they write them (bdg_warp_merge_running: the home
// sets are disjoint, so the valid keys of the lists are distinct and a key's
// final rank is its index plus the number of smaller keys in the other list);
// what remains is turning the running keys into graph rows.
#include "common.cuh"

namespace {

// running keys -> graph rows: ids and distances, (bits + 1, -1) past the valid keys
__global__ void finalize_kernel(const uint64_t* __restrict__ running, int64_t n, int bits,
                                int32_t* __restrict__ ids, int32_t* __restrict__ dist) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const uint64_t key = running[x];
  const bool valid = key < bdg_pad_key(bits);
  ids[x] = valid ? bdg_key_id(key) : -1;
  dist[x] = valid ? bdg_key_d(key) : bits + 1;
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

bdg_status bdg_launch_finalize(const uint64_t* running, int64_t N, int k, int bits, int32_t* ids,
                               int32_t* dist, cudaStream_t st) {
  const int64_t n = N * (int64_t)k;
  if (n == 0) return BDG_OK;
  bdg_prof_scope prof("merge", st);
  finalize_kernel<<<bdg_cdiv(n, 256), 256, 0, st>>>(running, n, bits, ids, dist);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}
