// rerank.cu -- the real-valued re-rank of Section 3.5 (d = l2 of Section 3):
// the binary candidates recalled by the graph search are re-scored by squared
// Euclidean distance of their float32 features to the query's, and the best k
// by (distance, id) are kept.
//
// One warp per query. The query vector lives in registers (D / 32 floats per
// lane, 16-byte loads); candidate rows are read 512 B per warp-wide load
// (coalesced, 4 candidates in flight per warp), reduced across lanes by
// butterfly shuffles, and inserted into a warp-wide sorted top-k held one entry
// per lane. HBM-bound: R * D * 4 bytes per query.
#include "common.cuh"


namespace {

constexpr int kWarps = 8;
constexpr int kBatch = 4;  // candidates scored per warp iteration

// Insert (s, id) into the sorted warp list (lane r holds the r-th best).
__device__ __forceinline__ void topk_insert(float& ls, int32_t& li, float s, int32_t id, int k,
                                            int lane) {
  const bool less = (ls < s) || (ls == s && li < id);  // entry r precedes the new one
  const unsigned before = __ballot_sync(0xffffffffu, lane < k && less);
  const int pos = __popc(before);
  if (pos >= k) return;
  const float ps = __shfl_up_sync(0xffffffffu, ls, 1);
  const int32_t pi = __shfl_up_sync(0xffffffffu, li, 1);
  if (lane > pos) { ls = ps; li = pi; }
  if (lane == pos) { ls = s; li = id; }
}

template <int V4>  // float4 per lane: D = 128 * V4
__global__ void __launch_bounds__(kWarps * 32)
rerank_kernel(const float* __restrict__ feats, int64_t N, const float* __restrict__ qfeats,
              const int32_t* __restrict__ cand, int64_t nq, int R, int k,
              int32_t* __restrict__ out_ids, float* __restrict__ out_d2) {
  constexpr int D = 128 * V4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int64_t q = (int64_t)blockIdx.x * kWarps + warp; q < nq; q += (int64_t)gridDim.x * kWarps) {
    float4 qv[V4];
#pragma unroll
    for (int u = 0; u < V4; ++u)
      qv[u] = reinterpret_cast<const float4*>(qfeats + q * D)[u * 32 + lane];
    float ls = __int_as_float(0x7f800000);  // +inf
    int32_t li = 0x7fffffff;
    for (int r0 = 0; r0 < R; r0 += kBatch) {
      int32_t id[kBatch];
      float s[kBatch];
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        id[b] = (r0 + b < R) ? cand[q * R + r0 + b] : -1;
        s[b] = 0.f;
      }
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
        if (id[b] >= 0 && id[b] < N) {
          const float4* row = reinterpret_cast<const float4*>(feats + (int64_t)id[b] * D);
#pragma unroll
          for (int u = 0; u < V4; ++u) {
            const float4 x = row[u * 32 + lane];
            const float d0 = qv[u].x - x.x, d1 = qv[u].y - x.y, d2 = qv[u].z - x.z,
                        d3 = qv[u].w - x.w;
            s[b] = fmaf(d0, d0, s[b]);
            s[b] = fmaf(d1, d1, s[b]);
            s[b] = fmaf(d2, d2, s[b]);
            s[b] = fmaf(d3, d3, s[b]);
          }
        }
      }
#pragma unroll
      for (int b = 0; b < kBatch; ++b) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s[b] += __shfl_xor_sync(0xffffffffu, s[b], o);
      }
#pragma unroll
      for (int b = 0; b < kBatch; ++b)
        if (id[b] >= 0 && id[b] < N) topk_insert(ls, li, s[b], id[b], k, lane);
    }
    if (lane < k) {
      const bool valid = li != 0x7fffffff;
      out_ids[q * k + lane] = valid ? li : -1;
      out_d2[q * k + lane] = ls;
    }
  }
}

template <int V4>
bdg_status launch_v(const float* feats, int64_t N, const float* qfeats, const int32_t* cand,
                    int64_t nq, int R, int k, int32_t* out_ids, float* out_d2, cudaStream_t st) {
  const int64_t need = (nq + kWarps - 1) / kWarps;
  const int64_t cap = (int64_t)bdg_num_sms() * 8;
  const int grid = (int)(need < cap ? need : cap);
  bdg_prof_scope prof("rerank", st);
  rerank_kernel<V4><<<grid, kWarps * 32, 0, st>>>(feats, N, qfeats, cand, nq, R, k, out_ids, out_d2);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

}  // namespace

bdg_status bdg_launch_rerank(const float* feats, int64_t N, int D, const float* qfeats,
                             const int32_t* cand, int64_t nq, int R, int k, int32_t* out_ids,
                             float* out_d2, cudaStream_t st) {
  if (nq == 0) return BDG_OK;
  switch (D) {
    case 128: return launch_v<1>(feats, N, qfeats, cand, nq, R, k, out_ids, out_d2, st);
    case 256: return launch_v<2>(feats, N, qfeats, cand, nq, R, k, out_ids, out_d2, st);
    case 512: return launch_v<4>(feats, N, qfeats, cand, nq, R, k, out_ids, out_d2, st);
    case 1024: return launch_v<8>(feats, N, qfeats, cand, nq, R, k, out_ids, out_d2, st);
    default:
      return bdg_set_error(BDG_EUNSUPPORTED, "feature dimension %d not built (128/256/512/1024)", D);
  }
}
