// mlp.cu -- the learned partition router: a BF16 MLP d_in -> h1 -> h2 -> m with
// FP32 accumulation, trained on the GPU with hand-written forward and backward
// kernels, that picks the partitions a point is compared against. The paper
// routes every point to its t nearest binary centres (Section 3.2); the router
// keeps that nearest centre as the home and replaces the other t - 1 probes by
// the partitions where the point's neighbours are predicted to live.
//
//   h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2), z = [h2 | s] W3^T + b3
// where s in {-1, +1}^cb is the point's code (cb = 0: no code input). Through
// the code columns of W3 the logits can carry the Hamming prior of the method's
// own routing: with W3 = [0 | c_p / 2] and b3 = 0, z_p = bits / 2 - d(y, c_p),
// whose top-P order is exactly the nearest-centre order (ties by p).
//   loss = -(1/B) sum_i sum_p q_ip log softmax(z_i)_p,
//   q_ip = #{labels of i equal to p} / #{valid labels of i}
// (a row without a valid label contributes neither loss nor gradient)
// Gradients by the chain rule (all products on the tcgen05 BF16 GEMM of
// gemm_tc.cu with fused bias / ReLU / ReLU-mask / bias-gradient epilogues),
// Adam with FP32 master weights and BF16 working copies.
//
// BF16 is stored exactly where the network's tensors are stored: the inputs,
// the weight copies, h1, h2, the logit gradient and the hidden-layer
// gradients; bias gradients are summed from the FP32 values before rounding.
#include <cuda_bf16.h>

#include <cmath>

#include "common.cuh"


struct bdg_router {
  int d_in, h1, h2, m;
  int cb;            // code bits appended to h2 as +-1 inputs of the last layer (0 = none)
  int h2s;           // h2 + cb: row length of the last layer's input
  int64_t n_params;
  float* w;          // fp32 master, packed W1 b1 W2 b2 W3 b3
  float* grad;       // same layout: gradients of the last training step
  float* adam_m;
  float* adam_v;
  __nv_bfloat16* wb; // bf16 copies of W1, W2, W3 (packed, no biases)
  int64_t step;
  int32_t* err;
  float* loss;       // device scalar: loss of the last step
  // training workspace for batches up to cap_b rows (h2 rows are h2s long)
  int cap_b;
  void* ws;
  size_t ws_bytes;
};

namespace {

inline size_t al(size_t b) { return (b + 255) & ~size_t(255); }

struct Offs {
  int64_t W1, b1, W2, b2, W3, b3, n;
};
// W3 is m x h2s (h2s = h2 + cb)
Offs param_offsets(int d_in, int h1, int h2, int h2s, int m) {
  Offs o;
  o.W1 = 0;
  o.b1 = o.W1 + (int64_t)h1 * d_in;
  o.W2 = o.b1 + h1;
  o.b2 = o.W2 + (int64_t)h2 * h1;
  o.W3 = o.b2 + h2;
  o.b3 = o.W3 + (int64_t)m * h2s;
  o.n = o.b3 + m;
  return o;
}

__global__ void f32_to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b,
                            int64_t n) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < n) b[x] = __float2bfloat16_rn(a[x]);
}

// out[c][r] = in[r][c] for a rows x cols bf16 matrix (32 x 32 tiles)
__global__ void transpose_bf16(const __nv_bfloat16* __restrict__ in, int rows, int cols,
                               __nv_bfloat16* __restrict__ out) {
  __shared__ __nv_bfloat16 t[32][33];
  const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[(int64_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(int64_t)c * rows + r] = t[threadIdx.x][i];
  }
}

// out[i][col0 + b] = +1 if bit b of code i is set, else -1 (BF16), for i < rows
__global__ void code_pm_bf16(const uint64_t* __restrict__ codes, int64_t rows, int W,
                             __nv_bfloat16* __restrict__ out, int ld, int col0) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int bits = 64 * W;
  if (x >= rows * bits) return;
  const int64_t i = x / bits;
  const int b = (int)(x - i * bits);
  const uint64_t w = codes[i * W + (b >> 6)];
  out[i * ld + col0 + b] = __float2bfloat16_rn(((w >> (b & 63)) & 1ull) ? 1.f : -1.f);
}

// Softmax cross-entropy against the neighbour-partition targets, one block per
// row: dz = (softmax(z) - q) / B as FP32 and BF16, loss accumulated. With
// `exclude`, partition exclude[i] is left out of row i's softmax (it gets
// probability 0 and gradient 0; its labels are ignored).
__global__ void __launch_bounds__(256)
softmax_ce(const float* __restrict__ z, int m, int B, const int32_t* __restrict__ labels, int kt,
           const int32_t* __restrict__ exclude, float* __restrict__ dz32,
           __nv_bfloat16* __restrict__ dz16, float* __restrict__ loss) {
  const int i = blockIdx.x;
  const float* zr = z + (int64_t)i * m;
  const int ex = exclude ? exclude[i] : -1;
  __shared__ float red[32];
  __shared__ float s_max, s_sum;
  float mx = -INFINITY;
  for (int p = threadIdx.x; p < m; p += blockDim.x)
    if (p != ex) mx = fmaxf(mx, zr[p]);
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = fmaxf(v, red[w]);
    s_max = v;
  }
  __syncthreads();
  const float zmax = s_max;
  float sum = 0.f;
  for (int p = threadIdx.x; p < m; p += blockDim.x)
    if (p != ex) sum += expf(zr[p] - zmax);
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float v = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[w];
    s_sum = v;
  }
  __syncthreads();
  const float lse = zmax + logf(s_sum);
  const int32_t* lab = labels + (int64_t)i * kt;
  int nval = 0;  // labels inside [0, m): the row's target is their empirical distribution
  for (int j = 0; j < kt; ++j) nval += (lab[j] >= 0 && lab[j] < m && lab[j] != ex);
  const float inv_b = 1.f / (float)B;
  float* dzr = dz32 + (int64_t)i * m;
  if (nval == 0) {  // no target: the row contributes neither loss nor gradient
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
      dzr[p] = 0.f;
      dz16[(int64_t)i * m + p] = __float2bfloat16_rn(0.f);
    }
    return;
  }
  const float inv_k = 1.f / (float)nval;
  for (int p = threadIdx.x; p < m; p += blockDim.x)
    dzr[p] = p == ex ? 0.f : expf(zr[p] - lse) * inv_b;
  __syncthreads();
  for (int j = threadIdx.x; j < kt; j += blockDim.x) {
    const int32_t p = lab[j];
    if (p >= 0 && p < m && p != ex) atomicAdd(&dzr[p], -inv_k * inv_b);  // - q_ip / B
  }
  __syncthreads();
  for (int p = threadIdx.x; p < m; p += blockDim.x)
    dz16[(int64_t)i * m + p] = __float2bfloat16_rn(dzr[p]);
  if (threadIdx.x == 0) {
    float l = 0.f;
    for (int j = 0; j < kt; ++j)
      if (lab[j] >= 0 && lab[j] < m && lab[j] != ex) l -= inv_k * (zr[lab[j]] - lse);
    atomicAdd(loss, l * inv_b);
  }
}

__global__ void colsum_f32(const float* __restrict__ a, int rows, int cols,
                           float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += a[(int64_t)r * cols + c];
  out[c] = s;
}

__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ mom, float* __restrict__ vel, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const float gx = g[x];
  const float mm = b1 * mom[x] + (1.f - b1) * gx;
  const float vv = b2 * vel[x] + (1.f - b2) * gx * gx;
  mom[x] = mm;
  vel[x] = vv;
  w[x] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// Partition choice per row: slot 0 = the given home, then the P - 1 best other
// partitions by (-logit, p). One warp per row; each lane keeps its best P - 1
// candidates and the warp pops the best across lanes P - 1 times.
constexpr int kMaxP = 16;
__device__ __forceinline__ bool better(float a, int pa, float b, int pb) {
  return a > b || (a == b && pa < pb);
}
__global__ void topp_kernel(const float* __restrict__ z, int rows, int m,
                            const int32_t* __restrict__ home, int P, int32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= rows) return;
  const float* zr = z + (int64_t)i * m;
  const int hm = home[i];
  const int need = P - 1;
  float bv[kMaxP];
  int bp[kMaxP];
#pragma unroll
  for (int s = 0; s < kMaxP; ++s) { bv[s] = -INFINITY; bp[s] = 0x7fffffff; }
  float wv = -INFINITY;  // the lane's current worst kept entry (slot need - 1)
  int wpp = 0x7fffffff;
  for (int p = lane; p < m && need > 0; p += 32) {
    if (p == hm) continue;
    const float v = zr[p];
    if (!better(v, p, wv, wpp)) continue;
#pragma unroll
    for (int s = kMaxP - 1; s >= 0; --s) {
      if (s < need && better(v, p, bv[s], bp[s])) {
        const int sp = s > 0 ? s - 1 : 0;
        if (s > 0 && better(v, p, bv[sp], bp[sp])) { bv[s] = bv[sp]; bp[s] = bp[sp]; }
        else { bv[s] = v; bp[s] = p; }
      }
    }
#pragma unroll
    for (int s = 0; s < kMaxP; ++s)
      if (s == need - 1) { wv = bv[s]; wpp = bp[s]; }
  }
  if (lane == 0) out[(int64_t)i * P] = hm;
  int head = 0;  // next unused entry of this lane's list
  for (int r = 0; r < need; ++r) {
    float v = -INFINITY;
    int p = 0x7fffffff;
#pragma unroll
    for (int s = 0; s < kMaxP; ++s)
      if (s == head) { v = bv[s]; p = bp[s]; }
    float bvw = v;
    int bpw = p;
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bvw, o);
      const int op = __shfl_xor_sync(0xffffffffu, bpw, o);
      if (better(ov, op, bvw, bpw)) { bvw = ov; bpw = op; }
    }
    if (p == bpw) ++head;
    if (lane == 0) out[(int64_t)i * P + 1 + r] = bpw;
  }
}

// ---------------------------------------------------------------------------
// Shortlist head: the last layer evaluated only on each point's shortlist of
// Q candidate partitions (its Q nearest centres, slot 0 = its home; -1 = none):
//   z_ij = [h2_i | s_i] . W3[cand_ij] + b3[cand_ij],
// softmax cross-entropy over the shortlist against q_ij = the share of the
// point's labels (homes of its exact neighbours) naming cand_ij among its labels
// found in the shortlist, and the probe choice: the home, then the other
// shortlisted partitions within theta of the largest shortlisted logit, by
// (-z, partition), at most pmax - 1 of them. One warp per point; the point's
// input row u = [h2 | s] (BF16) stays in registers, W3 rows are read from L2 in
// 16-byte chunks (8 BF16 values), products accumulate in FP32.
constexpr int kMaxQ = 16;
constexpr int kUChunks = 8;  // 16-byte chunks of u per lane: rows up to 8 * 32 * 8 = 2048 values

__device__ __forceinline__ float dot8(const uint4& a, const uint4& b) {
  const __nv_bfloat162* x = reinterpret_cast<const __nv_bfloat162*>(&a);
  const __nv_bfloat162* y = reinterpret_cast<const __nv_bfloat162*>(&b);
  float acc = 0.f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const float2 fx = __bfloat1622float2(x[e]), fy = __bfloat1622float2(y[e]);
    acc = fmaf(fx.x, fy.x, acc);
    acc = fmaf(fx.y, fy.y, acc);
  }
  return acc;
}

// z[j] of one row for j < Q (every lane ends with every value); the row's u
// chunks are loaded into uc
__device__ __forceinline__ void head_logits(const __nv_bfloat16* __restrict__ urow, int nch,
                                            const __nv_bfloat16* __restrict__ W3, int h2s,
                                            const float* __restrict__ b3,
                                            const int32_t* __restrict__ cand, int Q, int lane,
                                            uint4 (&uc)[kUChunks], float (&z)[kMaxQ]) {
#pragma unroll
  for (int q = 0; q < kUChunks; ++q) {
    const int c = lane + 32 * q;
    uc[q] = c < nch ? reinterpret_cast<const uint4*>(urow)[c] : make_uint4(0, 0, 0, 0);
  }
#pragma unroll
  for (int j = 0; j < kMaxQ; ++j) {
    z[j] = -INFINITY;
    if (j >= Q) continue;
    const int32_t p = cand[j];
    if (p < 0) continue;
    const uint4* wr = reinterpret_cast<const uint4*>(W3 + (int64_t)p * h2s);
    float acc = 0.f;
#pragma unroll
    for (int q = 0; q < kUChunks; ++q) {
      const int c = lane + 32 * q;
      if (c < nch) acc += dot8(uc[q], wr[c]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    z[j] = acc + b3[p];
  }
}

// Inference head: UC 16-byte chunks of u per lane (u held as FP32 in registers),
// a candidate's W3 chunks requested before its products are summed, and the
// probe choice made by all lanes at once (lane j ranks candidate j).
template <int UC>
__global__ void __launch_bounds__(256)
head_route_kernel(const __nv_bfloat16* __restrict__ u, int h2s,
                  const __nv_bfloat16* __restrict__ W3, const float* __restrict__ b3,
                  const int32_t* __restrict__ cand, int Q, int rows, float* __restrict__ z_out,
                  float theta, int pmax, int32_t* __restrict__ routes,
                  const int32_t* __restrict__ out_row, int64_t n_out) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= rows) return;
  // the output row of this input row (out_row: a processing order's rows)
  const int64_t orow = out_row ? (int64_t)out_row[i] : (int64_t)i;
  if (orow < 0 || orow >= n_out) return;
  const int nch = h2s / 8;
  const int32_t* cr = cand + (int64_t)i * Q;
  const int32_t myp = lane < Q ? cr[lane] : -1;  // lane j's candidate
  float uf[UC][8];
  {
    const uint4* urow = reinterpret_cast<const uint4*>(u + (int64_t)i * h2s);
#pragma unroll
    for (int q = 0; q < UC; ++q) {
      const int c = lane + 32 * q;
      const uint4 x = c < nch ? urow[c] : make_uint4(0, 0, 0, 0);
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&x);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(h[e]);
        uf[q][2 * e] = f.x;
        uf[q][2 * e + 1] = f.y;
      }
    }
  }
  float zl = -INFINITY;  // lane j ends with z_j
  for (int j0 = 0; j0 < Q; j0 += 2) {  // two candidates' W3 rows in flight at once
    int32_t p2[2];
    uint4 w[2][UC];
#pragma unroll
    for (int u2 = 0; u2 < 2; ++u2) {
      const int j = j0 + u2;
      p2[u2] = __shfl_sync(0xffffffffu, myp, j < Q ? j : 0);
      if (j >= Q) p2[u2] = -1;
      const uint4* wr = reinterpret_cast<const uint4*>(W3 + (int64_t)(p2[u2] < 0 ? 0 : p2[u2]) * h2s);
#pragma unroll
      for (int q = 0; q < UC; ++q) {
        const int c = lane + 32 * q;
        w[u2][q] = (p2[u2] >= 0 && c < nch) ? wr[c] : make_uint4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int u2 = 0; u2 < 2; ++u2) {
      float acc = 0.f;
#pragma unroll
      for (int q = 0; q < UC; ++q) {
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&w[u2][q]);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float2 f = __bfloat1622float2(h[e]);
          acc = fmaf(uf[q][2 * e], f.x, acc);
          acc = fmaf(uf[q][2 * e + 1], f.y, acc);
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (p2[u2] >= 0 && lane == j0 + u2) zl = acc + b3[p2[u2]];
    }
  }
  if (z_out && lane < Q) z_out[orow * Q + lane] = zl;
  if (routes == nullptr) return;
  // probe choice: the home, then the others within theta of the best, by (-z, p)
  float zmax = myp >= 0 ? zl : -INFINITY;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) zmax = fmaxf(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
  const float thr = zmax - theta;
  const bool kept = lane >= 1 && myp >= 0 && zl >= thr;
  int rank = 0;  // kept candidates ahead of this one
  for (int j = 1; j < Q; ++j) {
    const float zj = __shfl_sync(0xffffffffu, zl, j);
    const int32_t pj = __shfl_sync(0xffffffffu, myp, j);
    const bool kj = pj >= 0 && zj >= thr;
    rank += (kj && (zj > zl || (zj == zl && pj < myp))) ? 1 : 0;
  }
  const int nkept = __popc(__ballot_sync(0xffffffffu, kept));
  int32_t* out = routes + orow * pmax;
  if (lane == 0) out[0] = myp;
  if (kept && rank < pmax - 1) out[1 + rank] = myp;
  if (lane >= nkept && lane < pmax - 1) out[1 + lane] = -1;
}

// dst[j] = src[idx[j]] for rows of row_words 32-bit words; an index outside
// [0, n_src) gives a zero row
__global__ void gather_words(const uint32_t* __restrict__ src, int64_t n_src, int row_words,
                             const int32_t* __restrict__ idx, int64_t n,
                             uint32_t* __restrict__ dst) {
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n * row_words) return;
  const int64_t j = x / row_words;
  const int w = (int)(x - j * row_words);
  const int32_t r = idx[j];
  dst[x] = (r >= 0 && r < n_src) ? src[(int64_t)r * row_words + w] : 0u;
}

bdg_status gather_rows_words(const void* src, int64_t n_src, int row_words, const int32_t* idx,
                             int64_t n, void* dst, cudaStream_t st) {
  if (n == 0) return BDG_OK;
  gather_words<<<bdg_cdiv(n * row_words, 256), 256, 0, st>>>(
      (const uint32_t*)src, n_src, row_words, idx, n, (uint32_t*)dst);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

bdg_status launch_head_route(const __nv_bfloat16* u, int h2s, const __nv_bfloat16* W3,
                             const float* b3, const int32_t* cand, int Q, int rows, float* z_out,
                             float theta, int pmax, int32_t* routes, cudaStream_t st,
                             const int32_t* out_row = nullptr, int64_t n_out = -1) {
  const int uc = (h2s / 8 + 31) / 32;
  const int grid = bdg_cdiv(rows, 8);
  if (n_out < 0) n_out = rows;
  if (uc <= 1)
    head_route_kernel<1><<<grid, 256, 0, st>>>(u, h2s, W3, b3, cand, Q, rows, z_out, theta, pmax, routes, out_row, n_out);
  else if (uc <= 2)
    head_route_kernel<2><<<grid, 256, 0, st>>>(u, h2s, W3, b3, cand, Q, rows, z_out, theta, pmax, routes, out_row, n_out);
  else if (uc <= 3)
    head_route_kernel<3><<<grid, 256, 0, st>>>(u, h2s, W3, b3, cand, Q, rows, z_out, theta, pmax, routes, out_row, n_out);
  else if (uc <= 4)
    head_route_kernel<4><<<grid, 256, 0, st>>>(u, h2s, W3, b3, cand, Q, rows, z_out, theta, pmax, routes, out_row, n_out);
  else
    head_route_kernel<8><<<grid, 256, 0, st>>>(u, h2s, W3, b3, cand, Q, rows, z_out, theta, pmax, routes, out_row, n_out);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

// Shortlist cross-entropy and its backward through the last layer, one warp per
// row: dz_j = (softmax_j - q_j) / B (FP32); dW3[cand_j] += dz_j u, db3[cand_j] +=
// dz_j (FP32 atomics); dh2 = (sum_j dz_j W3[cand_j][:h2]) * [h2 > 0], written as
// BF16 for the layer-2 GEMMs and summed (FP32) into db2.
__global__ void __launch_bounds__(256)
head_bwd_kernel(const __nv_bfloat16* __restrict__ u, int h2s, int h2,
                const __nv_bfloat16* __restrict__ W3, const float* __restrict__ b3,
                const int32_t* __restrict__ cand, int Q, const int32_t* __restrict__ labels,
                int kt, int B, float* __restrict__ gW3, float* __restrict__ gb3,
                float* __restrict__ gb2, __nv_bfloat16* __restrict__ dh2,
                float* __restrict__ loss) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= B) return;
  const int32_t* cr = cand + (int64_t)i * Q;
  const int nch = h2s / 8, nch2 = h2 / 8;
  uint4 uc[kUChunks];
  float z[kMaxQ];
  head_logits(u + (int64_t)i * h2s, nch, W3, h2s, b3, cr, Q, lane, uc, z);
  // targets: labels found in the shortlist, counted per slot
  int32_t cp[kMaxQ];
#pragma unroll
  for (int j = 0; j < kMaxQ; ++j) cp[j] = j < Q ? cr[j] : -1;
  float cnt[kMaxQ];
#pragma unroll
  for (int j = 0; j < kMaxQ; ++j) cnt[j] = 0.f;
  for (int l = lane; l < kt; l += 32) {
    const int32_t lab = labels[(int64_t)i * kt + l];
#pragma unroll
    for (int j = 0; j < kMaxQ; ++j) cnt[j] += (cp[j] >= 0 && lab == cp[j]) ? 1.f : 0.f;
  }
  float hits = 0.f;
#pragma unroll
  for (int j = 0; j < kMaxQ; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) cnt[j] += __shfl_xor_sync(0xffffffffu, cnt[j], o);
    hits += cnt[j];
  }
  __nv_bfloat16* drow = dh2 + (int64_t)i * h2;
  if (hits == 0.f) {  // no target: neither loss nor gradient
    for (int c = lane; c < h2; c += 32) drow[c] = __float2bfloat16_rn(0.f);
    return;
  }
  float zmax = -INFINITY;
#pragma unroll
  for (int j = 0; j < kMaxQ; ++j)
    if (cp[j] >= 0) zmax = fmaxf(zmax, z[j]);
  float sum = 0.f;
#pragma unroll
  for (int j = 0; j < kMaxQ; ++j)
    if (cp[j] >= 0) sum += expf(z[j] - zmax);
  const float lse = zmax + logf(sum);
  const float inv_b = 1.f / (float)B;
  float dz[kMaxQ];
  float l = 0.f;
#pragma unroll
  for (int j = 0; j < kMaxQ; ++j) {
    dz[j] = 0.f;
    if (cp[j] < 0) continue;
    const float qj = cnt[j] / hits;
    dz[j] = (expf(z[j] - lse) - qj) * inv_b;
    if (qj > 0.f) l -= qj * (z[j] - lse);
  }
  if (lane == 0) atomicAdd(loss, l * inv_b);
  // last layer: bias and weight gradients of every shortlisted row of W3
#pragma unroll
  for (int j = 0; j < kMaxQ; ++j) {
    if (cp[j] < 0) continue;
    if (lane == 0) atomicAdd(&gb3[cp[j]], dz[j]);
    float4* gr = reinterpret_cast<float4*>(gW3 + (int64_t)cp[j] * h2s);
#pragma unroll
    for (int q = 0; q < kUChunks; ++q) {
      const int c = lane + 32 * q;
      if (c >= nch) continue;
      const __nv_bfloat162* x = reinterpret_cast<const __nv_bfloat162*>(&uc[q]);
      const float2 a0 = __bfloat1622float2(x[0]), a1 = __bfloat1622float2(x[1]);
      const float2 a2 = __bfloat1622float2(x[2]), a3 = __bfloat1622float2(x[3]);
      atomicAdd(&gr[2 * c], make_float4(dz[j] * a0.x, dz[j] * a0.y, dz[j] * a1.x, dz[j] * a1.y));
      atomicAdd(&gr[2 * c + 1], make_float4(dz[j] * a2.x, dz[j] * a2.y, dz[j] * a3.x, dz[j] * a3.y));
    }
  }
  // hidden gradient through the h2 columns of the shortlisted rows, ReLU mask
#pragma unroll
  for (int q = 0; q < kUChunks; ++q) {
    const int c = lane + 32 * q;
    if (c >= nch2) continue;
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0.f;
#pragma unroll
    for (int j = 0; j < kMaxQ; ++j) {
      if (cp[j] < 0) continue;
      const uint4 w = reinterpret_cast<const uint4*>(W3 + (int64_t)cp[j] * h2s)[c];
      const __nv_bfloat162* wv = reinterpret_cast<const __nv_bfloat162*>(&w);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float2 f = __bfloat1622float2(wv[e]);
        acc[2 * e] = fmaf(dz[j], f.x, acc[2 * e]);
        acc[2 * e + 1] = fmaf(dz[j], f.y, acc[2 * e + 1]);
      }
    }
    const __nv_bfloat162* hv = reinterpret_cast<const __nv_bfloat162*>(&uc[q]);
    __align__(16) __nv_bfloat16 outv[8];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const float2 h = __bfloat1622float2(hv[e]);
      const float d0 = h.x > 0.f ? acc[2 * e] : 0.f;
      const float d1 = h.y > 0.f ? acc[2 * e + 1] : 0.f;
      atomicAdd(&gb2[8 * c + 2 * e], d0);
      atomicAdd(&gb2[8 * c + 2 * e + 1], d1);
      outv[2 * e] = __float2bfloat16_rn(d0);
      outv[2 * e + 1] = __float2bfloat16_rn(d1);
    }
    reinterpret_cast<uint4*>(drow)[c] = *reinterpret_cast<const uint4*>(outv);
  }
}

}  // namespace

extern "C" {

bdg_status bdg_router_create(int32_t d_in, int32_t h1, int32_t h2, int32_t m, int32_t code_bits,
                             const float* init_params, int32_t max_batch, bdg_router** out) {
  if (!out) return bdg_set_error(BDG_EINVAL, "router_create: out is NULL");
  *out = nullptr;
  if (d_in < 8 || h1 < 8 || h2 < 8 || m < 2 || (d_in & 7) || (h1 & 7) || (h2 & 7) || (m & 7) ||
      max_batch < 8 || (max_batch & 7) || !init_params)
    return bdg_set_error(BDG_EINVAL,
                         "router_create: sizes must be multiples of 8 (d_in=%d h1=%d h2=%d m=%d "
                         "max_batch=%d) and init_params given", d_in, h1, h2, m, max_batch);
  if (code_bits < 0 || code_bits > 1024 || (code_bits & 63))
    return bdg_set_error(BDG_EINVAL, "router_create: code_bits = %d (0 or 64..1024, multiple of 64)",
                         code_bits);
  const int h2s = h2 + code_bits;
  const Offs o = param_offsets(d_in, h1, h2, h2s, m);
  bdg_router* r = new bdg_router();
  r->d_in = d_in; r->h1 = h1; r->h2 = h2; r->m = m; r->n_params = o.n; r->cap_b = max_batch;
  r->cb = code_bits; r->h2s = h2s;
  const int64_t nw = (int64_t)h1 * d_in + (int64_t)h2 * h1 + (int64_t)m * h2s;
  const int64_t B = max_batch;
  // workspace: h1, [h2 | s] (bf16), z (f32), dz32, dz16, transposes, dh1, dh2
  r->ws_bytes = al(B * h1 * 2) + al(B * h2s * 2) + al(B * m * 4) * 2 + al(B * m * 2) +
                al(B * m * 2) /* dzT */ + al(B * h2s * 2) /* h2T */ + al(B * h2 * 2) /* dh2 */ +
                al(B * h1 * 2) * 2 /* h1T, dh1 */ + al(B * d_in * 2) /* xT */ +
                al(B * h2 * 2) /* dh2T */ + al(B * h1 * 2) /* dh1T */ +
                al((int64_t)h2s * m * 2) /* W3T */ + al((int64_t)h1 * h2 * 2) /* W2T */;
  cudaError_t e = cudaSuccess;
  e = e == cudaSuccess ? cudaMalloc(&r->w, o.n * 4) : e;
  e = e == cudaSuccess ? cudaMalloc(&r->grad, o.n * 4) : e;
  e = e == cudaSuccess ? cudaMalloc(&r->adam_m, o.n * 4) : e;
  e = e == cudaSuccess ? cudaMalloc(&r->adam_v, o.n * 4) : e;
  e = e == cudaSuccess ? cudaMalloc(&r->wb, nw * 2) : e;
  e = e == cudaSuccess ? cudaMalloc(&r->err, 64) : e;
  e = e == cudaSuccess ? cudaMalloc(&r->loss, 64) : e;
  e = e == cudaSuccess ? cudaMalloc(&r->ws, r->ws_bytes) : e;
  if (e != cudaSuccess) {
    cudaGetLastError();
    bdg_router_free(r);
    return bdg_set_error(BDG_ENOMEM, "router_create: device allocation failed");
  }
  cudaMemcpy(r->w, init_params, o.n * 4, cudaMemcpyDeviceToDevice);
  cudaMemset(r->grad, 0, o.n * 4);
  cudaMemset(r->adam_m, 0, o.n * 4);
  cudaMemset(r->adam_v, 0, o.n * 4);
  cudaMemset(r->err, 0, 64);
  cudaMemset(r->loss, 0, 64);
  // bf16 working copies
  f32_to_bf16<<<bdg_cdiv((int64_t)h1 * d_in, 256), 256>>>(r->w + o.W1, r->wb, (int64_t)h1 * d_in);
  f32_to_bf16<<<bdg_cdiv((int64_t)h2 * h1, 256), 256>>>(r->w + o.W2, r->wb + (int64_t)h1 * d_in,
                                                         (int64_t)h2 * h1);
  f32_to_bf16<<<bdg_cdiv((int64_t)m * h2s, 256), 256>>>(
      r->w + o.W3, r->wb + (int64_t)h1 * d_in + (int64_t)h2 * h1, (int64_t)m * h2s);
  bdg_note_launch(3);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    bdg_router_free(r);
    return bdg_set_error(BDG_ECUDA, "router_create: initialisation failed");
  }
  *out = r;
  return BDG_OK;
}

void bdg_router_free(bdg_router* r) {
  if (!r) return;
  cudaFree(r->w); cudaFree(r->grad); cudaFree(r->adam_m); cudaFree(r->adam_v);
  cudaFree(r->wb); cudaFree(r->err); cudaFree(r->loss); cudaFree(r->ws);
  delete r;
}

bdg_status bdg_router_info(const bdg_router* r, float** params, float** grads, int64_t* n_params,
                           float** loss, int32_t** err) {
  if (!r) return bdg_set_error(BDG_EINVAL, "router is NULL");
  if (params) *params = r->w;
  if (grads) *grads = r->grad;
  if (n_params) *n_params = r->n_params;
  if (loss) *loss = r->loss;
  if (err) *err = r->err;
  return BDG_OK;
}

// Hidden layers into caller-provided buffers: h1b [B][h1], h2b [B][h2s] (h2,
// then the +-1 code).
static bdg_status router_hidden(bdg_router* r, const void* x, const uint64_t* codes, int B,
                                void* h1b, void* h2b, cudaStream_t st) {
  const Offs o = param_offsets(r->d_in, r->h1, r->h2, r->h2s, r->m);
  const __nv_bfloat16* W1 = r->wb;
  const __nv_bfloat16* W2 = W1 + (int64_t)r->h1 * r->d_in;
  BDG_TRY(bdg_gemm_bf16_ld(x, W1, B, r->h1, r->d_in, r->w + o.b1, nullptr, r->h1, 1, nullptr,
                           h1b, r->h1, nullptr, r->err, st));
  BDG_TRY(bdg_gemm_bf16_ld(h1b, W2, B, r->h2, r->h1, r->w + o.b2, nullptr, r->h2, 1, nullptr,
                           h2b, r->h2s, nullptr, r->err, st));
  if (r->cb) {
    const int64_t n = (int64_t)B * r->cb;
    code_pm_bf16<<<bdg_cdiv(n, 256), 256, 0, st>>>(codes, B, r->cb / 64, (__nv_bfloat16*)h2b,
                                                   r->h2s, r->h2);
    BDG_CUDA_TRY(cudaGetLastError());
    bdg_note_launch();
  }
  return BDG_OK;
}

// Forward pass into caller-provided buffers: h1b [B][h1], h2b [B][h2s], z [B][m].
static bdg_status router_fwd(bdg_router* r, const void* x, const uint64_t* codes, int B, float* z,
                             void* h1b, void* h2b, cudaStream_t st) {
  const Offs o = param_offsets(r->d_in, r->h1, r->h2, r->h2s, r->m);
  const __nv_bfloat16* W3 = r->wb + (int64_t)r->h1 * r->d_in + (int64_t)r->h2 * r->h1;
  BDG_TRY(router_hidden(r, x, codes, B, h1b, h2b, st));
  BDG_TRY(bdg_gemm_bf16_ld(h2b, W3, B, r->m, r->h2s, r->w + o.b3, nullptr, r->m, 0, z, nullptr,
                           r->m, nullptr, r->err, st));
  return BDG_OK;
}

// One Adam step on the FP32 master weights from r->grad, then fresh BF16 copies.
static bdg_status router_adam(bdg_router* r, float lr, cudaStream_t st) {
  const int d = r->d_in, H1 = r->h1, H2 = r->h2, H2S = r->h2s, m = r->m;
  const Offs o = param_offsets(d, H1, H2, H2S, m);
  r->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)r->step), c2 = 1.f - powf(b2, (float)r->step);
  adam_kernel<<<bdg_cdiv(r->n_params, 256), 256, 0, st>>>(r->w, r->grad, r->adam_m, r->adam_v,
                                                          r->n_params, lr, b1, b2, 1e-8f, c1, c2);
  bdg_note_launch();
  f32_to_bf16<<<bdg_cdiv((int64_t)H1 * d, 256), 256, 0, st>>>(r->w + o.W1, r->wb,
                                                              (int64_t)H1 * d);
  f32_to_bf16<<<bdg_cdiv((int64_t)H2 * H1, 256), 256, 0, st>>>(
      r->w + o.W2, r->wb + (int64_t)H1 * d, (int64_t)H2 * H1);
  f32_to_bf16<<<bdg_cdiv((int64_t)m * H2S, 256), 256, 0, st>>>(
      r->w + o.W3, r->wb + (int64_t)H1 * d + (int64_t)H2 * H1, (int64_t)m * H2S);
  bdg_note_launch(3);
  BDG_CUDA_TRY(cudaGetLastError());
  return BDG_OK;
}

bdg_status bdg_router_forward(bdg_router* r, const void* x, const uint64_t* codes, int32_t B,
                              float* logits, void* stream) {
  if (!r || !x || !logits || B < 1 || B > r->cap_b || (r->cb && !codes))
    return bdg_set_error(BDG_EINVAL, "router_forward: B = %d (1..%d)%s", B, r ? r->cap_b : 0,
                         r && r->cb && !codes ? ", codes required" : "");
  cudaStream_t st = (cudaStream_t)stream;
  char* p = (char*)r->ws;
  void* h1b = p; p += al((int64_t)r->cap_b * r->h1 * 2);
  void* h2b = p;
  return router_fwd(r, x, codes, B, logits, h1b, h2b, st);
}

bdg_status bdg_router_train_step(bdg_router* r, const void* x, const uint64_t* codes,
                                 const int32_t* labels, int32_t kt, const int32_t* exclude,
                                 int32_t B, float lr, int32_t apply_update, void* stream) {
  if (!r || !x || !labels || B < 8 || B > r->cap_b || (B & 7) || kt < 1 || (r->cb && !codes))
    return bdg_set_error(BDG_EINVAL,
                         "router_train_step: B = %d (8..%d, multiple of 8), kt = %d%s", B,
                         r ? r->cap_b : 0, kt, r && r->cb && !codes ? ", codes required" : "");
  cudaStream_t st = (cudaStream_t)stream;
  const int d = r->d_in, H1 = r->h1, H2 = r->h2, H2S = r->h2s, m = r->m;
  const int64_t cap = r->cap_b;
  const Offs o = param_offsets(d, H1, H2, H2S, m);
  char* p = (char*)r->ws;
  __nv_bfloat16* h1b = (__nv_bfloat16*)p; p += al(cap * H1 * 2);
  __nv_bfloat16* h2b = (__nv_bfloat16*)p; p += al(cap * H2S * 2);
  float* z = (float*)p;                   p += al(cap * m * 4);
  float* dz32 = (float*)p;                p += al(cap * m * 4);
  __nv_bfloat16* dz16 = (__nv_bfloat16*)p; p += al(cap * m * 2);
  __nv_bfloat16* dzT = (__nv_bfloat16*)p;  p += al(cap * m * 2);
  __nv_bfloat16* h2T = (__nv_bfloat16*)p;  p += al(cap * H2S * 2);
  __nv_bfloat16* dh2 = (__nv_bfloat16*)p;  p += al(cap * H2 * 2);
  __nv_bfloat16* h1T = (__nv_bfloat16*)p;  p += al(cap * H1 * 2);
  __nv_bfloat16* dh1 = (__nv_bfloat16*)p;  p += al(cap * H1 * 2);
  __nv_bfloat16* xT = (__nv_bfloat16*)p;   p += al(cap * d * 2);
  __nv_bfloat16* dh2T = (__nv_bfloat16*)p; p += al(cap * H2 * 2);
  __nv_bfloat16* dh1T = (__nv_bfloat16*)p; p += al(cap * H1 * 2);
  __nv_bfloat16* W3T = (__nv_bfloat16*)p;  p += al((int64_t)H2S * m * 2);
  __nv_bfloat16* W2T = (__nv_bfloat16*)p;
  const __nv_bfloat16* W2 = r->wb + (int64_t)H1 * d;
  const __nv_bfloat16* W3 = W2 + (int64_t)H2 * H1;
  auto T = [&](const __nv_bfloat16* in, int rows, int cols, __nv_bfloat16* out) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    transpose_bf16<<<grid, block, 0, st>>>(in, rows, cols, out);
    bdg_note_launch();
  };
  BDG_CUDA_TRY(cudaMemsetAsync(r->grad, 0, r->n_params * 4, st));
  BDG_CUDA_TRY(cudaMemsetAsync(r->loss, 0, 4, st));
  // forward
  BDG_TRY(router_fwd(r, x, codes, B, z, h1b, h2b, st));
  // loss and logit gradient
  softmax_ce<<<B, 256, 0, st>>>(z, m, B, labels, kt, exclude, dz32, dz16, r->loss);
  bdg_note_launch();
  colsum_f32<<<bdg_cdiv(m, 256), 256, 0, st>>>(dz32, B, m, r->grad + o.b3);
  bdg_note_launch();
  // layer 3: dW3 = dz^T [h2 | s], dh2 = (dz W3[:, :h2]) * [h2 > 0], db2 = colsum(dh2)
  T(dz16, B, m, dzT);
  T(h2b, B, H2S, h2T);
  T(W3, m, H2S, W3T);  // its first h2 rows are W3[:, :h2]^T
  BDG_TRY(bdg_gemm_bf16(dzT, h2T, m, H2S, B, nullptr, nullptr, 0, r->grad + o.W3, nullptr,
                        nullptr, r->err, (void*)st));
  BDG_TRY(bdg_gemm_bf16_ld(dz16, W3T, B, H2, m, nullptr, h2b, H2S, 0, nullptr, dh2, H2,
                           r->grad + o.b2, r->err, st));
  // layer 2: dW2 = dh2^T h1, dh1 = (dh2 W2) * [h1 > 0], db1 = colsum(dh1)
  T(dh2, B, H2, dh2T);
  T(h1b, B, H1, h1T);
  T(W2, H2, H1, W2T);
  BDG_TRY(bdg_gemm_bf16(dh2T, h1T, H2, H1, B, nullptr, nullptr, 0, r->grad + o.W2, nullptr,
                        nullptr, r->err, (void*)st));
  BDG_TRY(bdg_gemm_bf16(dh2, W2T, B, H1, H2, nullptr, h1b, 0, nullptr, dh1, r->grad + o.b1,
                        r->err, (void*)st));
  // layer 1: dW1 = dh1^T x
  T(dh1, B, H1, dh1T);
  T((const __nv_bfloat16*)x, B, d, xT);
  BDG_TRY(bdg_gemm_bf16(dh1T, xT, H1, d, B, nullptr, nullptr, 0, r->grad + o.W1, nullptr, nullptr,
                        r->err, (void*)st));
  if (apply_update) BDG_TRY(router_adam(r, lr, st));
  BDG_CUDA_TRY(cudaGetLastError());
  return BDG_OK;
}

bdg_status bdg_router_route(bdg_router* r, const void* x, const uint64_t* codes, int64_t N,
                            const int32_t* home, int32_t P, int32_t* routes, void* stream) {
  if (!r || !x || !home || !routes || N < 0 || P < 1 || P > kMaxP + 1 || P > r->m ||
      (r->cb && !codes))
    return bdg_set_error(BDG_EINVAL, "router_route: N = %lld, P = %d (1..%d)%s", (long long)N, P,
                         kMaxP + 1, r && r->cb && !codes ? ", codes required" : "");
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t cap = r->cap_b;
  char* p = (char*)r->ws;
  void* h1b = p; p += al(cap * r->h1 * 2);
  void* h2b = p; p += al(cap * r->h2s * 2);
  float* z = (float*)p;
  for (int64_t s = 0; s < N; s += cap) {
    const int B = (int)((N - s) < cap ? (N - s) : cap);
    BDG_TRY(router_fwd(r, (const __nv_bfloat16*)x + s * r->d_in,
                       r->cb ? codes + s * (r->cb / 64) : nullptr, B, z, h1b, h2b, st));
    topp_kernel<<<bdg_cdiv(B, 8), 256, 0, st>>>(z, B, r->m, home + s, P, routes + s * P);
    BDG_CUDA_TRY(cudaGetLastError());
    bdg_note_launch();
  }
  return BDG_OK;
}


// ---- shortlist head (see head_route_kernel / head_bwd_kernel)
static bdg_status check_shortlist(const bdg_router* r, int32_t Q, const char* who) {
  if (!r) return bdg_set_error(BDG_EINVAL, "%s: router is NULL", who);
  if (Q < 1 || Q > kMaxQ)
    return bdg_set_error(BDG_EINVAL, "%s: Q = %d (1..%d)", who, Q, kMaxQ);
  if (r->h2s > kUChunks * 32 * 8)
    return bdg_set_error(BDG_EUNSUPPORTED, "%s: last-layer input of %d values (at most %d)", who,
                         r->h2s, kUChunks * 32 * 8);
  return BDG_OK;
}

bdg_status bdg_router_forward_shortlist(bdg_router* r, const void* x, const uint64_t* codes,
                                        const int32_t* cand, int32_t Q, int32_t B,
                                        float* logits, void* stream) {
  BDG_TRY(check_shortlist(r, Q, "router_forward_shortlist"));
  if (!x || !cand || !logits || B < 1 || B > r->cap_b || (r->cb && !codes))
    return bdg_set_error(BDG_EINVAL, "router_forward_shortlist: B = %d (1..%d)%s", B, r->cap_b,
                         r->cb && !codes ? ", codes required" : "");
  cudaStream_t st = (cudaStream_t)stream;
  char* p = (char*)r->ws;
  void* h1b = p; p += al((int64_t)r->cap_b * r->h1 * 2);
  void* h2b = p;
  BDG_TRY(router_hidden(r, x, codes, B, h1b, h2b, st));
  const Offs o = param_offsets(r->d_in, r->h1, r->h2, r->h2s, r->m);
  const __nv_bfloat16* W3 = r->wb + (int64_t)r->h1 * r->d_in + (int64_t)r->h2 * r->h1;
  return launch_head_route((const __nv_bfloat16*)h2b, r->h2s, W3, r->w + o.b3, cand, Q, B, logits,
                           0.f, 1, nullptr, st);
}

bdg_status bdg_router_train_step_shortlist(bdg_router* r, const void* x, const uint64_t* codes,
                                           const int32_t* cand, int32_t Q, const int32_t* labels,
                                           int32_t kt, int32_t B, float lr, int32_t apply_update,
                                           void* stream) {
  BDG_TRY(check_shortlist(r, Q, "router_train_step_shortlist"));
  if (!x || !cand || !labels || B < 8 || B > r->cap_b || (B & 7) || kt < 1 ||
      (r->cb && !codes))
    return bdg_set_error(BDG_EINVAL,
                         "router_train_step_shortlist: B = %d (8..%d, multiple of 8), kt = %d%s",
                         B, r->cap_b, kt, r->cb && !codes ? ", codes required" : "");
  cudaStream_t st = (cudaStream_t)stream;
  const int d = r->d_in, H1 = r->h1, H2 = r->h2, H2S = r->h2s, m = r->m;
  const int64_t cap = r->cap_b;
  const Offs o = param_offsets(d, H1, H2, H2S, m);
  char* p = (char*)r->ws;
  __nv_bfloat16* h1b = (__nv_bfloat16*)p; p += al(cap * H1 * 2);
  __nv_bfloat16* h2b = (__nv_bfloat16*)p; p += al(cap * H2S * 2);
  p += al(cap * m * 4) * 2 + al(cap * m * 2) * 2 + al(cap * H2S * 2);  // dense-head buffers
  __nv_bfloat16* dh2 = (__nv_bfloat16*)p;  p += al(cap * H2 * 2);
  __nv_bfloat16* h1T = (__nv_bfloat16*)p;  p += al(cap * H1 * 2);
  __nv_bfloat16* dh1 = (__nv_bfloat16*)p;  p += al(cap * H1 * 2);
  __nv_bfloat16* xT = (__nv_bfloat16*)p;   p += al(cap * d * 2);
  __nv_bfloat16* dh2T = (__nv_bfloat16*)p; p += al(cap * H2 * 2);
  __nv_bfloat16* dh1T = (__nv_bfloat16*)p; p += al(cap * H1 * 2);
  p += al((int64_t)H2S * m * 2);           // W3T (dense head only)
  __nv_bfloat16* W2T = (__nv_bfloat16*)p;
  const __nv_bfloat16* W2 = r->wb + (int64_t)H1 * d;
  const __nv_bfloat16* W3 = W2 + (int64_t)H2 * H1;
  auto T = [&](const __nv_bfloat16* in, int rows, int cols, __nv_bfloat16* out) {
    dim3 grid((cols + 31) / 32, (rows + 31) / 32), block(32, 8);
    transpose_bf16<<<grid, block, 0, st>>>(in, rows, cols, out);
    bdg_note_launch();
  };
  BDG_CUDA_TRY(cudaMemsetAsync(r->grad, 0, r->n_params * 4, st));
  BDG_CUDA_TRY(cudaMemsetAsync(r->loss, 0, 4, st));
  BDG_TRY(router_hidden(r, x, codes, B, h1b, h2b, st));
  head_bwd_kernel<<<bdg_cdiv(B, 8), 256, 0, st>>>(h2b, H2S, H2, W3, r->w + o.b3, cand, Q, labels,
                                                  kt, B, r->grad + o.W3, r->grad + o.b3,
                                                  r->grad + o.b2, dh2, r->loss);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  // layer 2: dW2 = dh2^T h1, dh1 = (dh2 W2) * [h1 > 0], db1 = colsum(dh1)
  T(dh2, B, H2, dh2T);
  T(h1b, B, H1, h1T);
  T(W2, H2, H1, W2T);
  BDG_TRY(bdg_gemm_bf16(dh2T, h1T, H2, H1, B, nullptr, nullptr, 0, r->grad + o.W2, nullptr,
                        nullptr, r->err, (void*)st));
  BDG_TRY(bdg_gemm_bf16(dh2, W2T, B, H1, H2, nullptr, h1b, 0, nullptr, dh1, r->grad + o.b1,
                        r->err, (void*)st));
  // layer 1: dW1 = dh1^T x
  T(dh1, B, H1, dh1T);
  T((const __nv_bfloat16*)x, B, d, xT);
  BDG_TRY(bdg_gemm_bf16(dh1T, xT, H1, d, B, nullptr, nullptr, 0, r->grad + o.W1, nullptr, nullptr,
                        r->err, (void*)st));
  if (apply_update) BDG_TRY(router_adam(r, lr, st));
  BDG_CUDA_TRY(cudaGetLastError());
  return BDG_OK;
}

bdg_status bdg_router_route_shortlist(bdg_router* r, const void* x, const uint64_t* codes,
                                      const int32_t* cand, int32_t Q, int64_t N, float theta,
                                      int32_t pmax, const int32_t* order, int32_t* routes,
                                      float* logits, void* stream) {
  BDG_TRY(check_shortlist(r, Q, "router_route_shortlist"));
  if (!x || !cand || !routes || N < 0 || pmax < 1 || pmax > Q || (r->cb && !codes) ||
      !(theta >= 0.f))
    return bdg_set_error(BDG_EINVAL, "router_route_shortlist: N = %lld, pmax = %d (1..Q = %d), "
                         "theta = %g (>= 0)%s", (long long)N, pmax, Q, (double)theta,
                         r->cb && !codes ? ", codes required" : "");
  if (N == 0) return BDG_OK;
  cudaStream_t st = (cudaStream_t)stream;
  // inference runs in chunks of 2^18 points with its own stream-ordered
  // workspace: h1 and [h2 | s] of one chunk (640 MB at 512-wide layers and
  // 256-bit codes), and with an order the chunk's gathered inputs. Chunks of
  // 2^16 (whose activations stay in L2) took 9 % longer: each launch then
  // carries too little work for the persistent GEMM to fill the GPU
  const int64_t chunk = N < (1 << 18) ? N : (1 << 18);
  const int cw = r->cb / 64;
  void* ws = nullptr;
  const size_t b1 = al(chunk * r->h1 * 2), b2 = al(chunk * r->h2s * 2);
  const size_t bx = order ? al(chunk * r->d_in * 2) : 0, bc = order && cw ? al(chunk * cw * 8) : 0,
               bq = order ? al(chunk * Q * 4) : 0;
  if (cudaMallocAsync(&ws, b1 + b2 + bx + bc + bq, st) != cudaSuccess) {
    cudaGetLastError();
    return bdg_set_error(BDG_ENOMEM, "router_route_shortlist: workspace of %zu bytes",
                         b1 + b2 + bx + bc + bq);
  }
  const Offs o = param_offsets(r->d_in, r->h1, r->h2, r->h2s, r->m);
  const __nv_bfloat16* W3 = r->wb + (int64_t)r->h1 * r->d_in + (int64_t)r->h2 * r->h1;
  char* gx = (char*)ws + b1 + b2;
  char* gc = gx + bx;
  char* gq = gc + bc;
  bdg_status s = BDG_OK;
  for (int64_t c0 = 0; c0 < N && s == BDG_OK; c0 += chunk) {
    const int B = (int)((N - c0) < chunk ? (N - c0) : chunk);
    void* h1b = ws;
    void* h2b = (char*)ws + b1;
    const void* xc = (const __nv_bfloat16*)x + c0 * r->d_in;
    const uint64_t* cc = cw ? codes + c0 * cw : nullptr;
    const int32_t* qc = cand + c0 * Q;
    if (order) {  // this chunk's rows of the processing order, gathered
      s = gather_rows_words(x, N, r->d_in / 2, order + c0, B, gx, st);
      if (s == BDG_OK && cw) s = gather_rows_words(codes, N, cw * 2, order + c0, B, gc, st);
      if (s == BDG_OK) s = gather_rows_words(cand, N, Q, order + c0, B, gq, st);
      if (s != BDG_OK) break;
      xc = gx;
      cc = cw ? (const uint64_t*)gc : nullptr;
      qc = (const int32_t*)gq;
    }
    s = router_hidden(r, xc, cc, B, h1b, h2b, st);
    if (s != BDG_OK) break;
    bdg_prof_scope prof("router_head", st);
    if (order)
      s = launch_head_route((const __nv_bfloat16*)h2b, r->h2s, W3, r->w + o.b3, qc, Q, B, logits,
                            theta, pmax, routes, st, order + c0, N);
    else
      s = launch_head_route((const __nv_bfloat16*)h2b, r->h2s, W3, r->w + o.b3, qc, Q, B,
                            logits ? logits + c0 * Q : nullptr, theta, pmax, routes + c0 * pmax,
                            st);
  }
  cudaFreeAsync(ws, st);
  return s;
}

}  // extern "C"
