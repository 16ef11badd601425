// route_small.cu -- nearest-centre routing (Map step, Section 3.2) on the
// tensor cores when the centres are few (m <= 256, 256- or 512-bit codes,
// t <= 8).
//
// All m centres, expanded to E4M3 +-1 (one byte per code bit), stay in shared
// memory for the whole launch: at most 256 x 512 bytes. A 128-point tile is
// then one chain of bits / 32 MMAs (M = 128, N = m rounded up to 16, K = 32)
// into one TMEM accumulator: the dot product of two +-1 codes is
// bits - 2 d(x, c), exact in FP32. Each epilogue thread owns one point (one TMEM
// lane) and keeps its 8 best keys (d << 16 | c) in registers, of which the first t
// are its routes, so ties fall by centre index exactly as in the ALU routing
// kernel: the results are identical.
//
// One CTA per SM, persistent over the point tiles (static round robin). Warps
// 0-3 write the next tile's points into the second of two TMEM operand buffers
// while the MMAs of the current tile run; warp 4 loads the centres once and
// issues the MMAs. Every mbarrier wait is bounded: a wait that gives up sets the
// error word and the CTA stops issuing work, drains its MMAs and frees TMEM.
#include "common.cuh"
#include "tc05.cuh"

namespace {

constexpr int kRsThreads = 160;          // warps 0-3 epilogue (TMEM lanes 0-127), warp 4 MMA
constexpr int kRsMaxT = 8;
constexpr uint32_t kRsTmemCols = 512;    // accumulator [0, 256), operands from column 256
constexpr uint32_t kRsOperand0 = 256;
constexpr uint32_t kRsPolls = 1u << 20;

int padded_centres(int m) { return m < 16 ? 16 : (m + 15) / 16 * 16; }

__device__ __forceinline__ void cas(uint32_t& a, uint32_t& b) {
  const uint32_t lo = min(a, b);
  b = max(a, b);
  a = lo;
}
// ascending sort of 8 keys (Batcher's odd-even merge network, 19 comparators)
__device__ __forceinline__ void sort8(uint32_t (&x)[8]) {
  cas(x[0], x[1]); cas(x[2], x[3]); cas(x[4], x[5]); cas(x[6], x[7]);
  cas(x[0], x[2]); cas(x[1], x[3]); cas(x[4], x[6]); cas(x[5], x[7]);
  cas(x[1], x[2]); cas(x[5], x[6]);
  cas(x[0], x[4]); cas(x[1], x[5]); cas(x[2], x[6]); cas(x[3], x[7]);
  cas(x[2], x[4]); cas(x[3], x[5]);
  cas(x[1], x[2]); cas(x[3], x[4]); cas(x[5], x[6]);
}
// ascending sort of a bitonic sequence of 8 keys (half-cleaners at distance 4, 2, 1)
__device__ __forceinline__ void clean8(uint32_t (&x)[8]) {
  cas(x[0], x[4]); cas(x[1], x[5]); cas(x[2], x[6]); cas(x[3], x[7]);
  cas(x[0], x[2]); cas(x[1], x[3]); cas(x[4], x[6]); cas(x[5], x[7]);
  cas(x[0], x[1]); cas(x[2], x[3]); cas(x[4], x[5]); cas(x[6], x[7]);
}

// Centre c < np as KB bytes of E4M3 (zeros for c >= m) in the K-major
// core-matrix layout the MMA reads B in: 8-row groups of KB * 8 bytes, 16-byte
// chunks of one row 128 bytes apart within a group.
template <int W>
__global__ void expand_centres_kernel(const uint64_t* __restrict__ cent, int m, int np,
                                      uint8_t* __restrict__ out) {
  constexpr int KB = 64 * W, Q = 4 * W;  // 16-bit chunks per code
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int rr = (int)(x & 7);
  const int64_t rest = x >> 3;
  const int q = (int)(rest % Q);
  const int64_t grp = rest / Q;
  const int64_t row = grp * 8 + rr;
  if (row >= np) return;
  uint4 v = make_uint4(0, 0, 0, 0);
  if (row < m) v = tc05::expand16((uint32_t)(cent[row * W + (q >> 2)] >> (16 * (q & 3))) & 0xFFFFu);
  *reinterpret_cast<uint4*>(out + grp * (int64_t)(KB * 8) + (int64_t)q * 128 + rr * 16) = v;
}

template <int W>
__global__ void __launch_bounds__(kRsThreads, 1)
route_small_kernel(const uint64_t* __restrict__ codes, int64_t n,
                   const uint8_t* __restrict__ cexp, int m, int np, int t,
                   int32_t* __restrict__ routes, int32_t* __restrict__ rdist,
                   unsigned long long* __restrict__ loss, int32_t* __restrict__ err) {
  constexpr int KB = 64 * W;               // bytes of one expanded code
  constexpr uint32_t kOpCols = KB / 4;     // TMEM columns of one point operand
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + (size_t)np * KB);
  uint64_t* b_full = bars;          // the centres landed
  uint64_t* a_full = bars + 1;      // [2] a point operand written (4 epilogue warps)
  uint64_t* a_free = bars + 3;      // [2] the MMAs reading an operand completed
  uint64_t* acc_full = bars + 5;    // a tile's MMAs completed
  uint64_t* acc_free = bars + 6;    // the accumulator was read (4 epilogue warps)
  uint64_t* drain = bars + 7;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 8);
  volatile int32_t* s_abort = reinterpret_cast<int32_t*>(bars + 8) + 1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t ntile = (n + 127) / 128;
  const int nmine = blockIdx.x < ntile ? (int)((ntile - 1 - blockIdx.x) / gridDim.x) + 1 : 0;

  if (warp == 0) tc05::tmem_alloc(tmem_slot, kRsTmemCols);
  if (tid == 0) {
    tc05::mbar_init(b_full, 1);
    for (int i = 0; i < 2; ++i) {
      tc05::mbar_init(&a_full[i], 4);
      tc05::mbar_init(&a_free[i], 1);
    }
    tc05::mbar_init(acc_full, 1);
    tc05::mbar_init(acc_free, 4);
    tc05::mbar_init(drain, 1);
    *s_abort = 0;
    tc05::mbar_fence_init();
  }
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    // ---------------- centres (once) and MMA issue
    if (lane == 0) {
      const uint32_t b0 = tc05::smem_u32(sm);
      tc05::arrive_expect_tx(b_full, (uint32_t)np * KB);
      tc05::bulk_g2s(b0, cexp, (uint32_t)np * KB, b_full);
      bool ok = tc05::mbar_wait(b_full, 0, kRsPolls);
      const uint32_t id = tc05::idesc(0u, 0u, 128, np);  // E4M3 x E4M3 -> F32
      for (int s = 0; s < nmine && ok && !*s_abort; ++s) {
        const int a = s & 1;
        ok = tc05::mbar_wait(&a_full[a], (s >> 1) & 1, kRsPolls) &&
             (s == 0 || tc05::mbar_wait(acc_free, (s - 1) & 1, kRsPolls));
        if (!ok) break;
        tc05::fence_after();
        const uint32_t a0 = tmem + kRsOperand0 + a * kOpCols;
#pragma unroll
        for (int kk = 0; kk < KB / 32; ++kk)  // K = 32 per MMA: 8 TMEM columns of A
          tc05::mma_f8_ts(tmem, a0 + kk * 8, tc05::sdesc(b0 + kk * 256, 128, KB * 8), id,
                          kk > 0 ? 1u : 0u);
        tc05::commit(&a_free[a]);
        tc05::commit(acc_full);
      }
      if (!ok) { atomicExch(err, 1); *s_abort = 1; }
      // every MMA issued has completed before TMEM is released
      tc05::commit(drain);
      if (!tc05::mbar_wait(drain, 0, kRsPolls)) atomicExch(err, 1);
    }
  } else {
    // ---------------- epilogue: thread tid owns row tid of each tile
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    // the points of this CTA's s-th tile into operand buffer s & 1 (E4M3 +-1,
    // column c of a lane holding code bits 4c .. 4c + 3, one byte each)
    auto write_operand = [&](int s) {
      const int64_t i = ((int64_t)blockIdx.x + (int64_t)s * gridDim.x) * 128 + tid;
      uint64_t cw[W];
#pragma unroll
      for (int w = 0; w < W; ++w) cw[w] = i < n ? codes[i * W + w] : 0ull;
#pragma unroll
      for (int ch = 0; ch < W / 2; ++ch) {  // 32 columns = 128 code bits per store
        uint32_t col[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const uint64_t word = cw[2 * ch + (q >> 4)];
          const uint32_t nib = (uint32_t)(word >> (4 * (q & 15))) & 0xFu;
          col[q] = i < n ? 0xB8B8B8B8u ^ (((nib * 0x00204081u) & 0x01010101u) << 7) : 0u;
        }
        tc05::st32(tmem + lane_base + kRsOperand0 + (s & 1) * kOpCols + 32 * ch, col);
      }
      tc05::wait_st();
      tc05::fence_before();
      __syncwarp();
      if (lane == 0) tc05::mbar_arrive(&a_full[s & 1]);
    };
    // d = (bits - dot) / 2 sits in the low mantissa bits of dot * -1/2 + bits / 2
    // + 2^23, and those bits times 2^16 (mod 2^32) leave d << 16: the key of
    // centre c is one FFMA and one IMAD
    const int bits = 64 * W;
    const float hmagic = 0.5f * (float)bits + 8388608.0f;
    bool ok = true;
    if (nmine > 0) write_operand(0);
    for (int s = 0; s < nmine && ok; ++s) {
      if (s + 1 < nmine) {  // the next tile's operand, while the MMAs of this one run
        ok = s + 1 < 2 || tc05::mbar_wait(&a_free[(s + 1) & 1], ((s - 1) >> 1) & 1, kRsPolls);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        write_operand(s + 1);
      }
      ok = __all_sync(0xffffffffu, !*s_abort && tc05::mbar_wait(acc_full, s & 1, kRsPolls));
      if (!ok) break;
      tc05::fence_after();
      // the 8 smallest keys so far, ascending; eight new keys at a time are
      // sorted by a 19-comparator network, the elementwise minimum with the
      // kept keys in reverse order leaves the 8 smallest of both as a bitonic
      // sequence, and 12 comparators sort it: no branches, and the comparators
      // of a step are independent
      uint32_t best[kRsMaxT];
#pragma unroll
      for (int j = 0; j < kRsMaxT; ++j) best[j] = 0xFFFFFFFFu;
      for (int c0 = 0; c0 < np; c0 += 32) {
        uint32_t v[32];
        tc05::ld32(tmem + lane_base + (uint32_t)c0, v);
        tc05::wait_ld();
#pragma unroll
        for (int g = 0; g < 32; g += 8) {
          uint32_t x[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const uint32_t fb = __float_as_uint(fmaf(__uint_as_float(v[g + j]), -0.5f, hmagic));
            x[j] = c0 + g + j < m ? fb * 65536u + (uint32_t)(c0 + g + j) : 0xFFFFFFFFu;
          }
          sort8(x);
          uint32_t y[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) y[j] = min(best[j], x[7 - j]);
          clean8(y);
#pragma unroll
          for (int j = 0; j < 8; ++j) best[j] = y[j];
        }
      }
      tc05::fence_before();
      __syncwarp();
      if (lane == 0) tc05::mbar_arrive(acc_free);
      const int64_t i = ((int64_t)blockIdx.x + (int64_t)s * gridDim.x) * 128 + tid;
      if (loss) {  // Bk-means objective (Eq. 1): distance to the nearest centre, one atomic per warp
        unsigned long long dsum = i < n ? (unsigned long long)(best[0] >> 16) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dsum += __shfl_down_sync(0xffffffffu, dsum, o);
        if (lane == 0) atomicAdd(loss, dsum);
      }
      if (i < n) {
#pragma unroll
        for (int j = 0; j < kRsMaxT; ++j) {
          if (j < t) {
            routes[i * t + j] = (int32_t)(best[j] & 0xFFFFu);
            if (rdist) rdist[i * t + j] = (int32_t)(best[j] >> 16);
          }
        }
      }
    }
    if (!ok && lane == 0) { atomicExch(err, 1); *s_abort = 1; }
  }
  tc05::fence_before();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, kRsTmemCols);
}

template <int W>
bdg_status launch_w(const uint64_t* codes, int64_t n, const uint64_t* cent, int m, int t,
                    int32_t* routes, int32_t* rdist, unsigned long long* loss, uint8_t* cexp,
                    int32_t* err, cudaStream_t st) {
  constexpr int KB = 64 * W;
  const int np = padded_centres(m);
  const int64_t nthreads = (int64_t)np * 4 * W;  // one thread per 16-bit chunk
  expand_centres_kernel<W><<<bdg_cdiv(nthreads, 256), 256, 0, st>>>(cent, m, np, cexp);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  const size_t smem = (size_t)np * KB + 8 * 8 + 16;
  BDG_CUDA_TRY(cudaFuncSetAttribute(route_small_kernel<W>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t ntile = (n + 127) / 128;
  const int grid = (int)std::min<int64_t>(ntile, bdg_num_sms());
  route_small_kernel<W><<<grid, kRsThreads, smem, st>>>(codes, n, cexp, m, np, t, routes, rdist,
                                                         loss, err);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

}  // namespace

bool bdg_route_small_ok(int W, int m, int t) {
  return (W == 4 || W == 8) && m >= 1 && m <= 256 && t >= 1 && t <= kRsMaxT && t <= m;
}

size_t bdg_route_small_bytes(int m, int W) {
  return ((size_t)padded_centres(m) * 64 * W + 255) / 256 * 256 + 256;
}

bdg_status bdg_launch_route_small(const uint64_t* codes, int64_t n, int W, const uint64_t* cent,
                                  int m, int t, int32_t* routes, int32_t* rdist, void* scratch,
                                  size_t scratch_bytes, cudaStream_t st, unsigned long long* loss,
                                  const char* prof_name) {
  if (n == 0) return BDG_OK;
  if (!bdg_route_small_ok(W, m, t))
    return bdg_set_error(BDG_EINVAL, "route: W=%d m=%d t=%d outside the small tensor path", W, m, t);
  if (scratch_bytes < bdg_route_small_bytes(m, W))
    return bdg_set_error(BDG_EINVAL, "route: small tensor-path scratch too small");
  uint8_t* cexp = (uint8_t*)scratch;
  int32_t* err = (int32_t*)((char*)scratch + bdg_route_small_bytes(m, W) - 256);
  BDG_CUDA_TRY(cudaMemsetAsync(err, 0, 4, st));
  bdg_prof_scope prof(prof_name, st);
  if (W == 4) return launch_w<4>(codes, n, cent, m, t, routes, rdist, loss, cexp, err, st);
  return launch_w<8>(codes, n, cent, m, t, routes, rdist, loss, cexp, err, st);
}
