// gemm_tc.cu -- BF16 GEMM on the 5th-generation tensor cores for the MLP router:
//   C[M, N] = epilogue( A[M, K] * B[N, K]^T ),  A and B row-major with K contiguous.
// FP32 accumulation in tensor memory; epilogues: + bias[N], ReLU, multiply by
// the ReLU derivative of a mask tensor (backward of a ReLU layer), column sums
// of the result (bias gradients), output FP32 or BF16.
//
// Persistent: one CTA per SM walks the 128 x 128 output tiles (n fastest, so
// consecutive tiles of a CTA share their A rows in L2). Warps 4-7 stream 64-wide
// K slabs of A and B into a 4-stage shared-memory ring with 16-byte cp.async
// (zero-filled past the matrix edges) in the K-major no-swizzle core-matrix
// layout; one thread of warp 8 issues tcgen05.mma kind::f16 (M = 128, N = 128,
// K = 16 per instruction) into one of two TMEM accumulators, so the MMAs of the
// next tile run while warps 0-3 drain the previous one. The epilogue reads its
// accumulator rows (thread = row = TMEM lane) into a per-warp shared-memory
// tile, hands the accumulator back, and then writes the tile row by row with
// the 32 lanes on 32 consecutive columns: coalesced stores, coalesced bias and
// mask reads, per-column sums in registers. Every mbarrier wait is bounded and
// reports through an error word.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc05.cuh"

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;   // tile; K slab = 64 bf16 = 128 bytes
constexpr int kStages = 4;
constexpr int kAcc = 2;                         // TMEM accumulators (128 columns each)
constexpr int kThreads = 288;                   // 0-3 epilogue, 4-7 producer, 8 MMA
constexpr uint32_t kSlab = kBM * kBK * 2;       // 16 KB per operand per stage
constexpr uint32_t kRing = kStages * 2 * kSlab;  // 128 KB
constexpr int kLd = kBN + 1;                    // staging row stride (floats): no bank conflicts
constexpr uint32_t kStageBytes = 4u * 32 * kLd * 4;  // 4 warps x 32 rows x 129 floats
constexpr uint32_t kPolls = 1u << 20;

struct GemmArgs {
  const __nv_bfloat16* A;  // [M][K]
  const __nv_bfloat16* B;  // [N][K]
  int M, N, K;
  const float* bias;       // [N] or NULL
  const __nv_bfloat16* mask;  // [M][ldm] or NULL: multiply by (mask > 0)
  int ldm;                 // row stride of mask (elements)
  int relu;
  float* out_f32;          // [M][ldo] or NULL
  __nv_bfloat16* out_bf16; // [M][ldo] or NULL
  int ldo;                 // row stride of the output (elements)
  float* colsum;           // [N] or NULL: += column sums of the result (before rounding)
  int32_t* err;
};

// byte offset of (row r, 16-byte chunk c) inside one 128 x 128 B slab (K-major, no swizzle)
__device__ __forceinline__ uint32_t slab_off(int r, int c) {
  return (uint32_t)((r >> 3) * 1024 + c * 128 + (r & 7) * 16);
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(src_bytes)
               : "memory");
}

__global__ void __launch_bounds__(kThreads, 1) gemm_bf16_kernel(GemmArgs g) {
  extern __shared__ __align__(1024) uint8_t sm[];
  float* stage = reinterpret_cast<float*>(sm + kRing);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kRing + kStageBytes);
  uint64_t* full = bars;                  // [kStages], 128 producer arrivals
  uint64_t* empty = bars + kStages;       // [kStages], MMA commit
  uint64_t* tfull = bars + 2 * kStages;   // [kAcc], MMA commit: accumulator ready
  uint64_t* tempty = tfull + kAcc;        // [kAcc], 4 epilogue warps: accumulator read
  uint64_t* drain = tempty + kAcc;        // MMA drain before TMEM is freed
  uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = (g.K + kBK - 1) / kBK;
  const int tiles_n = (g.N + kBN - 1) / kBN;
  const int ntiles = ((g.M + kBM - 1) / kBM) * tiles_n;

  if (warp == 0) tc05::tmem_alloc(tslot, kAcc * kBN);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      tc05::mbar_init(&full[s], 128);
      tc05::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kAcc; ++b) {
      tc05::mbar_init(&tfull[b], 1);
      tc05::mbar_init(&tempty[b], 4);
    }
    tc05::mbar_init(drain, 1);
    tc05::mbar_fence_init();
  }
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  const uint32_t tmem = *tslot;

  if (warp >= 4 && warp < 8) {
    // ---------------- producers: 128 threads, 2 x 1024 16-byte chunks per stage
    const int p = tid - 128;
    uint32_t gs = 0;  // slabs issued by this CTA so far (ring position)
    bool ok = true;
    for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
      const int m0 = (tile / tiles_n) * kBM, n0 = (tile % tiles_n) * kBN;
      for (int j = 0; j < nk; ++j, ++gs) {
        const uint32_t s = gs % kStages, use = gs / kStages;
        if (use > 0 && !tc05::mbar_wait(&empty[s], (use - 1) & 1, kPolls)) {
          atomicExch(g.err, 11);
          ok = false;
          break;
        }
        const uint32_t sa = tc05::smem_u32(sm + s * 2 * kSlab), sb = sa + kSlab;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int x = p + 128 * q;                   // 0..1023
          const int rr = x & 7, c = (x >> 3) & 7, grp = x >> 6;  // row-in-group fastest
          const int r = grp * 8 + rr;
          const int kk = j * kBK + c * 8;              // first element of the chunk
          const int kv = max(0, min(8, g.K - kk));     // valid elements in this chunk
          {
            const int gr = m0 + r;
            const bool in = gr < g.M && kv > 0;
            const __nv_bfloat16* src = in ? g.A + (int64_t)gr * g.K + kk : g.A;
            cp16(sa + slab_off(r, c), src, in ? kv * 2 : 0);
          }
          {
            const int gr = n0 + r;
            const bool in = gr < g.N && kv > 0;
            const __nv_bfloat16* src = in ? g.B + (int64_t)gr * g.K + kk : g.B;
            cp16(sb + slab_off(r, c), src, in ? kv * 2 : 0);
          }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        if (gs > 0) {  // the previous slab has landed: publish it to the tensor core
          asm volatile("cp.async.wait_group 1;" ::: "memory");
          tc05::fence_proxy_async();
          tc05::mbar_arrive(&full[(gs - 1) % kStages]);
        }
      }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (ok && gs > 0) {
      tc05::fence_proxy_async();
      tc05::mbar_arrive(&full[(gs - 1) % kStages]);
    }
  } else if (warp == 8) {
    // ---------------- MMA issuer
    if (lane == 0) {
      constexpr uint32_t id = tc05::idesc(1u, 1u, kBM, kBN);  // BF16 x BF16 -> F32
      uint32_t gs = 0, it = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
        const uint32_t b = it % kAcc;
        if (it >= kAcc && !tc05::mbar_wait(&tempty[b], ((it / kAcc) - 1) & 1, kPolls)) {
          atomicExch(g.err, 14);
          break;
        }
        tc05::fence_after();
        for (int j = 0; j < nk; ++j, ++gs) {
          const uint32_t s = gs % kStages;
          if (!tc05::mbar_wait(&full[s], (gs / kStages) & 1, kPolls)) {
            atomicExch(g.err, 12);
            ok = false;
            break;
          }
          tc05::fence_after();
          const uint32_t sa = tc05::smem_u32(sm + s * 2 * kSlab), sb = sa + kSlab;
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {  // 16 bf16 = 32 bytes = 2 core matrices
            const uint64_t ad = tc05::sdesc(sa + kk * 256, 128, 1024);
            const uint64_t bd = tc05::sdesc(sb + kk * 256, 128, 1024);
            tc05::mma_f16(tmem + b * kBN, ad, bd, id, (j > 0 || kk > 0) ? 1u : 0u);
          }
          tc05::commit(&empty[s]);
        }
        if (ok) tc05::commit(&tfull[b]);
      }
      tc05::commit(drain);
      if (!tc05::mbar_wait(drain, 0, kPolls)) atomicExch(g.err, 15);
    }
  } else {
    // ---------------- epilogue: warp w owns rows 32w .. 32w + 31 of each tile
    float* st = stage + warp * 32 * kLd;
    uint32_t it = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++it) {
      const int m0 = (tile / tiles_n) * kBM, n0 = (tile % tiles_n) * kBN;
      const uint32_t b = it % kAcc;
      const bool ok = tc05::mbar_wait(&tfull[b], (it / kAcc) & 1, kPolls * 4);
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) atomicExch(g.err, 13);
        break;
      }
      tc05::fence_after();
      // accumulator rows -> this warp's staging tile (thread = row)
#pragma unroll 1
      for (int c0 = 0; c0 < kBN; c0 += 32) {
        uint32_t v[32];
        tc05::ld32(tmem + ((uint32_t)(32 * warp) << 16) + b * kBN + c0, v);
        tc05::wait_ld();
#pragma unroll
        for (int j = 0; j < 32; ++j) st[lane * kLd + c0 + j] = __uint_as_float(v[j]);
      }
      tc05::fence_before();
      __syncwarp();
      if (lane == 0) tc05::mbar_arrive(&tempty[b]);  // the accumulator is free again
      // staging tile -> output, row by row, lanes on consecutive columns
      const int row0 = m0 + 32 * warp;
#pragma unroll 1
      for (int c0 = 0; c0 < kBN; c0 += 32) {
        const int col = n0 + c0 + lane;
        const bool cin = col < g.N;
        const float bv = (g.bias && cin) ? g.bias[col] : 0.f;
        float csum = 0.f;
        for (int r = 0; r < 32; ++r) {
          const int row = row0 + r;
          if (row >= g.M) break;
          float x = st[r * kLd + c0 + lane] + bv;
          if (g.relu) x = fmaxf(x, 0.f);
          if (g.mask && cin && !(__bfloat162float(g.mask[(int64_t)row * g.ldm + col]) > 0.f))
            x = 0.f;
          if (cin) {
            if (g.out_f32) g.out_f32[(int64_t)row * g.ldo + col] = x;
            if (g.out_bf16) g.out_bf16[(int64_t)row * g.ldo + col] = __float2bfloat16_rn(x);
            csum += x;
          }
        }
        if (g.colsum && cin) atomicAdd(&g.colsum[col], csum);
      }
      __syncwarp();  // the staging tile is reused by the next tile
    }
  }
  tc05::fence_before();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, kAcc * kBN);
}

}  // namespace

size_t bdg_gemm_smem_bytes() { return (size_t)kRing + kStageBytes + 256; }

// C = epilogue(A * B^T) with row strides for the mask and the output; see GemmArgs.
// K % 8 == 0 (16-byte rows); ldm, ldo >= N.
bdg_status bdg_gemm_bf16_ld(const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                            const float* bias, const void* mask, int32_t ldm, int32_t relu,
                            float* out_f32, void* out_bf16, int32_t ldo, float* colsum,
                            int32_t* err, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0 || (K & 7) || ldm < N || ldo < N)
    return bdg_set_error(BDG_EINVAL, "gemm: M=%d N=%d K=%d ldm=%d ldo=%d (K %% 8 == 0)", M, N,
                         K, ldm, ldo);
  GemmArgs g{(const __nv_bfloat16*)A, (const __nv_bfloat16*)B, M, N, K, bias,
             (const __nv_bfloat16*)mask, ldm, relu, out_f32, (__nv_bfloat16*)out_bf16, ldo,
             colsum, err};
  const size_t smem = bdg_gemm_smem_bytes();
  BDG_CUDA_TRY(cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  const int64_t ntiles = (int64_t)((N + kBN - 1) / kBN) * ((M + kBM - 1) / kBM);
  const int grid = (int)(ntiles < bdg_num_sms() ? ntiles : bdg_num_sms());
  bdg_prof_scope prof("gemm", st);
  gemm_bf16_kernel<<<grid, kThreads, smem, st>>>(g);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

// C = epilogue(A * B^T) with contiguous rows; see GemmArgs. K % 8 == 0 (16-byte rows).
extern "C" bdg_status bdg_gemm_bf16(const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                                    const float* bias, const void* mask, int32_t relu,
                                    float* out_f32, void* out_bf16, float* colsum, int32_t* err,
                                    void* stream) {
  return bdg_gemm_bf16_ld(A, B, M, N, K, bias, mask, N, relu, out_f32, out_bf16, N, colsum, err,
                          (cudaStream_t)stream);
}
