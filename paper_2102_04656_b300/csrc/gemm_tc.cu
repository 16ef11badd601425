// gemm_tc.cu -- BF16 GEMM on the 5th-generation tensor cores for the MLP router:
//   C[M, N] = epilogue( A[M, K] * B[N, K]^T ),  A and B row-major with K contiguous.
// FP32 accumulation in tensor memory; epilogues: + bias[N], ReLU, multiply by
// the ReLU derivative of a mask tensor (backward of a ReLU layer), column sums
// of the result (bias gradients), output FP32 or BF16.
//
// Persistent: one CTA per SM walks the 128 x 128 output tiles (n fastest, so
// consecutive tiles of a CTA share their A rows in L2). One thread of warp 4
// streams 64-wide K slabs of A and B into a 4-stage shared-memory ring with TMA
// tensor copies (cp.async.bulk.tensor, 128-byte swizzle, zero fill past the
// matrix edges) completing on mbarriers; one thread of warp 5 issues
// tcgen05.mma kind::f16 (M = 128, N = 128, K = 16 per instruction) into one of
// two TMEM accumulators, so the MMAs of the next tile run while eight epilogue
// warps (two per scheduler: each reads its TMEM lane quarter and one half of
// the columns) drain the previous one. Inference layers (bias, ReLU, BF16 out,
// whole tiles) are written straight from the accumulator, each thread storing
// its own row 16 bytes at a time; the general epilogue stages a warp's block in
// shared memory and writes it row by row, each lane on 4 consecutive columns
// (coalesced stores, bias and mask reads, per-column sums in registers). Every
// mbarrier wait is bounded and reports through an error word.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "tc05.cuh"

namespace {

constexpr int kBM = 128, kBN = 128, kBK = 64;   // tile; K slab = 64 bf16 = 128 bytes
constexpr int kStages = 4;
constexpr int kAcc = 2;                         // TMEM accumulators (128 columns each)
constexpr int kThreads = 320;  // warps 0-3 and 6-9 epilogue, 4 producer, 5 MMA
constexpr uint32_t kSlab = kBM * kBK * 2;       // 16 KB per operand per stage
constexpr uint32_t kRing = kStages * 2 * kSlab;  // 192 KB: the copies in flight
// the epilogue stages half a tile (64 columns) at a time; row stride 68 floats:
// 16-byte aligned rows, and a thread writing its row 16 bytes at a time or half
// a warp reading one row 16 bytes per lane meet no bank conflicts
constexpr int kHalfN = kBN / 2;
constexpr int kLd = kHalfN + 4;
constexpr int kEpiWarps = 8;
constexpr uint32_t kStageBytes = kEpiWarps * 32u * kLd * 4;  // 8 warps x 32 rows x 68 floats
static_assert(kRing + kStageBytes + 256 <= 232448, "shared memory per block exceeds 227 KB");
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
  int vec_out;             // outputs 16-byte aligned with ldo % 4 == 0: 4-column stores
  int direct;              // bias, BF16 output only (no mask, FP32 or column sums), M and N
                           // multiples of the tile, ldo % 8 == 0, 16-byte aligned bias and
                           // output: every thread stores its own row
};

// One 2D TMA box (64 K-elements x 128 rows of BF16) into shared memory.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst), "l"(map), "r"(x), "r"(y),
      "r"(tc05::smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
          tc05::smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: 8-row groups 1024 bytes apart (stride byte offset), the
// leading byte offset unused, swizzle mode 2 (128 bytes).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused): 16 bytes
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 1024 bytes
  d |= (uint64_t)1 << 46;                  // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                  // 128-byte swizzle
  return d;
}

__global__ void __launch_bounds__(kThreads, 1)
gemm_bf16_kernel(GemmArgs g, const __grid_constant__ CUtensorMap mapA,
                 const __grid_constant__ CUtensorMap mapB) {
  extern __shared__ __align__(1024) uint8_t sm[];
  float* stage = reinterpret_cast<float*>(sm + kRing);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kRing + kStageBytes);
  uint64_t* full = bars;                  // [kStages], producer expect-tx + TMA bytes
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
      tc05::mbar_init(&full[s], 1);
      tc05::mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < kAcc; ++b) {
      tc05::mbar_init(&tfull[b], 1);
      tc05::mbar_init(&tempty[b], kEpiWarps);
    }
    tc05::mbar_init(drain, 1);
    tc05::mbar_fence_init();
  }
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 4) {
    // ---------------- producer: one thread, two TMA boxes per stage
    if (lane == 0) {
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
          expect_tx(&full[s], 2 * kSlab);
          tma_load_2d(sa, &mapA, j * kBK, m0, &full[s]);
          tma_load_2d(sb, &mapB, j * kBK, n0, &full[s]);
        }
      }
      // copies issued but possibly never consumed (an MMA wait gave up): wait
      // for them, bounded, before the CTA exits
      for (uint32_t q = gs > kStages ? gs - kStages : 0; q < gs; ++q)
        tc05::mbar_wait(&full[q % kStages], (q / kStages) & 1, kPolls);
    }
  } else if (warp == 5) {
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
          for (int kk = 0; kk < kBK / 16; ++kk) {  // 16 bf16 = 32 bytes within the swizzle atom
            const uint64_t ad = sdesc_sw128(sa + kk * 32);
            const uint64_t bd = sdesc_sw128(sb + kk * 32);
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
    // ---------------- epilogue: 8 warps; warp w reads TMEM lanes 32 (w % 4) ..
    // + 31 (the rows it may access) and one half of the tile's columns: warps
    // 0-3 columns 0-63, warps 6-9 columns 64-127
    const int quad = warp & 3, half = warp >= 6 ? 1 : 0;
    const int ew = quad + 4 * half;  // 0..7
    float* st = stage + ew * 32 * kLd;
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
      const int row0 = m0 + 32 * quad;
      const int cb = n0 + kHalfN * half;  // first column of this warp's half
      const uint32_t tbase = tmem + ((uint32_t)(32 * quad) << 16) + b * kBN + kHalfN * half;
      if (g.direct) {
        // inference layers (bias, optional ReLU, BF16 out, whole tile inside the
        // matrix): each thread converts its own row and stores it, 8 values per
        // 16-byte store, straight from the accumulator
        __nv_bfloat16* orow = g.out_bf16 + (int64_t)(row0 + lane) * g.ldo + cb;
#pragma unroll
        for (int c0 = 0; c0 < kHalfN; c0 += 32) {
          uint32_t v[32];
          tc05::ld32(tbase + c0, v);
          tc05::wait_ld();
          if (c0 == kHalfN - 32) {  // this warp's part of the accumulator is read
            tc05::fence_before();
            __syncwarp();
            if (lane == 0) tc05::mbar_arrive(&tempty[b]);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float4 b0 = *reinterpret_cast<const float4*>(g.bias + cb + c0 + 8 * q);
            const float4 b1 = *reinterpret_cast<const float4*>(g.bias + cb + c0 + 8 * q + 4);
            float x[8] = {__uint_as_float(v[8 * q]) + b0.x, __uint_as_float(v[8 * q + 1]) + b0.y,
                          __uint_as_float(v[8 * q + 2]) + b0.z, __uint_as_float(v[8 * q + 3]) + b0.w,
                          __uint_as_float(v[8 * q + 4]) + b1.x, __uint_as_float(v[8 * q + 5]) + b1.y,
                          __uint_as_float(v[8 * q + 6]) + b1.z, __uint_as_float(v[8 * q + 7]) + b1.w};
            if (g.relu) {
#pragma unroll
              for (int e = 0; e < 8; ++e) x[e] = fmaxf(x[e], 0.f);
            }
            uint4 pk;
            __nv_bfloat162 h0 = __floats2bfloat162_rn(x[0], x[1]);
            __nv_bfloat162 h1 = __floats2bfloat162_rn(x[2], x[3]);
            __nv_bfloat162 h2 = __floats2bfloat162_rn(x[4], x[5]);
            __nv_bfloat162 h3 = __floats2bfloat162_rn(x[6], x[7]);
            pk.x = *reinterpret_cast<uint32_t*>(&h0);
            pk.y = *reinterpret_cast<uint32_t*>(&h1);
            pk.z = *reinterpret_cast<uint32_t*>(&h2);
            pk.w = *reinterpret_cast<uint32_t*>(&h3);
            *reinterpret_cast<uint4*>(orow + c0 + 8 * q) = pk;
          }
        }
        continue;
      }
      // the general epilogue: this warp's 32 x 64 block of the accumulator into
      // its staging tile (thread = row), the accumulator handed back, then the
      // block written row by row with half-warps on rows and each lane on 4
      // consecutive columns: coalesced stores, bias and mask reads, per-column
      // sums in registers
#pragma unroll
      for (int c0 = 0; c0 < kHalfN; c0 += 32) {
        uint32_t v[32];
        tc05::ld32(tbase + c0, v);
        tc05::wait_ld();
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *reinterpret_cast<float4*>(&st[lane * kLd + c0 + 4 * q]) =
              make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                          __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
      }
      tc05::fence_before();
      __syncwarp();
      if (lane == 0) tc05::mbar_arrive(&tempty[b]);
      const int col = cb + 4 * (lane & 15);
      const int nc = max(0, min(4, g.N - col));  // valid columns of this lane
      float bv[4], csum[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int e = 0; e < 4; ++e) bv[e] = (g.bias && e < nc) ? g.bias[col + e] : 0.f;
      for (int r2 = 0; r2 < 32; r2 += 2) {
        const int r = r2 + (lane >> 4);
        const int row = row0 + r;
        if (row0 + r2 >= g.M) break;
        const float4 a4 = *reinterpret_cast<const float4*>(&st[r * kLd + 4 * (lane & 15)]);
        float x[4] = {a4.x + bv[0], a4.y + bv[1], a4.z + bv[2], a4.w + bv[3]};
        const bool rin = row < g.M;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          if (g.relu) x[e] = fmaxf(x[e], 0.f);
          if (g.mask && rin && e < nc &&
              !(__bfloat162float(g.mask[(int64_t)row * g.ldm + col + e]) > 0.f))
            x[e] = 0.f;
          if (e >= nc || !rin) x[e] = 0.f;
          csum[e] += x[e];
        }
        if (nc == 0 || !rin) continue;
        const int64_t o = (int64_t)row * g.ldo + col;
        if (g.vec_out && nc == 4) {
          if (g.out_f32)
            *reinterpret_cast<float4*>(g.out_f32 + o) = make_float4(x[0], x[1], x[2], x[3]);
          if (g.out_bf16) {
            __nv_bfloat162 p0 = __floats2bfloat162_rn(x[0], x[1]);
            __nv_bfloat162 p1 = __floats2bfloat162_rn(x[2], x[3]);
            uint2 pk;
            pk.x = *reinterpret_cast<uint32_t*>(&p0);
            pk.y = *reinterpret_cast<uint32_t*>(&p1);
            *reinterpret_cast<uint2*>(g.out_bf16 + o) = pk;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if (e >= nc) break;
            if (g.out_f32) g.out_f32[o + e] = x[e];
            if (g.out_bf16) g.out_bf16[o + e] = __float2bfloat16_rn(x[e]);
          }
        }
      }
      if (g.colsum) {  // the two half-warps' sums of each column, one atomic per column
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float tot = csum[e] + __shfl_xor_sync(0xffffffffu, csum[e], 16);
          if (lane < 16 && col + e < g.N) atomicAdd(&g.colsum[col + e], tot);
        }
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

namespace {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

// Tensor map of a row-major [rows][K] BF16 matrix: boxes of 64 K-elements
// (128 bytes) x 128 rows, 128-byte swizzle, zeros outside the matrix.
bdg_status encode_operand(CUtensorMap* map, const void* base, int rows, int K) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return bdg_set_error(BDG_ECUDA, "gemm: cuTensorMapEncodeTiled is unavailable");
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)kBM};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                         strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return bdg_set_error(BDG_EINVAL, "gemm: tensor map of a %d x %d operand refused (%d)", rows,
                         K, (int)r);
  return BDG_OK;
}

}  // namespace

// C = epilogue(A * B^T) with row strides for the mask and the output; see GemmArgs.
// K % 8 == 0 (16-byte rows), A and B 16-byte aligned; ldm, ldo >= N.
bdg_status bdg_gemm_bf16_ld(const void* A, const void* B, int32_t M, int32_t N, int32_t K,
                            const float* bias, const void* mask, int32_t ldm, int32_t relu,
                            float* out_f32, void* out_bf16, int32_t ldo, float* colsum,
                            int32_t* err, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0 || (K & 7) || ldm < N || ldo < N)
    return bdg_set_error(BDG_EINVAL, "gemm: M=%d N=%d K=%d ldm=%d ldo=%d (K %% 8 == 0)", M, N,
                         K, ldm, ldo);
  if (((uintptr_t)A & 15) || ((uintptr_t)B & 15))
    return bdg_set_error(BDG_EINVAL, "gemm: A and B must be 16-byte aligned");
  CUtensorMap mapA, mapB;
  BDG_TRY(encode_operand(&mapA, A, M, K));
  BDG_TRY(encode_operand(&mapB, B, N, K));
  const bool vec = (ldo % 4 == 0) && ((uintptr_t)out_f32 % 16 == 0) &&
                   ((uintptr_t)out_bf16 % 16 == 0);
  const bool direct = bias && out_bf16 && !out_f32 && !mask && !colsum && (M % kBM == 0) &&
                      (N % kBN == 0) && (ldo % 8 == 0) && ((uintptr_t)bias % 16 == 0) &&
                      ((uintptr_t)out_bf16 % 16 == 0);
  GemmArgs g{(const __nv_bfloat16*)A, (const __nv_bfloat16*)B, M, N, K, bias,
             (const __nv_bfloat16*)mask, ldm, relu, out_f32, (__nv_bfloat16*)out_bf16, ldo,
             colsum, err, vec ? 1 : 0, direct ? 1 : 0};
  const size_t smem = bdg_gemm_smem_bytes();
  BDG_CUDA_TRY(cudaFuncSetAttribute(gemm_bf16_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  const int64_t ntiles = (int64_t)((N + kBN - 1) / kBN) * ((M + kBM - 1) / kBM);
  const int grid = (int)(ntiles < bdg_num_sms() ? ntiles : bdg_num_sms());
  bdg_prof_scope prof("gemm", st);
  gemm_bf16_kernel<<<grid, kThreads, smem, st>>>(g, mapA, mapB);
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
