// knn_tc.cu -- Reduce 1 of Section 3.2 on the 5th-generation tensor cores.
//
// Hamming distance as a +-1 dot product: with s = 2y - 1 in {-1, +1}^bits,
// <s_a, s_b> = bits - 2 d(a, b). Codes become FP8 E4M3 +-1.0 and one
// tcgen05.mma kind::f8f6f4 (M = 128 visitors x N = 64 homes x K = 32 bits)
// accumulates in FP32 in tensor memory; every partial sum is an integer of
// magnitude <= 1024, so the result is exact.
//
// Work item = (partition p, 128 visitors of V_p). Roles inside a CTA:
//   * producer (one thread): streams 64-home tiles of the pre-expanded home
//     operand of p from HBM/L2 into a 2-stage shared-memory ring with
//     cp.async.bulk (TMA bulk copies completing on mbarriers);
//   * MMA issuer (one thread): K / 32 MMAs per tile into one of two TMEM
//     accumulators (64 columns each), then tcgen05.commit frees the stage and
//     hands the accumulator to the epilogue;
//   * epilogue (4 warps, one thread per visitor row = TMEM lane): reads the 64
//     dot products of its row and appends the values under its threshold as
//     words (d << 21 | home position) to a per-row candidate list in shared
//     memory. The homes of a partition are stored in ascending id order, so
//     word order is (d, id) order. An exact per-row histogram of the listed
//     distances (d < 256) lowers the threshold to the k-th smallest distance
//     seen so far after every 16 values; it only tightens, so every final
//     neighbour is kept. When a row's list is nearly full, the warp compacts
//     all its rows together against their thresholds (with an exact word
//     threshold if ties at the k-th distance fill the list); a row whose list
//     still overflows is flagged and recomputed by the popcount kernel.
// At the end of the item each warp selects, row by row, the k smallest
// (d, id) keys among the candidates inside the final threshold (bitonic sort
// of at most 128 keys) and writes the row's partial list.
//
// Every mbarrier wait is bounded; a wait that gives up sets the device error
// word and the CTA drains (waits for its own copies and MMAs, bounded) and
// frees its tensor memory before returning.
#include "common.cuh"
#include "tc05.cuh"

namespace {

constexpr int kM = 128;         // visitors per item (TMEM lanes)
constexpr int kNT = 64;         // homes per tile (TMEM columns per accumulator)
constexpr int kStages = 2;
constexpr int kCap = 124;       // candidate slots per row
constexpr int kHalf = 16;       // compaction is checked every 16 columns
constexpr int kHB = 256;        // exact distance histogram over d in [0, 256)
constexpr int kSortN = 128;     // keys sorted per row at selection
constexpr int kCandStride = kM + 1;  // words between candidate slots (odd: no bank conflicts)
constexpr int kThreads = 192;   // warps 0-3 epilogue, warp 4 producer, warp 5 MMA
constexpr uint32_t kPolls = 1u << 20;
constexpr int kPosBits = 21;    // home position bits in a candidate word
constexpr uint32_t kPosMask = (1u << kPosBits) - 1;

template <int W>
struct TcCfg {
  static constexpr int KB = 64 * W;               // bytes of one expanded code
  static constexpr int NB = kHB;                   // distance histogram bins (width 1)
  static constexpr uint32_t A_BYTES = kM * KB;
  static constexpr uint32_t B_BYTES = kNT * KB;
  static constexpr uint32_t HIST_BYTES = ((NB * kM) + 15) & ~15u;
  static constexpr uint32_t CAND_BYTES = ((kCap * kCandStride * 4) + 15) & ~15u;
  static constexpr uint32_t OFF_B = A_BYTES;
  static constexpr uint32_t OFF_HIST = OFF_B + kStages * B_BYTES;
  static constexpr uint32_t OFF_CAND = OFF_HIST + HIST_BYTES;
  static constexpr uint32_t OFF_SORT = OFF_CAND + CAND_BYTES;     // 4 warps x 128 keys
  static constexpr uint32_t OFF_BAR = OFF_SORT + 4 * kSortN * 8;
  static constexpr uint32_t SMEM = OFF_BAR + 256;
  static_assert(OFF_B % 16 == 0 && OFF_HIST % 16 == 0 && OFF_CAND % 16 == 0 &&
                    OFF_SORT % 16 == 0 && OFF_BAR % 16 == 0,
                "shared-memory regions must be 16-byte aligned");
  static_assert(SMEM <= 232448, "shared memory per block exceeds 227 KB");
};

// offset of (row r, byte kb) in a K-major no-swizzle operand whose rows are KB bytes
template <int KB>
__device__ __forceinline__ uint32_t cm_off(int r, int kb) {
  return (uint32_t)((r >> 3) * (KB * 8) + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15));
}

// 16 code bits -> 16 bytes of E4M3 (+1.0 = 0x38 for a set bit, -1.0 = 0xB8 otherwise)
__device__ __forceinline__ uint4 expand16(uint32_t bits16) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const uint32_t nib = (bits16 >> (4 * i)) & 0xFu;
    const uint32_t spread = ((nib * 0x00204081u) & 0x01010101u) << 7;  // bit j -> bit 8j+7
    w[i] = 0xB8B8B8B8u ^ spread;
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst), "l"(src), "r"(bytes), "r"(tc05::smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
          tc05::smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

// Expanded home operand: row e of the 64-padded order of partition p holds
// home_codes[home_off[p] + (e - eoff[p])] (zeros past |H_p|) as KB bytes of
// E4M3 in the K-major core-matrix layout (8-row groups of KB * 8 bytes).
template <int W>
__global__ void expand_homes_kernel(const uint64_t* __restrict__ home_codes,
                                    const int32_t* __restrict__ home_off,
                                    const int32_t* __restrict__ eoff, int m, int64_t max_rows,
                                    uint8_t* __restrict__ hexp) {
  constexpr int KB = 64 * W, Q = 4 * W;  // 16-bit chunks per code
  const int64_t x = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  // thread order: row-in-group fastest, then chunk, then group (contiguous 16-byte stores)
  const int rr = (int)(x & 7);
  const int64_t rest = x >> 3;
  const int q = (int)(rest % Q);
  const int64_t grp = rest / Q;
  const int64_t e = grp * 8 + rr;
  if (e >= max_rows || e >= eoff[m]) return;
  int lo = 0, hi = m;  // partition with eoff[lo] <= e < eoff[lo + 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (eoff[mid] <= e) lo = mid; else hi = mid;
  }
  const int64_t local = e - eoff[lo];
  const int32_t nh = home_off[lo + 1] - home_off[lo];
  uint4 v = make_uint4(0, 0, 0, 0);
  if (local < nh) {
    const uint64_t word = home_codes[(int64_t)(home_off[lo] + local) * W + (q >> 2)];
    v = expand16((uint32_t)(word >> (16 * (q & 3))) & 0xFFFFu);
  }
  *reinterpret_cast<uint4*>(hexp + grp * (int64_t)(KB * 8) + (int64_t)q * 128 + rr * 16) = v;
}

__device__ __forceinline__ uint32_t cidx(int c, int r) {  // candidate slot c of row r
  return (uint32_t)(c * kCandStride + r);
}

// Keep the row's candidates below thr_w, in order; the histogram of listed
// distances (d < kHB) loses the dropped ones. Returns the new count.
__device__ __forceinline__ int compact_row(uint32_t* crow, int cnt, uint32_t thr_w,
                                           uint8_t* hist, int r) {
  int w = 0;
  for (int x = 0; x < cnt; ++x) {
    const uint32_t e = crow[x * kCandStride];
    if (e < thr_w) {
      crow[(w++) * kCandStride] = e;
    } else {
      const uint32_t d = e >> kPosBits;
      if (d < (uint32_t)kHB) hist[d * kM + r] = (uint8_t)(hist[d * kM + r] - 1);
    }
  }
  return w;
}

template <int W>
__global__ void __launch_bounds__(kThreads, 1)
knn_tc_kernel(bdg_knn_tc_args ta) {
  using C = TcCfg<W>;
  constexpr int KB = C::KB, NB = C::NB;
  extern __shared__ __align__(1024) uint8_t sm[];
  uint8_t* sA = sm;
  uint8_t* hist = sm + C::OFF_HIST;
  uint32_t* cand = reinterpret_cast<uint32_t*>(sm + C::OFF_CAND);
  uint64_t* sortbuf = reinterpret_cast<uint64_t*>(sm + C::OFF_SORT);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + C::OFF_BAR);
  uint64_t* full = bars;            // [2]
  uint64_t* empty = bars + 2;       // [2]
  uint64_t* tfull = bars + 4;       // [2]
  uint64_t* tempty = bars + 6;      // [2]
  uint64_t* drain = bars + 8;       // MMA drain at exit
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 9);
  int32_t* s_item = reinterpret_cast<int32_t*>(bars + 10);
  volatile int32_t* s_abort = reinterpret_cast<int32_t*>(bars + 11);

  const bdg_knn_args& a = ta.base;
  const bdg_csr& c = a.csr;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = a.m, k = a.k, bits = a.bits;
  const int32_t total_items = c.item_off[m];

  if (warp == 0) tc05::tmem_alloc(tmem_slot, 128);
  if (tid == 0) {
    for (int i = 0; i < 2; ++i) {
      tc05::mbar_init(&full[i], 1);
      tc05::mbar_init(&empty[i], 1);
      tc05::mbar_init(&tfull[i], 1);
      tc05::mbar_init(&tempty[i], 4);
    }
    tc05::mbar_init(drain, 1);
    *s_abort = 0;
    tc05::mbar_fence_init();
  }
  tc05::fence_before();
  __syncthreads();
  tc05::fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t id_mma = tc05::idesc(0u, 0u, kM, kNT);  // E4M3 x E4M3 -> F32
  uint32_t g = 0;       // tiles processed by this CTA so far (drives barrier phases)
  uint32_t nprod = 0;   // tiles whose copies the producer issued

  for (;;) {
    __syncthreads();
    if (tid == 0) *s_item = atomicAdd(a.item_counter, 1);
    __syncthreads();
    const int item = *s_item;
    if (item >= total_items || *s_abort) break;
    int lo = 0, hi = m;
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (c.item_off[mid] <= item) lo = mid; else hi = mid;
    }
    const int p = c.part_order[lo];
    const int tile = item - c.item_off[lo];
    const int v0 = c.visit_off[p] + tile * kM;
    const int nv = min(kM, c.visit_off[p + 1] - v0);
    const int h0 = c.home_off[p];
    const int nh = c.home_off[p + 1] - h0;
    const int ntiles = (nh + kNT - 1) / kNT;
    const int64_t e0 = c.eoff[p];
    if (nh > (int)kPosMask) {  // positions do not fit a candidate word: popcount fixup
      for (int r = tid; r < nv; r += kThreads) ta.fixflag[v0 + r] = 1;
      continue;
    }

    // ---- A operand: the item's visitor codes (staged in the candidate area,
    // which is free between items) expanded to E4M3 +-1 by all threads
    uint64_t* vwords = reinterpret_cast<uint64_t*>(cand);
    for (int x = tid; x < kM * W; x += kThreads) {
      const int r = x / W, w = x - r * W;
      uint64_t word = 0ull;
      if (r < nv) {
        const int32_t vid = c.visit_ids[v0 + r];
        if (vid >= 0) word = a.codes[(int64_t)vid * W + w];
      }
      vwords[x] = word;
    }
    __syncthreads();
    for (int x = tid; x < kM * 4 * W; x += kThreads) {
      const int rr = x & 7, rest = x >> 3;
      const int q = rest % (4 * W), grp = rest / (4 * W);
      const int r = grp * 8 + rr;
      const uint64_t word = vwords[r * W + (q >> 2)];
      *reinterpret_cast<uint4*>(sA + cm_off<KB>(r, q * 16)) =
          expand16((uint32_t)(word >> (16 * (q & 3))) & 0xFFFFu);
    }
    for (int x = tid; x < NB * kM / 4; x += kThreads) reinterpret_cast<uint32_t*>(hist)[x] = 0u;
    tc05::fence_proxy_async();
    __syncthreads();

    if (warp == 4) {
      // ---------------- producer
      if (lane == 0) {
        for (int j = 0; j < ntiles && !*s_abort; ++j) {
          const uint32_t gg = g + j, st = gg & 1, use = gg >> 1;
          if (use > 0 && !tc05::mbar_wait(&empty[st], (use - 1) & 1, kPolls)) {
            atomicExch(ta.err, 1); *s_abort = 1; break;
          }
          arrive_expect_tx(&full[st], C::B_BYTES);
          bulk_g2s(tc05::smem_u32(sm + C::OFF_B + st * C::B_BYTES),
                   ta.hexp + (e0 + (int64_t)j * kNT) * KB, C::B_BYTES, &full[st]);
          ++nprod;
        }
      }
    } else if (warp == 5) {
      // ---------------- MMA issuer
      if (lane == 0) {
        const uint32_t a0 = tc05::smem_u32(sA);
        for (int j = 0; j < ntiles && !*s_abort; ++j) {
          const uint32_t gg = g + j, st = gg & 1, b = gg & 1;
          if (!tc05::mbar_wait(&full[st], (gg >> 1) & 1, kPolls) ||
              (gg >= 2 && !tc05::mbar_wait(&tempty[b], ((gg >> 1) - 1) & 1, kPolls))) {
            atomicExch(ta.err, 2); *s_abort = 1; break;
          }
          tc05::fence_after();
          const uint32_t b0 = tc05::smem_u32(sm + C::OFF_B + st * C::B_BYTES);
#pragma unroll
          for (int kk = 0; kk < KB / 32; ++kk) {
            const uint64_t ad = tc05::sdesc(a0 + kk * 256, 128, KB * 8);
            const uint64_t bd = tc05::sdesc(b0 + kk * 256, 128, KB * 8);
            tc05::mma_f8(tmem + b * kNT, ad, bd, id_mma, kk > 0 ? 1u : 0u);
          }
          tc05::commit(&empty[st]);
          tc05::commit(&tfull[b]);
        }
      }
    } else {
      // ---------------- epilogue: thread r owns visitor row r (TMEM lane r)
      // A candidate word is (d << 21) | position of the home in H_p. The homes of
      // a partition are stored in ascending id order, so word order is exactly
      // (d, id) order: the row keeps an exact threshold on words.
      const int r = tid;
      const bool live = r < nv && c.visit_ids[v0 + r] >= 0;
      // v is one of its own partition's homes: its self pair (d = 0) is counted
      // like any other value and dropped at selection, so k + 1 values are needed
      const int need_k = k + ((live && c.visit_slot[v0 + r] == 0) ? 1 : 0);
      uint32_t thr_w = live ? 0xFFFFFFFFu : 0u;  // accept word < thr_w
      if (live && a.home_kth != nullptr) {  // sub-round: the running k-th key bounds d
        const uint64_t kth = a.home_kth[(int64_t)c.visit_ids[v0 + r] * k + (k - 1)];
        if (kth < bdg_pad_key(bits)) thr_w = (uint32_t)(bdg_key_d(kth) + 1) << kPosBits;
      }
      int cnt = 0;   // entries in the row's candidate list
      int cle = 0;   // entries with word < thr_w (every value seen below thr_w is listed)
      bool overflow = false;
      const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
      const float hbits = 0.5f * (float)bits;  // d = (bits - dot) / 2 = dot * -0.5 + bits / 2
      uint32_t* crow = cand + r;
      for (int j = 0; j < ntiles; ++j) {
        const uint32_t gg = g + j, b = gg & 1;
        bool ok = !*s_abort && tc05::mbar_wait(&tfull[b], (gg >> 1) & 1, kPolls);
        ok = __all_sync(0xffffffffu, ok);  // the warp leaves together
        if (!ok) {
          if (lane == 0) { atomicExch(ta.err, 3); *s_abort = 1; }
          break;
        }
        tc05::fence_after();
        uint32_t v[64];
        tc05::ld32(tmem + lane_base + b * kNT, *reinterpret_cast<uint32_t(*)[32]>(&v[0]));
        tc05::ld32(tmem + lane_base + b * kNT + 32, *reinterpret_cast<uint32_t(*)[32]>(&v[32]));
        tc05::wait_ld();
        tc05::fence_before();
        __syncwarp();
        if (lane == 0) tc05::mbar_arrive(&tempty[b]);
        const uint32_t pos0 = (uint32_t)(j * kNT);
        const int nvalid = min(kNT, nh - j * kNT);
#pragma unroll
        for (int half = 0; half < kNT / kHalf; ++half) {
          // compaction, taken by the whole warp at once as soon as one row's list
          // could not take another 16 values (lanes compacting one by one would
          // serialise the warp)
          if (__any_sync(0xffffffffu, cnt > kCap - kHalf)) {
            int td = (int)((thr_w - 1u) >> kPosBits);
            if (cle >= need_k && td >= kHB) {
              // outside the histogram: binary search of the k-th distance over the list
              int lo = 0, hi = min(td, bits);
              while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                int c2 = 0;
                for (int x = 0; x < cnt; ++x) {
                  const uint32_t e = crow[x * kCandStride];
                  c2 += (e < thr_w && (int)(e >> kPosBits) <= mid);
                }
                if (c2 >= need_k) hi = mid; else lo = mid + 1;
              }
              thr_w = min(thr_w, (uint32_t)(lo + 1) << kPosBits);
            }
            cnt = compact_row(crow, cnt, thr_w, hist, r);
            cle = cnt;
            if (cnt > kCap - kHalf) {
              // heavy ties at the k-th distance: the exact need_k-th smallest word
              // becomes the threshold, leaving exactly need_k entries
              td = (int)((thr_w - 1u) >> kPosBits);
              int c_lt = 0;
              for (int x = 0; x < cnt; ++x)
                c_lt += ((int)(crow[x * kCandStride] >> kPosBits) < td);
              const int want = need_k - c_lt - 1;  // rank among the entries at td
              uint32_t wk = thr_w - 1u;
              for (int x = 0; x < cnt; ++x) {
                const uint32_t e = crow[x * kCandStride];
                if ((int)(e >> kPosBits) != td) continue;
                int below = 0;
                for (int y = 0; y < cnt; ++y) {
                  const uint32_t f = crow[y * kCandStride];
                  below += (f < e && (int)(f >> kPosBits) == td);
                }
                if (below == want) wk = e;
              }
              thr_w = wk + 1u;
              cnt = compact_row(crow, cnt, thr_w, hist, r);
              cle = cnt;
            }
            if (cnt > kCap - kHalf) {  // still full: the popcount kernel redoes this row
              overflow = true;
              thr_w = 0u;  // accept nothing more
              cnt = 0;     // (the row's list is no longer used)
            }
          }
          // branch-free append: every value is written at the running slot, only
          // words below the threshold advance it
          const int c_before = cnt;
          uint32_t* wp = crow + cnt * kCandStride;
          const uint32_t posq = pos0 + (uint32_t)(half * kHalf);
          if (nvalid == kNT) {
#pragma unroll
            for (int c2 = 0; c2 < kHalf; ++c2) {
              const float dot = __uint_as_float(v[half * kHalf + c2]);
              const uint32_t d = (uint32_t)__float2int_rz(fmaf(dot, -0.5f, hbits));
              const uint32_t word = d * (1u << kPosBits) + (posq + c2);
              *wp = word;
              wp += (word < thr_w) ? kCandStride : 0;
            }
          } else {
#pragma unroll
            for (int c2 = 0; c2 < kHalf; ++c2) {
              const int cc = half * kHalf + c2;
              const float dot = __uint_as_float(v[cc]);
              const uint32_t d = (uint32_t)__float2int_rz(fmaf(dot, -0.5f, hbits));
              const uint32_t word = d * (1u << kPosBits) + (posq + c2);
              *wp = word;
              wp += (word < thr_w && cc < nvalid) ? kCandStride : 0;
            }
          }
          cnt = (int)((wp - crow) / kCandStride);
          if (cnt > c_before) {
            cle += cnt - c_before;
            for (int x = c_before; x < cnt; ++x) {
              const uint32_t d = crow[x * kCandStride] >> kPosBits;
              if (d > (uint32_t)bits) {  // cannot happen for +-1 operands
                atomicExch(ta.err, 5);
                continue;
              }
              if (d < (uint32_t)kHB) hist[d * kM + r] = (uint8_t)(hist[d * kM + r] + 1);
            }
            // lower the bound one distance at a time while need_k listed words
            // stay below it; every listed word at the bound's distance is below
            // the bound, so hist counts them exactly
            int td = (int)((thr_w - 1u) >> kPosBits);
            while (td > 0 && td < kHB) {
              const int h = hist[td * kM + r];
              if (cle - h < need_k) break;
              cle -= h;
              thr_w = (uint32_t)td << kPosBits;
              --td;
            }
          }
        }
      }
      // ---- final compaction: only candidates inside the final threshold remain
      if (!overflow) {
        cnt = compact_row(crow, cnt, thr_w, hist, r);
        if (cnt > kSortN) overflow = true;  // cannot happen: cnt <= kCap
      }
      // ---- selection: k smallest (d, id) among candidates inside the threshold
      uint64_t* sb = sortbuf + warp * 128;
      const uint64_t pad = bdg_pad_key(bits);
      for (int rr = 0; rr < 32; ++rr) {
        const int row = warp * 32 + rr;
        const int n_r = __shfl_sync(0xffffffffu, cnt, rr);
        const uint32_t tb = __shfl_sync(0xffffffffu, thr_w, rr);
        const int ovf = __shfl_sync(0xffffffffu, overflow ? 1 : 0, rr);
        if (row >= nv) continue;
        const int32_t vid = c.visit_ids[v0 + row];
        if (vid < 0) {  // an invalid id: its row (written by position) is padding
          if (a.t == 1 && a.out_by_pos) {
            const int64_t orow = (int64_t)(tile * kM + row);
            for (int j2 = lane; j2 < k; j2 += 32) {
              a.out_ids[orow * k + j2] = -1;
              a.out_dist[orow * k + j2] = bits + 1;
            }
          }
          continue;
        }
        if (ovf) {  // recomputed by the popcount kernel
          if (lane == 0) ta.fixflag[v0 + row] = 1;
          continue;
        }
        if (n_r <= 32) {
          // few candidates: one key per lane, bitonic sort across the warp in registers
          uint64_t key = BDG_KEY_INF;
          if (lane < n_r) {
            const uint32_t e = cand[cidx(lane, row)];
            const int d = (int)(e >> kPosBits);
            if (e < tb) {
              const int32_t hid = c.home_ids[h0 + (int)(e & kPosMask)];
              if (hid != vid) key = bdg_key((uint32_t)d, (uint32_t)hid);
            }
          }
#pragma unroll
          for (int k2 = 2; k2 <= 32; k2 <<= 1) {
#pragma unroll
            for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
              const uint64_t o = __shfl_xor_sync(0xffffffffu, key, j2);
              const bool up = (lane & k2) == 0, low = (lane & j2) == 0;
              key = (low == up) ? (key < o ? key : o) : (key < o ? o : key);
            }
          }
          sb[lane] = key;
          sb[lane + 32] = BDG_KEY_INF;
          sb[lane + 64] = BDG_KEY_INF;
          sb[lane + 96] = BDG_KEY_INF;
          __syncwarp();
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int x = lane + 32 * q;
            uint64_t key = BDG_KEY_INF;
            if (x < n_r) {
              const uint32_t e = cand[cidx(x, row)];
              const int d = (int)(e >> kPosBits);
              if (e < tb) {
                const int32_t hid = c.home_ids[h0 + (int)(e & kPosMask)];
                if (hid != vid) key = bdg_key((uint32_t)d, (uint32_t)hid);
              }
            }
            sb[x] = key;
          }
          __syncwarp();
          // bitonic sort of 128 keys, ascending
          for (int size = 2; size <= 128; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
              for (int q = 0; q < 2; ++q) {
                const int i = lane + 32 * q;                           // pair index 0..63
                const int lo2 = (i / stride) * (2 * stride) + (i % stride);
                const int hi2 = lo2 + stride;
                const bool up = (lo2 & size) == 0;
                const uint64_t x0 = sb[lo2], x1 = sb[hi2];
                if ((x0 > x1) == up) { sb[lo2] = x1; sb[hi2] = x0; }
              }
              __syncwarp();
            }
          }
        }
        if (a.t == 1) {
          const int64_t orow = a.out_by_pos ? (int64_t)(tile * kM + row) : (int64_t)vid;
          for (int j2 = lane; j2 < k; j2 += 32) {
            const uint64_t key = sb[j2] < pad ? sb[j2] : pad;
            a.out_ids[orow * k + j2] = key < pad ? bdg_key_id(key) : -1;
            a.out_dist[orow * k + j2] = bdg_key_d(key);
          }
        } else if (!a.merge_running) {  // round A: the running list starts as this row
          uint64_t* out = a.partial + (int64_t)vid * k;
          for (int j2 = lane; j2 < k; j2 += 32) out[j2] = sb[j2] < pad ? sb[j2] : pad;
        } else {
          bdg_warp_merge_running(a.partial + (int64_t)vid * k, sb, k, k, pad, lane);
        }
        __syncwarp();
      }
    }
    g += ntiles;
    __syncthreads();
  }

  // ---- drain: own copies and MMAs finished before TMEM is released
  if (warp == 5 && lane == 0) {
    tc05::commit(drain);
    if (!tc05::mbar_wait(drain, 0, kPolls)) atomicExch(ta.err, 4);
  }
  if (warp == 4 && lane == 0 && *s_abort) {
    // copies issued but possibly never consumed: wait for their completion
    for (uint32_t gg = (nprod > 2 ? nprod - 2 : 0); gg < nprod; ++gg)
      tc05::mbar_wait(&full[gg & 1], (gg >> 1) & 1, kPolls);
  }
  tc05::fence_before();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, 128);
}

template <int W>
bdg_status launch_w(const bdg_knn_tc_args& ta, bool expand, cudaStream_t st) {
  using C = TcCfg<W>;
  const bdg_knn_args& a = ta.base;
  if (expand) {  // expanded home operand (rows are bounded by N + 64 m)
    const int64_t max_rows = a.N + 64LL * a.m;
    const int64_t nthreads = ((max_rows + 7) / 8) * 8 * (4 * W);
    expand_homes_kernel<W><<<bdg_cdiv(nthreads, 256), 256, 0, st>>>(
        a.csr.home_codes, a.csr.home_off, a.csr.eoff, a.m, max_rows, ta.hexp);
    BDG_CUDA_TRY(cudaGetLastError());
    bdg_note_launch();
  }
  BDG_CUDA_TRY(cudaFuncSetAttribute(knn_tc_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)C::SMEM));
  const int grid = bdg_num_sms();
  {
    bdg_prof_scope prof("knn", st);
    knn_tc_kernel<W><<<grid, kThreads, C::SMEM, st>>>(ta);
    BDG_CUDA_TRY(cudaGetLastError());
    bdg_note_launch();
  }
  // rows whose candidate list overflowed: exact recomputation by the popcount kernel
  BDG_CUDA_TRY(cudaMemsetAsync(a.item_counter, 0, sizeof(int32_t), st));
  bdg_knn_args fx = a;
  fx.fixflag = ta.fixflag;
  return bdg_launch_knn_popc(fx, W, st);
}

}  // namespace

bool bdg_knn_tc_supported(int W, int k) { return (W == 4 || W == 8) && k >= 1 && k <= 64; }

size_t bdg_knn_tc_hexp_bytes(int64_t N, int m, int W) {
  return (size_t)(N + 64LL * m) * 64 * W;
}

bdg_status bdg_launch_knn_tc(const bdg_knn_tc_args& a, int W, bool expand, cudaStream_t st) {
  if (W == 4) return launch_w<4>(a, expand, st);
  if (W == 8) return launch_w<8>(a, expand, st);
  return bdg_set_error(BDG_EUNSUPPORTED, "tensor k-NN path needs 256- or 512-bit codes");
}
