// knn_tc.cu -- Reduce 1 of Section 3.2 on the 5th-generation tensor cores.
//
// Hamming distance as a +-1 dot product: with s = 2y - 1 in {-1, +1}^bits,
// <s_a, s_b> = bits - 2 d(a, b). Codes become FP8 E4M3 +-1.0 and one
// tcgen05.mma kind::f8f6f4 (M = 128 visitors x N = 128 homes x K = 32 bits)
// accumulates in FP32 in tensor memory; every partial sum is an integer of
// magnitude <= 1024, so the result is exact.
//
// Work item = (partition p, 128 visitors of V_p). The visitors' codes are the
// A operand: each epilogue thread writes its visitor's code, expanded to E4M3,
// into its tensor-memory lane, and the MMAs read A from there (shared memory
// holds only the home tiles, so its bandwidth serves B alone). Roles:
//   * producer (one thread): streams 128-home tiles of the pre-expanded home
//     operand of p from HBM/L2 into a shared-memory ring (2 stages of 64 KB at
//     512 bits, 4 at 256) with
//     cp.async.bulk (TMA bulk copies completing on mbarriers);
//   * MMA issuer (one thread): K / 32 MMAs per tile into one of three TMEM
//     accumulators (128 columns each), then tcgen05.commit frees the stage and
//     hands the accumulator to the epilogue;
//   * epilogue (4 warps, one thread per visitor row = TMEM lane): reads its
//     row's dot products, 64 at a time, and appends the values under its threshold as
//     words (d << 21 | id rank of the home in H_p) to a per-row candidate list
//     in shared memory, so word order is (d, id) order. When a row's list is
//     nearly full, the warp compacts all its rows together: the threshold of
//     each row becomes its exact k-th smallest distance so far (counted into
//     16 bins just below the current threshold, usually in one pass over the
//     list), or its exact k-th smallest word when ties at that distance fill
//     the list. The threshold only tightens, so every final neighbour is kept;
//   * lookup (one thread of warp 6): takes the next work item from the round's
//     counter and reads its partition's offsets while the current item runs.
// The homes are streamed in id order, or in locality order (sorted by nearest
// pivot home, with every tile's id ranks copied beside it); in locality order
// a round-A item starts at its own tile and spirals out.
// At the end of an item, in round A (and in a single-round build) each thread
// cuts its row's list to its k + 1 best words, ranks them by counting and
// writes its row without the self pair; in the sub-rounds each warp sorts, row
// by row, the few candidates below the running list's k-th key and merges them
// into that list. Round A and the sub-rounds are separate instantiations (RUN).
//
// Every mbarrier wait is bounded; a wait that gives up sets the device error
// word and the CTA drains (waits for its own copies and MMAs, bounded) and
// frees its tensor memory before returning.
#include "common.cuh"
#include "tc05.cuh"

namespace {

constexpr int kM = 128;         // visitors per item (TMEM lanes)
constexpr int kNT = BDG_TC_TILE;  // homes per tile (TMEM columns per accumulator)
constexpr int kSub = 64;        // columns the epilogue reads from TMEM at a time
constexpr int kMaxStages = 4;   // home-tile ring in shared memory (2 stages of 64 KB at 512 bits)
// candidate slots per row: 188 with the homes in id order; 180 in locality order,
// whose tiles' id ranks take 4 KB of shared memory
template <bool LOC>
struct CapOf { static constexpr int v = LOC ? 180 : 188; };
constexpr int kHalf = 16;       // compaction is checked every 16 columns
constexpr int kSortN = 128;     // keys sorted per row at selection (sub-rounds)
constexpr int kOutSlot = 96;    // first slot of a row's ranked words (round A / one round)
constexpr int kNeedMax = 65;    // k + 1 for the largest k the kernel takes
static_assert(kOutSlot >= kNeedMax && kOutSlot + kNeedMax <= CapOf<true>::v &&
                  kOutSlot + kNeedMax <= CapOf<false>::v,
              "ranked words need k + 1 free slots after the list");
// words between a row's candidate slots: slot c of row r is word c * (kM + 1) + r,
// so the 32 lanes of a warp touch 32 different banks both when they are 32 rows
// (whatever slot each row is at) and when they are 32 consecutive slots of one
// row (the write-out)
constexpr int kCandStride = kM + 1;
constexpr int kThreads = 224;   // warps 0-3 epilogue, 4 producer, 5 MMA, 6 next-item lookup
constexpr int kIdrSlots = 8;    // tiles of home id ranks in flight (locality order)
constexpr uint32_t kPolls = 1u << 20;
constexpr int kPosBits = 21;    // home position bits in a candidate word
constexpr uint32_t kPosMask = (1u << kPosBits) - 1;

constexpr int kAcc = 3;                  // accumulators: the MMAs run up to 2 tiles ahead
constexpr uint32_t kAccCols = kAcc * kNT;  // accumulators in TMEM columns [0, 384)
constexpr uint32_t kTmemCols = 512;        // + the visitors' operand in [384, 384 + KB / 4)
// barriers (full/empty per stage, tfull/tempty per accumulator, drain, id-rank
// slots), the TMEM address, the abort flag and two item records
constexpr uint32_t kBarBytes = 272;
static_assert((2 * kMaxStages + 2 * kAcc + 1 + kIdrSlots) * 8 + 16 + 2 * 8 * 4 <= kBarBytes,
              "barrier area too small");

template <int W, bool LOC>
struct TcCfg {
  static constexpr int KB = 64 * W;               // bytes of one expanded code
  static constexpr uint32_t B_BYTES = kNT * KB;
  static constexpr int STAGES = W >= 8 ? 2 : kMaxStages;
  static constexpr int CAP = CapOf<LOC>::v;
  static constexpr uint32_t CAND_BYTES = ((CAP * kCandStride * 4) + 15) & ~15u;
  static constexpr uint32_t OFF_B = 0;
  static constexpr uint32_t OFF_CAND = OFF_B + STAGES * B_BYTES;
  static constexpr uint32_t OFF_SORT = OFF_CAND + CAND_BYTES;     // 4 warps x 128 keys
  static constexpr uint32_t OFF_IDR = OFF_SORT + 4 * kSortN * 8;   // kIdrSlots x 128 id ranks
  static constexpr uint32_t OFF_BAR = OFF_IDR + (LOC ? kIdrSlots * kNT * 4 : 0);
  static constexpr uint32_t SMEM = OFF_BAR + kBarBytes;
  static_assert(OFF_B % 16 == 0 && OFF_CAND % 16 == 0 && OFF_SORT % 16 == 0 &&
                    OFF_IDR % 16 == 0 && OFF_BAR % 16 == 0,
                "shared-memory regions must be 16-byte aligned");
  static_assert(SMEM <= 232448, "shared memory per block exceeds 227 KB");
  static_assert(kAccCols + KB / 4 <= kTmemCols, "visitor operand does not fit in TMEM");
};

// Expanded home operand: row e of the 128-padded order of partition p holds
// home_codes[home_off[p] + r] with r = e - eoff[p] (id order) or r = loc_idr[e]
// (locality order), zeros past |H_p|, as KB bytes of E4M3 in the K-major
// core-matrix layout (8-row groups of KB * 8 bytes).
template <int W>
__global__ void expand_homes_kernel(const uint64_t* __restrict__ home_codes,
                                    const int32_t* __restrict__ home_off,
                                    const int32_t* __restrict__ eoff,
                                    const int32_t* __restrict__ loc_idr, int m, int64_t max_rows,
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
  if (local < nh) {  // locality order: row e holds the home of id rank loc_idr[e]
    const int64_t src = home_off[lo] + (loc_idr ? (int64_t)loc_idr[e] : local);
    const uint64_t word = home_codes[src * W + (q >> 2)];
    v = tc05::expand16((uint32_t)(word >> (16 * (q & 3))) & 0xFFFFu);
  }
  *reinterpret_cast<uint4*>(hexp + grp * (int64_t)(KB * 8) + (int64_t)q * 128 + rr * 16) = v;
}

// The j-th tile an item visits in locality order: tile `own` first, then
// alternately the next tile to the right and to the left while both sides have
// tiles, then the rest of the longer side (a bijection on [0, n)).
__device__ __forceinline__ int spiral_tile(int j, int own, int n) {
  if (j == 0) return own;
  const int s = min(own, n - 1 - own);  // tiles on the shorter side
  if (j <= 2 * s) return own + ((j & 1) ? (j + 1) / 2 : -(j / 2));
  return own + (n - 1 - own > own ? j - s : -(j - s));
}

__device__ __forceinline__ uint32_t cidx(int c, int r) {  // candidate slot c of row r
  return (uint32_t)(c * kCandStride + r);
}

// Keep the row's candidates below thr_w, in order. Returns the new count.
// Words are read eight at a time into registers before any is written back: a
// kept word only moves down (to a slot already read), and the loads of a batch
// do not wait for the stores of the previous one.
__device__ __forceinline__ int compact_row(uint32_t* crow, int cnt, uint32_t thr_w) {
  int w = 0;
  for (int x = 0; x < cnt; x += 8) {
    uint32_t e[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) e[q] = x + q < cnt ? crow[(x + q) * kCandStride] : 0xFFFFFFFFu;
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (e[q] < thr_w) crow[(w++) * kCandStride] = e[q];
  }
  return w;
}

// 16 byte counters in four words (counter s is byte s % 4 of c[s / 4]): adds
// one to counter sb, nothing for sb >= 16. PTX shl yields 0 for a shift of 32
// or more, so each word takes its one-hot byte without a select.
__device__ __forceinline__ uint32_t shl_clamp(uint32_t a, uint32_t n) {
  uint32_t r;
  asm("shl.b32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(n));
  return r;
}
__device__ __forceinline__ void bin16_add(uint32_t (&c)[4], uint32_t sb) {
  const uint32_t x = min(sb, 16u) << 3;  // bit of counter sb in the 128-bit row
  c[0] += shl_clamp(1u, x);
  c[1] += shl_clamp(1u, x - 32u);
  c[2] += shl_clamp(1u, x - 64u);
  c[3] += shl_clamp(1u, x - 96u);
}
__device__ __forceinline__ int bin16_get(const uint32_t (&c)[4], int s) {
  return (int)((c[s >> 2] >> (8 * (s & 3))) & 0xFFu);
}

// The smallest distance lo with at least need_k listed words at distance <= lo
// (every listed word has d <= td, and there are at least need_k of them). One
// pass over the list counts the words in 16 bins of 2^shift distances below
// `base`; the words above the bins are known from earlier passes, so the words
// below them follow, and the running count from the bottom names the bin
// holding lo. A bin of one distance is the answer; a wider bin is split again
// into 16, and when lo lies below every bin the bins move down. After a small
// drop of the bound one pass suffices; an open bound (td = bits) takes three.
__device__ __forceinline__ int kth_dist(const uint32_t* crow, int cnt, int need_k, int td,
                                        int bits) {
  int base = td;
  int shift = td >= bits ? 5 : 0;  // an open bound: bins of 32 distances first
  int above = 0;                   // words with d > base
  for (int pass = 0; pass < 12; ++pass) {
    uint32_t c[4] = {0u, 0u, 0u, 0u};  // counter s: words with (base - d) >> shift == s
    for (int x = 0; x < cnt; x += 8) {
      uint32_t e[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) e[q] = x + q < cnt ? crow[(x + q) * kCandStride] : 0xFFFFFFFFu;
#pragma unroll
      for (int q = 0; q < 8; ++q)  // above base (or no word): t < 0, a huge bin
        bin16_add(c, (uint32_t)(base - (int)(e[q] >> kPosBits)) >> shift);
    }
    int binned = 0;
#pragma unroll
    for (int sb = 0; sb < 16; ++sb) binned += bin16_get(c, sb);
    const int below = cnt - above - binned;  // (base - d) >> shift >= 16
    if (below >= need_k) {  // below every bin: move the bins down
      above += binned;
      base -= 16 << shift;
      shift = min(shift + 4, 6);
      continue;
    }
    int run = below, bin = 0;
#pragma unroll
    for (int sb = 15; sb >= 0; --sb) {  // the highest bin (lowest d) reaching need_k
      const int before = run;
      run += bin16_get(c, sb);
      if (before < need_k && run >= need_k) bin = sb;
    }
    if (shift == 0) return base - bin;
#pragma unroll
    for (int sb = 0; sb < 16; ++sb) above += sb < bin ? bin16_get(c, sb) : 0;
    base -= bin << shift;  // the bin (base - 2^shift, base]: split it into 16
    shift = max(shift - 4, 0);
  }
  return 0;  // not reached: every pass narrows the range or moves below it
}

// The need_k-th smallest listed word, known to lie in [wbase, wbase + 2^rb)
// (the words of one distance, rb the bits of their low field; no listed word
// lies above that range): the same search over 16 bins of the low field, four
// bits at a time from the top, the words below the bins following from the
// count.
__device__ __forceinline__ uint32_t kth_word(const uint32_t* crow, int cnt, int need_k,
                                            uint32_t wbase, int rb) {
  uint32_t lo = wbase;
  // a multiple of 4, so that the 16 bins of a split cover exactly the bin split
  int shift = rb > 4 ? (rb - 1) / 4 * 4 : 0;
  int above = 0;  // words at or above the top of the bins
  for (int pass = 0; pass < 8; ++pass) {
    uint32_t c[4] = {0u, 0u, 0u, 0u};  // counter s: words with (w - lo) >> shift == s
    for (int x = 0; x < cnt; x += 8) {
      uint32_t e[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) e[q] = x + q < cnt ? crow[(x + q) * kCandStride] : 0xFFFFFFFFu;
#pragma unroll
      for (int q = 0; q < 8; ++q)  // below lo: no bin
        bin16_add(c, e[q] >= lo ? (e[q] - lo) >> shift : 16u);
    }
    int binned = 0;
#pragma unroll
    for (int sb = 0; sb < 16; ++sb) binned += bin16_get(c, sb);
    int run = cnt - above - binned, bin = 0;  // starts with the words below lo
#pragma unroll
    for (int sb = 0; sb < 16; ++sb) {  // the lowest bin whose running count reaches need_k
      const int before = run;
      run += bin16_get(c, sb);
      if (before < need_k && run >= need_k) bin = sb;
    }
    if (shift == 0) return lo + (uint32_t)bin;
#pragma unroll
    for (int sb = 0; sb < 16; ++sb) above += sb > bin ? bin16_get(c, sb) : 0;
    lo += (uint32_t)bin << shift;
    shift = max(shift - 4, 0);
  }
  return lo;  // not reached: the last pass has single-word bins
}

// Exact compaction of one row's list. Every listed word is below thr_w. Once
// the list holds need_k words, the bound becomes the need_k-th smallest
// distance and the words above it are dropped; if ties at that distance still
// leave more than `limit` words, the need_k-th smallest word itself becomes the
// bound, leaving exactly need_k. `ordered`: the list is in word order within a
// distance (homes in id order: words are appended by increasing position and
// compaction keeps their order); otherwise (locality order) the word is found
// by a search over the low `rank_bits` bits of the words at that distance.
// Returns the new count.
__device__ __forceinline__ int compact_exact(uint32_t* crow, int cnt, uint32_t& thr_w, int need_k,
                                             int bits, int limit, bool ordered, int rank_bits) {
  if (cnt < need_k) return cnt;
  // the k-th distance, found below td, the bound's distance
  const int td = min((int)((thr_w - 1u) >> kPosBits), bits);
  const int lo = kth_dist(crow, cnt, need_k, td, bits);
  thr_w = min(thr_w, (uint32_t)(lo + 1) << kPosBits);
  cnt = compact_row(crow, cnt, thr_w);
  if (cnt > limit) {
    uint32_t wk;
    if (ordered) {
      // words at distance lo are in position order: the bound is the
      // (need_k - #{d < lo})-th of them
      int c_lt = 0;
#pragma unroll 8
      for (int x = 0; x < cnt; ++x) c_lt += ((int)(crow[x * kCandStride] >> kPosBits) < lo);
      const int want = need_k - c_lt;  // 1-based rank among the words at distance lo
      wk = thr_w - 1u;
      int seen = 0;
      for (int x = 0; x < cnt; ++x) {
        const uint32_t e = crow[x * kCandStride];
        if ((int)(e >> kPosBits) == lo && ++seen == want) { wk = e; break; }
      }
    } else {
      // the need_k-th smallest word: among those at distance lo, whose low
      // fields (id ranks) have rank_bits bits
      wk = kth_word(crow, cnt, need_k, (uint32_t)lo << kPosBits, rank_bits);
    }
    thr_w = wk + 1u;
    cnt = compact_row(crow, cnt, thr_w);
  }
  return cnt;
}

// RUN: a sub-round (rows merge into running lists) or round A / a single round;
// compiled apart so that each path gets its own register allocation
template <int W, bool LOC, bool RUN>
__global__ void __launch_bounds__(kThreads, 1)
knn_tc_kernel(bdg_knn_tc_args ta) {
  using C = TcCfg<W, LOC>;
  constexpr int kCap = C::CAP;
  constexpr int KB = C::KB;
  extern __shared__ __align__(1024) uint8_t sm[];
  uint32_t* cand = reinterpret_cast<uint32_t*>(sm + C::OFF_CAND);
  uint64_t* sortbuf = reinterpret_cast<uint64_t*>(sm + C::OFF_SORT);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + C::OFF_BAR);
  constexpr int kStages = C::STAGES;
  uint64_t* full = bars;                  // [kStages]
  uint64_t* empty = bars + kMaxStages;    // [kStages]
  uint64_t* tfull = bars + 2 * kMaxStages;  // [kAcc]
  uint64_t* tempty = tfull + kAcc;        // [kAcc]
  uint64_t* drain = tempty + kAcc;        // MMA drain at exit
  uint64_t* idr_full = drain + 1;         // [kIdrSlots] a tile's home id ranks landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(idr_full + kIdrSlots);
  volatile int32_t* s_abort = reinterpret_cast<int32_t*>(idr_full + kIdrSlots) + 1;
  // two item records (item, p, tile, v0, nv, h0, nh, eoff[p]): the current one
  // and the next, looked up by warp 6 while the current item runs
  int32_t* s_info = reinterpret_cast<int32_t*>(idr_full + kIdrSlots) + 4;  // [2][8]
  int32_t* idr_sm = reinterpret_cast<int32_t*>(sm + C::OFF_IDR);

  const bdg_knn_args& a = ta.base;
  const bdg_csr& c = a.csr;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m = a.m, k = a.k, bits = a.bits;
  int32_t item_begin, item_end;
  bdg_item_range(c, m, a.size_lo, a.size_hi, &item_begin, &item_end);

  if (warp == 0) tc05::tmem_alloc(tmem_slot, kTmemCols);
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      tc05::mbar_init(&full[i], 1);
      tc05::mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < kAcc; ++i) {
      tc05::mbar_init(&tfull[i], 1);
      tc05::mbar_init(&tempty[i], 4);
    }
    tc05::mbar_init(drain, 1);
    for (int i = 0; i < kIdrSlots; ++i) tc05::mbar_init(&idr_full[i], 1);
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
  // Locality order (loc_idr set): the operand rows are the homes sorted by pivot,
  // each tile comes with the id ranks of its 128 homes, and candidate words
  // carry those ranks. In round A an item visits the tiles in a spiral from its
  // own tile (its visitors are that tile's homes); sub-round items visit the
  // tiles in order.
  const int32_t* loc_idr = LOC ? c.loc_idr : nullptr;
  const bool ordered = !LOC;

  // the next work item from the round's counter, and its partition's offsets
  auto lookup = [&](int32_t* dst) {
    const int item = item_begin + atomicAdd(a.item_counter, 1);
    dst[0] = item;
    if (item < item_end) {
      const int lo = c.item_lo[item];  // rank of the item's partition in part_order
      const int p = c.part_order[lo];
      const int tile = item - c.item_off[lo];
      const int v0 = c.visit_off[p] + tile * kM;
      dst[1] = p;
      dst[2] = tile;
      dst[3] = v0;
      dst[4] = min(kM, c.visit_off[p + 1] - v0);
      dst[5] = c.home_off[p];
      dst[6] = c.home_off[p + 1] - dst[5];
      dst[7] = c.eoff[p];
    }
  };
  if (tid == 6 * 32) lookup(s_info);

  for (uint32_t it = 0;; ++it) {
    __syncthreads();
    const int32_t* inf = s_info + 8 * (it & 1);
    const int item = inf[0];
    if (item >= item_end || *s_abort) break;
    const int p = inf[1], tile = inf[2], v0 = inf[3], nv = inf[4], h0 = inf[5], nh = inf[6];
    const int64_t e0 = inf[7];
    const int ntiles = (nh + kNT - 1) / kNT;
    // warp 6 looks up the next item meanwhile (read after the next barrier)
    if (tid == 6 * 32) lookup(s_info + 8 * ((it + 1) & 1));
    const int rank_bits = nh > 1 ? 32 - __clz(nh - 1) : 1;  // bits of an id rank in H_p
    const int start = loc_idr != nullptr && !RUN ? tile : -1;  // spiral start
    if (nh > (int)kPosMask) {  // positions do not fit a candidate word: popcount fixup
      for (int r = tid; r < nv; r += kThreads) ta.fixflag[v0 + r] = 1;
      if (tid == 0) ta.err[1] = 1;
      continue;
    }

    // ---- A operand: each epilogue thread writes its visitor's code, as E4M3
    // +-1 (+1 for a set bit), into its TMEM lane: column c holds code bits
    // 4c .. 4c + 3, one byte each (the layout tcgen05.mma reads A from TMEM in)
    if (warp < 4) {
      const int r = tid;
      uint64_t cw[W];
      const int32_t vid = r < nv ? c.visit_ids[v0 + r] : -1;
#pragma unroll
      for (int w = 0; w < W; ++w) cw[w] = vid >= 0 ? a.codes[(int64_t)vid * W + w] : 0ull;
#pragma unroll
      for (int ch = 0; ch < W / 2; ++ch) {  // 32 columns = 128 code bits per store
        uint32_t col[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const uint64_t word = cw[2 * ch + (q >> 4)];
          const uint32_t nib = (uint32_t)(word >> (4 * (q & 15))) & 0xFu;
          col[q] = vid >= 0 ? 0xB8B8B8B8u ^ (((nib * 0x00204081u) & 0x01010101u) << 7) : 0u;
        }
        tc05::st32(tmem + ((uint32_t)(32 * warp) << 16) + kAccCols + 32 * ch, col);
      }
      tc05::wait_st();
    }
    tc05::fence_before();
    __syncthreads();

    if (warp == 4) {
      // ---------------- producer
      if (lane == 0) {
        for (int j = 0; j < ntiles && !*s_abort; ++j) {
          const uint32_t gg = g + j, st = gg % kStages, use = gg / kStages;
          if (use > 0 && !tc05::mbar_wait(&empty[st], (use - 1) & 1, kPolls)) {
            atomicExch(ta.err, 1); *s_abort = 1; break;
          }
          const int jt = start >= 0 ? spiral_tile(j, start, ntiles) : j;  // the home tile
          tc05::arrive_expect_tx(&full[st], C::B_BYTES);
          tc05::bulk_g2s(tc05::smem_u32(sm + C::OFF_B + st * C::B_BYTES),
                   ta.hexp + (e0 + (int64_t)jt * kNT) * KB, C::B_BYTES, &full[st]);
          if (loc_idr) {
            // slot gg % kIdrSlots is free: the epilogue is at most kIdrSlots - 1
            // tiles behind (this copy needed the MMAs of tile gg - kStages, those
            // needed the accumulator of tile gg - kStages - kAcc read)
            const uint32_t is = gg % kIdrSlots;
            tc05::arrive_expect_tx(&idr_full[is], kNT * 4);
            tc05::bulk_g2s(tc05::smem_u32(idr_sm + is * kNT), loc_idr + e0 + (int64_t)jt * kNT,
                     kNT * 4, &idr_full[is]);
          }
          ++nprod;
        }
      }
    } else if (warp == 5) {
      // ---------------- MMA issuer
      if (lane == 0) {
        const uint32_t a0 = tmem + kAccCols;  // visitors' operand (TMEM columns)
        for (int j = 0; j < ntiles && !*s_abort; ++j) {
          const uint32_t gg = g + j, st = gg % kStages, b = gg % kAcc;
          if (!tc05::mbar_wait(&full[st], (gg / kStages) & 1, kPolls) ||
              (gg >= kAcc && !tc05::mbar_wait(&tempty[b], ((gg / kAcc) - 1) & 1, kPolls))) {
            atomicExch(ta.err, 2); *s_abort = 1; break;
          }
          tc05::fence_after();
          const uint32_t b0 = tc05::smem_u32(sm + C::OFF_B + st * C::B_BYTES);
#pragma unroll
          for (int kk = 0; kk < KB / 32; ++kk) {  // K = 32 per MMA: 8 TMEM columns of A
            const uint64_t bd = tc05::sdesc(b0 + kk * 256, 128, KB * 8);
            tc05::mma_f8_ts(tmem + b * kNT, a0 + kk * 8, bd, id_mma, kk > 0 ? 1u : 0u);
          }
          tc05::commit(&empty[st]);
          tc05::commit(&tfull[b]);
        }
      }
    } else if (warp < 4) {
      // ---------------- epilogue: thread r owns visitor row r (TMEM lane r)
      // A candidate word is (d << 21) | position of the home in H_p. The homes of
      // a partition are stored in ascending id order, so word order is exactly
      // (d, id) order: the row keeps an exact threshold on words.
      const int r = tid;
      const int32_t myvid = r < nv ? c.visit_ids[v0 + r] : -1;  // this row's point
      const bool live = myvid >= 0;
      // a visitor of its own home set (slot 0) is one of the homes: its self pair
      // (d = 0) is counted like any other value and dropped at selection, so
      // k + 1 values are needed
      const bool excl = live && c.visit_slot[v0 + r] == 0;
      const int need_k = k + (excl ? 1 : 0);
      // accept word < thr_w; (bits + 1) << 21 accepts every real distance and no
      // missing home of a ragged tile (those read as d = bits + 1)
      uint32_t thr_w = live ? (uint32_t)(bits + 1) << kPosBits : 0u;
      uint64_t kth = BDG_KEY_INF;  // sub-round: the running list's k-th key
      if (RUN && live && a.home_kth != nullptr) {  // it bounds d, and no key above it can enter
        kth = a.home_kth[(int64_t)myvid * k + (k - 1)];
        if (kth < bdg_pad_key(bits)) thr_w = (uint32_t)(bdg_key_d(kth) + 1) << kPosBits;
      }
      int cnt = 0;   // entries in the row's candidate list
      bool overflow = false;
      const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
      // d = (bits - dot) / 2; adding 2^23 places the integer d in the low mantissa
      // bits of the FP32 result (exact: |dot| <= 1024), and multiplying those bits
      // by 2^21 (mod 2^32) leaves d << 21: the word is one FFMA and one IMAD
      const float hmagic = 0.5f * (float)bits + 8388608.0f;
      uint32_t* crow = cand + r;
      // a value can enter only if its distance is at most the threshold's distance
      // part td, i.e. if its dot product is at least bits - 2 td: the skip test's
      // limit, recomputed only when the threshold changes
      auto lim_of = [bits](uint32_t t) {
        return t ? (float)(bits - 2 * (int)((t - 1u) >> kPosBits)) : 3.0e38f;
      };
      float lim = lim_of(thr_w);
      // a row's list is compacted once it holds more than trig words: at most
      // kCap - 16 (room for the next 16 values); with small k (routing: the t
      // nearest centres) after a few dozen, so that the bound tightens early.
      // trig is also the compaction's tie limit, so a compaction always leaves
      // at most trig words and never has to run again at once
      const int trig = k <= 16 ? 2 * (k + 1) + 16 : min(kCap - kHalf, 4 * (k + 1) + 16);
      for (int j = 0; j < ntiles; ++j) {
        const uint32_t gg = g + j, b = gg % kAcc;
        const int jt = start >= 0 ? spiral_tile(j, start, ntiles) : j;  // the home tile
        bool ok = !*s_abort && tc05::mbar_wait(&tfull[b], (gg / kAcc) & 1, kPolls) &&
                  (!loc_idr ||
                   tc05::mbar_wait(&idr_full[gg % kIdrSlots], (gg / kIdrSlots) & 1, kPolls));
        ok = __all_sync(0xffffffffu, ok);  // the warp leaves together
        if (!ok) {
          if (lane == 0) { atomicExch(ta.err, 3); *s_abort = 1; }
          break;
        }
        tc05::fence_after();
#pragma unroll 1
        for (int sub = 0; sub < kNT / kSub; ++sub) {  // 64 columns at a time
          uint32_t v[kSub];
          const uint32_t tcol = tmem + lane_base + b * kNT + sub * kSub;
          tc05::ld32(tcol, *reinterpret_cast<uint32_t(*)[32]>(&v[0]));
          tc05::ld32(tcol + 32, *reinterpret_cast<uint32_t(*)[32]>(&v[32]));
          tc05::wait_ld();
          if (sub == kNT / kSub - 1) {  // the accumulator is read: hand it back
            tc05::fence_before();
            __syncwarp();
            if (lane == 0) tc05::mbar_arrive(&tempty[b]);
          }
          const uint32_t pos0 = (uint32_t)(jt * kNT + sub * kSub);
          const int nvalid = min(kSub, nh - (int)pos0);
          if (nvalid <= 0) continue;  // past the partition's last home
          if (nvalid < kSub) {  // ragged last columns: missing homes read as d = bits + 1
            const uint32_t padv = __float_as_uint(-(float)(bits + 2));
  #pragma unroll
            for (int cc = 0; cc < kSub; ++cc)
              if (cc >= nvalid) v[cc] = padv;
          }
  #pragma unroll
          for (int half = 0; half < kSub / kHalf; ++half) {
            // skip the 16 values when no row of the warp can take one of them: a value
            // can enter only if its distance is at most td, the bound's distance part
            {
              float f[kHalf];
  #pragma unroll
              for (int c2 = 0; c2 < kHalf; ++c2) f[c2] = __uint_as_float(v[half * kHalf + c2]);
              const float m0 = fmaxf(fmaxf(f[0], f[1]), fmaxf(f[2], f[3]));
              const float m1 = fmaxf(fmaxf(f[4], f[5]), fmaxf(f[6], f[7]));
              const float m2 = fmaxf(fmaxf(f[8], f[9]), fmaxf(f[10], f[11]));
              const float m3 = fmaxf(fmaxf(f[12], f[13]), fmaxf(f[14], f[15]));
              if (!__any_sync(0xffffffffu, fmaxf(fmaxf(m0, m1), fmaxf(m2, m3)) >= lim)) continue;
            }
            // compaction, taken by the whole warp at once as soon as one row's list
            // holds more than trig words (lanes compacting one by one would
            // serialise the warp); only needed before an append, so skipped groups
            // do not pay for the check
            if (__any_sync(0xffffffffu, cnt > trig)) {
              cnt = compact_exact(crow, cnt, thr_w, need_k, bits, trig, ordered, rank_bits);
              if (cnt > trig) {  // cannot happen (need_k <= 65); kept as a guard:
                overflow = true;         // the popcount kernel redoes this row
                thr_w = 0u;
                cnt = 0;
              }
              lim = lim_of(thr_w);
            }
            // branch-free append: every value is written at the running slot, only
            // words below the threshold advance it
            uint32_t* const wp0 = crow + cnt * kCandStride;
            uint32_t* wp = wp0;
            // the low bits of a word: the home's position (id order) or its id
            // rank (locality order, from the tile's ranks in shared memory)
            uint32_t lw[kHalf];
            if (loc_idr) {
              const uint4* ir = reinterpret_cast<const uint4*>(
                  idr_sm + (gg % kIdrSlots) * kNT + sub * kSub + half * kHalf);
  #pragma unroll
              for (int q = 0; q < kHalf / 4; ++q) {
                const uint4 t4 = ir[q];
                lw[4 * q] = (uint32_t)t4.x; lw[4 * q + 1] = (uint32_t)t4.y;
                lw[4 * q + 2] = (uint32_t)t4.z; lw[4 * q + 3] = (uint32_t)t4.w;
              }
            } else {
              const uint32_t posq = pos0 + (uint32_t)(half * kHalf);
  #pragma unroll
              for (int c2 = 0; c2 < kHalf; ++c2) lw[c2] = posq + c2;
            }
  #pragma unroll
            for (int c2 = 0; c2 < kHalf; ++c2) {
              const float dot = __uint_as_float(v[half * kHalf + c2]);
              const uint32_t fb = __float_as_uint(fmaf(dot, -0.5f, hmagic));
              const uint32_t word = fb * (1u << kPosBits) + lw[c2];
              *wp = word;
              wp += (word < thr_w) ? kCandStride : 0;
            }
            cnt += (int)((wp - wp0) / kCandStride);
          }
        }
      }
      const uint64_t pad = bdg_pad_key(bits);
      if constexpr (!RUN) {
        // ---- round A or a single round. Each thread cuts its row's list to
        // exactly its need_k best words, ranks them by counting (word order is
        // (d, id) order) into slots kOutSlot.., and looks up their ids into
        // slots 0..; then each warp writes its 32 rows, coalesced, without the
        // self pair.
        if (__any_sync(0xffffffffu, !overflow && cnt > need_k)) {
          if (!overflow && cnt > need_k) cnt = compact_exact(crow, cnt, thr_w, need_k, bits, need_k, ordered, rank_bits);
        }
        if (cnt > need_k) overflow = true;  // cannot happen; the popcount kernel would redo it
        int self_j = kNeedMax;  // sorted index of the self pair (none: kNeedMax)
        if (!overflow) {
          uint32_t wv[kNeedMax];  // the row's words in registers (missing ones: never below)
#pragma unroll
          for (int j = 0; j < kNeedMax; ++j) wv[j] = j < cnt ? crow[j * kCandStride] : 0xFFFFFFFFu;
          static_assert(kNeedMax % 4 == 1, "four partial counts + one");
          for (int i = 0; i < cnt; ++i) {
            const uint32_t wi = crow[i * kCandStride];
            int r0 = wv[kNeedMax - 1] < wi ? 1 : 0, r1 = 0, r2 = 0, r3 = 0;  // four short chains
#pragma unroll
            for (int j = 0; j < kNeedMax - 1; j += 4) {
              r0 += wv[j] < wi ? 1 : 0;
              r1 += wv[j + 1] < wi ? 1 : 0;
              r2 += wv[j + 2] < wi ? 1 : 0;
              r3 += wv[j + 3] < wi ? 1 : 0;
            }
            crow[(kOutSlot + (r0 + r1) + (r2 + r3)) * kCandStride] = wi;
          }
          for (int j0 = 0; j0 < cnt; j0 += 8) {
            int32_t h8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {  // eight id loads in flight
              const int j = j0 + q;
              h8[q] = j < cnt ? c.home_ids[h0 + (int)(crow[(kOutSlot + j) * kCandStride] & kPosMask)]
                              : -1;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              const int j = j0 + q;
              if (j < cnt) {
                crow[j * kCandStride] = (uint32_t)h8[q];
                if (excl && h8[q] == myvid && self_j == kNeedMax) self_j = j;
              }
            }
          }
        }
        __syncwarp();
#pragma unroll 2
        for (int rr = 0; rr < 32; ++rr) {
          const int row = warp * 32 + rr;
          const int n_r = __shfl_sync(0xffffffffu, cnt, rr);
          const int sj = __shfl_sync(0xffffffffu, self_j, rr);
          const int ovf = __shfl_sync(0xffffffffu, overflow ? 1 : 0, rr);
          const int32_t vid = __shfl_sync(0xffffffffu, myvid, rr);
          if (row >= nv) continue;
          const int64_t orow = a.out_by_pos ? (int64_t)(tile * kM + row) : (int64_t)vid;
          if (vid < 0) {  // an invalid id: its row (written by position) is padding
            if (a.t == 1 && a.out_by_pos) {
              for (int j2 = lane; j2 < k; j2 += 32) {
                a.out_ids[orow * k + j2] = -1;
                a.out_dist[orow * k + j2] = bits + 1;
              }
            }
            continue;
          }
          if (ovf) {  // recomputed by the popcount kernel
            if (lane == 0) { ta.fixflag[v0 + row] = 1; ta.err[1] = 1; }
            continue;
          }
          const int n_out = min(k, n_r - (sj < n_r ? 1 : 0));
          for (int o = lane; o < k; o += 32) {
            if (o < n_out) {
              const int e = o + (o >= sj ? 1 : 0);  // sorted index, the self pair skipped
              const int32_t hid = (int32_t)cand[cidx(e, row)];
              const uint32_t d = cand[cidx(kOutSlot + e, row)] >> kPosBits;
              if (a.t == 1) {
                a.out_ids[orow * k + o] = hid;
                a.out_dist[orow * k + o] = (int32_t)d;
              } else {
                a.partial[(int64_t)vid * k + o] = bdg_key(d, (uint32_t)hid);
              }
            } else {  // fewer than k candidates: padding
              if (a.t == 1) {
                a.out_ids[orow * k + o] = -1;
                a.out_dist[orow * k + o] = bits + 1;
              } else {
                a.partial[(int64_t)vid * k + o] = pad;
              }
            }
          }
        }
      } else {
        // ---- sub-round. Each thread cuts its row's list to its k best words and
        // turns them into keys (d, id), dropping those at or above the running
        // list's k-th key (they cannot enter); then each warp sorts, row by row,
        // the few surviving keys and merges them into the running list.
        if (__any_sync(0xffffffffu, !overflow && cnt > need_k)) {
          if (!overflow && cnt > need_k) cnt = compact_exact(crow, cnt, thr_w, need_k, bits, need_k, ordered, rank_bits);
        }
        if (cnt > need_k) overflow = true;  // cannot happen; the popcount kernel would redo it
        if (!overflow) {
          int w = 0;
          for (int j0 = 0; j0 < cnt; j0 += 8) {
            uint32_t w8[8];
            int32_t h8[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {  // eight id loads in flight
              const int j = j0 + q;
              w8[q] = j < cnt ? crow[j * kCandStride] : 0u;
              h8[q] = j < cnt ? c.home_ids[h0 + (int)(w8[q] & kPosMask)] : -1;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              if (j0 + q >= cnt || h8[q] == myvid) continue;
              if (bdg_key(w8[q] >> kPosBits, (uint32_t)h8[q]) >= kth) continue;
              crow[w * kCandStride] = w8[q];
              crow[(kOutSlot + w) * kCandStride] = (uint32_t)h8[q];
              ++w;
            }
          }
          cnt = w;
        }
        __syncwarp();
        uint64_t* sb = sortbuf + warp * 128;
        // only rows with keys to merge (or flagged) need the warp: most have none
        unsigned todo = __ballot_sync(0xffffffffu, r < nv && live && (overflow || cnt > 0));
        while (todo) {
          const int rr = __ffs(todo) - 1;
          todo &= todo - 1;
          const int row = warp * 32 + rr;
          const int n_r = __shfl_sync(0xffffffffu, cnt, rr);
          const int ovf = __shfl_sync(0xffffffffu, overflow ? 1 : 0, rr);
          const uint64_t kb = __shfl_sync(0xffffffffu, kth, rr);
          const int32_t vid = __shfl_sync(0xffffffffu, myvid, rr);
          if (ovf) {  // recomputed by the popcount kernel
            if (lane == 0) { ta.fixflag[v0 + row] = 1; ta.err[1] = 1; }
            continue;
          }
          // keys ascending: n_r <= 32 by one bitonic sort across the warp in
          // registers, else (n_r <= 64) two such sorts merged by ranks
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            const int x = lane + 32 * q;
            uint64_t key = BDG_KEY_INF;
            if (x < n_r)
              key = bdg_key(cand[cidx(x, row)] >> kPosBits, cand[cidx(kOutSlot + x, row)]);
            if (q == 1 && n_r <= 32) break;
#pragma unroll
            for (int k2 = 2; k2 <= 32; k2 <<= 1) {
#pragma unroll
              for (int j2 = k2 >> 1; j2 > 0; j2 >>= 1) {
                const uint64_t o = __shfl_xor_sync(0xffffffffu, key, j2);
                const bool up = (lane & k2) == 0, low = (lane & j2) == 0;
                key = (low == up) ? (key < o ? key : o) : (key < o ? o : key);
              }
            }
            sb[32 * q + lane] = key;
          }
          __syncwarp();
          if (n_r > 32) {  // merge the two sorted halves by ranks
            const uint64_t x0 = sb[lane], x1 = sb[32 + lane];
            int lo = 0, hi = 32;  // rank of x0 among the second half
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (sb[32 + mid] < x0) lo = mid + 1; else hi = mid;
            }
            int lo1 = 0, hi1 = 32;  // rank of x1 among the first half
            while (lo1 < hi1) {
              const int mid = (lo1 + hi1) >> 1;
              if (sb[mid] < x1) lo1 = mid + 1; else hi1 = mid;
            }
            __syncwarp();
            sb[64 + lane + lo] = x0;
            sb[64 + lane + lo1] = x1;
            __syncwarp();
            bdg_warp_merge_running(a.partial + (int64_t)vid * k, sb + 64, n_r, k, pad, kb, lane);
          } else {
            bdg_warp_merge_running(a.partial + (int64_t)vid * k, sb, n_r, k, pad, kb, lane);
          }
          __syncwarp();
        }
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
    for (uint32_t gg = (nprod > kStages ? nprod - kStages : 0); gg < nprod; ++gg)
      tc05::mbar_wait(&full[gg % kStages], (gg / kStages) & 1, kPolls);
    if (loc_idr)
      for (uint32_t gg = (nprod > kIdrSlots ? nprod - kIdrSlots : 0); gg < nprod; ++gg)
        tc05::mbar_wait(&idr_full[gg % kIdrSlots], (gg / kIdrSlots) & 1, kPolls);
  }
  tc05::fence_before();
  __syncthreads();
  if (warp == 0) tc05::tmem_dealloc(tmem, kTmemCols);
}

template <int W, bool LOC, bool RUN>
bdg_status launch_main(const bdg_knn_tc_args& ta, cudaStream_t st) {
  using C = TcCfg<W, LOC>;
  BDG_CUDA_TRY(cudaFuncSetAttribute(knn_tc_kernel<W, LOC, RUN>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM));
  bdg_prof_scope prof(ta.base.prof ? ta.base.prof : "knn", st);
  knn_tc_kernel<W, LOC, RUN><<<bdg_num_sms(), kThreads, C::SMEM, st>>>(ta);
  BDG_CUDA_TRY(cudaGetLastError());
  bdg_note_launch();
  return BDG_OK;
}

template <int W>
bdg_status launch_w(const bdg_knn_tc_args& ta, bool expand, cudaStream_t st) {
  const bdg_knn_args& a = ta.base;
  if (expand) {  // expanded home operand (rows are bounded by N + BDG_TC_TILE m)
    const int64_t max_rows = a.N + (int64_t)BDG_TC_TILE * a.m;
    const int64_t nthreads = ((max_rows + 7) / 8) * 8 * (4 * W);
    bdg_prof_scope prof(a.prof ? a.prof : "expand", st);
    expand_homes_kernel<W><<<bdg_cdiv(nthreads, 256), 256, 0, st>>>(
        a.csr.home_codes, a.csr.home_off, a.csr.eoff, a.csr.loc_idr, a.m, max_rows, ta.hexp);
    BDG_CUDA_TRY(cudaGetLastError());
    bdg_note_launch();
  }
  // homes in locality order (id ranks with every tile) or in id order
  if (a.csr.loc_idr) {
    if (a.merge_running) BDG_TRY((launch_main<W, true, true>(ta, st)));
    else BDG_TRY((launch_main<W, true, false>(ta, st)));
  } else {
    if (a.merge_running) BDG_TRY((launch_main<W, false, true>(ta, st)));
    else BDG_TRY((launch_main<W, false, false>(ta, st)));
  }
  // rows whose candidate list overflowed: exact recomputation by the popcount kernel
  BDG_CUDA_TRY(cudaMemsetAsync(a.item_counter, 0, sizeof(int32_t), st));
  bdg_knn_args fx = a;
  fx.fixflag = ta.fixflag;
  fx.fix_any = ta.err + 1;
  return bdg_launch_knn_popc(fx, W, st);
}

}  // namespace

bool bdg_knn_tc_supported(int W, int k) { return (W == 4 || W == 8) && k >= 1 && k <= 64; }

size_t bdg_knn_tc_hexp_bytes(int64_t N, int m, int W) {
  return (size_t)(N + (int64_t)BDG_TC_TILE * m) * 64 * W;
}

bdg_status bdg_launch_knn_tc(const bdg_knn_tc_args& a, int W, bool expand, cudaStream_t st) {
  if (W == 4) return launch_w<4>(a, expand, st);
  if (W == 8) return launch_w<8>(a, expand, st);
  return bdg_set_error(BDG_EUNSUPPORTED, "tensor k-NN path needs 256- or 512-bit codes");
}
