// Wedge aggregation: the hot loop of ExactBFC (Algorithm 1, the loops over
// v, u in Gamma_v, w in Gamma_u), of vBFC (Algorithm 2) and of the per-edge
// counts.
//
// For a start vertex v (rank r) the multiplicity c(v, w) = |Gamma_v ^ Gamma_w|
// of every later start vertex w (rank > r) is counted, then sum_w C(c, 2) is
// the number of butterflies with v and w as their start-side pair (Lemma 1,
// Eq. (2)-(3)); every unordered pair is seen once, from its lower rank.
//
// Start vertices are split into classes by the wedges they walk (Lemma 3:
// vBFC costs O(|Gamma^2_v|)) and by their degree (which bounds every c(v, w)):
//   skip   degree < 2 or nothing after it: every c <= 1, contributes 0
//   warp   <= 512 wedges: one warp per vertex, open addressing in shared memory
//   small windows (<= 128 wedge-list segments of 512 targets, or at most 64
//          rows with longer segments): a 128-thread CTA (eleven per SM) with
//          4,096 counter words in shared memory
//   large windows (<= 1,280 segments, or at most 640 rows): a 512-thread CTA
//          (three per SM) with 12,288 words
//   big    more: the large CTA with its segment cursors in global memory and a
//          32-bit window
// The window classes pack their counters by degree, 32 / b fields of b bits
// to a word: small windows 2 bits for degree <= 3, 3 for <= 7, 4 for <= 15,
// 5 for <= 31, else 8 (a small-class vertex has at most 127 rows); large
// windows 2, 4, 5 and 8 bits likewise up to degree 255, else 16 (at most
// 1,279 rows).  A 4,096-word window spans 65,536 ranks at 2 bits, 24,576 at
// 5 and 16,384 at 8.  Ranks ascend with degree, so the low-rank vertices,
// which walk the most of the rank space, are exactly the ones with the
// narrowest counters and the widest windows.
// The thresholds are scheduling settings (bfc_tuning); the counts do not
// depend on them.
//
// A window kernel walks the ranks after r window by window; a window starts at
// the lowest rank still pending in any of the vertex's (rank-sorted) wedge
// lists, so empty rank ranges cost nothing.  Each window has a count sweep
// (shared-memory atomic increments whose old values sum to sum_w C(c, 2)), in
// EDGE and LOCAL modes a read sweep of the same pieces against the final
// counts, and a clear of the counter words.  A vertex whose later ranks all
// fit in one window and whose lists are short skips the walk and expands its
// lists 32 targets at a time (count_flat).  In the ordered TOTAL and EDGE
// modes a vertex first tries the heavy-light split (count_hl): its lists other
// than the longest in a small hash table, the longest streamed once against
// it; in EDGE mode a vertex whose other lists are too long for the table walks
// the windows with the longest list as their heavy list, walked by the whole
// CTA after each window's count (heavy_walk).
//
// Modes: TOTAL (B only), EDGE (b_e; the vertex counts follow from b_e),
// SINGLE (Algorithm 2 on a batch of vertices: every w != v, whole midpoint
// rows), LOCAL (Algorithm 2 for every start vertex, with the row sums b_e).
// Per wedge v - x - w of a pair with c = c(v, w):
//   start side  b_v += sum_w C(c(v,w), 2), b_w += C(c(v,w), 2)
//   mid side    b_x += c(v,w) - 1 for each wedge v - x - w (pairs through x)
//   edges       b_(v,x) += c(v,w) - 1, b_(w,x) += c(v,w) - 1 for each wedge v - x - w
// which are the definitions of Section 2 written per wedge: a butterfly
// {v, w} x {x, y} is seen from the wedge v - x - w once for each of its two
// midpoints.
#include <algorithm>
#include <string>
#include <vector>

#include "bfc_internal.cuh"

namespace bfc {

constexpr uint32_t EMPTY_KEY = 0xFFFFFFFFu;
constexpr uint32_t INF_RANK = 0xFFFFFFFFu;
// class ids: skip, warp, then small windows for counter widths 2/4/8/16/32,
// large windows for the same widths, then big
enum Cls : uint32_t { CLS_SKIP = 0, CLS_WARP = 1, CLS_S0 = 2, CLS_L0 = 7, CLS_BIG = 12 };
static_assert(CLS_BIG + 1 == Plan::NCLS, "class count");
// counter bits of each window class slot, small and large (class_of)
constexpr int CW_SMALL[5] = {2, 4, 8, 6, 5};
constexpr int CW_LARGE[5] = {2, 4, 8, 16, 10};

// warp class
constexpr int WH_WARPS = 8;
constexpr int WH_SLOTS = 1024;                    // per warp
constexpr uint64_t WH_MAX_WORK = WH_SLOTS / 2;    // load factor <= 1/2
// window kernels come in two sizes (tag P_SMALL / P_LARGE).  A CTA runs one
// start vertex at a time through a chain of dependent phases (row loads,
// segment table, each window's count, read and clear, each closed by a CTA
// barrier), so many small CTAs per SM hide that chain better than a few large
// ones.  Small: eleven 128-thread CTAs per SM, each with 4,096 counter words
// and room for 128 wedge-list segments; measured faster than six 256-thread
// CTAs with 8,192 words, three 512-thread ones with 16,384 words, four
// 384-thread ones or eight 192-thread ones.  A vertex of at most half as many
// rows as segments fits any window class whatever its wedge count: its
// segments are lengthened (seg_len_for).  Large: three
// 512-thread CTAs per SM with 12,288 words and 1,280 segments, for the
// vertices whose wedge lists need more segments (one 1,024-thread CTA per SM
// measured twice as slow).
template <int P>
struct WinCfg;
template <>
struct WinCfg<4> {  // small: 11 CTAs of 4 warps per SM, 16 KB windows
  static constexpr int THREADS = 128;
  static constexpr int MINB = 11;  // 11 x (18.9 KB + 1 KB reserved) fit the SM's 228 KB, 12 do not
  static constexpr uint32_t WORDS = 4 * 1024;
  static constexpr uint32_t SMAX = 128;
  static constexpr size_t SMEM = (size_t)WORDS * 4 + (size_t)SMAX * 5 * 4;
};
template <>
struct WinCfg<1> {  // large: 3 CTAs of 16 warps per SM, 48 KB windows
  static constexpr int THREADS = 512;
  static constexpr int MINB = 3;
  static constexpr uint32_t WORDS = 12 * 1024;
  static constexpr uint32_t SMAX = 1280;
  static constexpr size_t SMEM = (size_t)WORDS * 4 + (size_t)SMAX * 5 * 4;
};
constexpr int P_SMALL = 4, P_LARGE = 1;
constexpr uint32_t SEG = 512;                     // wedge-list segment (elements)
// Segment length of an ordered-sweep start vertex with d rows and w wedges in
// a window class of smax segments: SEG, or longer so that the segments fit
// (sum_rows ceil(len / L) <= d + w / L <= smax for L >= w / (smax - d)).
__host__ __device__ __forceinline__ uint32_t seg_len_for(uint64_t w, uint64_t d, uint32_t smax) {
  if (d >= smax) return SEG;
  const uint64_t need = (w + (smax - d) - 1) / (smax - d);
  return need <= SEG ? SEG : (uint32_t)(need < 0x40000000ull ? need : 0x40000000ull);
}

// big class (segment cursors in global memory)
constexpr int CT_THREADS = 1024;
constexpr uint32_t CT_WORDS = 48 * 1024;          // 192 KB of counter words
constexpr uint32_t BIG_SEG = 256;
constexpr uint32_t BIG_Z = CT_WORDS;
// single-window vertices take the flat expansion (count_flat) only when their
// wedge lists are short: by default at most this many targets per start-row
// entry on average (bfc_tuning.flat_max_avg).  Longer lists keep the segment
// path, whose 256-wedge segments spread a few long lists over every warp of
// the CTA.
constexpr uint32_t FLAT_MAX_AVG = 64;

struct WArgs {
  uint32_t nS;
  const uint64_t *offR;
  const uint32_t *sX, *sEid, *sB;
  const uint64_t *offM;
  const uint32_t *mR, *mEid;
  const uint32_t *vert_of;
  const uint64_t *work;  // wedges walked from each start rank (the ordered suffixes)
  uint32_t flat_max;     // flat expansion limit (targets per start-row entry), BFC_TUNE_NO_FLAT: never
  uint32_t hl_max;       // heavy-light split limit (light wedges per start vertex), 0: never
  const uint32_t *list;
  uint32_t list_n;
  unsigned int *queue;
  unsigned long long *B;
  unsigned long long *bS, *be;  // LOCAL mode: b of the start vertex (by id); LOCAL / EDGE: b_e (canonical ids)
  // ordered EDGE mode: the far edge's updates go to beM (per midpoint-row
  // entry, so lanes of a warp hit consecutive words); one pass then adds
  // them to be by canonical edge id
  unsigned long long *beM;
  uint32_t *err;
  // big class: segment scratch (per CTA, seg_cap entries each)
  uint32_t *seg;        // 5 u32 per segment: begin, end, cur, pstart, next
  uint32_t *seg_row;    // row index per segment
  uint32_t seg_cap;
  // MODE_SINGLE (Algorithm 2 on a batch): list holds item ids
  const uint32_t *item_rank;
  unsigned long long *bitem;
  // TOTAL mode over a disjoint union of graphs: each start vertex's pair sum
  // also goes to gB[grp[rank]] (its graph's count)
  const uint32_t *grp;
  unsigned long long *gB;
  uint32_t cls;
  // start ranks >= rank_end walk nothing (their pairs are counted by the
  // hub block); nS otherwise
  uint32_t rank_end;
};


__device__ __forceinline__ uint64_t umin64(uint64_t x, uint64_t y) { return x < y ? x : y; }
__device__ __forceinline__ uint32_t umax32(uint32_t x, uint32_t y) { return x > y ? x : y; }
// modes that walk whole midpoint rows (every w != v) rather than the part after v
template <int MODE>
struct Full { static constexpr bool value = (MODE == MODE_SINGLE || MODE == MODE_LOCAL); };
__device__ __forceinline__ uint64_t pairs_of(uint32_t c) { return (uint64_t)c * (c - (c > 0)) / 2; }

__device__ __forceinline__ uint32_t warp_incl_scan_u32(uint32_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}
__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;  // valid in lane 0
}
// The same sum, by one 32-bit warp reduction when every lane's value is below
// 2^27 (the per-piece sums nearly always are); valid in lane 0.
__device__ __forceinline__ uint64_t warp_sum_u64_small(uint64_t x) {
  if (__all_sync(0xffffffffu, x < (1ull << 27))) return __reduce_add_sync(0xffffffffu, (uint32_t)x);
  return warp_sum_u64(x);
}

// ---------------------------------------------------------------------------
// warp class: open addressing in shared memory (keys = start ranks)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t wh_hash(uint32_t w) { return (w * 0x9E3779B1u) >> (32 - 10); }
static_assert(WH_SLOTS == 1024, "wh_hash assumes 1024 slots");

// (the class limit keeps a table at most half full, so the probe sequence
// always ends; a full table would be an internal error, reported, not dropped)
__device__ __forceinline__ void wh_insert(uint32_t *keys, uint32_t *cnts, uint32_t w, uint32_t *err) {
  uint32_t h = wh_hash(w);
  for (int probe = 0; probe < WH_SLOTS; probe++) {
    uint32_t k = keys[h];
    if (k == w) { atomicAdd(&cnts[h], 1u); return; }
    if (k == EMPTY_KEY) {
      uint32_t old = atomicCAS(&keys[h], EMPTY_KEY, w);
      if (old == EMPTY_KEY || old == w) { atomicAdd(&cnts[h], 1u); return; }
    }
    h = (h + 1) & (WH_SLOTS - 1);
  }
  atomicOr(err, DERR_CAPACITY);
}
__device__ __forceinline__ uint32_t wh_lookup(const uint32_t *keys, const uint32_t *cnts, uint32_t w) {
  uint32_t h = wh_hash(w);
  for (int probe = 0; probe < WH_SLOTS; probe++) {
    uint32_t k = keys[h];
    if (k == w) return cnts[h];
    if (k == EMPTY_KEY) return 0;
    h = (h + 1) & (WH_SLOTS - 1);
  }
  return 0;
}

// Expand the wedges of start-row entries [rb, re) 32 rows at a time and call
// f(i, j) for every wedge target index i (into mR) of row entry j.  All 32
// lanes must call this together.  FULL: the whole midpoint row (Algorithm 2:
// every w != v) instead of the part after v.
template <bool FULL, class F>
__device__ __forceinline__ void warp_for_each_wedge(const WArgs &a, uint64_t rb, uint64_t re, F f) {
  const int lane = threadIdx.x & 31;
  for (uint64_t chunk = rb; chunk < re; chunk += 32) {
    uint64_t j = chunk + lane;
    uint32_t b = 0, len = 0;
    if (j < re) {
      const uint32_t x = a.sX[j];
      b = FULL ? (uint32_t)a.offM[x] : a.sB[j];
      uint32_t e = (uint32_t)a.offM[x + 1];
      len = e - b;
    }
    uint32_t incl = warp_incl_scan_u32(len);
    uint32_t excl = incl - len;
    uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
    for (uint32_t base = 0; base < T; base += 32) {
      uint32_t t = base + lane;
      int l = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        int c = l + step;
        uint32_t ex = __shfl_sync(0xffffffffu, excl, c);
        if (ex <= t) l = c;
      }
      uint32_t sb = __shfl_sync(0xffffffffu, b, l);
      uint32_t sx = __shfl_sync(0xffffffffu, excl, l);
      if (t < T) f(sb + (t - sx), chunk + l);
    }
  }
}

template <int MODE>
__global__ void __launch_bounds__(WH_WARPS * 32) k_warp_class(WArgs a) {
  extern __shared__ uint32_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *keys = smem + (size_t)warp * 2 * WH_SLOTS;
  uint32_t *cnts = keys + WH_SLOTS;
  for (int i = lane; i < WH_SLOTS; i += 32) { keys[i] = EMPTY_KEY; cnts[i] = 0; }
  __syncwarp();
  uint64_t localB = 0;
  while (true) {
    uint32_t idx = 0;
    if (lane == 0) idx = atomicAdd(a.queue, 1u);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= a.list_n) break;
    const uint32_t item = a.list[idx];
    const uint32_t r = (MODE == MODE_SINGLE) ? a.item_rank[item] : item;
    const uint64_t rb = a.offR[r], re = (r < a.rank_end) ? a.offR[r + 1] : rb;  // ranks >= rank_end: done elsewhere
    warp_for_each_wedge<Full<MODE>::value>(a, rb, re, [&](uint32_t i, uint64_t) {
      const uint32_t w = a.mR[i];
      if (!Full<MODE>::value || w != r) wh_insert(keys, cnts, w, a.err);
    });
    __syncwarp();
    if (MODE == MODE_EDGE) {
      // second sweep: every wedge learns its final multiplicity
      warp_for_each_wedge<false>(a, rb, re, [&](uint32_t i, uint64_t j) {
        uint32_t c = wh_lookup(keys, cnts, a.mR[i]);
        if (c > 1) {
          if (a.be) {
            atomicAdd(&a.beM[i], (unsigned long long)(c - 1));
            atomicAdd(&a.be[a.sEid[j]], (unsigned long long)(c - 1));
          }
        }
      });
      __syncwarp();
    }
    if (MODE == MODE_LOCAL && a.be) {
      // b_(v,x) = sum over w in Gamma_x, w != v, of (c(v, w) - 1)
      warp_for_each_wedge<true>(a, rb, re, [&](uint32_t i, uint64_t j) {
        const uint32_t c = wh_lookup(keys, cnts, a.mR[i]);
        if (c > 1) atomicAdd(&a.be[a.sEid[j]], (unsigned long long)(c - 1));
      });
      __syncwarp();
    }
    uint64_t acc = 0;
    for (int i = lane; i < WH_SLOTS; i += 32) {
      uint32_t k = keys[i];
      if (k != EMPTY_KEY) {
        uint64_t p = pairs_of(cnts[i]);
        acc += p;
        keys[i] = EMPTY_KEY;
        cnts[i] = 0;
      }
    }
    acc = warp_sum_u64(acc);
    if (lane == 0) {
      localB += acc;
      if (MODE == MODE_SINGLE) a.bitem[item] = acc;
      if (MODE == MODE_LOCAL && a.bS) a.bS[a.vert_of[r]] = acc;
      if (MODE == MODE_TOTAL && a.gB && acc) atomicAdd(&a.gB[a.grp[r]], (unsigned long long)acc);
    }
    __syncwarp();
  }
  if (lane == 0 && localB) atomicAdd(a.B, (unsigned long long)localB);
}

// ---------------------------------------------------------------------------
// window classes: packed dense counters in shared memory
// Predicated atomics: the sweeps' per-target updates are issued under a
// predicate instead of inside a branch, so a warp whose lanes disagree does
// not diverge around them.
// shared-memory add returning the old word; 0 (and no add) where p is false
__device__ __forceinline__ uint32_t atom_add_if(bool p, uint32_t *addr, uint32_t v) {
  uint32_t old = 0;
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(addr);
  asm volatile(
      "{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %1, 0;\n\t@q atom.shared.add.u32 %0, [%2], %3;\n\t}"
      : "+r"(old)
      : "r"((uint32_t)p), "r"(sa), "r"(v)
      : "memory");
  return old;
}
// global 64-bit add where p is true (no return value)
__device__ __forceinline__ void red_add_if(bool p, unsigned long long *addr, unsigned long long v) {
  asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %0, 0;\n\t@q red.global.add.u64 [%1], %2;\n\t}"
               :
               : "r"((uint32_t)p), "l"(addr), "l"(v)
               : "memory");
}

// ---------------------------------------------------------------------------
// Counter of window offset idx: word idx mod WIN_WORDS, field idx / WIN_WORDS,
// so consecutive ranks (a sorted wedge list) fall in consecutive words and
// different banks.  A CW-bit field cannot overflow because every c(v, w) is at
// most the degree of v, which the class bounds by 2^CW - 1.
template <int CW, uint32_t WIN_WORDS>
struct Ctr {
  static constexpr uint32_t PER = 32 / CW;
  static constexpr uint32_t MASK = (CW == 32) ? 0xFFFFFFFFu : ((1u << CW) - 1u);
  static constexpr uint32_t Z = WIN_WORDS * PER;
  __device__ static __forceinline__ void at(uint32_t idx, uint32_t &wi, uint32_t &sh) {
    const uint32_t q = (PER == 1) ? 0u : idx / WIN_WORDS;
    wi = idx - q * WIN_WORDS;
    sh = q * CW;
  }
  // increment and return the field's old value
  __device__ static __forceinline__ uint32_t inc_get(uint32_t *c, uint32_t idx) {
    uint32_t wi, sh;
    at(idx, wi, sh);
    return (atomicAdd(&c[wi], 1u << sh) >> sh) & MASK;
  }
  // the same under a predicate, with no branch around it: 0 where p is false
  __device__ static __forceinline__ uint32_t inc_get_if(bool p, uint32_t *c, uint32_t idx) {
    uint32_t wi, sh;
    at(idx, wi, sh);
    return (atom_add_if(p, &c[wi], 1u << sh) >> sh) & MASK;
  }
  __device__ static __forceinline__ uint32_t peek(const uint32_t *c, uint32_t idx) {
    uint32_t wi, sh;
    at(idx, wi, sh);
    return (c[wi] >> sh) & MASK;
  }
};

// Count the wedge targets of one segment that fall in [lo, hi), starting at
// cur; one 32-element load first (most pieces end within it), then four in
// flight per warp.  Targets are ascending, so the
// in-window ones are a prefix.  On return cur is the first target >= hi (or
// end) and nx that target's rank (INF_RANK at the end of the segment).
// Raising a counter from c to c + 1 adds exactly c new pairs (C(c+1, 2) -
// C(c, 2) = c), so the old field values are summed into acc: after the
// window acc holds sum_w C(c(v, w), 2) over its targets.
template <int MODE, int CW, uint32_t WIN_WORDS>
__device__ __forceinline__ void count_segment(const uint32_t *__restrict__ mR, uint32_t &cur, uint32_t end,
                                              uint32_t lo, uint32_t hi, uint32_t r, uint32_t *ctr, uint32_t &nx,
                                              uint64_t &acc) {
  const int lane = threadIdx.x & 31;
  using C = Ctr<CW, WIN_WORDS>;
  {
    // the first 32 alone: most pieces end within them
    const uint32_t i = cur + lane;
    const uint32_t w = (i < end) ? __ldg(&mR[i]) : INF_RANK;
    const bool in = w < hi;
    const uint32_t n = __popc(__ballot_sync(0xffffffffu, in));
    acc += C::inc_get_if(in && (!Full<MODE>::value || w != r), ctr, w - lo);
    cur += n;
    if (n < 32) {
      const uint32_t first_out = __shfl_sync(0xffffffffu, w, n & 31);
      nx = (cur < end) ? first_out : INF_RANK;
      return;
    }
  }
  while (true) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t i = cur + k * 32 + lane;
      w[k] = (i < end) ? __ldg(&mR[i]) : INF_RANK;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const bool in = w[k] < hi;
      const uint32_t bal = __ballot_sync(0xffffffffu, in);
      acc += C::inc_get_if(in && (!Full<MODE>::value || w[k] != r), ctr, w[k] - lo);
      const uint32_t n = __popc(bal);
      cur += n;
      if (n < 32) {
        const uint32_t first_out = __shfl_sync(0xffffffffu, w[k], n & 31);
        nx = (cur < end) ? first_out : INF_RANK;
        return;
      }
    }
  }
}

// The heavy list in a window (the split of count_hl with windows): the
// vertex's longest wedge list is not counted and not segmented; after the
// window's light counts are final, every warp of the CTA walks it from cur
// (mR[cur, end)), warp k taking the 128-entry chunks k, k + NW, ... .
// Targets below lo lie where no light list has a target (c_L = 0) and are
// passed over; a target w in [lo, hi) adds c_L(w) = peek(w - lo) to rs (this
// lane's near-edge sum, which is also the vertex's B share), and in EDGE mode
// raises its counter by one (so the read sweep sees c = c_L + 1) and adds c_L
// to the far edge (staged at beM[i]); hit records some c_L > 0.  Targets are
// ascending, so each warp stops at its first chunk with a target >= hi (or at
// end) and reports that position to *pos_min: their minimum is the list's
// first target >= hi, its cursor for the next window.
template <int MODE, int CW, uint32_t WIN_WORDS, int NW>
__device__ __forceinline__ void heavy_walk(const uint32_t *__restrict__ mR, unsigned long long *beM, uint32_t cur,
                                           uint32_t end, uint32_t lo, uint32_t hi, uint32_t *ctr, uint32_t *pos_min,
                                           uint64_t &rs, bool &hit) {
  using C = Ctr<CW, WIN_WORDS>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr uint32_t STRIDE = NW * 128u;
  uint32_t c0 = cur + (uint32_t)warp * 128u;
  while (c0 < end) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t i = c0 + k * 32 + lane;
      w[k] = (i < end) ? __ldg(&mR[i]) : INF_RANK;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const bool in = w[k] < hi;
      const uint32_t bal = __ballot_sync(0xffffffffu, in);
      if (in && w[k] >= lo) {
        const uint32_t c = C::peek(ctr, w[k] - lo);
        if (c) {
          rs += c;
          hit = true;
          if (MODE == MODE_EDGE) {
            C::inc_get(ctr, w[k] - lo);
            atomicAdd(&beM[c0 + k * 32 + lane], (unsigned long long)c);
          }
        }
      }
      const uint32_t n = __popc(bal);
      if (n < 32) {
        if (lane == 0) atomicMin(pos_min, c0 + k * 32 + n);
        return;
      }
    }
    if (end - c0 <= STRIDE) break;
    c0 += STRIDE;
  }
  if (lane == 0) atomicMin(pos_min, end);
}

// Read sweep of one counted piece mR[ps, pe) of a wedge list (EDGE and
// LOCAL modes), after the window's counts are final: the target w of entry i
// has multiplicity c = peek(w - lo) = c(v, w), and the wedge v - x - w adds
// c - 1 to the far edge (w, x) (EDGE: staged at beM[i]) and to the near edge
// (v, x) (the returned warp sum, valid in lane 0).  Four 32-element loads in
// flight per warp, as in the count sweep.
template <int MODE, class Peek>
__device__ __forceinline__ uint64_t read_piece(const uint32_t *__restrict__ mR, unsigned long long *beM, uint32_t ps,
                                               uint32_t pe, uint32_t lo, Peek peek) {
  const int lane = threadIdx.x & 31;
  uint64_t rowsum = 0;
  uint32_t i0 = ps;
  for (; i0 + 32 < pe; i0 += 128) {
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t i = i0 + k * 32 + lane;
      w[k] = (i < pe) ? __ldg(&mR[i]) : 0u;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t i = i0 + k * 32 + lane;
      const uint32_t c = (i < pe) ? peek(w[k] - lo) : 0u;
      const bool p = c > 1;
      rowsum += p ? c - 1 : 0u;
      if (MODE != MODE_LOCAL) red_add_if(p, &beM[i], (unsigned long long)(c - 1));
    }
  }
  if (i0 < pe) {
    // the last (often the only) 32 targets
    const uint32_t i = i0 + lane;
    const uint32_t w = (i < pe) ? __ldg(&mR[i]) : 0u;
    const uint32_t c = (i < pe) ? peek(w - lo) : 0u;
    const bool p = c > 1;
    rowsum += p ? c - 1 : 0u;
    if (MODE != MODE_LOCAL) red_add_if(p, &beM[i], (unsigned long long)(c - 1));
  }
  return warp_sum_u64_small(rowsum);
}

// Expand the wedge lists of start-row entries [cb, ce) (at most 32, one per
// lane) and call f(i, w, l) for every target index i (into mR), its target
// w = mR[i] and its row cb + l.  The warp takes 32 consecutive elements of
// the concatenated lists at a time (prefix sum of the lengths + shuffle
// search), four of them in flight; each lane's row index never decreases.
// All 32 lanes must call this together.  FULL: whole midpoint rows.
template <bool FULL, class F>
__device__ __forceinline__ void expand_rows(const WArgs &a, uint64_t cb, uint64_t ce, F f) {
  const int lane = threadIdx.x & 31;
  const uint64_t j = cb + lane;
  uint32_t b = 0, len = 0;
  if (j < ce) {
    const uint32_t x = a.sX[j];
    b = FULL ? (uint32_t)a.offM[x] : a.sB[j];
    len = (uint32_t)a.offM[x + 1] - b;
  }
  const uint32_t incl = warp_incl_scan_u32(len);
  const uint32_t excl = incl - len;
  const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
  for (uint32_t base = 0; base < T; base += 128) {
    uint32_t idx[4], w[4];
    int row[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
      const uint32_t t = base + k * 32 + lane;
      int l = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        const int c = l + step;
        const uint32_t ex = __shfl_sync(0xffffffffu, excl, c);
        if (ex <= t) l = c;
      }
      const uint32_t sb = __shfl_sync(0xffffffffu, b, l);
      const uint32_t sx = __shfl_sync(0xffffffffu, excl, l);
      idx[k] = (t < T) ? sb + (t - sx) : 0xFFFFFFFFu;
      row[k] = l;
    }
#pragma unroll
    for (int k = 0; k < 4; k++) w[k] = (idx[k] != 0xFFFFFFFFu) ? __ldg(&a.mR[idx[k]]) : 0u;
#pragma unroll
    for (int k = 0; k < 4; k++)
      if (idx[k] != 0xFFFFFFFFu) f(idx[k], w[k], row[k]);
  }
}

// A start vertex whose later ranks (every rank, in the whole-row modes) fit in
// one counter window: no segments and no window walk.  Each warp takes the
// start-row entries in chunks of 32 and counts their targets by expand_rows,
// so short wedge lists (the top-ranked vertices' suffixes hold a few targets
// each) keep every lane busy.  EDGE / LOCAL: after a barrier the same
// expansion reads the final counts; the near edge's sum is gathered per row in
// rs (32 u64 per warp, shared memory) and the far edge's update staged at
// beM[i], as in the windowed path.  inc(idx) increments a counter and returns
// its old value, peek(idx) reads it.  Ends with a barrier; the caller clears
// the counters and reduces acc.
template <int MODE, int NW, class Inc, class Peek>
__device__ __forceinline__ void count_flat(const WArgs &a, uint32_t r, uint64_t rb, uint64_t re, uint32_t lo,
                                           unsigned long long *rs_all, uint64_t &acc, Inc inc, Peek peek) {
  constexpr bool FULL = Full<MODE>::value;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint64_t acc_before = acc;
  for (uint64_t cb = rb + (uint64_t)warp * 32; cb < re; cb += (uint64_t)NW * 32)
    expand_rows<FULL>(a, cb, umin64(cb + 32, re), [&](uint32_t, uint32_t w, int) {
      if (!FULL || w != r) acc += inc(w - lo);
    });
  // the read sweep adds c - 1 > 0 only where some counter reached 2
  const bool any2 = __syncthreads_or(acc != acc_before);
  if ((MODE == MODE_EDGE || (MODE == MODE_LOCAL && a.be)) && any2) {
    unsigned long long *rs = rs_all + warp * 32;
    for (uint64_t cb = rb + (uint64_t)warp * 32; cb < re; cb += (uint64_t)NW * 32) {
      rs[lane] = 0;
      __syncwarp();
      int cur = -1;
      unsigned long long part = 0;
      expand_rows<FULL>(a, cb, umin64(cb + 32, re), [&](uint32_t i, uint32_t w, int l) {
        const uint32_t c = peek(w - lo);  // 0 for w = v itself (never incremented)
        if (c > 1) {
          if (l != cur) {
            if (part) atomicAdd(&rs[cur], part);
            cur = l;
            part = 0;
          }
          part += c - 1;
          if (MODE != MODE_LOCAL) atomicAdd(&a.beM[i], (unsigned long long)(c - 1));
        }
      });
      if (part) atomicAdd(&rs[cur], part);
      __syncwarp();
      const uint64_t j = cb + lane;
      if (j < re && rs[lane]) atomicAdd(&a.be[a.sEid[j]], rs[lane]);
      __syncwarp();
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// heavy-light split of one start vertex (ordered TOTAL and EDGE modes)
// ---------------------------------------------------------------------------
// On power-law midpoint sides most of a low-degree start vertex's wedges come
// from one wedge list: its heaviest midpoint row.  A target w with c(v, w) >= 2
// lies in at least one of the other ("light") lists, so with c_L(w) the count
// over the light lists and h(w) = [w in the heavy list],
//   sum_w C(c, 2) = sum_w C(c_L, 2) + sum_{w in heavy} c_L(w)      (Eq. (3))
// The light lists are counted in a shared-memory hash table (keys w + 1, so
// an all-zero table is empty); the heavy list is streamed once against it
// with read-only lookups: a miss (c_L = 0) adds nothing to any output.  EDGE:
// a heavy hit flags its slot (h = 1), then the light lists read back
// c = c_L + h; a heavy wedge v - x - w adds c - 1 = c_L to both its edges.
// The table holds at most half as many keys as slots, so every probe
// sequence ends at an empty slot or the key.
constexpr uint32_t HL_FLAG = 0x80000000u;
// light wedges of the split at most: HL_FILL quarters of the largest table
// (its bitmap still turns most heavy-list misses away at that load; the light
// lookups walk somewhat longer probe sequences)
#ifndef HL_FILL
#define HL_FILL 3
#endif
#ifndef HL_U
#define HL_U 4
#endif
#ifndef HL_UL
#define HL_UL 4
#endif
__device__ __forceinline__ uint32_t hl_slot(uint32_t key, int shift) { return (key * 0x9E3779B1u) >> shift; }
__device__ __forceinline__ int hl_insert(uint32_t *keys, uint32_t mask, int shift, uint32_t key) {
  uint32_t s = hl_slot(key, shift);
  for (uint32_t p = 0; p <= mask; p++) {
    uint32_t k = reinterpret_cast<volatile uint32_t *>(keys)[s];
    if (k == key) return (int)s;
    if (k == 0u) {
      k = atomicCAS(&keys[s], 0u, key);
      if (k == 0u || k == key) return (int)s;
    }
    s = (s + 1) & mask;
  }
  return -1;
}
__device__ __forceinline__ int hl_find(const uint32_t *keys, uint32_t mask, int shift, uint32_t key) {
  uint32_t s = hl_slot(key, shift);
  for (uint32_t p = 0; p <= mask; p++) {
    const uint32_t k = keys[s];
    if (k == key) return (int)s;
    if (k == 0u) return -1;
    s = (s + 1) & mask;
  }
  return -1;
}
// row of light element t: the last row l with pre[l] <= t (pre[d] = total)
__device__ __forceinline__ uint32_t hl_row(const uint32_t *pre, uint32_t d, uint32_t t) {
  uint32_t lo = 0, hi = d;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (pre[mid] <= t) lo = mid; else hi = mid;
  }
  return lo;
}

// Count start vertex r (rows [rb, re), 1 <= re - rb <= THREADS) by the split
// above if its light lists hold at most wmax wedges (below tmax, the power of
// two of table slots that fits); returns false (after a barrier, nothing
// written) otherwise.  ctr: the WORDS zeroed counter words (left
// zeroed); area: 4 THREADS + 4 free words (8-byte aligned); sh_hmax: a shared
// word the caller zeroed before the vertex.  All threads call it together.
template <int MODE, int THREADS, uint32_t WORDS>
__device__ __forceinline__ bool count_hl(const WArgs &a, uint64_t rb, uint64_t re, uint64_t work, uint32_t *ctr,
                                         uint32_t tmax, uint32_t wmax, uint32_t *area, unsigned long long *sh_hmax,
                                         uint32_t *sh_wt, uint64_t &acc) {
  constexpr int NW = THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t d = (uint32_t)(re - rb), j = threadIdx.x;
  uint32_t b = 0, len = 0;
  if (j < d) {
    const uint32_t x = a.sX[rb + j];
    b = a.sB[rb + j];
    len = (uint32_t)a.offM[x + 1] - b;
  }
  // the heaviest row, the lowest index among equals
  unsigned long long key = (j < d) ? (((unsigned long long)len << 16) | (0xFFFFu - j)) : 0ull;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, key, o);
    key = y > key ? y : key;
  }
  if (lane == 0) atomicMax(sh_hmax, key);
  __syncthreads();
  const unsigned long long hk = *sh_hmax;
  const uint32_t hlen = (uint32_t)(hk >> 16), hj = 0xFFFFu - (uint32_t)(hk & 0xFFFFu);
  const uint64_t wl = work - hlen;
  if (wl > wmax) return false;
  // T: the smallest power of two >= max(2 wl, 64), at most tmax (so the table
  // is at most half full, or up to wmax / tmax in the largest one)
  const uint32_t need = min(tmax, umax32(2u * (uint32_t)wl, 64u));
  const int logT = 32 - __clz(need - 1u);
  const uint32_t T = 1u << logT;
  const uint32_t mask = T - 1;
  const int shift = 32 - logT;
  uint32_t *keys = ctr, *cnt = ctr + T;
  // a bitmap of the light keys after the table (the largest power of two of
  // words that fits, at most 8,192): most heavy targets are not light, and one
  // bit test turns them away without walking a probe sequence
  const int lognbw = min(31 - __clz(WORDS - 2 * T), 13);
  const uint32_t nbw = 1u << lognbw;
  uint32_t *bits = ctr + 2 * T;
  const int bshift = 32 - (lognbw + 5);
  uint32_t *pre = area, *beg = area + THREADS + 2;
  unsigned long long *rs = reinterpret_cast<unsigned long long *>(area + 2 * THREADS + 4);
  // prefix sums of the light rows' lengths
  const uint32_t ll = (j < d && j != hj) ? len : 0u;
  const uint32_t inc = warp_incl_scan_u32(ll);
  if (lane == 31) sh_wt[warp] = inc;
  if (j < d) {
    beg[j] = b;
    if (MODE == MODE_EDGE) rs[j] = 0;
  }
  __syncthreads();
  // warp totals -> this warp's base and the grand total, by one warp scan
  const uint32_t wt = (lane < NW) ? sh_wt[lane] : 0u;
  const uint32_t wincl = warp_incl_scan_u32(wt);
  const uint32_t base = __shfl_sync(0xffffffffu, wincl - wt, warp);
  const uint32_t total = __shfl_sync(0xffffffffu, wincl, 31);
  if (j < d) pre[j] = base + inc - ll;
  if (j == 0) pre[d] = total;
  __syncthreads();
  // count sweep over the light lists, HL_UL elements in flight per thread
  for (uint32_t t0 = j; t0 < total; t0 += HL_UL * THREADS) {
    uint32_t w[HL_UL];
#pragma unroll
    for (int k = 0; k < HL_UL; k++) {
      const uint32_t t = t0 + k * THREADS;
      w[k] = 0xFFFFFFFFu;
      if (t < total) {
        const uint32_t l = hl_row(pre, d, t);
        w[k] = __ldg(&a.mR[beg[l] + (t - pre[l])]);
      }
    }
#pragma unroll
    for (int k = 0; k < HL_UL; k++) {
      if (w[k] == 0xFFFFFFFFu) continue;
      const int sl = hl_insert(keys, mask, shift, w[k] + 1u);
      if (sl >= 0) acc += atomicAdd(&cnt[sl], 1u);
      else atomicOr(a.err, DERR_CAPACITY);
      const uint32_t bi = ((w[k] + 1u) * 0x85EBCA6Bu) >> bshift;
      atomicOr(&bits[bi >> 5], 1u << (bi & 31));
    }
  }
  __syncthreads();
  // the heavy list, HL_U loads in flight per thread
  const uint32_t hb = beg[hj];
  uint64_t rsh = 0;
  for (uint32_t t0 = j; t0 < hlen; t0 += HL_U * THREADS) {
    uint32_t w[HL_U];
#pragma unroll
    for (int k = 0; k < HL_U; k++) {
      const uint32_t t = t0 + k * THREADS;
      w[k] = (t < hlen) ? __ldg(&a.mR[hb + t]) : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int k = 0; k < HL_U; k++) {
      if (w[k] == 0xFFFFFFFFu) continue;
      const uint32_t bi = ((w[k] + 1u) * 0x85EBCA6Bu) >> bshift;
      if (!((bits[bi >> 5] >> (bi & 31)) & 1u)) continue;
      const int sl = hl_find(keys, mask, shift, w[k] + 1u);
      if (sl >= 0) {
        const uint32_t c = cnt[sl];
        acc += c;
        if (MODE == MODE_EDGE) {
          cnt[sl] = c | HL_FLAG;
          rsh += c;
          atomicAdd(&a.beM[hb + t0 + k * THREADS], (unsigned long long)c);
        }
      }
    }
  }
  if (MODE == MODE_EDGE) {
    rsh = warp_sum_u64(rsh);
    if (lane == 0 && rsh) atomicAdd(&rs[hj], (unsigned long long)rsh);
    // the read sweep adds c - 1 > 0 only where some c reached 2
    if (__syncthreads_or(acc != 0)) {
      for (uint32_t t = j; t < total; t += THREADS) {
        const uint32_t l = hl_row(pre, d, t);
        const uint32_t i = beg[l] + (t - pre[l]);
        const int sl = hl_find(keys, mask, shift, __ldg(&a.mR[i]) + 1u);
        if (sl < 0) { atomicOr(a.err, DERR_CAPACITY); continue; }
        const uint32_t v = cnt[sl];
        const uint32_t c = (v & ~HL_FLAG) + (v >> 31);
        if (c > 1) {
          atomicAdd(&rs[l], (unsigned long long)(c - 1));
          atomicAdd(&a.beM[i], (unsigned long long)(c - 1));
        }
      }
      __syncthreads();
      if (j < d && rs[j]) atomicAdd(&a.be[a.sEid[rb + j]], rs[j]);
    }
  } else {
    __syncthreads();
  }
  // back to an all-zero table
  uint4 *c4 = reinterpret_cast<uint4 *>(ctr);
  for (uint32_t i = j; i < (2 * T + nbw) / 4; i += THREADS) c4[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();
  return true;
}

// (the whole-row modes, off the default path, are compiled for two fewer resident
// CTAs: their read sweep needs a few more registers than the 46 that eleven
// 128-thread CTAs leave)
template <int MODE, int CW, int P>
__global__ void __launch_bounds__(WinCfg<P>::THREADS, (Full<MODE>::value && WinCfg<P>::MINB > 4) ? WinCfg<P>::MINB - 2 : WinCfg<P>::MINB) k_cta_win(WArgs a) {
  constexpr int WIN_THREADS = WinCfg<P>::THREADS;
  constexpr uint32_t WIN_WORDS = WinCfg<P>::WORDS;
  constexpr uint32_t WIN_SMAX = WinCfg<P>::SMAX;
  using C = Ctr<CW, WIN_WORDS>;
  extern __shared__ uint32_t sm[];
  uint32_t *ctr = sm;
  uint32_t *s_cur = sm + WIN_WORDS, *s_end = s_cur + WIN_SMAX, *s_ps = s_end + WIN_SMAX, *s_nx = s_ps + WIN_SMAX;
  uint32_t *s_row = s_nx + WIN_SMAX;  // canonical id of the segment's start-row edge
  // window state, double buffered by window parity so that a window needs
  // two barriers: one after counting, one after clearing
  __shared__ uint32_t sh_min[2];
  __shared__ unsigned long long sh_win[2];
  __shared__ uint32_t sh_idx, sh_carry;
  __shared__ unsigned long long sh_acc, sh_hmax;
  __shared__ uint32_t sh_hj;  // the vertex's heavy list (row index), INF_RANK: none
  __shared__ uint32_t sh_heid;  // its start-row edge id, INF_RANK: none
  __shared__ uint32_t sh_hb, sh_he;  // its wedge list mR[sh_hb, sh_he) (not segmented)
  __shared__ uint32_t sh_hpos[2];  // per window parity: where its walk stopped
  __shared__ uint32_t sh_seglen;  // segment length of the vertex (ordered modes)
  __shared__ uint32_t wtot[32];
  constexpr int NW = WIN_THREADS / 32;
  // heavy-light table slots: the largest power of two <= a quarter of the
  // counter words (keys and counts take half, the bitmap at least a quarter)
  constexpr uint32_t HL_TMAX = (WIN_WORDS / 4 >= 4096) ? 4096u : (WIN_WORDS / 4 >= 2048) ? 2048u : 1024u;
  static_assert(2 * HL_TMAX + 4 <= WIN_WORDS, "table and bitmap fit the counter words");
  static_assert(5 * WIN_SMAX >= 4 * WIN_THREADS + 4, "heavy-light scratch fits the segment tables");
  constexpr uint32_t Z = C::Z;
  // B accumulates at increment time (the sum of old values is C(c, 2))
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint32_t i = threadIdx.x; i < WIN_WORDS; i += WIN_THREADS) ctr[i] = 0;
  uint64_t localB = 0;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) {
      sh_idx = atomicAdd(a.queue, 1u);
      sh_carry = 0;
      sh_acc = 0;
      sh_hmax = 0;
      sh_hj = INF_RANK;
      sh_heid = INF_RANK;
      sh_hb = sh_he = 0;
      sh_hpos[0] = sh_hpos[1] = INF_RANK;
      sh_min[0] = INF_RANK; sh_win[0] = 0;
      sh_min[1] = INF_RANK; sh_win[1] = 0;
    }
    __syncthreads();
    const uint32_t idx = sh_idx;
    if (idx >= a.list_n) break;
    const uint32_t item = a.list[idx];
    const uint32_t r = (MODE == MODE_SINGLE) ? a.item_rank[item] : item;
    const uint64_t rb = a.offR[r], re = (r < a.rank_end) ? a.offR[r + 1] : rb;  // ranks >= rank_end: done elsewhere
    const uint32_t lo0 = Full<MODE>::value ? 0u : r + 1;
    uint64_t acc = 0;  // per thread, over the whole vertex
    bool done = false;
    if (!Full<MODE>::value && threadIdx.x == 0) sh_seglen = seg_len_for(a.work[r], re - rb, WIN_SMAX);
    if ((MODE == MODE_TOTAL || MODE == MODE_EDGE) && a.hl_max && re > rb && re - rb <= (uint64_t)WIN_THREADS) {
      done = count_hl<MODE, WIN_THREADS, WIN_WORDS>(a, rb, re, a.work[r], ctr, HL_TMAX,
                                         (uint32_t)umin64(HL_TMAX / 4 * HL_FILL, a.hl_max), sm + WIN_WORDS,
                                         &sh_hmax, wtot, acc);
      // otherwise, in EDGE mode, the longest list is walked as the heavy list of
      // the windows (it spares the read sweep of that list; in TOTAL mode the
      // extra barrier per window measured slower)
      if (MODE == MODE_EDGE && !done && re - rb > 1 && threadIdx.x == 0)
        sh_hj = 0xFFFFu - (uint32_t)(sh_hmax & 0xFFFFu);
    } else if (!Full<MODE>::value) {
      __syncthreads();  // sh_seglen (count_hl's first barrier publishes it otherwise)
    }
    if (done) {
      // counted by the heavy-light split
    } else if ((uint64_t)a.nS <= (uint64_t)lo0 + Z && a.flat_max != BFC_TUNE_NO_FLAT &&
        a.work[r] <= (uint64_t)a.flat_max * (re - rb)) {
      // ---- every later rank fits in one window and the lists are short:
      // no segments, no window walk
      count_flat<MODE, NW>(a, r, rb, re, lo0, reinterpret_cast<unsigned long long *>(s_cur), acc,
                           [&](uint32_t i) { return C::inc_get(ctr, i); },
                           [&](uint32_t i) { return C::peek(ctr, i); });
      const uint32_t used = (uint32_t)umin64((uint64_t)WIN_WORDS, (uint64_t)a.nS - lo0);
      uint4 *c4 = reinterpret_cast<uint4 *>(ctr);
      for (uint32_t i = threadIdx.x; i < (used + 3) / 4; i += WIN_THREADS) c4[i] = make_uint4(0, 0, 0, 0);
    } else {
    // ---- segments of the vertex's wedge lists
    const uint32_t seglen = Full<MODE>::value ? SEG : sh_seglen;
    for (uint64_t base = rb; base < re; base += WIN_THREADS) {
      const uint64_t j = base + threadIdx.x;
      uint32_t b = 0, e = 0, ns = 0, eid = 0;
      if (j < re) {
        const uint32_t x = a.sX[j];
        b = Full<MODE>::value ? (uint32_t)a.offM[x] : a.sB[j];
        e = (uint32_t)a.offM[x + 1];
        ns = (e - b + seglen - 1) / seglen;
        eid = a.sEid[j];
        if ((uint32_t)(j - rb) == sh_hj) {
          // the heavy list is walked by the whole CTA after each window's count
          sh_heid = eid;
          sh_hb = b;
          sh_he = e;
          ns = 0;
        }
      }
      const uint32_t incl = warp_incl_scan_u32(ns);
      if (lane == 31) wtot[warp] = incl;
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t run = sh_carry;
        for (int w = 0; w < NW; w++) { const uint32_t t = wtot[w]; wtot[w] = run; run += t; }
        sh_carry = run;
      }
      __syncthreads();
      const uint32_t first = wtot[warp] + incl - ns;
      for (uint32_t k = 0; k < ns; k++) {
        const uint32_t s = first + k;
        if (s >= WIN_SMAX) { atomicOr(a.err, DERR_CAPACITY); break; }
        const uint32_t sb = b + k * seglen;
        s_cur[s] = sb;
        s_end[s] = min(e, sb + seglen);
        s_ps[s] = sb;
        s_nx[s] = 0;  // unknown: load it
        s_row[s] = eid;
      }
      __syncthreads();
    }
    const uint32_t nseg = min(sh_carry, WIN_SMAX);
    uint32_t hcur = sh_hb;  // the heavy list's cursor (the same in every thread)
    const uint32_t hend = sh_he;
    uint32_t lo = lo0;
    uint32_t hi = (uint32_t)umin64((uint64_t)a.nS, (uint64_t)lo + Z);
    for (uint32_t par = 0;; par ^= 1) {
      // ---- count: warp w owns segments w, w + NW, ...; its lanes test 32 of them
      // at once and the whole warp counts each one that has targets below hi
      uint32_t wcount = 0, wmin = INF_RANK;
      const uint64_t acc_before = acc;  // unchanged over the window: every counter ended at 1
      for (uint32_t s0 = warp; s0 < nseg; s0 += NW * 32) {
        const uint32_t sl = s0 + (uint32_t)lane * NW;  // this lane's segment
        uint32_t my_nx = INF_RANK;
        bool act = false;
        if (sl < nseg) {
          const uint32_t c0 = s_cur[sl];
          my_nx = (c0 < s_end[sl]) ? s_nx[sl] : INF_RANK;
          act = my_nx < hi;  // 0: next target not loaded yet
          s_ps[sl] = c0;     // nothing of it counted in this window yet
        }
        uint32_t bal = __ballot_sync(0xffffffffu, act);
        while (bal) {
          const int l = __ffs(bal) - 1;
          bal &= bal - 1;
          const uint32_t sg = s0 + (uint32_t)l * NW;
          uint32_t cur = s_cur[sg], nx = INF_RANK;
          const uint32_t ps = cur;
          count_segment<MODE, CW, WIN_WORDS>(a.mR, cur, s_end[sg], lo, hi, r, ctr, nx, acc);
          if (lane == 0) {
            s_cur[sg] = cur;
            s_nx[sg] = nx;
          }
          if (lane == l) my_nx = nx;
          wcount += cur - ps;
        }
        wmin = min(wmin, my_nx);
      }
      for (int o = 16; o > 0; o >>= 1) wmin = min(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
      if (lane == 0 && wmin != INF_RANK) atomicMin(&sh_min[par], wmin);
      // the read sweep adds c - 1 > 0 only where a counter reached 2, i.e.
      // where an increment met an old value >= 1 (acc grew)
      if (MODE == MODE_EDGE || MODE == MODE_LOCAL) {
        const bool any2 = __any_sync(0xffffffffu, acc != acc_before);
        if ((MODE == MODE_EDGE || a.be) && lane == 0 && wcount && any2)
          atomicAdd(&sh_win[par], (unsigned long long)wcount);
      }
      __syncthreads();
      // the other parity's state was last read before this barrier: reset it
      if (threadIdx.x == 0) {
        sh_min[par ^ 1] = INF_RANK;
        sh_win[par ^ 1] = 0;
      }
      const uint32_t nm = sh_min[par];
      // ---- the heavy list against the window's final light counts
      if (sh_hj != INF_RANK) {
        if (threadIdx.x == 0) sh_hpos[par ^ 1] = INF_RANK;
        bool hit = false;
        uint64_t rs = 0;
        heavy_walk<MODE, CW, WIN_WORDS, NW>(a.mR, a.beM, hcur, hend, lo, hi, ctr, &sh_hpos[par], rs, hit);
        acc += rs;
        if (MODE == MODE_EDGE) {
          const uint64_t t = warp_sum_u64_small(rs);
          if (lane == 0 && t) atomicAdd(&a.be[sh_heid], (unsigned long long)t);
          if (__any_sync(0xffffffffu, hit) && lane == 0) atomicAdd(&sh_win[par], 1ull);
        }
        __syncthreads();
        hcur = sh_hpos[par];
      }
      // ---- EDGE / LOCAL: every wedge of the window reads its final count
      if (MODE == MODE_EDGE || MODE == MODE_LOCAL) {
        if (sh_win[par]) {
          // the same ownership: each warp reads back the pieces it counted
          for (uint32_t s0 = warp; s0 < nseg; s0 += NW * 32) {
            const uint32_t sl = s0 + (uint32_t)lane * NW;
            const bool act = sl < nseg && s_ps[sl] < s_cur[sl];
            uint32_t bal = __ballot_sync(0xffffffffu, act);
            while (bal) {
              const int l = __ffs(bal) - 1;
              bal &= bal - 1;
              const uint32_t sg = s0 + (uint32_t)l * NW;
              const uint64_t rowsum = read_piece<MODE>(a.mR, a.beM, s_ps[sg], s_cur[sg], lo,
                                                        [&](uint32_t idx) { return C::peek(ctr, idx); });
              if (lane == 0 && rowsum)
                atomicAdd(&a.be[s_row[sg]], (unsigned long long)rowsum);
            }
          }
          __syncthreads();
        }
      }
      // ---- every target of the window has been counted: zero the words in use
      {
        const uint32_t used = (uint32_t)umin64((uint64_t)WIN_WORDS, (uint64_t)(hi - lo));
        uint4 *c4 = reinterpret_cast<uint4 *>(ctr);
        const uint32_t n4 = (used + 3) / 4;
        for (uint32_t i = threadIdx.x; i < n4; i += WIN_THREADS) c4[i] = make_uint4(0, 0, 0, 0);
      }
      __syncthreads();
      if (nm == INF_RANK) break;
      lo = nm;
      hi = (uint32_t)umin64((uint64_t)a.nS, (uint64_t)lo + Z);
    }
    }
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(&sh_acc, (unsigned long long)acc);
    __syncthreads();
    if (threadIdx.x == 0) {
      localB += sh_acc;
      if (MODE == MODE_SINGLE) a.bitem[item] = sh_acc;
      if (MODE == MODE_LOCAL && a.bS) a.bS[a.vert_of[r]] = sh_acc;
      if (MODE == MODE_TOTAL && a.gB && sh_acc) atomicAdd(&a.gB[a.grp[r]], sh_acc);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && localB) atomicAdd(a.B, (unsigned long long)localB);
}

// ---------------------------------------------------------------------------
// big class: 32-bit window, segment cursors in global memory (any degree,
// any number of segments)
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(CT_THREADS, 1) k_cta_big(WArgs a) {
  extern __shared__ uint32_t ctr[];  // BIG_Z counters, then 32 u64 per warp (count_flat's row sums)
  unsigned long long *rs_all = reinterpret_cast<unsigned long long *>(ctr + BIG_Z);
  __shared__ uint32_t s_idx, s_next_min, s_carry;
  __shared__ unsigned long long s_acc;
  __shared__ uint32_t wtot[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = CT_THREADS / 32;
  uint32_t *seg = a.seg + (size_t)blockIdx.x * a.seg_cap * 5;
  uint32_t *seg_row = a.seg_row + (size_t)blockIdx.x * a.seg_cap;
  for (uint32_t i = threadIdx.x; i < BIG_Z; i += CT_THREADS) ctr[i] = 0;
  uint64_t localB = 0;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) {
      s_idx = atomicAdd(a.queue, 1u);
      s_carry = 0;
      s_acc = 0;
      s_next_min = INF_RANK;
    }
    __syncthreads();
    const uint32_t idx = s_idx;
    if (idx >= a.list_n) break;
    const uint32_t item = a.list[idx];
    const uint32_t r = (MODE == MODE_SINGLE) ? a.item_rank[item] : item;
    const uint64_t rb = a.offR[r], re = (r < a.rank_end) ? a.offR[r + 1] : rb;  // ranks >= rank_end: done elsewhere
    const uint32_t lo0 = Full<MODE>::value ? 0u : r + 1;
    uint64_t acc = 0;  // per thread: sum of old counter values = sum C(c, 2)
    if ((uint64_t)a.nS <= (uint64_t)lo0 + BIG_Z && a.flat_max != BFC_TUNE_NO_FLAT &&
        a.work[r] <= (uint64_t)a.flat_max * (re - rb)) {
      // ---- every later rank fits in one window and the lists are short:
      // no segments, no window walk
      count_flat<MODE, NW>(a, r, rb, re, lo0, rs_all, acc, [&](uint32_t i) { return atomicAdd(&ctr[i], 1u); },
                           [&](uint32_t i) { return ctr[i]; });
      const uint32_t used = (uint32_t)umin64((uint64_t)BIG_Z, (uint64_t)a.nS - lo0);
      uint4 *c4 = reinterpret_cast<uint4 *>(ctr);
      for (uint32_t i = threadIdx.x; i < (used + 3) / 4; i += CT_THREADS) c4[i] = make_uint4(0, 0, 0, 0);
    } else {
    for (uint64_t base = rb; base < re; base += CT_THREADS) {
      uint64_t j = base + threadIdx.x;
      uint32_t b = 0, e = 0, ns = 0;
      if (j < re) {
        const uint32_t x = a.sX[j];
        b = Full<MODE>::value ? (uint32_t)a.offM[x] : a.sB[j];
        e = (uint32_t)a.offM[x + 1];
        ns = (e - b + BIG_SEG - 1) / BIG_SEG;
      }
      uint32_t incl = warp_incl_scan_u32(ns);
      if (lane == 31) wtot[warp] = incl;
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t run = s_carry;
        for (int w = 0; w < NW; w++) { uint32_t t = wtot[w]; wtot[w] = run; run += t; }
        s_carry = run;
      }
      __syncthreads();
      uint32_t first = wtot[warp] + incl - ns;
      if (first + ns > a.seg_cap) {
        atomicOr(a.err, DERR_CAPACITY);
        ns = (first < a.seg_cap) ? a.seg_cap - first : 0;
      }
      for (uint32_t k = 0; k < ns; k++) {
        uint32_t sb = b + k * BIG_SEG;
        uint32_t se = min(e, sb + BIG_SEG);
        uint32_t *sg = seg + (size_t)(first + k) * 5;
        sg[0] = sb; sg[1] = se; sg[2] = sb; sg[3] = sb; sg[4] = 0;
        seg_row[first + k] = (uint32_t)j;
      }
      __syncthreads();
    }
    const uint32_t nseg = min(s_carry, a.seg_cap);
    uint32_t lo = lo0;
    uint32_t hi = (uint32_t)umin64((uint64_t)a.nS, (uint64_t)lo + BIG_Z);
    while (true) {
      // ---- count: warp w owns segments w, w + NW, ...; 32 tested per ballot
      uint32_t wmin = INF_RANK;
      for (uint32_t s0 = warp; s0 < nseg; s0 += NW * 32) {
        const uint32_t sl = s0 + (uint32_t)lane * NW;
        uint32_t my_nx = INF_RANK;
        bool act = false;
        if (sl < nseg) {
          uint32_t *sg = seg + (size_t)sl * 5;
          const uint32_t pos = sg[2];
          my_nx = (pos < sg[1]) ? sg[4] : INF_RANK;
          act = my_nx < hi;  // 0: next target not loaded yet
          sg[3] = pos;       // nothing of it counted in this window yet
        }
        uint32_t bal = __ballot_sync(0xffffffffu, act);
        while (bal) {
          const int l = __ffs(bal) - 1;
          bal &= bal - 1;
          uint32_t *sg = seg + (size_t)(s0 + (uint32_t)l * NW) * 5;
          uint32_t pos = sg[2], nxt = INF_RANK;
          count_segment<MODE, 32, BIG_Z>(a.mR, pos, sg[1], lo, hi, r, ctr, nxt, acc);
          if (lane == 0) { sg[2] = pos; sg[4] = nxt; }
          if (lane == l) my_nx = nxt;
        }
        wmin = min(wmin, my_nx);
      }
      for (int o = 16; o > 0; o >>= 1) wmin = min(wmin, __shfl_xor_sync(0xffffffffu, wmin, o));
      if (lane == 0 && wmin != INF_RANK) atomicMin(&s_next_min, wmin);
      __syncthreads();
      if (MODE == MODE_EDGE || (MODE == MODE_LOCAL && a.be)) {
        for (uint32_t s0 = warp; s0 < nseg; s0 += NW * 32) {
          const uint32_t sl = s0 + (uint32_t)lane * NW;
          const bool act = sl < nseg && seg[(size_t)sl * 5 + 3] < seg[(size_t)sl * 5 + 2];
          uint32_t bal = __ballot_sync(0xffffffffu, act);
          while (bal) {
            const int l = __ffs(bal) - 1;
            bal &= bal - 1;
            const uint32_t sidx = s0 + (uint32_t)l * NW;
            const uint32_t *sg = seg + (size_t)sidx * 5;
            const uint64_t rowsum = read_piece<MODE>(a.mR, a.beM, sg[3], sg[2], lo,
                                                      [&](uint32_t idx) { return ctr[idx]; });
            if (lane == 0 && rowsum) atomicAdd(&a.be[a.sEid[seg_row[sidx]]], (unsigned long long)rowsum);
          }
        }
        __syncthreads();
      }
      // ---- every target of the window has been counted: zero the words in use
      {
        const uint32_t used = (uint32_t)umin64((uint64_t)BIG_Z, (uint64_t)(hi - lo));
        uint4 *c4 = reinterpret_cast<uint4 *>(ctr);
        for (uint32_t i = threadIdx.x; i < (used + 3) / 4; i += CT_THREADS) c4[i] = make_uint4(0, 0, 0, 0);
      }
      const uint32_t nm = s_next_min;
      __syncthreads();
      if (nm == INF_RANK) break;
      if (threadIdx.x == 0) s_next_min = INF_RANK;
      lo = nm;
      hi = (uint32_t)umin64((uint64_t)a.nS, (uint64_t)lo + BIG_Z);
      __syncthreads();
    }
    }
    acc = warp_sum_u64(acc);
    if (lane == 0 && acc) atomicAdd(&s_acc, (unsigned long long)acc);
    __syncthreads();
    if (threadIdx.x == 0) {
      localB += s_acc;
      if (MODE == MODE_SINGLE) a.bitem[item] = s_acc;
      if (MODE == MODE_LOCAL && a.bS) a.bS[a.vert_of[r]] = s_acc;
      if (MODE == MODE_TOTAL && a.gB && s_acc) atomicAdd(&a.gB[a.grp[r]], s_acc);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && localB) atomicAdd(a.B, (unsigned long long)localB);
}

// ---------------------------------------------------------------------------
// classification
// ---------------------------------------------------------------------------
// Class limits of a plan (tunable, see bfc_set_tuning): start vertices with
// at most warp_max wedges take the warp class, those with at most small_max
// segments the small windows.  Both are capped by the tables' capacities.
struct ClsLimits {
  uint32_t warp_max, small_max;
  // ordered plans: a window class also takes any vertex of at most half its
  // segment capacity in rows, with segments lengthened to fit (seg_len_for)
  bool adaptive;
};
static ClsLimits limits_of(const Plan &p, bool adaptive = true) {
  return ClsLimits{std::min<uint32_t>(p.warp_max, (uint32_t)WH_MAX_WORK),
                   std::min<uint32_t>(std::max<uint32_t>(p.small_max, 1u), WinCfg<P_SMALL>::SMAX), adaptive};
}

__device__ __forceinline__ uint32_t class_of(uint64_t d, uint64_t w, ClsLimits lim) {
  if (d < 2 || w == 0) return CLS_SKIP;
  if (w <= lim.warp_max) return CLS_WARP;
  const uint64_t segs = d + w / SEG + 1;
  constexpr uint32_t LMAX = WinCfg<P_LARGE>::SMAX;
  uint32_t base;
  if (segs <= lim.small_max || (lim.adaptive && 2 * d <= lim.small_max)) base = CLS_S0;
  else if (segs <= LMAX || (lim.adaptive && 2 * d <= LMAX)) base = CLS_L0;
  else return CLS_BIG;
  // counter width (CW_SMALL / CW_LARGE): every c(v, w) <= degree of v
  if (d <= 3) return base + 0;
  if (d <= 15) return base + 1;
  if (base == CLS_S0) return d <= 31 ? base + 4 : d <= 63 ? base + 3 : base + 2;  // (d <= 127 here)
  if (d <= 255) return base + 2;
  if (d <= 1023) return base + 4;
  if (d <= 65535) return base + 3;
  return CLS_BIG;  // (not reached: a large-class vertex has d <= 1,279)
}

// Class of every start rank, with per-class vertex counts, wedge and row
// sums gathered in shared memory first (one global atomic per block and
// class instead of one per vertex on the same few words).
__global__ void k_classify(const uint64_t *offR, const uint64_t *work, uint32_t nS, ClsLimits lim, uint32_t *cls_of,
                           unsigned int *counts, unsigned long long *maxseg, unsigned long long *sums) {
  constexpr int N = Plan::NCLS;
  __shared__ unsigned int s_cnt[N];
  __shared__ unsigned long long s_sum[2 * N];
  __shared__ unsigned long long s_max;
  for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) {
    if (i < N) s_cnt[i] = 0;
    s_sum[i] = 0;
  }
  if (threadIdx.x == 0) s_max = 0;
  __syncthreads();
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nS; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t d = offR[r + 1] - offR[r], w = work[r];
    const uint32_t c = class_of(d, w, lim);
    cls_of[r] = c;
    atomicAdd(&s_cnt[c], 1u);
    if (w) atomicAdd(&s_sum[c], (unsigned long long)w);
    if (d) atomicAdd(&s_sum[N + c], (unsigned long long)d);
    if (c == CLS_BIG) atomicMax(&s_max, (unsigned long long)(d + w / BIG_SEG + 1));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * N; i += blockDim.x) {
    if (i < N && s_cnt[i]) atomicAdd(&counts[i], s_cnt[i]);
    if (s_sum[i]) atomicAdd(&sums[i], s_sum[i]);
  }
  if (threadIdx.x == 0 && s_max) atomicMax(maxseg, s_max);
}
__global__ void k_scatter_class(const uint32_t *cls_of, uint32_t nS, const unsigned int *begin, unsigned int *cursor,
                                uint32_t *list) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nS; r += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t c = cls_of[r];
    uint32_t p = atomicAdd(&cursor[c], 1u);
    list[begin[c] + p] = (uint32_t)r;
  }
}
// 16-bit sort key for "heaviest first": the work's float exponent and top 7
// mantissa bits (order within 1%), complemented so that an ascending sort
// puts the largest work first
__global__ void k_work_keys(const uint32_t *list, uint32_t n, const uint64_t *work, uint32_t *keys, uint32_t *vals) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t r = list[i];
    keys[i] = 0xFFFFu - (__float_as_uint((float)work[r]) >> 16);
    vals[i] = r;
  }
}

static unsigned grid_for(uint64_t n, unsigned threads, unsigned cap = 152 * 16) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

int plan_classify(bfc_graph *g, Plan &p, cudaStream_t s) {
  constexpr int N = Plan::NCLS;
  const uint32_t nS = p.nS;
  BFC_TRY(dalloc(p.cls, (uint64_t)std::max<uint32_t>(nS, 1) * 4, s));
  DBuf cls_of, cnt, k1, k2, v2;
  auto cleanup = [&]() { dfree(cls_of, s); dfree(cnt, s); dfree(k1, s); dfree(k2, s); dfree(v2, s); };
  int rc = BFC_OK;
#define PC_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
  PC_TRY(dalloc(cls_of, (uint64_t)std::max<uint32_t>(nS, 1) * 4, s));
  PC_TRY(dalloc(cnt, 512, s));
  BFC_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, 512, s));
  static_assert(N <= 16, "class arrays below hold 16 entries");
  unsigned int *counts = ptr<unsigned int>(cnt);                                      // [0, 16)
  unsigned int *cursor = counts + 16;                                                 // [16, 32)
  unsigned long long *maxseg = reinterpret_cast<unsigned long long *>(counts + 32);  // 1
  unsigned long long *sums = reinterpret_cast<unsigned long long *>(counts + 34);    // 2 N (<= 32)
  k_classify<<<grid_for(nS, 256), 256, 0, s>>>(ptr<uint64_t>(p.offR), ptr<uint64_t>(p.work), nS, limits_of(p),
                                              ptr<uint32_t>(cls_of), counts, maxseg, sums);
  count_launch();
  unsigned int hc[16];
  unsigned long long hmax = 0, hs[2 * N];
  BFC_CUDA_TRY(cudaMemcpyAsync(hc, counts, 64, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaMemcpyAsync(&hmax, maxseg, 8, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaMemcpyAsync(hs, sums, sizeof(hs), cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  unsigned int hb[16] = {};
  for (int c = 0; c < N; c++) {
    p.cls_count[c] = hc[c];
    p.cls_begin[c] = (c == 0) ? 0 : p.cls_begin[c - 1] + p.cls_count[c - 1];
    hb[c] = p.cls_begin[c];
    p.cls_work[c] = hs[c];
    p.cls_rows[c] = hs[N + c];
  }
  p.big_seg_cap = (uint32_t)std::min<unsigned long long>(hmax, 0xFFFFFFFFull);
  BFC_CUDA_TRY(cudaMemcpyAsync(counts, hb, 64, cudaMemcpyHostToDevice, s));
  k_scatter_class<<<grid_for(nS, 256), 256, 0, s>>>(ptr<uint32_t>(cls_of), nS, counts, cursor, ptr<uint32_t>(p.cls));
  count_launch();
  // heaviest first inside each window class (better load balance at the tail)
  uint32_t maxn = 0;
  for (int c = CLS_S0; c < N; c++) maxn = std::max(maxn, p.cls_count[c]);
  if (maxn > 1) {
    PC_TRY(dalloc(k1, (uint64_t)maxn * 4, s));
    PC_TRY(dalloc(k2, (uint64_t)maxn * 4, s));
    PC_TRY(dalloc(v2, (uint64_t)maxn * 4, s));
    for (int c = CLS_S0; c < N; c++) {
      const uint32_t nc = p.cls_count[c];
      if (nc < 2) continue;
      uint32_t *list = ptr<uint32_t>(p.cls) + p.cls_begin[c];
      k_work_keys<<<grid_for(nc, 256), 256, 0, s>>>(list, nc, ptr<uint64_t>(p.work), ptr<uint32_t>(k1), list);
      count_launch();
      PC_TRY(radix_sort_u32(ptr<uint32_t>(k1), ptr<uint32_t>(k2), list, ptr<uint32_t>(v2), nc, 16, g->scr, s));
      BFC_CUDA_TRY(cudaMemcpyAsync(list, v2.p, (uint64_t)nc * 4, cudaMemcpyDeviceToDevice, s));
    }
  }
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  cleanup();
#undef PC_TRY
  return BFC_OK;
}

// ---------------------------------------------------------------------------
// launch
// ---------------------------------------------------------------------------
static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

static const char *tag_of(int kind, int mode) {
  static const char *tags[3][4] = {{"warp.total", "warp.edge", "warp.single", "warp.local"},
                                   {"win.total", "win.edge", "win.single", "win.local"},
                                   {"big.total", "big.edge", "big.single", "big.local"}};
  return tags[kind][mode];
}

// class lists: lists[c], counts[c] for c in [0, NCLS).
template <int MODE>
static int launch_lists(bfc_graph *g, WArgs a, const uint32_t *const *lists, const uint32_t *counts, uint32_t big_cap,
                        cudaStream_t s) {
  const int sms = sm_count();
  unsigned int *queues = ptr<unsigned int>(g->acc) + 16;  // one counter per class
  static_assert(64 + 4 * Plan::NCLS <= 256, "queues live in the 256-byte accumulator block");
  BFC_CUDA_TRY(cudaMemsetAsync(queues, 0, 4 * Plan::NCLS, s));
  auto have = [&](int c) { return counts[c] != 0; };
  auto setup = [&](WArgs &w, int c) {
    w.cls = (uint32_t)c;
    w.queue = queues + c;
    w.list = lists[c];
    w.list_n = counts[c];
  };
  auto cap = [&](unsigned full, int c) -> unsigned {
    return std::max(1u, std::min<unsigned>(full, counts[c]));
  };
  if (have(CLS_WARP)) {
    WArgs w = a;
    setup(w, CLS_WARP);
    const size_t smem = (size_t)WH_WARPS * 2 * WH_SLOTS * 4;
    BFC_CUDA_TRY(cudaFuncSetAttribute(k_warp_class<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    BFC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_warp_class<MODE>, WH_WARPS * 32, smem));
    const unsigned full = (unsigned)std::max(1, occ) * sms;
    const unsigned grid = std::min<unsigned>(full, (counts[CLS_WARP] + WH_WARPS - 1) / WH_WARPS);
    profile_begin(tag_of(0, MODE), s);
    k_warp_class<MODE><<<grid, WH_WARPS * 32, smem, s>>>(w);
    BFC_LAUNCHED();
    profile_end(tag_of(0, MODE), s);
  }
  bool any_win = false;
  for (int c = CLS_S0; c < CLS_BIG; c++) any_win = any_win || have(c);
  if (any_win) profile_begin(tag_of(1, MODE), s);
  for (int c = CLS_S0; c < CLS_BIG; c++) {
    if (!have(c)) continue;
    WArgs w = a;
    setup(w, c);
    const bool small = c < CLS_L0;
    const int cw = small ? CW_SMALL[c - CLS_S0] : CW_LARGE[c - CLS_L0];
    void (*kern)(WArgs) = nullptr;
    if (small) {
      kern = cw == 2 ? k_cta_win<MODE, 2, P_SMALL> : cw == 4 ? k_cta_win<MODE, 4, P_SMALL>
           : cw == 5 ? k_cta_win<MODE, 5, P_SMALL> : cw == 6 ? k_cta_win<MODE, 6, P_SMALL>
                                                            : k_cta_win<MODE, 8, P_SMALL>;
    } else {
      kern = cw == 2 ? k_cta_win<MODE, 2, P_LARGE> : cw == 4 ? k_cta_win<MODE, 4, P_LARGE>
           : cw == 8 ? k_cta_win<MODE, 8, P_LARGE> : cw == 10 ? k_cta_win<MODE, 10, P_LARGE>
                                                             : k_cta_win<MODE, 16, P_LARGE>;
    }
    const int per_sm = small ? WinCfg<P_SMALL>::MINB : WinCfg<P_LARGE>::MINB;
    const int threads = small ? WinCfg<P_SMALL>::THREADS : WinCfg<P_LARGE>::THREADS;
    const size_t smem = small ? WinCfg<P_SMALL>::SMEM : WinCfg<P_LARGE>::SMEM;
    BFC_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // per-class timing as well ("win.edge.s8": the 8-bit small-window class)
    static const char *cls_names[10] = {"s2", "s4", "s8", "s6", "s5", "l2", "l4", "l8", "l16", "l10"};
    const std::string ctag = std::string(tag_of(1, MODE)) + "." + cls_names[c - CLS_S0];
    profile_begin(ctag.c_str(), s);
    kern<<<cap((unsigned)(sms * per_sm), c), threads, smem, s>>>(w);
    BFC_LAUNCHED();
    profile_end(ctag.c_str(), s);
  }
  if (any_win) profile_end(tag_of(1, MODE), s);
  if (have(CLS_BIG) && big_cap > 0) {
    WArgs c = a;
    setup(c, CLS_BIG);
    const size_t smem = (size_t)BIG_Z * 4 + (size_t)CT_THREADS * 8;  // counters + per-warp row sums
    BFC_CUDA_TRY(cudaFuncSetAttribute(k_cta_big<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = cap((unsigned)sms, CLS_BIG);
    c.seg_cap = big_cap;
    const uint64_t need = (uint64_t)grid * c.seg_cap * 6 * 4;
    BFC_TRY(g->scr.reserve(need, s));
    c.seg = static_cast<uint32_t *>(g->scr.base());
    c.seg_row = c.seg + (uint64_t)grid * c.seg_cap * 5;
    profile_begin(tag_of(2, MODE), s);
    k_cta_big<MODE><<<grid, CT_THREADS, smem, s>>>(c);
    BFC_LAUNCHED();
    profile_end(tag_of(2, MODE), s);
  }
  return BFC_OK;
}

template <int MODE>
static int launch_classes(bfc_graph *g, Plan &p, WArgs a, cudaStream_t s) {
  const uint32_t *cls = ptr<uint32_t>(p.cls);
  const uint32_t *lists[Plan::NCLS];
  for (int c = 0; c < Plan::NCLS; c++) lists[c] = cls + p.cls_begin[c];
  return launch_lists<MODE>(g, a, lists, p.cls_count, std::max<uint32_t>(p.big_seg_cap, 1), s);
}

static WArgs args_of(bfc_graph *g, Plan &p) {
  WArgs a{};
  a.nS = p.nS;
  a.rank_end = p.nS;
  a.offR = ptr<uint64_t>(p.offR);
  a.sX = ptr<uint32_t>(p.sX);
  a.sEid = ptr<uint32_t>(p.sEid);
  a.sB = ptr<uint32_t>(p.sB);
  a.offM = p.offM;
  a.mR = ptr<uint32_t>(p.mR);
  a.mEid = ptr<uint32_t>(p.mEid);
  a.vert_of = ptr<uint32_t>(p.vert_of);
  a.work = ptr<uint64_t>(p.work);
  a.flat_max = g->tune.flat_max_avg ? g->tune.flat_max_avg : FLAT_MAX_AVG;
  a.hl_max = g->tune.hl_max_light == BFC_TUNE_NO_HL ? 0u : g->tune.hl_max_light ? g->tune.hl_max_light : 0xFFFFFFFFu;
  a.err = ptr<uint32_t>(g->err);
  return a;
}

// ---------------------------------------------------------------------------
// batched Algorithm 2
// ---------------------------------------------------------------------------
__global__ void k_item_classify(const uint32_t *item_rank, uint32_t n, const uint64_t *offR, const uint32_t *sX,
                                const uint64_t *offM, ClsLimits lim, uint32_t *cls_of, unsigned int *counts,
                                unsigned long long *maxseg, unsigned long long *out) {
  const int lane = threadIdx.x & 31;
  uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = warp; i < n; i += nw) {
    const uint32_t r = item_rank ? item_rank[i] : (uint32_t)i;
    const uint64_t b = offR[r], e = offR[r + 1];
    uint64_t w = 0;
    for (uint64_t j = b + lane; j < e; j += 32) {
      const uint32_t x = sX[j];
      w += offM[x + 1] - offM[x] - 1;
    }
    w = warp_sum_u64(w);
    if (lane == 0) {
      const uint64_t d = e - b;
      const uint32_t c = class_of(d, w, lim);
      cls_of[i] = c;
      atomicAdd(&counts[c], 1u);
      if (out) out[i] = 0;
      if (c == CLS_BIG) atomicMax(maxseg, (unsigned long long)(d + w / BIG_SEG + 1));
    }
  }
}
__global__ void k_item_scatter(const uint32_t *cls_of, uint32_t n, const unsigned int *begin, unsigned int *cursor,
                               uint32_t *lists) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = cls_of[i];
    if (c == CLS_SKIP) continue;
    lists[begin[c] + atomicAdd(&cursor[c], 1u)] = (uint32_t)i;
  }
}

// Whole-row counting for a batch of start ranks (item_rank, or every rank when
// null): SINGLE writes b of each item to out; LOCAL writes b_v to bS, the row
// sums b_e to be, and adds 2B to d_B.
static int full_rows_batch(bfc_graph *g, Plan &p, int mode, const uint32_t *item_rank, uint32_t n_items,
                           unsigned long long *out, unsigned long long *d_B, unsigned long long *bS,
                           unsigned long long *be, cudaStream_t s) {
  constexpr int N = Plan::NCLS;
  if (n_items == 0) return BFC_OK;
  DBuf cls_of, lists, cnt;
  auto cleanup = [&]() { dfree(cls_of, s); dfree(lists, s); dfree(cnt, s); };
  int rc = BFC_OK;
#define VB_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
  VB_TRY(dalloc(cls_of, (uint64_t)n_items * 4, s));
  VB_TRY(dalloc(lists, (uint64_t)n_items * 4, s));
  VB_TRY(dalloc(cnt, 256, s));
  BFC_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, 256, s));
  static_assert(N <= 16, "class arrays below hold 16 entries");
  unsigned int *counts = ptr<unsigned int>(cnt);                                      // [0, 16)
  unsigned int *begin = counts + 16;                                                  // [16, 32)
  unsigned int *cursor = counts + 32;                                                 // [32, 48)
  unsigned long long *maxseg = reinterpret_cast<unsigned long long *>(counts + 48);
  k_item_classify<<<grid_for((uint64_t)n_items * 32, 256), 256, 0, s>>>(item_rank, n_items, ptr<uint64_t>(p.offR),
                                                                        ptr<uint32_t>(p.sX), p.offM, limits_of(p, false),
                                                                        ptr<uint32_t>(cls_of), counts, maxseg, out);
  count_launch();
  unsigned int hc[16];
  unsigned long long hmax = 0;
  BFC_CUDA_TRY(cudaMemcpyAsync(hc, counts, 64, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaMemcpyAsync(&hmax, maxseg, 8, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  unsigned int hb[16] = {};
  uint32_t run = 0;
  for (int c = 1; c < N; c++) { hb[c] = run; run += hc[c]; }
  BFC_CUDA_TRY(cudaMemcpyAsync(begin, hb, 64, cudaMemcpyHostToDevice, s));
  k_item_scatter<<<grid_for(n_items, 256), 256, 0, s>>>(ptr<uint32_t>(cls_of), n_items, begin, cursor,
                                                       ptr<uint32_t>(lists));
  count_launch();
  WArgs a = args_of(g, p);
  a.item_rank = item_rank;
  a.bitem = out;
  a.B = d_B;
  a.bS = bS;
  a.be = be;
  const uint32_t *L[N];
  uint32_t C[N];
  for (int c = 0; c < N; c++) { L[c] = ptr<uint32_t>(lists) + hb[c]; C[c] = (c == 0) ? 0 : hc[c]; }
  const uint32_t cap = std::max<uint32_t>(1, (uint32_t)std::min<unsigned long long>(hmax, 0xFFFFFFFFull));
  if (mode == MODE_LOCAL) VB_TRY(launch_lists<MODE_LOCAL>(g, a, L, C, cap, s));
  else VB_TRY(launch_lists<MODE_SINGLE>(g, a, L, C, cap, s));
  cleanup();
#undef VB_TRY
  return BFC_OK;
}

int vbfc_batch(bfc_graph *g, Plan &p, const uint32_t *item_rank, uint32_t n_items, unsigned long long *out,
               cudaStream_t s) {
  // B is not read back here: it lands in the second accumulator word
  return full_rows_batch(g, p, MODE_SINGLE, item_rank, n_items, out, ptr<unsigned long long>(g->acc) + 1, nullptr,
                         nullptr, s);
}

// b_x of a midpoint vertex: half the sum of b_e over its edges (each butterfly
// through x contains two of x's edges)
__global__ void k_mid_from_edges(const uint64_t *offM, uint32_t nM, const uint32_t *mEid,
                                 const unsigned long long *be, unsigned long long *bM) {
  const int lane = threadIdx.x & 31;
  uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t x = warp; x < nM; x += nw) {
    uint64_t t = 0;
    for (uint64_t i = offM[x] + lane; i < offM[x + 1]; i += 32) t += be[mEid[i]];
    t = warp_sum_u64(t);
    if (lane == 0) bM[x] = t / 2;
  }
}

int wedge_local(bfc_graph *g, Plan &p, unsigned long long *d_2B, uint64_t *bS, uint64_t *bM, uint64_t *be,
                cudaStream_t s) {
  if (bM && !be) return BFC_EINVAL;
  if (bS) BFC_CUDA_TRY(cudaMemsetAsync(bS, 0, (uint64_t)p.nS * 8, s));
  if (be && p.m) BFC_CUDA_TRY(cudaMemsetAsync(be, 0, p.m * 8, s));
  BFC_TRY(full_rows_batch(g, p, MODE_LOCAL, nullptr, p.nS, nullptr, d_2B,
                          reinterpret_cast<unsigned long long *>(bS), reinterpret_cast<unsigned long long *>(be), s));
  if (bM) {
    k_mid_from_edges<<<grid_for((uint64_t)p.nM * 32, 256), 256, 0, s>>>(
        p.offM, p.nM, ptr<uint32_t>(p.mEid), reinterpret_cast<const unsigned long long *>(be),
        reinterpret_cast<unsigned long long *>(bM));
    BFC_LAUNCHED();
  }
  return BFC_OK;
}

// b_x = 1/2 sum_{e containing x} b_e (every butterfly through x holds two of
// x's edges) over the rows off[x] .. off[x+1]; eid maps row entries to
// canonical edge ids (null: the row entries are the canonical ids)
__global__ void k_half_row_sums(const uint64_t *off, uint32_t n, const uint32_t *eid, const unsigned long long *be,
                                unsigned long long *out) {
  const int lane = threadIdx.x & 31;
  uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t x = warp; x < n; x += nw) {
    uint64_t t = 0;
    for (uint64_t i = off[x] + lane; i < off[x + 1]; i += 32) t += be[eid ? eid[i] : i];
    t = warp_sum_u64(t);
    if (lane == 0) out[x] = t / 2;
  }
}

int vertex_from_edges(const uint64_t *off, uint32_t n, const uint32_t *eid, const uint64_t *be, uint64_t *out,
                      cudaStream_t s) {
  if (n == 0) return BFC_OK;
  k_half_row_sums<<<grid_for((uint64_t)n * 32, 256), 256, 0, s>>>(
      off, n, eid, reinterpret_cast<const unsigned long long *>(be), reinterpret_cast<unsigned long long *>(out));
  BFC_LAUNCHED();
  return BFC_OK;
}

// move the staged sums to their outputs: be[canonical id] += beM[row entry]
__global__ void k_finish_edges(const uint32_t *mEid, uint64_t m, const unsigned long long *beM,
                               unsigned long long *be) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    be[mEid[i]] += beM[i];  // every canonical edge appears once in midpoint-row order
}

// ---------------------------------------------------------------------------
// counting entry points
// ---------------------------------------------------------------------------
int wedge_count_groups(bfc_graph *g, Plan &p, const uint32_t *grp_of_rank, unsigned long long *gB,
                       unsigned long long *d_B, cudaStream_t s) {
  WArgs a = args_of(g, p);
  a.B = d_B;
  a.grp = grp_of_rank;
  a.gB = gB;
  return launch_classes<MODE_TOTAL>(g, p, a, s);
}

int wedge_count_below(bfc_graph *g, Plan &p, uint32_t rank_end, unsigned long long *d_B, cudaStream_t s) {
  WArgs a = args_of(g, p);
  a.B = d_B;
  a.rank_end = rank_end;
  return launch_classes<MODE_TOTAL>(g, p, a, s);
}

int wedge_count(bfc_graph *g, Plan &p, Mode mode, unsigned long long *d_B, uint64_t *be, cudaStream_t s) {
  WArgs a = args_of(g, p);
  a.B = d_B;
  a.be = reinterpret_cast<unsigned long long *>(be);
  if (be && p.m) {
    BFC_TRY(dalloc(g->beM, p.m * 8, s));
    BFC_CUDA_TRY(cudaMemsetAsync(g->beM.p, 0, p.m * 8, s));
    a.beM = ptr<unsigned long long>(g->beM);
  }
  int rc = BFC_EINVAL;
  switch (mode) {
    case MODE_TOTAL: rc = launch_classes<MODE_TOTAL>(g, p, a, s); break;
    case MODE_EDGE: rc = launch_classes<MODE_EDGE>(g, p, a, s); break;
    default: break;
  }
  if (rc) return rc;
  if (a.beM) {
    k_finish_edges<<<grid_for(p.m, 256), 256, 0, s>>>(ptr<uint32_t>(p.mEid), p.m, a.beM, a.be);
    BFC_LAUNCHED();
  }
  return BFC_OK;
}

}  // namespace bfc
