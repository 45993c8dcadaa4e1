// Batched sparsification trials (Section 6: ESpar, Algorithm 8; ClrSpar,
// Algorithm 9) in one persistent launch over the full graph's rank layout.
//
// A trial t keeps edge e with a predicate of (t, e): ESpar keeps it with
// probability p, ClrSpar when both endpoints drew the same of N colours.  The
// trial's beta is B of the kept subgraph.  Nothing is rebuilt per trial:
//   1. keep masks: for every trial and every position of the start-row and
//      midpoint-row arrays, one bit (the predicate of that entry's edge), laid
//      out interleaved by trial: 32-bit word (pos / 32) * T + t holds trial t's
//      bits of positions pos & ~31 .. (pos & ~31) + 31, so the words of all
//      trials for one stretch of a row are adjacent in memory;
//   2. one persistent kernel over (start vertex, trial range) items, heaviest
//      start vertices first: for each trial, Algorithm 1's loops for that start
//      vertex restricted to the kept entries (a start edge (v, x) with its bit
//      set, then the set bits of x's midpoint row after v), counting c(v, w) in
//      a per-warp hash table; sum_w C(c, 2) goes to beta[t] (Lemma 1, Eq. (3):
//      B of the kept subgraph, with the full graph's side and rank order, on
//      which B does not depend).
// A (start vertex, trial) pair whose kept targets overflow the warp table is
// put on a list that the same launch drains afterwards, a whole CTA at a time,
// with a larger table in global memory; the CTAs wait for that list with a
// bounded spin.
#include <algorithm>
#include <vector>

#include "bfc_internal.cuh"

namespace bfc {
namespace {

__device__ __forceinline__ uint64_t tr_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
// SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), counter based: output k of the
// sequence seeded by s; trial t uses the sequence seeded by output t + 1 of
// the caller's seed
__device__ __forceinline__ uint64_t tr_sm64(uint64_t s, uint64_t k) { return tr_mix(s + k * 0x9E3779B97F4A7C15ull); }
__device__ __forceinline__ uint32_t tr_colour(uint64_t ts, uint64_t k, uint32_t N) {
  return (uint32_t)(((tr_sm64(ts, k) >> 32) * (uint64_t)N) >> 32);
}

unsigned tr_grid(uint64_t n, unsigned threads, unsigned cap = 152 * 16) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

constexpr int KIND_ESPAR = 0, KIND_CLR = 1;

// ---------------------------------------------------------------------------
// keep masks
// ---------------------------------------------------------------------------
// One warp per 32-position block of a layout array (eid: the canonical edge
// id of each position); lane l owns position 32 b + l, and a ballot over the
// lanes gives trial t's word.  Lane (t mod 32) keeps that word, so every 32
// trials the warp writes 32 adjacent words at once.  ESpar: keep iff the top
// 32 bits of output e + 1 of trial tbase + t's sequence are < thr.  ClrSpar: keep iff
// the colours of u (counter u + 1) and of v (counter nU + v + 1) agree, with
// u_of / v_of the endpoints of each canonical edge.
template <int KIND>
__global__ void k_keep_bits(const uint32_t *eid, uint64_t m, uint64_t seed, uint32_t tbase, uint32_t T, uint32_t thr,
                            const uint32_t *u_of, const uint32_t *v_of, uint32_t nU, uint32_t N, uint32_t *bits) {
  const int lane = threadIdx.x & 31;
  const uint64_t nblk = (m + 31) / 32;
  const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t b = wid; b < nblk; b += nw) {
    const uint64_t pos = b * 32 + lane;
    const bool valid = pos < m;
    uint32_t e = 0, cu = 0, cv = 0;
    if (valid) {
      e = eid[pos];
      if (KIND == KIND_CLR) {
        cu = u_of[e] + 1;
        cv = nU + v_of[e] + 1;
      }
    }
    for (uint32_t t0 = 0; t0 < T; t0 += 32) {
      uint32_t mine = 0;
      const uint32_t tn = min(32u, T - t0);
      for (uint32_t k = 0; k < tn; k++) {
        const uint64_t ts = tr_sm64(seed, (uint64_t)tbase + t0 + k + 1);
        bool keep = false;
        if (valid) {
          if (KIND == KIND_ESPAR) keep = (uint32_t)(tr_sm64(ts, (uint64_t)e + 1) >> 32) < thr;
          else keep = tr_colour(ts, cu, N) == tr_colour(ts, cv, N);
        }
        const uint32_t wbits = __ballot_sync(0xffffffffu, keep);
        if (lane == (int)k) mine = wbits;
      }
      if ((uint32_t)lane < tn) bits[b * T + t0 + lane] = mine;
    }
  }
}

// bit of position pos for trial t
__device__ __forceinline__ uint32_t keep_bit(const uint32_t *bits, uint32_t T, uint64_t pos, uint32_t t) {
  return (bits[(pos >> 5) * T + t] >> (pos & 31)) & 1u;
}

// ---------------------------------------------------------------------------
// the persistent counting kernel
// ---------------------------------------------------------------------------
constexpr int TR_WARPS = 8, TR_THREADS = TR_WARPS * 32;
// per-warp table: one word a slot, (w + 1) << 7 | count, for start sides of
// fewer than 2^25 - 1 ranks and pairs of at most 127 kept start edges
constexpr uint32_t TR_SLOTS = 2048;
constexpr uint32_t TR_LIMIT = TR_SLOTS / 2;   // distinct targets a warp table takes
constexpr uint32_t TR_CMASK = 127;
constexpr uint32_t TR_TCHUNK = 32;            // trials per work item
constexpr size_t TR_WARP_BYTES = TR_SLOTS * 4 + TR_LIMIT * 2;
constexpr size_t TR_SMEM = TR_WARPS * TR_WARP_BYTES;
constexpr uint64_t TR_SPIN_MAX = 1ull << 23;  // bounded wait for the heavy list (about 2 s)

struct TArgs {
  const uint64_t *offR;
  const uint32_t *sX, *sB;
  const uint64_t *offM;
  const uint32_t *mR;
  const uint32_t *items;  // light start ranks (warp tables)
  uint32_t n_items;
  const uint32_t *heavy_items;  // start ranks whose pairs are counted by whole CTAs
  uint32_t n_heavy;
  const uint32_t *bitsS, *bitsM;  // keep masks (interleaved by trial)
  uint32_t T;
  unsigned long long *beta;  // [T]
  // q[0]: next light item, q[1]: overflowed pairs listed, q[2]: next overflowed pair,
  // q[3]: CTAs past the light phase, q[4]: next heavy-vertex item
  unsigned int *q;
  uint2 *heavy;  // (start rank, trial); entries start as (~0, ~0) and are written once
  uint32_t heavy_cap;
  unsigned long long *gt;  // per-CTA global tables ((w + 1) << 32 | count), 2^log_gslots each
  uint32_t log_gslots;
  uint32_t packed;  // start ranks + 1 fit 25 bits
  uint32_t *err;
};

__device__ __forceinline__ uint32_t tr_hash(uint32_t key, int shift) { return (key * 0x9E3779B1u) >> shift; }
__device__ __forceinline__ uint64_t warp_sum64(uint64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;  // valid in lane 0
}

// Count target key (= w + 1) in a warp table; returns the old count.  A slot
// newly claimed is listed (for the clear) while the table holds at most
// TR_LIMIT keys; past that the table is marked full (*over) and the pair is
// redone elsewhere.
__device__ __forceinline__ uint32_t wt_insert(uint32_t *slots, uint16_t *list, unsigned int *claimed, uint32_t key,
                                              bool &over) {
  uint32_t h = tr_hash(key, 21);
  for (uint32_t p = 0; p < TR_SLOTS; p++) {
    uint32_t v = reinterpret_cast<volatile uint32_t *>(slots)[h];
    if (v == 0u) {
      v = atomicCAS(&slots[h], 0u, (key << 7) | 1u);
      if (v == 0u) {
        const unsigned int c = atomicAdd(claimed, 1u);
        if (c < TR_LIMIT) list[c] = (uint16_t)h;
        else over = true;
        return 0;
      }
    }
    if ((v >> 7) == key) return atomicAdd(&slots[h], 1u) & TR_CMASK;
    h = (h + 1) & (TR_SLOTS - 1);
  }
  over = true;
  return 0;
}
__device__ __forceinline__ unsigned long long warp_max64(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xffffffffu, x, o);
    x = y > x ? y : x;
  }
  return x;  // in every lane
}
// count of key in a warp table (0 when absent); the table is not being written
__device__ __forceinline__ uint32_t wt_find(const uint32_t *slots, uint32_t key) {
  uint32_t h = tr_hash(key, 21);
  for (uint32_t p = 0; p < TR_SLOTS; p++) {
    const uint32_t v = slots[h];
    if ((v >> 7) == key) return v & TR_CMASK;
    if (v == 0u) return 0;
    h = (h + 1) & (TR_SLOTS - 1);
  }
  return 0;
}

// the bits of words k in [k_first, k_last] of a suffix [b, e) of a midpoint row
__device__ __forceinline__ uint32_t suffix_word(const uint32_t *bitsM, uint32_t T, uint32_t t, uint64_t k, uint64_t b,
                                                uint64_t e) {
  uint32_t word = bitsM[k * T + t];
  if (k == (b >> 5)) word &= 0xFFFFFFFFu << (b & 31);
  if (k == ((e - 1) >> 5)) {
    const uint32_t hi = (uint32_t)((e - 1) & 31);
    word &= (hi == 31) ? 0xFFFFFFFFu : ((2u << hi) - 1u);
  }
  return word;
}

// the kept bits of start-row word kb restricted to the row [rb, re)
__device__ __forceinline__ uint32_t start_word(const uint32_t *bitsS, uint32_t T, uint32_t t, uint64_t kb, uint64_t rb,
                                               uint64_t re) {
  uint32_t word = bitsS[kb * T + t];
  if (kb == (rb >> 5)) word &= 0xFFFFFFFFu << (rb & 31);
  if (kb == ((re - 1) >> 5)) {
    const uint32_t hi = (uint32_t)((re - 1) & 31);
    word &= (hi == 31) ? 0xFFFFFFFFu : ((2u << hi) - 1u);
  }
  return word;
}
// Call f(j) for every kept start edge j of rows [rb, re) in trial t: warp w
// reads bit words w, w + TR_WARPS, ... of the row and walks their set bits;
// all lanes of the warp call f together (a warp-cooperative body).
template <class F>
__device__ __forceinline__ void for_warp_starts(const uint32_t *bitsS, uint32_t T, uint32_t t, uint64_t rb,
                                                uint64_t re, F f) {
  if (re <= rb) return;
  const int warp = threadIdx.x >> 5;
  for (uint64_t kb = (rb >> 5) + warp; kb <= ((re - 1) >> 5); kb += TR_WARPS) {
    uint32_t word = start_word(bitsS, T, t, kb, rb, re);
    while (word) {
      const int bit = __ffs(word) - 1;
      word &= word - 1;
      f(kb * 32 + bit);
    }
  }
}
// count of key in a global table (0 when absent); the table is not being written
__device__ __forceinline__ uint32_t gt_find(const unsigned long long *gt, uint32_t mask, uint32_t key) {
  uint32_t h = (key * 0x9E3779B1u) & mask;
  for (uint32_t p = 0; p <= mask; p++) {
    const unsigned long long v = __ldcg(&gt[h]);
    if ((uint32_t)(v >> 32) == key) return (uint32_t)(v & 0xFFFFFFFFull);
    if (v == 0ull) return 0;
    h = (h + 1) & mask;
  }
  return 0;
}
// global-table insert for the heavy pairs; returns the old count
__device__ __forceinline__ uint32_t gt_insert(unsigned long long *gt, uint32_t mask, uint32_t key, uint32_t *err) {
  uint32_t h = (key * 0x9E3779B1u) & mask;
  const unsigned long long mine = ((unsigned long long)key << 32) | 1ull;
  for (uint32_t p = 0; p <= mask; p++) {
    unsigned long long v = __ldcg(&gt[h]);
    if (v == 0ull) {
      v = atomicCAS(&gt[h], 0ull, mine);
      if (v == 0ull) return 0;
    }
    if ((uint32_t)(v >> 32) == key) return (uint32_t)(atomicAdd(&gt[h], 1ull) & 0xFFFFFFFFull);
    h = (h + 1) & mask;
  }
  atomicOr(err, DERR_CAPACITY);
  return 0;
}

// One (start rank, trial) pair counted by the whole CTA.  A first pass finds
// the kept start edge with the longest suffix and counts the kept wedges of
// the other kept rows, which bound the table's distinct keys; the table is
// the CTA's shared memory when twice that count fits its SM_SLOTS, else the
// CTA's global table.  Adds the pair's sum_w C(c, 2) to beta[t].  All threads
// call it together; the shared words are in use only inside.
__device__ void cta_pair(const TArgs &a, uint32_t r, uint32_t t, uint32_t *sm, unsigned long long *gt,
                         unsigned long long *sh_red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t T = a.T;
  const uint64_t rb = a.offR[r], re = a.offR[r + 1];
  // the kept start edge with the longest suffix: its targets are looked up
  // afterwards (sum_w C(c, 2) = sum_w C(c_L, 2) + sum_{w in it} c_L(w), c_L
  // over the other kept rows), so the table holds the other rows' targets only
  // (the start row is read 32 positions per bit word: thread i takes words
  // i, i + TR_THREADS, ...; below, warp w takes words w, w + TR_WARPS, ...)
  unsigned long long best = 0;
  const uint64_t kb0 = rb >> 5, kb1 = (re - 1) >> 5;
  for (uint64_t kb = kb0 + threadIdx.x; re > rb && kb <= kb1; kb += TR_THREADS) {
    uint32_t word = start_word(a.bitsS, T, t, kb, rb, re);
    while (word) {
      const int bit = __ffs(word) - 1;
      word &= word - 1;
      const uint64_t j = kb * 32 + bit;
      const uint64_t len = a.offM[a.sX[j] + 1] - a.sB[j];
      const unsigned long long key = (len << 32) | (0xFFFFFFFFu - (uint32_t)(j - rb));
      best = key > best ? key : best;
    }
  }
  best = warp_max64(best);
  if (lane == 0) sh_red[warp] = best;
  __syncthreads();
  for (int w = 0; w < TR_WARPS; w++) best = sh_red[w] > best ? sh_red[w] : best;
  const uint64_t jh = best ? rb + (0xFFFFFFFFu - (uint32_t)(best & 0xFFFFFFFFu)) : ~0ull;
  __syncthreads();
  // kept wedges of the other rows bound the table's keys
  uint64_t kw = 0;
  for_warp_starts(a.bitsS, T, t, rb, re, [&](uint64_t j) {
    if (j == jh) return;
    const uint32_t x = a.sX[j];
    const uint64_t b = a.sB[j], e = a.offM[x + 1];
    if (e <= b) return;
    const uint64_t k_last = (e - 1) >> 5;
    for (uint64_t k = (b >> 5) + lane; k <= k_last; k += 32) kw += __popc(suffix_word(a.bitsM, T, t, k, b, e));
  });
  kw = warp_sum64(kw);
  if (lane == 0) sh_red[warp] = kw;
  __syncthreads();
  uint64_t kept = 0;
  for (int w = 0; w < TR_WARPS; w++) kept += sh_red[w];
  // slots of a shared-memory table: the largest power of two whose keys and
  // counts fit the CTA's dynamic shared memory
  constexpr uint32_t SM_SLOTS = (TR_SMEM / 8 >= 16384) ? 16384u : (TR_SMEM / 8 >= 8192) ? 8192u : 4096u;
  const bool in_smem = 2 * kept <= SM_SLOTS;
  uint32_t logT = 6;
  while (((uint64_t)1 << logT) < 2 * kept && logT < (in_smem ? 31u : a.log_gslots)) logT++;
  const uint32_t mask = (1u << logT) - 1u;
  const int shift = 32 - (int)logT;
  uint32_t *keys = sm, *cnts = sm + (mask + 1);
  if (in_smem) {
    for (uint32_t i = threadIdx.x; i < 2 * (mask + 1); i += TR_THREADS) sm[i] = 0;
  } else {
    for (uint32_t i = threadIdx.x; i <= mask; i += TR_THREADS) gt[i] = 0ull;
  }
  __syncthreads();
  uint64_t acc = 0;
  // pass 0: the other kept rows into the table; pass 1: the longest one looked up
  for (int pass = 0; pass < 2; pass++) {
    for_warp_starts(a.bitsS, T, t, rb, re, [&](uint64_t j) {
      if ((pass == 0) == (j == jh)) return;
      const uint32_t x = a.sX[j];
      const uint64_t b = a.sB[j], e = a.offM[x + 1];
      if (e <= b) return;
      const uint64_t k_last = (e - 1) >> 5;
      for (uint64_t k = (b >> 5) + lane; k <= k_last; k += 32) {
        uint32_t word = suffix_word(a.bitsM, T, t, k, b, e);
        while (word) {
          const int bit = __ffs(word) - 1;
          word &= word - 1;
          const uint32_t key = a.mR[k * 32 + bit] + 1u;
          if (!in_smem) {
            acc += pass == 0 ? gt_insert(gt, mask, key, a.err) : gt_find(gt, mask, key);
            continue;
          }
          uint32_t h = (key * 0x9E3779B1u) >> shift;
          for (uint32_t pr = 0;; pr++) {
            uint32_t kk = reinterpret_cast<volatile uint32_t *>(keys)[h];
            if (pass == 1) {
              if (kk == key) acc += cnts[h];
              if (kk == key || kk == 0u || pr == mask) break;
            } else {
              if (kk == 0u) kk = atomicCAS(&keys[h], 0u, key);
              if (kk == 0u || kk == key) {
                acc += atomicAdd(&cnts[h], 1u);
                break;
              }
              if (pr == mask) {  // cannot happen at half load
                atomicOr(a.err, DERR_CAPACITY);
                break;
              }
            }
            h = (h + 1) & mask;
          }
        }
      }
    });
    __syncthreads();
  }
  acc = warp_sum64(acc);
  if (lane == 0) sh_red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0;
    for (int w = 0; w < TR_WARPS; w++) s += sh_red[w];
    if (s) atomicAdd(&a.beta[t], s);
  }
  __syncthreads();
}

// Light phase: a warp takes (light start rank, 32 trials) items from q[0];
// for each trial it checks that at least two start edges are kept (fewer
// cannot close a butterfly), then walks the kept start edges and, for each,
// the set bits of its midpoint row after the start vertex, 32 words (1,024
// positions) per step.  Heavy phase: CTAs take (heavy start rank, 32 trials)
// items from q[4] (start vertices expected to overflow a warp table), then the
// pairs that did overflow one from q[2], and count them with cta_pair.
__global__ void __launch_bounds__(TR_THREADS, 2) k_trials(TArgs a) {
  extern __shared__ uint8_t tr_smem[];
  __shared__ unsigned int claimed[TR_WARPS];
  __shared__ unsigned long long sh_red[TR_WARPS];
  __shared__ uint32_t sh_state, sh_item;
  __shared__ uint2 sh_pair;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *slots = reinterpret_cast<uint32_t *>(tr_smem + (size_t)warp * TR_WARP_BYTES);
  uint16_t *list = reinterpret_cast<uint16_t *>(slots + TR_SLOTS);
  for (uint32_t i = lane; i < TR_SLOTS; i += 32) slots[i] = 0;
  if (lane == 0) claimed[warp] = 0;
  __syncwarp();
  const uint32_t T = a.T, nchunks = (T + TR_TCHUNK - 1) / TR_TCHUNK;
  const uint64_t n_work = (uint64_t)a.n_items * nchunks;
  // ---- light phase
  while (true) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(&a.q[0], 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if ((uint64_t)item >= n_work) break;
    const uint32_t r = a.items[item / nchunks];
    const uint32_t t_lo = (item % nchunks) * TR_TCHUNK, t_hi = min(T, t_lo + TR_TCHUNK);
    const uint64_t rb = a.offR[r], re = a.offR[r + 1];
    for (uint32_t t = t_lo; t < t_hi; t++) {
      // kept start edges, and the one with the longest suffix (its targets
      // are looked up, not inserted: see cta_pair)
      uint32_t nk = 0;
      unsigned long long best = 0;
      for (uint64_t c = rb; c < re; c += 32) {
        const uint64_t j = c + lane;
        const bool kept = j < re && keep_bit(a.bitsS, T, j, t);
        nk += __popc(__ballot_sync(0xffffffffu, kept));
        if (kept) {
          const uint64_t len = a.offM[a.sX[j] + 1] - a.sB[j];
          const unsigned long long key = (len << 32) | (0xFFFFFFFFu - (uint32_t)(j - rb));
          best = key > best ? key : best;
        }
      }
      if (nk < 2) continue;
      best = warp_max64(best);
      // counts above TR_CMASK or keys above 25 bits do not fit a slot: such a
      // pair goes to the whole-CTA path
      bool over = nk > TR_CMASK || !a.packed;
      const uint64_t jh = rb + (0xFFFFFFFFu - (uint32_t)(best & 0xFFFFFFFFu));
      uint64_t acc = 0;
      for (uint64_t c = rb; c < re && !over; c += 32) {
        const uint64_t j = c + lane;
        uint32_t bal = __ballot_sync(0xffffffffu, j < re && j != jh && keep_bit(a.bitsS, T, j, t));
        while (bal) {
          const int l = __ffs(bal) - 1;
          bal &= bal - 1;
          const uint64_t jj = c + l;
          const uint32_t x = a.sX[jj];
          const uint64_t b = a.sB[jj], e = a.offM[x + 1];
          if (e <= b) continue;
          const uint64_t k_last = (e - 1) >> 5;
          for (uint64_t k0 = b >> 5; k0 <= k_last; k0 += 32) {
            const uint64_t k = k0 + lane;
            uint32_t word = (k <= k_last) ? suffix_word(a.bitsM, T, t, k, b, e) : 0u;
            while (word) {
              const int bit = __ffs(word) - 1;
              word &= word - 1;
              const uint32_t w = a.mR[k * 32 + bit];
              acc += wt_insert(slots, list, &claimed[warp], w + 1u, over);
            }
            if (__any_sync(0xffffffffu, over)) break;
          }
          if (__any_sync(0xffffffffu, over)) break;
        }
        if (__any_sync(0xffffffffu, over)) break;
      }
      __syncwarp();
      if (!__any_sync(0xffffffffu, over)) {
        // the longest kept suffix against the table: a target met c times in
        // the other rows adds c pairs
        const uint32_t x = a.sX[jh];
        const uint64_t b = a.sB[jh], e = a.offM[x + 1];
        if (e > b) {
          const uint64_t k_last = (e - 1) >> 5;
          for (uint64_t k = (b >> 5) + lane; k <= k_last; k += 32) {
            uint32_t word = suffix_word(a.bitsM, T, t, k, b, e);
            while (word) {
              const int bit = __ffs(word) - 1;
              word &= word - 1;
              acc += wt_find(slots, a.mR[k * 32 + bit] + 1u);
            }
          }
        }
      }
      const bool full = __any_sync(0xffffffffu, over);
      __syncwarp();
      // back to an empty table: the listed slots, or all of them past the limit
      const unsigned int nc = claimed[warp];
      if (nc > TR_LIMIT) {
        for (uint32_t i = lane; i < TR_SLOTS; i += 32) slots[i] = 0;
      } else {
        for (uint32_t i = lane; i < nc; i += 32) slots[list[i]] = 0;
      }
      __syncwarp();
      if (lane == 0) claimed[warp] = 0;
      if (full) {
        if (lane == 0) {
          const unsigned int hi = atomicAdd(&a.q[1], 1u);
          if (hi < a.heavy_cap) {
            // the trial first, then the rank the readers test against ~0
            volatile uint32_t *hp = reinterpret_cast<volatile uint32_t *>(a.heavy + hi);
            hp[1] = t;
            __threadfence();
            hp[0] = r;
            __threadfence();
          } else {
            atomicOr(a.err, DERR_CAPACITY);
          }
        }
      } else {
        acc = warp_sum64(acc);
        if (lane == 0 && acc) atomicAdd(&a.beta[t], (unsigned long long)acc);
      }
      __syncwarp();
    }
  }
  // ---- heavy phase
  __syncthreads();
  // past the light phase: no more pairs will be listed by this CTA
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&a.q[3], 1u);
  }
  unsigned long long *gt = a.gt + ((uint64_t)blockIdx.x << a.log_gslots);
  uint32_t *sm = reinterpret_cast<uint32_t *>(tr_smem);
  const uint64_t n_heavy_work = (uint64_t)a.n_heavy * nchunks;
  while (true) {
    if (threadIdx.x == 0) sh_item = atomicAdd(&a.q[4], 1u);
    __syncthreads();
    const uint32_t item = sh_item;
    if ((uint64_t)item >= n_heavy_work) break;
    const uint32_t r = a.heavy_items[item / nchunks];
    const uint32_t t_lo = (item % nchunks) * TR_TCHUNK, t_hi = min(T, t_lo + TR_TCHUNK);
    for (uint32_t t = t_lo; t < t_hi; t++) cta_pair(a, r, t, sm, gt, sh_red);
  }
  while (true) {
    if (threadIdx.x == 0) {
      // claim the next overflowed pair; wait (bounded) until it is listed and
      // written, or until every CTA is past its light phase and the list
      // turns out shorter
      const uint32_t idx = atomicAdd(&a.q[2], 1u);
      uint32_t state = 2;  // 0: process, 2: done
      for (uint64_t spin = 0;; spin++) {
        const bool final_list = *(volatile unsigned int *)&a.q[3] == gridDim.x;
        __threadfence();
        const uint32_t listed = min(*(volatile unsigned int *)&a.q[1], a.heavy_cap);
        if (idx < listed) {
          const volatile uint32_t *hp = reinterpret_cast<const volatile uint32_t *>(a.heavy + idx);
          const uint32_t er = hp[0];
          if (er != 0xFFFFFFFFu) {
            __threadfence();
            sh_pair = make_uint2(er, hp[1]);
            state = 0;
            break;
          }
        } else if (final_list) {
          break;
        }
        if (spin >= TR_SPIN_MAX) {
          atomicOr(a.err, DERR_TIMEOUT);
          break;
        }
        __nanosleep(256);
      }
      sh_state = state;
    }
    __syncthreads();
    if (sh_state != 0) break;
    const uint2 pr = sh_pair;
    cta_pair(a, pr.x, pr.y, sm, gt, sh_red);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// the class list without the skip class, reversed (big class, then the
// window classes, then the warp class: roughly heaviest first), split into the
// start ranks whose expected kept wedges (work * kept fraction) exceed half a
// warp table (heavy: work > wthr) and the others; flag[k] = 1 for heavy
__global__ void k_heavy_flags(const uint32_t *cls, uint32_t begin, uint32_t n, const uint64_t *work, uint64_t wthr,
                              uint32_t *flag) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x)
    flag[k] = work[cls[begin + n - 1 - k]] > wthr ? 1u : 0u;
}
__global__ void k_split_items(const uint32_t *cls, uint32_t begin, uint32_t n, const uint32_t *flag,
                              const uint64_t *pos, uint32_t *heavy, uint32_t *light) {
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t r = cls[begin + n - 1 - k];
    if (flag[k]) heavy[pos[k]] = r;
    else light[k - pos[k]] = r;
  }
}
__global__ void k_u_of_edges(const uint64_t *offU, uint32_t nU, uint32_t *u_of) {
  const int lane = threadIdx.x & 31;
  const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = wid; u < nU; u += nw)
    for (uint64_t e = offU[u] + lane; e < offU[u + 1]; e += 32) u_of[e] = (uint32_t)u;
}
__global__ void k_max_work(const uint64_t *work, uint32_t n, unsigned long long *out) {
  unsigned long long mx = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    mx = max(mx, (unsigned long long)work[i]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

}  // namespace

// The trials of one estimator, [t0, t0 + T) of its trial sequence, in one
// launch of k_trials after the keep masks (the two launches and the clears
// before them are recorded into one CUDA graph on a capturable stream).
// beta: host, T entries.
int run_trials(bfc_graph *g, int kind, uint64_t seed, uint32_t thr, uint32_t colors, uint32_t trials, uint64_t *beta,
               cudaStream_t s) {
  const int side = choose_side(g, 0);
  BFC_TRY(plan_build(g, side, s));
  Plan &p = g->plan[side];
  const uint64_t m = p.m;
  for (uint32_t t = 0; t < trials; t++) beta[t] = 0;
  const uint32_t n_items = p.nS - p.cls_count[0];  // every class but skip
  if (m == 0 || n_items == 0) return BFC_OK;
  int occ = 0, dev = 0, sms = 0;
  BFC_CUDA_TRY(cudaFuncSetAttribute(k_trials, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TR_SMEM));
  BFC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_trials, TR_THREADS, TR_SMEM));
  BFC_CUDA_TRY(cudaGetDevice(&dev));
  BFC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // every CTA of the grid is resident at once (the heavy phase waits for all of them)
  const unsigned grid = (unsigned)std::max(1, occ) * (unsigned)std::max(1, sms);
  // trials per pass: keep masks of at most 24 GB
  const uint64_t nblk = (m + 31) / 32;
  const uint64_t per_trial = nblk * 4 * 2;
  const uint32_t batch = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(trials, (24ull << 30) / per_trial));
  DBuf bitsS, bitsM, items, hitems, flag, fpos, uof, q, heavy, gt, betas, mx;
  auto cleanup = [&]() {
    DBuf *bs[] = {&bitsS, &bitsM, &items, &hitems, &flag, &fpos, &uof, &q, &heavy, &gt, &betas, &mx};
    for (DBuf *b : bs) dfree(*b, s);
  };
  int rc = BFC_OK;
#define TR_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
#define TR_CUDA(x) do { if ((x) != cudaSuccess) { cleanup(); return BFC_ECUDA; } } while (0)
  TR_TRY(dalloc(bitsS, (uint64_t)batch * nblk * 4, s));
  TR_TRY(dalloc(bitsM, (uint64_t)batch * nblk * 4, s));
  TR_TRY(dalloc(items, (uint64_t)n_items * 4, s));
  TR_TRY(dalloc(q, 32, s));
  TR_TRY(dalloc(betas, (uint64_t)batch * 8, s));
  TR_TRY(dalloc(mx, 8, s));
  if (kind == KIND_CLR) {
    TR_TRY(dalloc(uof, m * 4, s));
    k_u_of_edges<<<tr_grid((uint64_t)g->nU * 32, 256), 256, 0, s>>>(ptr<uint64_t>(g->offU), g->nU, ptr<uint32_t>(uof));
    count_launch();
  }
  // kept fraction of the wedges: p^2 (ESpar), 1 / N^2 (ClrSpar)
  const double pk = (double)thr / 4294967296.0;
  const double kf = kind == KIND_ESPAR ? pk * pk : 1.0 / ((double)colors * (double)colors);
  const double wt = (double)(4 * TR_LIMIT) / std::max(kf, 1e-300);
  const uint64_t wthr = wt >= 1.8e19 ? ~0ull : (uint64_t)wt;
  TR_TRY(dalloc(hitems, (uint64_t)n_items * 4, s));
  TR_TRY(dalloc(flag, (uint64_t)n_items * 4, s));
  TR_TRY(dalloc(fpos, ((uint64_t)n_items + 1) * 8, s));
  k_heavy_flags<<<tr_grid(n_items, 256), 256, 0, s>>>(ptr<uint32_t>(p.cls), p.cls_count[0], n_items,
                                                      ptr<uint64_t>(p.work), wthr, ptr<uint32_t>(flag));
  count_launch();
  TR_TRY(exclusive_scan_u32_to_u64(ptr<uint32_t>(flag), ptr<uint64_t>(fpos), n_items, g->scr, s));
  k_split_items<<<tr_grid(n_items, 256), 256, 0, s>>>(ptr<uint32_t>(p.cls), p.cls_count[0], n_items,
                                                      ptr<uint32_t>(flag), ptr<uint64_t>(fpos),
                                                      ptr<uint32_t>(hitems), ptr<uint32_t>(items));
  count_launch();
  uint64_t n_heavy = 0;
  TR_CUDA(cudaMemcpyAsync(&n_heavy, ptr<uint64_t>(fpos) + n_items, 8, cudaMemcpyDeviceToHost, s));
  // global tables: twice the largest start vertex's wedge count, at most
  // 2^20 slots a CTA and 4 GB in all
  TR_CUDA(cudaMemsetAsync(mx.p, 0, 8, s));
  k_max_work<<<tr_grid(p.nS, 256), 256, 0, s>>>(ptr<uint64_t>(p.work), p.nS, ptr<unsigned long long>(mx));
  count_launch();
  unsigned long long maxw = 0;
  TR_CUDA(cudaMemcpyAsync(&maxw, mx.p, 8, cudaMemcpyDeviceToHost, s));
  TR_CUDA(cudaStreamSynchronize(s));
  uint32_t log_gslots = 10;
  while (log_gslots < 20 && (1ull << log_gslots) < 2 * maxw) log_gslots++;
  while (log_gslots > 10 && ((uint64_t)grid << log_gslots) * 8 > (4ull << 30)) log_gslots--;
  TR_TRY(dalloc(gt, ((uint64_t)grid << log_gslots) * 8, s));
  const uint64_t heavy_cap = std::min<uint64_t>((uint64_t)n_items * batch, 1ull << 24);
  TR_TRY(dalloc(heavy, heavy_cap * 8, s));
  TR_CUDA(cudaGetLastError());
  for (uint32_t t0 = 0; t0 < trials && !rc; t0 += batch) {
    const uint32_t T = std::min(batch, trials - t0);
    auto enqueue = [&]() -> int {
      if (cudaMemsetAsync(q.p, 0, 32, s) != cudaSuccess) return BFC_ECUDA;
      if (cudaMemsetAsync(betas.p, 0, (uint64_t)T * 8, s) != cudaSuccess) return BFC_ECUDA;
      if (cudaMemsetAsync(heavy.p, 0xFF, heavy_cap * 8, s) != cudaSuccess) return BFC_ECUDA;
      const unsigned kg = tr_grid(nblk * 32, 256);
      if (kind == KIND_ESPAR) {
        k_keep_bits<KIND_ESPAR><<<kg, 256, 0, s>>>(ptr<uint32_t>(p.sEid), m, seed, t0, T, thr, nullptr, nullptr, 0, 0,
                                                   ptr<uint32_t>(bitsS));
        k_keep_bits<KIND_ESPAR><<<kg, 256, 0, s>>>(ptr<uint32_t>(p.mEid), m, seed, t0, T, thr, nullptr, nullptr, 0, 0,
                                                   ptr<uint32_t>(bitsM));
      } else {
        k_keep_bits<KIND_CLR><<<kg, 256, 0, s>>>(ptr<uint32_t>(p.sEid), m, seed, t0, T, 0, ptr<uint32_t>(uof),
                                                 ptr<uint32_t>(g->nbrU), g->nU, colors, ptr<uint32_t>(bitsS));
        k_keep_bits<KIND_CLR><<<kg, 256, 0, s>>>(ptr<uint32_t>(p.mEid), m, seed, t0, T, 0, ptr<uint32_t>(uof),
                                                 ptr<uint32_t>(g->nbrU), g->nU, colors, ptr<uint32_t>(bitsM));
      }
      count_launch(2);
      TArgs a{};
      a.offR = ptr<uint64_t>(p.offR);
      a.sX = ptr<uint32_t>(p.sX);
      a.sB = ptr<uint32_t>(p.sB);
      a.offM = p.offM;
      a.mR = ptr<uint32_t>(p.mR);
      a.items = ptr<uint32_t>(items);
      a.n_items = n_items - (uint32_t)n_heavy;
      a.heavy_items = ptr<uint32_t>(hitems);
      a.n_heavy = (uint32_t)n_heavy;
      a.bitsS = ptr<uint32_t>(bitsS);
      a.bitsM = ptr<uint32_t>(bitsM);
      a.T = T;
      a.beta = ptr<unsigned long long>(betas);
      a.q = ptr<unsigned int>(q);
      a.heavy = ptr<uint2>(heavy);
      a.heavy_cap = (uint32_t)heavy_cap;
      a.gt = ptr<unsigned long long>(gt);
      a.log_gslots = log_gslots;
      a.packed = (uint64_t)p.nS + 1 < (1ull << 25) ? 1u : 0u;
      a.err = ptr<uint32_t>(g->err);
      profile_begin("trials", s);
      k_trials<<<grid, TR_THREADS, TR_SMEM, s>>>(a);
      count_launch();
      profile_end("trials", s);
      return cudaGetLastError() == cudaSuccess ? BFC_OK : BFC_ECUDA;
    };
    // record the pass into one CUDA graph and launch it once; a stream that
    // cannot be captured (the legacy default stream) or a profiled run (its
    // events) takes the launches directly
    bool ran = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (s != nullptr && !profile_on() && cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int r = enqueue();
      const cudaError_t e = cudaStreamEndCapture(s, &graph);
      if (r == BFC_OK && e == cudaSuccess && graph && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
        ran = cudaGraphLaunch(exec, s) == cudaSuccess;
      cudaGetLastError();  // a failed recording leaves no sticky error
    }
    if (!ran) rc = enqueue();
    if (!rc && cudaMemcpyAsync(beta + t0, betas.p, (uint64_t)T * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
      rc = BFC_ECUDA;
    if (!rc) rc = read_device_error(g, s);  // synchronises s
    else cudaStreamSynchronize(s);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
  cleanup();
#undef TR_TRY
#undef TR_CUDA
  return rc;
}

}  // namespace bfc
