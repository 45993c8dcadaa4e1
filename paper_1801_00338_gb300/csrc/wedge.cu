// Wedge aggregation: the hot loop of ExactBFC (Algorithm 1, the loops over
// v, u in Gamma_v, w in Gamma_u), of vBFC (Algorithm 2) and of the per-edge
// counts.
//
// For a start vertex v (rank r) the multiplicity c(v, w) = |Gamma_v ^ Gamma_w|
// of every later start vertex w (rank > r) is counted, then sum_w C(c, 2) is
// the number of butterflies with v and w as their start-side pair (Lemma 1,
// Eq. (2)-(3)); every unordered pair is seen once, from its lower rank.
//
// Start vertices are split into classes by the number of wedges they walk
// (Lemma 3: vBFC costs O(|Gamma^2_v|)):
//   skip  : degree < 2 or nothing after it; c <= 1 everywhere, contributes 0
//   warp  : few wedges; one warp per vertex, open-addressing table in shared memory
//   cta   : many wedges; one CTA per vertex, a dense counter array in shared
//           memory covering a window ("tile") of Z consecutive ranks; the rank
//           space is walked tile by tile from r+1 upwards, skipping empty tiles.
//
// Modes: TOTAL (B only), VERTEX (b for both sides), EDGE (b_e).
//   start side  b_v += sum_w C(c(v,w), 2), b_w += C(c(v,w), 2)
//   mid side    b_x += c(v,w) - 1 for each wedge v - x - w (pairs through x)
//   edges       b_(v,x) += c(v,w) - 1, b_(w,x) += c(v,w) - 1 for each wedge v - x - w
// which are the definitions of Section 2 written per wedge: a butterfly
// {v, w} x {x, y} is seen from the wedge v - x - w once for each of its two
// midpoints.
#include <algorithm>
#include <vector>

#include "bfc_internal.cuh"

namespace bfc {

constexpr uint32_t EMPTY_KEY = 0xFFFFFFFFu;
constexpr uint32_t CLS_SKIP = 0, CLS_WARP = 1, CLS_CTA = 2;

// warp class
constexpr int WH_WARPS = 8;
constexpr int WH_SLOTS = 1024;                    // per warp
constexpr uint64_t WH_MAX_WORK = WH_SLOTS / 2;    // load factor <= 1/2
// cta class
constexpr int CT_THREADS = 1024;
constexpr uint32_t CT_Z = 48 * 1024;              // u32 counters (192 KB)
constexpr uint32_t CT_SEG = 256;                  // elements per segment

struct WArgs {
  uint32_t nS;
  const uint64_t *offR;
  const uint32_t *sX, *sEid, *sB;
  const uint64_t *offM;
  const uint32_t *mR, *mEid;
  const uint32_t *vert_of;
  const uint32_t *list;
  uint32_t list_n;
  unsigned int *queue;
  unsigned long long *B;
  unsigned long long *bS, *bM, *be;
  uint32_t *err;
  // cta-class segment scratch (per CTA, seg_cap entries each)
  uint32_t *seg;        // 5 u32 per segment: begin, end, cur, pstart, next
  uint32_t *seg_row;    // row index per segment
  uint32_t seg_cap;
  // MODE_SINGLE (Algorithm 2 on a batch): list holds item ids
  const uint32_t *item_rank;
  unsigned long long *bitem;
};

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
__device__ __forceinline__ long long warp_sum_i64(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// ---------------------------------------------------------------------------
// warp class: open addressing in shared memory (keys = start ranks)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t wh_hash(uint32_t w) { return (w * 0x9E3779B1u) >> (32 - 10); }
static_assert(WH_SLOTS == 1024, "wh_hash assumes 1024 slots");

__device__ __forceinline__ void wh_insert(uint32_t *keys, uint32_t *cnts, uint32_t w) {
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
// lanes must call this together.
// FULL: the whole midpoint row (Algorithm 2: every w != v) instead of the
// part after v.
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
    const uint64_t rb = a.offR[r], re = a.offR[r + 1];
    warp_for_each_wedge<MODE == MODE_SINGLE>(a, rb, re, [&](uint32_t i, uint64_t) {
      const uint32_t w = a.mR[i];
      if (MODE != MODE_SINGLE || w != r) wh_insert(keys, cnts, w);
    });
    __syncwarp();
    if (MODE != MODE_TOTAL) {
      // second sweep: every wedge learns its final multiplicity
      for (uint64_t chunk = rb; chunk < re; chunk += 32) {
        // per-row sums: accumulate into per-lane slots then flush per row
        warp_for_each_wedge<false>(a, chunk, min(chunk + 32, re), [&](uint32_t i, uint64_t j) {
          uint32_t c = wh_lookup(keys, cnts, a.mR[i]);
          if (c > 1) {
            if (MODE == MODE_EDGE) {
              atomicAdd(&a.be[a.mEid[i]], (unsigned long long)(c - 1));
              atomicAdd(&a.be[a.sEid[j]], (unsigned long long)(c - 1));
            } else {
              atomicAdd(&a.bM[a.sX[j]], (unsigned long long)(c - 1));
            }
          }
        });
      }
      __syncwarp();
    }
    uint64_t acc = 0;
    for (int i = lane; i < WH_SLOTS; i += 32) {
      uint32_t k = keys[i];
      if (k != EMPTY_KEY) {
        uint64_t p = pairs_of(cnts[i]);
        acc += p;
        if (MODE == MODE_VERTEX && p) atomicAdd(&a.bS[a.vert_of[k]], (unsigned long long)p);
        keys[i] = EMPTY_KEY;
        cnts[i] = 0;
      }
    }
    acc = warp_sum_u64(acc);
    if (lane == 0) {
      localB += acc;
      if (MODE == MODE_VERTEX && acc) atomicAdd(&a.bS[a.vert_of[r]], (unsigned long long)acc);
      if (MODE == MODE_SINGLE) a.bitem[item] = acc;
    }
    __syncwarp();
  }
  if (lane == 0 && localB) atomicAdd(a.B, (unsigned long long)localB);
}

// ---------------------------------------------------------------------------
// cta class: dense counters over a window of CT_Z ranks
// ---------------------------------------------------------------------------
// tile of rank w: windows are aligned to the top of the rank space,
// window k covers [nS - (k+1) Z, nS - k Z)
__device__ __forceinline__ void tile_bounds(uint32_t nS, uint32_t w, uint32_t &lo, uint32_t &hi) {
  uint32_t k = (nS - 1 - w) / CT_Z;
  hi = nS - k * CT_Z;
  lo = hi > CT_Z ? hi - CT_Z : 0;
}

template <int MODE>
__global__ void __launch_bounds__(CT_THREADS, 1) k_cta_class(WArgs a) {
  extern __shared__ uint32_t ctr[];  // CT_Z counters
  __shared__ uint32_t s_idx, s_nseg, s_next_min, s_carry;
  __shared__ unsigned long long s_acc;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = CT_THREADS / 32;
  uint32_t *seg = a.seg + (size_t)blockIdx.x * a.seg_cap * 5;
  uint32_t *seg_row = a.seg_row + (size_t)blockIdx.x * a.seg_cap;
  for (uint32_t i = threadIdx.x; i < CT_Z; i += CT_THREADS) ctr[i] = 0;
  uint64_t localB = 0;
  __syncthreads();
  while (true) {
    if (threadIdx.x == 0) {
      s_idx = atomicAdd(a.queue, 1u);
      s_nseg = 0;
      s_carry = 0;
      s_acc = 0;
      s_next_min = 0xFFFFFFFFu;
    }
    __syncthreads();
    const uint32_t idx = s_idx;
    if (idx >= a.list_n) break;
    const uint32_t item = a.list[idx];
    const uint32_t r = (MODE == MODE_SINGLE) ? a.item_rank[item] : item;
    const uint64_t rb = a.offR[r], re = a.offR[r + 1];
    // ---- segments: each start-row entry's suffix cut into pieces of CT_SEG
    for (uint64_t base = rb; base < re; base += CT_THREADS) {
      uint64_t j = base + threadIdx.x;
      uint32_t b = 0, e = 0, ns = 0;
      if (j < re) {
        const uint32_t x = a.sX[j];
        b = (MODE == MODE_SINGLE) ? (uint32_t)a.offM[x] : a.sB[j];
        e = (uint32_t)a.offM[x + 1];
        ns = (e - b + CT_SEG - 1) / CT_SEG;
      }
      // block exclusive scan of ns
      uint32_t incl = warp_incl_scan_u32(ns);
      __shared__ uint32_t wtot[NW];
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
        uint32_t sb = b + k * CT_SEG;
        uint32_t se = min(e, sb + CT_SEG);
        uint32_t *sg = seg + (size_t)(first + k) * 5;
        sg[0] = sb; sg[1] = se; sg[2] = sb; sg[3] = sb; sg[4] = 0;  // next = 0: unknown, load it
        seg_row[first + k] = (uint32_t)j;
      }
      __syncthreads();
    }
    const uint32_t nseg = min(s_carry, a.seg_cap);
    // ---- walk the windows
    uint32_t lo, hi;
    tile_bounds(a.nS, (MODE == MODE_SINGLE) ? 0u : r + 1, lo, hi);
    while (true) {
      // count
      for (uint32_t sidx = warp; sidx < nseg; sidx += NW) {
        uint32_t *sg = seg + (size_t)sidx * 5;
        uint32_t pos = sg[2], end = sg[1], nxt = sg[4];
        uint32_t pstart = pos;
        if (pos < end && nxt < hi) {
          while (pos < end) {
            uint32_t i = pos + lane;
            uint32_t w = (i < end) ? a.mR[i] : 0xFFFFFFFFu;
            bool in = w < hi;
            uint32_t bal = __ballot_sync(0xffffffffu, in);
            if (in && (MODE != MODE_SINGLE || w != r)) atomicAdd(&ctr[w - lo], 1u);
            uint32_t n = __popc(bal);
            pos += n;
            if (n < 32) {
              nxt = __shfl_sync(0xffffffffu, w, n);  // first rank at or above hi (or 0xFFFFFFFF)
              break;
            }
          }
          if (pos >= end) nxt = 0xFFFFFFFFu;
          if (lane == 0) { sg[2] = pos; sg[3] = pstart; sg[4] = nxt; }
        } else {
          if (lane == 0) sg[3] = pos;  // nothing this window
          if (pos >= end) nxt = 0xFFFFFFFFu;
        }
        if (lane == 0 && nxt != 0xFFFFFFFFu) atomicMin(&s_next_min, nxt);
      }
      __syncthreads();
      // VERTEX / EDGE: every wedge of this window reads its final count
      if (MODE != MODE_TOTAL) {
        for (uint32_t sidx = warp; sidx < nseg; sidx += NW) {
          uint32_t *sg = seg + (size_t)sidx * 5;
          uint32_t ps = sg[3], pe = sg[2];
          if (ps >= pe) continue;
          uint32_t j = seg_row[sidx];
          long long rowsum = 0;
          for (uint32_t i = ps + lane; i < pe; i += 32) {
            uint32_t c = ctr[a.mR[i] - lo];
            if (c > 1) {
              rowsum += c - 1;
              if (MODE == MODE_EDGE) atomicAdd(&a.be[a.mEid[i]], (unsigned long long)(c - 1));
            }
          }
          rowsum = warp_sum_i64(rowsum);
          if (lane == 0 && rowsum) {
            if (MODE == MODE_EDGE) atomicAdd(&a.be[a.sEid[j]], (unsigned long long)rowsum);
            else atomicAdd(&a.bM[a.sX[j]], (unsigned long long)rowsum);
          }
        }
        __syncthreads();
      }
      // exchange: collect C(c, 2) once per distinct w and clear the window
      uint64_t acc = 0;
      for (uint32_t sidx = warp; sidx < nseg; sidx += NW) {
        uint32_t *sg = seg + (size_t)sidx * 5;
        uint32_t ps = sg[3], pe = sg[2];
        for (uint32_t i = ps + lane; i < pe; i += 32) {
          uint32_t w = a.mR[i];
          uint32_t c = atomicExch(&ctr[w - lo], 0u);
          if (c > 1) {
            uint64_t p = pairs_of(c);
            acc += p;
            if (MODE == MODE_VERTEX) atomicAdd(&a.bS[a.vert_of[w]], (unsigned long long)p);
          }
        }
      }
      acc = warp_sum_u64(acc);
      if (lane == 0 && acc) atomicAdd(&s_acc, (unsigned long long)acc);
      __syncthreads();
      const uint32_t nm = s_next_min;
      __syncthreads();
      if (nm == 0xFFFFFFFFu || nm >= a.nS) break;
      if (threadIdx.x == 0) s_next_min = 0xFFFFFFFFu;
      tile_bounds(a.nS, nm, lo, hi);
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      localB += s_acc;
      if (MODE == MODE_VERTEX && s_acc) atomicAdd(&a.bS[a.vert_of[r]], s_acc);
      if (MODE == MODE_SINGLE) a.bitem[item] = s_acc;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0 && localB) atomicAdd(a.B, (unsigned long long)localB);
}

// ---------------------------------------------------------------------------
// classification
// ---------------------------------------------------------------------------
__global__ void k_classify(const uint64_t *offR, const uint64_t *work, uint32_t nS, uint32_t *cls_of,
                           unsigned int *counts, unsigned long long *maxseg, unsigned long long *cls_sums) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nS; r += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t d = offR[r + 1] - offR[r], w = work[r];
    uint32_t c = (d < 2 || w == 0) ? CLS_SKIP : (w <= WH_MAX_WORK ? CLS_WARP : CLS_CTA);
    cls_of[r] = c;
    atomicAdd(&counts[c], 1u);
    if (w) atomicAdd(&cls_sums[c], (unsigned long long)w);
    if (d) atomicAdd(&cls_sums[3 + c], (unsigned long long)d);
    if (c == CLS_CTA) atomicMax(maxseg, (unsigned long long)(d + w / CT_SEG + 1));
  }
}
__global__ void k_scatter_class(const uint32_t *cls_of, uint32_t nS, const unsigned int *begin, unsigned int *cursor,
                                uint32_t *list) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nS; r += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t c = cls_of[r];
    uint32_t p = atomicAdd(&cursor[c], 1u);
    list[begin[c] + p] = (uint32_t)r;
  }
}
__global__ void k_work_keys(const uint32_t *list, uint32_t n, const uint64_t *work, uint64_t *keys, uint32_t *vals) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t r = list[i];
    keys[i] = ~work[r];  // ascending sort of ~work = descending work
    vals[i] = r;
  }
}

static unsigned grid_for(uint64_t n, unsigned threads, unsigned cap = 152 * 16) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

struct ClassMeta {
  uint32_t seg_cap = 0;
};
static ClassMeta g_meta_dummy;

int plan_classify(bfc_graph *g, Plan &p, cudaStream_t s) {
  const uint32_t nS = p.nS;
  BFC_TRY(dalloc(p.cls, (uint64_t)std::max<uint32_t>(nS, 1) * 4, s));
  DBuf cls_of, cnt, k1, k2, v2;
  auto cleanup = [&]() { dfree(cls_of, s); dfree(cnt, s); dfree(k1, s); dfree(k2, s); dfree(v2, s); };
  int rc = BFC_OK;
#define PC_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
  PC_TRY(dalloc(cls_of, (uint64_t)std::max<uint32_t>(nS, 1) * 4, s));
  PC_TRY(dalloc(cnt, 128, s));
  BFC_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, 128, s));
  unsigned int *counts = ptr<unsigned int>(cnt);
  unsigned long long *maxseg = reinterpret_cast<unsigned long long *>(counts + 8);
  unsigned long long *sums = reinterpret_cast<unsigned long long *>(counts + 16);  // 6 x u64
  k_classify<<<grid_for(nS, 256), 256, 0, s>>>(ptr<uint64_t>(p.offR), ptr<uint64_t>(p.work), nS,
                                              ptr<uint32_t>(cls_of), counts, maxseg, sums);
  count_launch();
  unsigned int hc[8];
  unsigned long long hmax = 0, hs[6];
  BFC_CUDA_TRY(cudaMemcpyAsync(hc, counts, 32, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaMemcpyAsync(&hmax, maxseg, 8, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaMemcpyAsync(hs, sums, 48, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  for (int c = 0; c < 3; c++) { p.cls_work[c] = hs[c]; p.cls_rows[c] = hs[3 + c]; }
  unsigned int hb[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int c = 0; c < 3; c++) {
    p.cls_count[c] = hc[c];
    p.cls_begin[c] = (c == 0) ? 0 : p.cls_begin[c - 1] + p.cls_count[c - 1];
    hb[c] = p.cls_begin[c];
  }
  p.cls_count[3] = (uint32_t)std::min<unsigned long long>(hmax, 0xFFFFFFFFull);  // segment capacity
  BFC_CUDA_TRY(cudaMemcpyAsync(counts, hb, 32, cudaMemcpyHostToDevice, s));
  BFC_CUDA_TRY(cudaMemsetAsync(counts + 8, 0, 32, s));
  k_scatter_class<<<grid_for(nS, 256), 256, 0, s>>>(ptr<uint32_t>(cls_of), nS, counts, counts + 8,
                                                   ptr<uint32_t>(p.cls));
  count_launch();
  // heaviest first inside the cta class
  const uint32_t nc = p.cls_count[CLS_CTA];
  if (nc > 1) {
    PC_TRY(dalloc(k1, (uint64_t)nc * 8, s));
    PC_TRY(dalloc(k2, (uint64_t)nc * 8, s));
    PC_TRY(dalloc(v2, (uint64_t)nc * 4, s));
    uint32_t *list = ptr<uint32_t>(p.cls) + p.cls_begin[CLS_CTA];
    k_work_keys<<<grid_for(nc, 256), 256, 0, s>>>(list, nc, ptr<uint64_t>(p.work), ptr<uint64_t>(k1), list);
    count_launch();
    PC_TRY(radix_sort_u64(ptr<uint64_t>(k1), ptr<uint64_t>(k2), list, ptr<uint32_t>(v2), nc, 64, g->scr, s));
    BFC_CUDA_TRY(cudaMemcpyAsync(list, v2.p, (uint64_t)nc * 4, cudaMemcpyDeviceToDevice, s));
  }
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  cleanup();
#undef PC_TRY
  (void)g_meta_dummy;
  return BFC_OK;
}

// ---------------------------------------------------------------------------
// driver
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

static const char *tag_of(int cls, int mode) {
  static const char *tags[2][3] = {{"warp.total", "warp.vertex", "warp.edge"}, {"cta.total", "cta.vertex", "cta.edge"}};
  return tags[cls == CLS_CTA ? 1 : 0][mode];
}

template <int MODE>
static int launch_lists(bfc_graph *g, WArgs a, const uint32_t *warp_list, uint32_t n_warp, const uint32_t *cta_list,
                        uint32_t n_cta, uint32_t seg_cap, cudaStream_t s) {
  const int sms = sm_count();
  unsigned int *queues = ptr<unsigned int>(g->acc) + 16;  // two counters
  BFC_CUDA_TRY(cudaMemsetAsync(queues, 0, 8, s));
  const int tmode = MODE == MODE_SINGLE ? 0 : MODE;
  if (n_warp) {
    WArgs w = a;
    w.list = warp_list;
    w.list_n = n_warp;
    w.queue = queues;
    const size_t smem = (size_t)WH_WARPS * 2 * WH_SLOTS * 4;
    BFC_CUDA_TRY(cudaFuncSetAttribute(k_warp_class<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    BFC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_warp_class<MODE>, WH_WARPS * 32, smem));
    unsigned grid = (unsigned)std::max(1, occ) * sms;
    grid = std::min<unsigned>(grid, (w.list_n + WH_WARPS - 1) / WH_WARPS);
    profile_begin(tag_of(CLS_WARP, tmode), s);
    k_warp_class<MODE><<<grid, WH_WARPS * 32, smem, s>>>(w);
    BFC_LAUNCHED();
    profile_end(tag_of(CLS_WARP, tmode), s);
  }
  if (n_cta) {
    WArgs c = a;
    c.list = cta_list;
    c.list_n = n_cta;
    c.queue = queues + 1;
    const size_t smem = (size_t)CT_Z * 4;
    BFC_CUDA_TRY(cudaFuncSetAttribute(k_cta_class<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    unsigned grid = std::min<unsigned>((unsigned)sms, c.list_n);
    c.seg_cap = std::max<uint32_t>(seg_cap, 1);
    const uint64_t need = (uint64_t)grid * c.seg_cap * 6 * 4;
    BFC_TRY(g->scr.reserve(need, s));
    c.seg = static_cast<uint32_t *>(g->scr.base());
    c.seg_row = c.seg + (uint64_t)grid * c.seg_cap * 5;
    profile_begin(tag_of(CLS_CTA, tmode), s);
    k_cta_class<MODE><<<grid, CT_THREADS, smem, s>>>(c);
    BFC_LAUNCHED();
    profile_end(tag_of(CLS_CTA, tmode), s);
  }
  return BFC_OK;
}

template <int MODE>
static int launch_classes(bfc_graph *g, Plan &p, WArgs a, cudaStream_t s) {
  const uint32_t *cls = ptr<uint32_t>(p.cls);
  return launch_lists<MODE>(g, a, cls + p.cls_begin[CLS_WARP], p.cls_count[CLS_WARP], cls + p.cls_begin[CLS_CTA],
                            p.cls_count[CLS_CTA], p.cls_count[3], s);
}

static WArgs args_of(bfc_graph *g, Plan &p) {
  WArgs a{};
  a.nS = p.nS;
  a.offR = ptr<uint64_t>(p.offR);
  a.sX = ptr<uint32_t>(p.sX);
  a.sEid = ptr<uint32_t>(p.sEid);
  a.sB = ptr<uint32_t>(p.sB);
  a.offM = p.offM;
  a.mR = ptr<uint32_t>(p.mR);
  a.mEid = ptr<uint32_t>(p.mEid);
  a.vert_of = ptr<uint32_t>(p.vert_of);
  a.err = ptr<uint32_t>(g->err);
  return a;
}

// ---------------------------------------------------------------------------
// batched Algorithm 2
// ---------------------------------------------------------------------------
__global__ void k_item_classify(const uint32_t *item_rank, uint32_t n, const uint64_t *offR, const uint32_t *sX,
                                const uint64_t *offM, uint32_t *cls_of, unsigned int *counts,
                                unsigned long long *maxseg, unsigned long long *out) {
  const int lane = threadIdx.x & 31;
  uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = warp; i < n; i += nw) {
    const uint32_t r = item_rank[i];
    const uint64_t b = offR[r], e = offR[r + 1];
    uint64_t w = 0;
    for (uint64_t j = b + lane; j < e; j += 32) {
      const uint32_t x = sX[j];
      w += offM[x + 1] - offM[x] - 1;
    }
    w = warp_sum_u64(w);
    if (lane == 0) {
      const uint64_t d = e - b;
      uint32_t c = (d < 2 || w == 0) ? CLS_SKIP : (w <= WH_MAX_WORK ? CLS_WARP : CLS_CTA);
      cls_of[i] = c;
      atomicAdd(&counts[c], 1u);
      out[i] = 0;
      if (c == CLS_CTA) atomicMax(maxseg, (unsigned long long)(d + w / CT_SEG + 1));
    }
  }
}
__global__ void k_item_scatter(const uint32_t *cls_of, uint32_t n, unsigned int *cursor, uint32_t *warp_list,
                               uint32_t *cta_list) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t c = cls_of[i];
    if (c == CLS_WARP) warp_list[atomicAdd(&cursor[0], 1u)] = (uint32_t)i;
    else if (c == CLS_CTA) cta_list[atomicAdd(&cursor[1], 1u)] = (uint32_t)i;
  }
}

int vbfc_batch(bfc_graph *g, Plan &p, const uint32_t *item_rank, uint32_t n_items, unsigned long long *out,
               cudaStream_t s) {
  if (n_items == 0) return BFC_OK;
  DBuf cls_of, lists, cnt;
  auto cleanup = [&]() { dfree(cls_of, s); dfree(lists, s); dfree(cnt, s); };
  int rc = BFC_OK;
#define VB_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
  VB_TRY(dalloc(cls_of, (uint64_t)n_items * 4, s));
  VB_TRY(dalloc(lists, (uint64_t)n_items * 8, s));
  VB_TRY(dalloc(cnt, 64, s));
  BFC_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, 64, s));
  unsigned int *counts = ptr<unsigned int>(cnt);
  unsigned long long *maxseg = reinterpret_cast<unsigned long long *>(counts + 4);
  k_item_classify<<<grid_for((uint64_t)n_items * 32, 256), 256, 0, s>>>(item_rank, n_items, ptr<uint64_t>(p.offR),
                                                                        ptr<uint32_t>(p.sX), p.offM,
                                                                        ptr<uint32_t>(cls_of), counts, maxseg, out);
  count_launch();
  unsigned int hc[4];
  unsigned long long hmax = 0;
  BFC_CUDA_TRY(cudaMemcpyAsync(hc, counts, 16, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaMemcpyAsync(&hmax, maxseg, 8, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  uint32_t *warp_list = ptr<uint32_t>(lists);
  uint32_t *cta_list = warp_list + n_items;
  BFC_CUDA_TRY(cudaMemsetAsync(counts + 8, 0, 8, s));
  k_item_scatter<<<grid_for(n_items, 256), 256, 0, s>>>(ptr<uint32_t>(cls_of), n_items, counts + 8, warp_list,
                                                       cta_list);
  count_launch();
  WArgs a = args_of(g, p);
  a.item_rank = item_rank;
  a.bitem = out;
  unsigned long long dummyB_off = 0;
  (void)dummyB_off;
  a.B = ptr<unsigned long long>(g->acc) + 1;  // not read back
  VB_TRY(launch_lists<MODE_SINGLE>(g, a, warp_list, hc[CLS_WARP], cta_list, hc[CLS_CTA],
                                   (uint32_t)std::min<unsigned long long>(hmax, 0xFFFFFFFFull), s));
  cleanup();
#undef VB_TRY
  return BFC_OK;
}

int wedge_count(bfc_graph *g, Plan &p, Mode mode, unsigned long long *d_B, uint64_t *bS, uint64_t *bM, uint64_t *be,
                cudaStream_t s) {
  WArgs a = args_of(g, p);
  a.B = d_B;
  a.bS = reinterpret_cast<unsigned long long *>(bS);
  a.bM = reinterpret_cast<unsigned long long *>(bM);
  a.be = reinterpret_cast<unsigned long long *>(be);
  switch (mode) {
    case MODE_TOTAL: return launch_classes<MODE_TOTAL>(g, p, a, s);
    case MODE_VERTEX: return launch_classes<MODE_VERTEX>(g, p, a, s);
    case MODE_EDGE: return launch_classes<MODE_EDGE>(g, p, a, s);
  }
  return BFC_EINVAL;
}

}  // namespace bfc
