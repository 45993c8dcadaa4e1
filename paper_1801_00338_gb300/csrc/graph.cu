// Graph preparation on the device.
//
// Section 2 ("Preliminaries" and "Networks and Experimental Setup"): the input
// is a simple bipartite graph; repeated edges are either rejected or dropped.
// Algorithm 1, first three lines: the start side is L unless
// sum_L d^2 < sum_R d^2.  Algorithm 1's coloured line counts each pair of
// start vertices once under a total order; here the order is the rank
// (ascending degree, ties by id), the reading that keeps the per-vertex tables
// of high-degree start vertices small.
//
// Layout built per start side S with midpoint side M (struct Plan):
//   start rows in rank order:  offR[r] .. offR[r+1]  ->  sX (midpoint x),
//                              sEid (canonical edge id), sB (suffix begin)
//   midpoint rows:             offM[x] .. offM[x+1]  ->  mR (start ranks,
//                              ascending), mEid (canonical edge id)
// For start rank r and an entry (r, x), the wedges r -> x -> w with w after r
// are exactly mR[sB .. offM[x+1]), because row x is sorted by rank and sB is
// one past r's own position in it.
#include <algorithm>

#include "bfc_internal.cuh"

namespace bfc {

static inline unsigned grid_for(uint64_t n, unsigned threads, unsigned cap = 152 * 16) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

// ---------------------------------------------------------------------------
// edge keys
// ---------------------------------------------------------------------------
__global__ void k_make_keys(const uint32_t *u, const uint32_t *v, uint64_t m, uint32_t nU, uint32_t nV, int bV,
                            uint64_t *key, uint32_t *err) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t a = u[e], x = v[e];
    if (a >= nU || x >= nV) {
      atomicOr(err, DERR_RANGE);
      a = 0;
      x = 0;
    }
    key[e] = ((uint64_t)a << bV) | x;
  }
}

__global__ void k_mark_unique(const uint64_t *key, uint64_t m, uint32_t *flag, unsigned long long *dups) {
  uint64_t local = 0;
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t f = (e == 0 || key[e] != key[e - 1]) ? 1u : 0u;
    flag[e] = f;
    local += 1 - f;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_down_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(dups, (unsigned long long)local);
}

__global__ void k_compact_keys(const uint64_t *key, const uint32_t *flag, const uint64_t *pos, uint64_t m,
                               uint64_t *out) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
    if (flag[e]) out[pos[e]] = key[e];
}

// Row offsets from a sorted row-id sequence: off[r] = first index whose row is >= r.
// rowid(e) = key[e] >> shift (64-bit keys) -- every offset entry written once.
__global__ void k_offsets_from_sorted64(const uint64_t *key, uint64_t m, int shift, uint32_t nrows, uint64_t *off) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= m; e += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t prev = (e == 0) ? 0 : (key[e - 1] >> shift) + 1;   // first row not yet started
    uint64_t cur = (e == m) ? (uint64_t)nrows : (key[e] >> shift);
    for (uint64_t r = prev; r <= cur && r <= nrows; r++) {
      if (e == 0 || r >= prev) off[r] = e;
    }
  }
}
__global__ void k_offsets_from_sorted32(const uint32_t *key, uint64_t m, uint32_t nrows, uint64_t *off) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= m; e += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t prev = (e == 0) ? 0 : (uint64_t)key[e - 1] + 1;
    uint64_t cur = (e == m) ? (uint64_t)nrows : (uint64_t)key[e];
    for (uint64_t r = prev; r <= cur && r <= nrows; r++) off[r] = e;
  }
}

__global__ void k_split_u_side(const uint64_t *key, uint64_t m, int bV, uint32_t *nbrU, uint32_t *vkey,
                               uint32_t *iota) {
  const uint64_t mask = (bV >= 64) ? ~0ull : ((1ull << bV) - 1);
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x = (uint32_t)(key[e] & mask);
    nbrU[e] = x;
    vkey[e] = x;
    iota[e] = (uint32_t)e;
  }
}

__global__ void k_fill_v_side(const uint64_t *key, const uint32_t *perm, uint64_t m, int bV, uint32_t *nbrV,
                              uint32_t *eidV) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t e = perm[j];
    nbrV[j] = (uint32_t)(key[e] >> bV);
    eidV[j] = e;
  }
}

__global__ void k_degrees(const uint64_t *off, uint32_t n, uint32_t *deg, unsigned long long *acc) {
  // acc[0] += sum d^2, acc[1] += sum C(d,2), acc[2] = max d
  uint64_t sq = 0, w = 0;
  uint32_t mx = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t d = off[i + 1] - off[i];
    deg[i] = (uint32_t)d;
    sq += d * d;
    w += d * (d - (d > 0)) / 2;
    mx = max(mx, (uint32_t)d);
  }
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_down_sync(0xffffffffu, sq, o);
    w += __shfl_down_sync(0xffffffffu, w, o);
    mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (sq) atomicAdd(&acc[0], (unsigned long long)sq);
    if (w) atomicAdd(&acc[1], (unsigned long long)w);
    if (mx) atomicMax(&acc[2], (unsigned long long)mx);
  }
}

static int read_err_word(bfc_graph *g, cudaStream_t s, uint32_t *out) {
  BFC_CUDA_TRY(cudaMemcpyAsync(out, g->err.p, 4, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  return BFC_OK;
}

int read_device_error(bfc_graph *g, cudaStream_t s) {
  uint32_t e = 0;
  BFC_TRY(read_err_word(g, s, &e));
  if (e == 0) return BFC_OK;
  BFC_CUDA_TRY(cudaMemsetAsync(g->err.p, 0, 4, s));
  if (e & DERR_RANGE) return BFC_ERANGE;
  if (e & DERR_DUP) return BFC_EDUP;
  if (e & DERR_TIMEOUT) return BFC_ETIMEOUT;
  if (e & DERR_OVERFLOW) return BFC_EOVERFLOW;
  if (e & DERR_INVALID) return BFC_EINVAL;
  return BFC_EINTERNAL;
}

// degrees, sum d^2, wedges C(d, 2) and maximum degree of both sides
static int degree_stats(bfc_graph *g, cudaStream_t s) {
  const uint32_t nU = g->nU, nV = g->nV;
  BFC_CUDA_TRY(cudaMemsetAsync(g->acc.p, 0, 256, s));
  unsigned long long *acc = ptr<unsigned long long>(g->acc);
  k_degrees<<<grid_for(nU, 256), 256, 0, s>>>(ptr<uint64_t>(g->offU), nU, ptr<uint32_t>(g->degU), acc);
  count_launch();
  k_degrees<<<grid_for(nV, 256), 256, 0, s>>>(ptr<uint64_t>(g->offV), nV, ptr<uint32_t>(g->degV), acc + 4);
  count_launch();
  unsigned long long h[8];
  BFC_CUDA_TRY(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  BFC_CUDA_TRY(cudaGetLastError());
  g->sqU = h[0]; g->wU = h[1]; g->maxU = (uint32_t)h[2];
  g->sqV = h[4]; g->wV = h[5]; g->maxV = (uint32_t)h[6];
  return BFC_OK;
}

int graph_build(bfc_graph *g, const uint32_t *u, const uint32_t *v, uint64_t m, uint32_t flags, cudaStream_t s) {
  const uint32_t nU = g->nU, nV = g->nV;
  const int bU = std::max(1, bits_for(nU - 1)), bV = std::max(1, bits_for(nV - 1));
  BFC_TRY(dalloc(g->err, 64, s));
  BFC_CUDA_TRY(cudaMemsetAsync(g->err.p, 0, 64, s));
  BFC_TRY(dalloc(g->acc, 256, s));

  // input on the device
  DBuf du, dv, key, key2, flag, pos;
  const uint32_t *pu = u, *pv = v;
  auto cleanup = [&]() {
    dfree(du, s); dfree(dv, s); dfree(key, s); dfree(key2, s); dfree(flag, s); dfree(pos, s);
  };
  if (!(flags & BFC_INPUT_DEVICE) && m > 0) {
    int rc = dalloc(du, m * 4, s);
    if (!rc) rc = dalloc(dv, m * 4, s);
    if (rc) { cleanup(); return rc; }
    if (cudaMemcpyAsync(du.p, u, m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(dv.p, v, m * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      cleanup();
      return BFC_ECUDA;
    }
    pu = ptr<uint32_t>(du);
    pv = ptr<uint32_t>(dv);
  }
  int rc = BFC_OK;
#define GB_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
  GB_TRY(dalloc(key, std::max<uint64_t>(m, 1) * 8, s));
  GB_TRY(dalloc(key2, std::max<uint64_t>(m, 1) * 8, s));
  if (m > 0) {
    k_make_keys<<<grid_for(m, 256), 256, 0, s>>>(pu, pv, m, nU, nV, bV, ptr<uint64_t>(key), ptr<uint32_t>(g->err));
    count_launch();
    GB_TRY(read_device_error(g, s));
    // canonical order: sort by (u, v)
    GB_TRY(radix_sort_u64(ptr<uint64_t>(key), ptr<uint64_t>(key2), nullptr, nullptr, m, bU + bV, g->scr, s));
    std::swap(key, key2);
    // duplicates
    GB_TRY(dalloc(flag, m * 4, s));
    GB_TRY(dalloc(pos, (m + 1) * 8, s));
    BFC_CUDA_TRY(cudaMemsetAsync(g->acc.p, 0, 256, s));
    k_mark_unique<<<grid_for(m, 256), 256, 0, s>>>(ptr<uint64_t>(key), m, ptr<uint32_t>(flag),
                                                  ptr<unsigned long long>(g->acc));
    count_launch();
    uint64_t dups = 0;
    BFC_CUDA_TRY(cudaMemcpyAsync(&dups, g->acc.p, 8, cudaMemcpyDeviceToHost, s));
    BFC_CUDA_TRY(cudaStreamSynchronize(s));
    if (dups) {
      if (!(flags & BFC_DEDUP)) { cleanup(); return BFC_EDUP; }
      GB_TRY(exclusive_scan_u32_to_u64(ptr<uint32_t>(flag), ptr<uint64_t>(pos), m, g->scr, s));
      k_compact_keys<<<grid_for(m, 256), 256, 0, s>>>(ptr<uint64_t>(key), ptr<uint32_t>(flag), ptr<uint64_t>(pos), m,
                                                     ptr<uint64_t>(key2));
      count_launch();
      std::swap(key, key2);
      m -= dups;
    }
  }
  g->m = m;
  if (m >= (1ull << 32)) { cleanup(); return BFC_ERANGE; }
  GB_TRY(dalloc(g->offU, ((uint64_t)nU + 1) * 8, s));
  GB_TRY(dalloc(g->offV, ((uint64_t)nV + 1) * 8, s));
  GB_TRY(dalloc(g->nbrU, std::max<uint64_t>(m, 1) * 4, s));
  GB_TRY(dalloc(g->nbrV, std::max<uint64_t>(m, 1) * 4, s));
  GB_TRY(dalloc(g->eidV, std::max<uint64_t>(m, 1) * 4, s));
  GB_TRY(dalloc(g->degU, (uint64_t)nU * 4, s));
  GB_TRY(dalloc(g->degV, (uint64_t)nV * 4, s));
  // U side: rows are runs of equal u in the sorted keys
  k_offsets_from_sorted64<<<grid_for(m + 1, 256), 256, 0, s>>>(ptr<uint64_t>(key), m, bV, nU, ptr<uint64_t>(g->offU));
  count_launch();
  // V side: stable sort of canonical ids by v keeps u ascending within a row
  DBuf vk, vk2, io, io2;
  auto cleanup2 = [&]() { dfree(vk, s); dfree(vk2, s); dfree(io, s); dfree(io2, s); };
  if ((rc = dalloc(vk, std::max<uint64_t>(m, 1) * 4, s)) || (rc = dalloc(vk2, std::max<uint64_t>(m, 1) * 4, s)) ||
      (rc = dalloc(io, std::max<uint64_t>(m, 1) * 4, s)) || (rc = dalloc(io2, std::max<uint64_t>(m, 1) * 4, s))) {
    cleanup2(); cleanup(); return rc;
  }
  if (m > 0) {
    k_split_u_side<<<grid_for(m, 256), 256, 0, s>>>(ptr<uint64_t>(key), m, bV, ptr<uint32_t>(g->nbrU),
                                                   ptr<uint32_t>(vk), ptr<uint32_t>(io));
    count_launch();
    rc = radix_sort_u32(ptr<uint32_t>(vk), ptr<uint32_t>(vk2), ptr<uint32_t>(io), ptr<uint32_t>(io2), m, bV, g->scr, s);
    if (rc) { cleanup2(); cleanup(); return rc; }
    k_fill_v_side<<<grid_for(m, 256), 256, 0, s>>>(ptr<uint64_t>(key), ptr<uint32_t>(io2), m, bV,
                                                  ptr<uint32_t>(g->nbrV), ptr<uint32_t>(g->eidV));
    count_launch();
  }
  k_offsets_from_sorted32<<<grid_for(m + 1, 256), 256, 0, s>>>(ptr<uint32_t>(vk2), m, nV, ptr<uint64_t>(g->offV));
  count_launch();
  cleanup2();
  cleanup();
#undef GB_TRY
  return degree_stats(g, s);
}

// ---------------------------------------------------------------------------
// graph from caller-owned rows
// ---------------------------------------------------------------------------
// offsets: start at 0, never decrease, end at m
__global__ void k_check_offsets(const uint64_t *off, uint32_t n, uint64_t m, uint32_t *err) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    if (off[i] > off[i + 1] || off[i + 1] > m || (i == 0 && off[0] != 0)) atomicOr(err, DERR_INVALID);
}
// every entry below `bound`; strictly ascending within its row (one warp per row)
__global__ void k_check_rows(const uint64_t *off, uint32_t n, const uint32_t *nbr, uint32_t bound, uint32_t *err) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = warp; r < n; r += nw) {
    for (uint64_t i = off[r] + lane; i < off[r + 1]; i += 32) {
      const uint32_t x = nbr[i];
      if (x >= bound) atomicOr(err, DERR_RANGE);
      if (i > off[r] && nbr[i - 1] >= x) atomicOr(err, DERR_INVALID);
    }
  }
}
// canonical id of each V-row entry (x's row holds a): the position of x in
// a's ascending row; with `given` ids, check them instead
__global__ void k_edge_ids(const uint64_t *offU, const uint32_t *nbrU, const uint64_t *offV, uint32_t nV,
                           const uint32_t *nbrV, const uint32_t *given, uint32_t *eidV, uint32_t *err) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t x = warp; x < nV; x += nw) {
    for (uint64_t i = offV[x] + lane; i < offV[x + 1]; i += 32) {
      const uint32_t a = nbrV[i];
      uint64_t lo = offU[a], hi = offU[a + 1];
      while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (nbrU[mid] < x) lo = mid + 1; else hi = mid;
      }
      const bool found = lo < offU[a + 1] && nbrU[lo] == (uint32_t)x;
      if (!found || (given && given[i] != lo)) atomicOr(err, DERR_INVALID);
      eidV[i] = (uint32_t)lo;
    }
  }
}

int graph_from_rows(bfc_graph *g, const uint64_t *offU, const uint32_t *nbrU, const uint64_t *offV,
                    const uint32_t *nbrV, const uint32_t *eidV, cudaStream_t s) {
  const uint32_t nU = g->nU, nV = g->nV;
  BFC_TRY(dalloc(g->err, 64, s));
  BFC_CUDA_TRY(cudaMemsetAsync(g->err.p, 0, 64, s));
  BFC_TRY(dalloc(g->acc, 256, s));
  uint64_t mm[2];
  BFC_CUDA_TRY(cudaMemcpyAsync(&mm[0], offU + nU, 8, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaMemcpyAsync(&mm[1], offV + nV, 8, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  if (mm[0] != mm[1]) return BFC_EINVAL;
  const uint64_t m = mm[0];
  if (m >= (1ull << 32)) return BFC_ERANGE;
  g->m = m;
  const uint64_t mb = std::max<uint64_t>(m, 1) * 4;
  BFC_TRY(dalloc(g->offU, ((uint64_t)nU + 1) * 8, s));
  BFC_TRY(dalloc(g->offV, ((uint64_t)nV + 1) * 8, s));
  BFC_TRY(dalloc(g->nbrU, mb, s));
  BFC_TRY(dalloc(g->nbrV, mb, s));
  BFC_TRY(dalloc(g->eidV, mb, s));
  BFC_TRY(dalloc(g->degU, (uint64_t)nU * 4, s));
  BFC_TRY(dalloc(g->degV, (uint64_t)nV * 4, s));
  BFC_CUDA_TRY(cudaMemcpyAsync(g->offU.p, offU, ((uint64_t)nU + 1) * 8, cudaMemcpyDeviceToDevice, s));
  BFC_CUDA_TRY(cudaMemcpyAsync(g->offV.p, offV, ((uint64_t)nV + 1) * 8, cudaMemcpyDeviceToDevice, s));
  if (m) {
    BFC_CUDA_TRY(cudaMemcpyAsync(g->nbrU.p, nbrU, m * 4, cudaMemcpyDeviceToDevice, s));
    BFC_CUDA_TRY(cudaMemcpyAsync(g->nbrV.p, nbrV, m * 4, cudaMemcpyDeviceToDevice, s));
  }
  uint32_t *err = ptr<uint32_t>(g->err);
  k_check_offsets<<<grid_for(nU, 256), 256, 0, s>>>(ptr<uint64_t>(g->offU), nU, m, err);
  count_launch();
  k_check_offsets<<<grid_for(nV, 256), 256, 0, s>>>(ptr<uint64_t>(g->offV), nV, m, err);
  count_launch();
  BFC_TRY(read_device_error(g, s));  // the row checks below index by these offsets
  k_check_rows<<<grid_for((uint64_t)nU * 32, 256), 256, 0, s>>>(ptr<uint64_t>(g->offU), nU, ptr<uint32_t>(g->nbrU),
                                                               nV, err);
  count_launch();
  k_check_rows<<<grid_for((uint64_t)nV * 32, 256), 256, 0, s>>>(ptr<uint64_t>(g->offV), nV, ptr<uint32_t>(g->nbrV),
                                                               nU, err);
  count_launch();
  BFC_TRY(read_device_error(g, s));  // ids in range before they index rows
  k_edge_ids<<<grid_for((uint64_t)nV * 32, 256), 256, 0, s>>>(ptr<uint64_t>(g->offU), ptr<uint32_t>(g->nbrU),
                                                             ptr<uint64_t>(g->offV), nV, ptr<uint32_t>(g->nbrV),
                                                             eidV, ptr<uint32_t>(g->eidV), err);
  count_launch();
  BFC_TRY(read_device_error(g, s));
  return degree_stats(g, s);
}

// Algorithm 1, first three lines: start from L (= U) unless sum_L d^2 < sum_R d^2.
int choose_side(const bfc_graph *g, uint32_t flags) {
  if (flags & BFC_SIDE_U) return 0;
  if (flags & BFC_SIDE_V) return 1;
  return (g->sqU < g->sqV) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
__global__ void k_iota_and_copy(const uint32_t *deg, uint32_t n, uint32_t *keys, uint32_t *iota) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    keys[i] = deg[i];
    iota[i] = (uint32_t)i;
  }
}
__global__ void k_group_keys(const uint32_t *vert_of, const uint32_t *group, uint32_t n, uint32_t *keys,
                             uint32_t *vals) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = vert_of[r];
    keys[r] = group[x];
    vals[r] = x;
  }
}
__global__ void k_rank_of(const uint32_t *vert_of, const uint32_t *deg, uint32_t n, uint32_t *rank_of, uint32_t *dR) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t x = vert_of[r];
    rank_of[x] = (uint32_t)r;
    dR[r] = deg[x];
  }
}
// one warp per start rank: copy its row in rank order
__global__ void k_fill_start_rows(const uint32_t *vert_of, uint32_t nS, const uint64_t *offS, const uint32_t *nbrS,
                                  const uint32_t *eidS /* null: eid = position */, const uint64_t *offR,
                                  uint32_t *sX, uint32_t *sEid, uint32_t *sRank) {
  const int lane = threadIdx.x & 31;
  uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = warp; r < nS; r += nwarps) {
    uint32_t x = vert_of[r];
    uint64_t src = offS[x], len = offS[x + 1] - src, dst = offR[r];
    for (uint64_t k = lane; k < len; k += 32) {
      sX[dst + k] = nbrS[src + k];
      sEid[dst + k] = eidS ? eidS[src + k] : (uint32_t)(src + k);
      sRank[dst + k] = (uint32_t)r;
    }
  }
}
__global__ void k_fill_mid_rows(const uint32_t *perm, uint64_t m, const uint32_t *sRank, const uint32_t *sEid,
                                uint32_t *mR, uint32_t *mEid, uint32_t *sB) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t j = perm[i];
    mR[i] = sRank[j];
    mEid[i] = sEid[j];
    sB[j] = (uint32_t)(i + 1);
  }
}
// work[r] = sum over the row of (offM[x+1] - sB): wedges walked from r
__global__ void k_work(const uint64_t *offR, uint32_t nS, const uint32_t *sX, const uint32_t *sB, const uint64_t *offM,
                       uint64_t *work) {
  const int lane = threadIdx.x & 31;
  uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = warp; r < nS; r += nwarps) {
    uint64_t b = offR[r], e = offR[r + 1];
    uint64_t t = 0;
    for (uint64_t j = b + lane; j < e; j += 32) t += offM[sX[j] + 1] - sB[j];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) work[r] = t;
  }
}

int plan_classify(bfc_graph *g, Plan &p, cudaStream_t s);  // wedge.cu

// class limits of the graph's tuning (0 = the default)
static void tuned_limits(const bfc_graph *g, uint32_t *warp_max, uint32_t *small_max) {
  *warp_max = g->tune.warp_max_wedges ? g->tune.warp_max_wedges : 512u;
  *small_max = g->tune.small_max_segs ? g->tune.small_max_segs : 128u;
}

int plan_build(bfc_graph *g, int side, cudaStream_t s) {
  Plan &p = g->plan[side];
  uint32_t wmax, smax;
  tuned_limits(g, &wmax, &smax);
  if (p.built) {
    if (p.warp_max == wmax && p.small_max == smax) return BFC_OK;
    // the tuning changed a class limit: redo the classification only
    dfree(p.cls, s);
    p.warp_max = wmax;
    p.small_max = smax;
    return plan_classify(g, p, s);
  }
  p.warp_max = wmax;
  p.small_max = smax;
  p.side = side;
  const uint32_t nS = side ? g->nV : g->nU, nM = side ? g->nU : g->nV;
  const uint64_t m = g->m;
  p.nS = nS; p.nM = nM; p.m = m;
  p.max_deg_S = side ? g->maxV : g->maxU;
  const uint32_t *degS = ptr<uint32_t>(side ? g->degV : g->degU);
  const uint64_t *offS = ptr<uint64_t>(side ? g->offV : g->offU);
  const uint32_t *nbrS = ptr<uint32_t>(side ? g->nbrV : g->nbrU);
  const uint32_t *eidS = side ? ptr<uint32_t>(g->eidV) : nullptr;
  p.offM = ptr<uint64_t>(side ? g->offU : g->offV);
  const uint64_t mm = std::max<uint64_t>(m, 1);

  BFC_TRY(dalloc(p.vert_of, (uint64_t)nS * 4, s));
  BFC_TRY(dalloc(p.rank_of, (uint64_t)nS * 4, s));
  BFC_TRY(dalloc(p.offR, ((uint64_t)nS + 1) * 8, s));
  BFC_TRY(dalloc(p.sX, mm * 4, s));
  BFC_TRY(dalloc(p.sEid, mm * 4, s));
  BFC_TRY(dalloc(p.sB, mm * 4, s));
  BFC_TRY(dalloc(p.mR, mm * 4, s));
  BFC_TRY(dalloc(p.mEid, mm * 4, s));
  BFC_TRY(dalloc(p.work, (uint64_t)nS * 8, s));

  DBuf k1, k2, i1, dR, sRank, perm;
  int rc = BFC_OK;
  auto cleanup = [&]() { dfree(k1, s); dfree(k2, s); dfree(i1, s); dfree(dR, s); dfree(sRank, s); dfree(perm, s); };
#define PB_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
  const uint64_t big = std::max<uint64_t>(mm, nS);
  PB_TRY(dalloc(k1, big * 4, s));
  PB_TRY(dalloc(k2, big * 4, s));
  PB_TRY(dalloc(i1, big * 4, s));
  PB_TRY(dalloc(dR, (uint64_t)nS * 4, s));
  // ranks: stable sort of ids by degree (ids start ascending, so ties stay by id)
  k_iota_and_copy<<<grid_for(nS, 256), 256, 0, s>>>(degS, nS, ptr<uint32_t>(k1), ptr<uint32_t>(i1));
  count_launch();
  PB_TRY(radix_sort_u32(ptr<uint32_t>(k1), ptr<uint32_t>(k2), ptr<uint32_t>(i1), ptr<uint32_t>(p.vert_of), nS,
                        bits_for(p.max_deg_S), g->scr, s));
  if (side == 0 && g->rank_group && nS > 0) {
    // grouped ranks: a second stable sort by group gives the order (group,
    // degree, id), so every group's start vertices hold consecutive ranks
    k_group_keys<<<grid_for(nS, 256), 256, 0, s>>>(ptr<uint32_t>(p.vert_of), g->rank_group, nS, ptr<uint32_t>(k1),
                                                   ptr<uint32_t>(i1));
    count_launch();
    PB_TRY(radix_sort_u32(ptr<uint32_t>(k1), ptr<uint32_t>(k2), ptr<uint32_t>(i1), ptr<uint32_t>(p.vert_of), nS,
                          std::max(1, bits_for(g->rank_group_max)), g->scr, s));
  }
  k_rank_of<<<grid_for(nS, 256), 256, 0, s>>>(ptr<uint32_t>(p.vert_of), degS, nS, ptr<uint32_t>(p.rank_of),
                                              ptr<uint32_t>(dR));
  count_launch();
  PB_TRY(exclusive_scan_u32_to_u64(ptr<uint32_t>(dR), ptr<uint64_t>(p.offR), nS, g->scr, s));
  PB_TRY(dalloc(sRank, mm * 4, s));
  if (m > 0) {
    k_fill_start_rows<<<grid_for((uint64_t)nS * 32, 256), 256, 0, s>>>(
        ptr<uint32_t>(p.vert_of), nS, offS, nbrS, eidS, ptr<uint64_t>(p.offR), ptr<uint32_t>(p.sX),
        ptr<uint32_t>(p.sEid), ptr<uint32_t>(sRank));
    count_launch();
    // midpoint rows: stable sort of start entries (rank order) by midpoint
    PB_TRY(dalloc(perm, mm * 4, s));
    k_iota_and_copy<<<grid_for(m, 256), 256, 0, s>>>(ptr<uint32_t>(p.sX), (uint32_t)m, ptr<uint32_t>(k1),
                                                    ptr<uint32_t>(i1));
    count_launch();
    PB_TRY(radix_sort_u32(ptr<uint32_t>(k1), ptr<uint32_t>(k2), ptr<uint32_t>(i1), ptr<uint32_t>(perm), m,
                          std::max(1, bits_for(nM - 1)), g->scr, s));
    k_fill_mid_rows<<<grid_for(m, 256), 256, 0, s>>>(ptr<uint32_t>(perm), m, ptr<uint32_t>(sRank),
                                                    ptr<uint32_t>(p.sEid), ptr<uint32_t>(p.mR), ptr<uint32_t>(p.mEid),
                                                    ptr<uint32_t>(p.sB));
    count_launch();
  }
  k_work<<<grid_for((uint64_t)nS * 32, 256), 256, 0, s>>>(ptr<uint64_t>(p.offR), nS, ptr<uint32_t>(p.sX),
                                                         ptr<uint32_t>(p.sB), p.offM, ptr<uint64_t>(p.work));
  count_launch();
  BFC_CUDA_TRY(cudaMemsetAsync(g->acc.p, 0, 8, s));
  PB_TRY(reduce_add_u64(ptr<uint64_t>(p.work), nS, ptr<unsigned long long>(g->acc), s));
  unsigned long long tw = 0;
  BFC_CUDA_TRY(cudaMemcpyAsync(&tw, g->acc.p, 8, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  p.total_work = tw;
  cleanup();
#undef PB_TRY
  BFC_TRY(plan_classify(g, p, s));
  p.built = true;
  return BFC_OK;
}

}  // namespace bfc
