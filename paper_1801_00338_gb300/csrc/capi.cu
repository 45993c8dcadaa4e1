// C ABI entry points (declared in include/bfc.h).
#include <algorithm>
#include <cmath>
#include <vector>
#include <new>

#include "bfc_internal.cuh"

using namespace bfc;

namespace {

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// device accumulator layout inside g->acc (256 bytes):
//   [0, 8)   B
//   [64, 72) work queues (2 x u32)
unsigned long long *acc_B(bfc_graph *g) { return ptr<unsigned long long>(g->acc); }

__global__ void k_rows_to_ids(const uint64_t *off, uint32_t n, uint32_t *out) {
  const int lane = threadIdx.x & 31;
  uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t r = warp; r < n; r += nw)
    for (uint64_t e = off[r] + lane; e < off[r + 1]; e += 32) out[e] = (uint32_t)r;
}

int finish_count(bfc_graph *g, uint64_t *out_B, cudaStream_t s) {
  unsigned long long hB = 0;
  if (out_B) BFC_CUDA_TRY(cudaMemcpyAsync(&hB, acc_B(g), 8, cudaMemcpyDeviceToHost, s));
  BFC_TRY(read_device_error(g, s));  // synchronises s
  if (out_B) *out_B = hB;
  return BFC_OK;
}

int prepare(bfc_graph *g, uint32_t flags, cudaStream_t s, int *side) {
  if (!g) return BFC_EINVAL;
  if ((flags & BFC_SIDE_U) && (flags & BFC_SIDE_V)) return BFC_EINVAL;
  if (flags & ~(BFC_SIDE_U | BFC_SIDE_V | BFC_WHOLE_ROWS)) return BFC_EINVAL;
  *side = choose_side(g, flags);
  BFC_TRY(plan_build(g, *side, s));
  g->last_stream = s;
  BFC_CUDA_TRY(cudaMemsetAsync(acc_B(g), 0, 8, s));
  return BFC_OK;
}

}  // namespace

extern "C" {

int bfc_graph_from_edges(const uint32_t *u, const uint32_t *v, uint64_t m, uint32_t nU, uint32_t nV, uint32_t flags,
                         void *stream, bfc_graph **out) {
  if (!out || nU == 0 || nV == 0) return BFC_EINVAL;
  if (m > 0 && (!u || !v)) return BFC_EINVAL;
  if (flags & ~(BFC_INPUT_DEVICE | BFC_DEDUP)) return BFC_EINVAL;
  if (m >= (1ull << 32)) return BFC_ERANGE;
  *out = nullptr;
  bfc_graph *g = new (std::nothrow) bfc_graph();
  if (!g) return BFC_ENOMEM;
  g->nU = nU;
  g->nV = nV;
  cudaStream_t s = as_stream(stream);
  g->last_stream = s;
  int rc = graph_build(g, u, v, m, flags, s);
  if (rc != BFC_OK) {
    bfc_graph_free(g);
    return rc;
  }
  *out = g;
  return BFC_OK;
}

int bfc_graph_from_csr(const uint64_t *offU, const uint32_t *nbrU, uint32_t nU, const uint64_t *offV,
                       const uint32_t *nbrV, const uint32_t *eidV, uint32_t nV, void *stream, bfc_graph **out) {
  if (!out || !offU || !nbrU || !offV || !nbrV || nU == 0 || nV == 0) return BFC_EINVAL;
  *out = nullptr;
  bfc_graph *g = new (std::nothrow) bfc_graph();
  if (!g) return BFC_ENOMEM;
  g->nU = nU;
  g->nV = nV;
  cudaStream_t s = as_stream(stream);
  g->last_stream = s;
  int rc = graph_from_rows(g, offU, nbrU, offV, nbrV, eidV, s);
  if (rc != BFC_OK) {
    bfc_graph_free(g);
    return rc;
  }
  *out = g;
  return BFC_OK;
}

int bfc_graph_free(bfc_graph *g) {
  if (!g) return BFC_EINVAL;
  cudaStream_t s = g->last_stream;
  cudaStreamSynchronize(s);
  for (int side = 0; side < 2; side++) {
    Plan &p = g->plan[side];
    DBuf *bufs[] = {&p.vert_of, &p.rank_of, &p.offR, &p.sX, &p.sEid, &p.sB, &p.mR, &p.mEid, &p.work, &p.cls};
    for (DBuf *b : bufs) dfree(*b, s);
  }
  DBuf *gb[] = {&g->offU, &g->nbrU, &g->offV, &g->nbrV, &g->eidV, &g->degU, &g->degV, &g->err, &g->acc, &g->scr.buf,
                &g->beM};
  for (DBuf *b : gb) dfree(*b, s);
  cudaStreamSynchronize(s);
  delete g;
  return BFC_OK;
}

int bfc_graph_stats(const bfc_graph *g, uint64_t *m, uint64_t *sq_u, uint64_t *sq_v, uint64_t *wedges_u,
                    uint64_t *wedges_v) {
  if (!g) return BFC_EINVAL;
  if (m) *m = g->m;
  if (sq_u) *sq_u = g->sqU;
  if (sq_v) *sq_v = g->sqV;
  if (wedges_u) *wedges_u = g->wU;
  if (wedges_v) *wedges_v = g->wV;
  return BFC_OK;
}

int bfc_graph_edges(const bfc_graph *g, uint32_t *u_out, uint32_t *v_out, void *stream) {
  if (!g) return BFC_EINVAL;
  cudaStream_t s = as_stream(stream);
  if (g->m == 0) return BFC_OK;
  if (u_out) {
    unsigned grid = (unsigned)std::min<uint64_t>(((uint64_t)g->nU * 32 + 255) / 256, 152 * 16);
    k_rows_to_ids<<<grid ? grid : 1, 256, 0, s>>>(ptr<uint64_t>(g->offU), g->nU, u_out);
    BFC_LAUNCHED();
  }
  if (v_out) BFC_CUDA_TRY(cudaMemcpyAsync(v_out, g->nbrU.p, g->m * 4, cudaMemcpyDeviceToDevice, s));
  return BFC_OK;
}

int bfc_exact_hub(bfc_graph *g, uint32_t flags, uint32_t hubs, uint32_t tau, uint64_t *out_B, int *out_side,
                  uint64_t *out_stats, void *stream) {
  if (!out_B || tau == 1) return BFC_EINVAL;
  cudaStream_t s = as_stream(stream);
  int side = 0;
  BFC_TRY(prepare(g, flags & ~BFC_HUB_MMA, s, &side));
  Plan &p = g->plan[side];
  uint32_t h = hubs;
  if (h == 0) BFC_TRY(hub_auto_size(p, BFC_HUB_MAX, &h, s));
  if (h % 128 || h > p.nS) return BFC_EINVAL;
  if (h) {
    BFC_TRY(hub_block_count(g, p, h, tau, acc_B(g), out_stats, s));
  } else if (out_stats) {
    for (int i = 0; i < 4; i++) out_stats[i] = 0;
  }
  BFC_TRY(wedge_count_below(g, p, p.nS - h, acc_B(g), s));
  BFC_TRY(finish_count(g, out_B, s));
  if (out_side) *out_side = side;
  return BFC_OK;
}

int bfc_exact(bfc_graph *g, uint32_t flags, uint64_t *out_B, int *out_side, void *stream) {
  if (!out_B) return BFC_EINVAL;
  if (g && (flags & BFC_HUB_MMA) && g->tune.hubs != BFC_TUNE_NO_HUBS) {
    // a tuned hub count is capped at the start side's size (whole tiles)
    const uint32_t nS = choose_side(g, flags) ? g->nV : g->nU;
    const uint32_t h = std::min<uint32_t>(g->tune.hubs, nS / 128 * 128);
    if (g->tune.hubs == 0 || h > 0)
      return bfc_exact_hub(g, flags, h, g->tune.tau, out_B, out_side, nullptr, stream);
  }
  flags &= ~BFC_HUB_MMA;
  cudaStream_t s = as_stream(stream);
  int side = 0;
  BFC_TRY(prepare(g, flags, s, &side));
  BFC_TRY(wedge_count(g, g->plan[side], MODE_TOTAL, acc_B(g), nullptr, s));
  BFC_TRY(finish_count(g, out_B, s));
  if (out_side) *out_side = side;
  return BFC_OK;
}

// The whole-row sweep (BFC_WHOLE_ROWS).
static int whole_rows(bfc_graph *g, uint32_t flags, uint64_t *bU, uint64_t *bV, uint64_t *be, uint64_t *out_B,
                      cudaStream_t s) {
  int side = 0;
  BFC_TRY(prepare(g, flags, s, &side));
  uint64_t *bS = side ? bV : bU;
  uint64_t *bM = side ? bU : bV;
  DBuf tmp;
  uint64_t *pe = be;
  if (bM && !be) {
    BFC_TRY(dalloc(tmp, std::max<uint64_t>(g->m, 1) * 8, s));
    pe = ptr<uint64_t>(tmp);
  }
  int rc = wedge_local(g, g->plan[side], acc_B(g), bS, bM, pe, s);
  uint64_t twoB = 0;
  if (rc == BFC_OK) rc = finish_count(g, &twoB, s);
  dfree(tmp, s);
  if (rc != BFC_OK) return rc;
  if (twoB & 1) return BFC_EINTERNAL;  // Eq. (1): the start side counts every butterfly twice
  if (out_B) *out_B = twoB / 2;
  return BFC_OK;
}

// The ordered one-sided sweep (each pair once, Algorithm 1's order) in EDGE
// mode: b_e for every edge (both edges of every counted wedge pair are
// credited), then b_x = 1/2 sum_{e containing x} b_e on both sides.
static int ordered_local(bfc_graph *g, uint32_t flags, uint64_t *bU, uint64_t *bV, uint64_t *be, uint64_t *out_B,
                         cudaStream_t s) {
  int side = 0;
  BFC_TRY(prepare(g, flags, s, &side));
  DBuf tmpE;
  uint64_t *pe = be;
  if (!pe && g->m > 0) {
    BFC_TRY(dalloc(tmpE, g->m * 8, s));
    pe = ptr<uint64_t>(tmpE);
  }
  int rc = BFC_OK;
  if (g->m > 0 && cudaMemsetAsync(pe, 0, g->m * 8, s) != cudaSuccess) rc = BFC_ECUDA;
  if (!rc) rc = wedge_count(g, g->plan[side], MODE_EDGE, acc_B(g), pe, s);
  if (!rc && bU) rc = vertex_from_edges(ptr<uint64_t>(g->offU), g->nU, nullptr, pe, bU, s);
  if (!rc && bV) rc = vertex_from_edges(ptr<uint64_t>(g->offV), g->nV, ptr<uint32_t>(g->eidV), pe, bV, s);
  if (!rc) rc = finish_count(g, out_B, s);
  dfree(tmpE, s);
  return rc;
}

// the sweep of the local counts: BFC_WHOLE_ROWS, or the graph's tuned default
static uint32_t local_flags(const bfc_graph *g, uint32_t flags) {
  return (g->tune.local_sweep == 1) ? (flags | BFC_WHOLE_ROWS) : flags;
}

int bfc_set_tuning(bfc_graph *g, const bfc_tuning *t) {
  if (!g) return BFC_EINVAL;
  if (!t) {
    g->tune = bfc_tuning{};
    return BFC_OK;
  }
  if (t->warp_max_wedges > 512 || t->small_max_segs > 128 || t->tau == 1 || t->local_sweep > 1) return BFC_EINVAL;
  if (t->hubs != 0 && t->hubs != BFC_TUNE_NO_HUBS && (t->hubs % 128 || t->hubs > BFC_HUB_MAX)) return BFC_EINVAL;
  g->tune = *t;
  return BFC_OK;
}

int bfc_get_tuning(const bfc_graph *g, bfc_tuning *t) {
  if (!g || !t) return BFC_EINVAL;
  *t = g->tune;
  if (!t->warp_max_wedges) t->warp_max_wedges = 512;
  if (!t->small_max_segs) t->small_max_segs = 128;
  if (!t->flat_max_avg) t->flat_max_avg = 64;
  return BFC_OK;
}

int bfc_local_counts(bfc_graph *g, uint32_t flags, uint64_t *bU, uint64_t *bV, uint64_t *be, uint64_t *out_B,
                     void *stream) {
  if (!g) return BFC_EINVAL;
  cudaStream_t s = as_stream(stream);
  flags = local_flags(g, flags);
  if (flags & BFC_WHOLE_ROWS) return whole_rows(g, flags, bU, bV, be, out_B, s);
  return ordered_local(g, flags, bU, bV, be, out_B, s);
}

int bfc_per_vertex(bfc_graph *g, uint32_t flags, uint64_t *bU, uint64_t *bV, uint64_t *out_B, void *stream) {
  if (!g) return BFC_EINVAL;
  cudaStream_t s = as_stream(stream);
  flags = local_flags(g, flags);
  if (!(flags & BFC_WHOLE_ROWS)) return ordered_local(g, flags, bU, bV, nullptr, out_B, s);
  DBuf tU, tV;
  uint64_t *pU = bU, *pV = bV;
  if (!pU) { BFC_TRY(dalloc(tU, (uint64_t)g->nU * 8, s)); pU = ptr<uint64_t>(tU); }
  if (!pV) { BFC_TRY(dalloc(tV, (uint64_t)g->nV * 8, s)); pV = ptr<uint64_t>(tV); }
  int rc = whole_rows(g, flags, pU, pV, nullptr, out_B, s);
  dfree(tU, s);
  dfree(tV, s);
  return rc;
}

int bfc_per_edge(bfc_graph *g, uint32_t flags, uint64_t *be, uint64_t *out_B, void *stream) {
  if (!g || (!be && g->m > 0)) return BFC_EINVAL;
  cudaStream_t s = as_stream(stream);
  flags = local_flags(g, flags);
  if (flags & BFC_WHOLE_ROWS) return whole_rows(g, flags, nullptr, nullptr, be, out_B, s);
  return ordered_local(g, flags, nullptr, nullptr, be, out_B, s);
}

int bfc_plan_stats(bfc_graph *g, int side, uint64_t *out, void *stream) {
  if (!g || !out || (side != 0 && side != 1)) return BFC_EINVAL;
  cudaStream_t s = as_stream(stream);
  BFC_TRY(plan_build(g, side, s));
  const Plan &p = g->plan[side];
  out[0] = p.nS;
  for (int c = 0; c < Plan::NCLS; c++) {
    out[1 + c] = p.cls_count[c];
    out[1 + Plan::NCLS + c] = p.cls_work[c];
    out[1 + 2 * Plan::NCLS + c] = p.cls_rows[c];
  }
  out[1 + 3 * Plan::NCLS] = p.total_work;
  return BFC_OK;
}

int bfc_median_of_means(const double *y, uint64_t n, uint32_t groups, double *out) {
  if (!y || !out || groups == 0 || n == 0 || n % groups) return BFC_EINVAL;
  const uint64_t per = n / groups;
  std::vector<double> mean(groups);
  for (uint32_t gi = 0; gi < groups; gi++) {
    double sum = 0.0;
    for (uint64_t i = 0; i < per; i++) sum += y[(uint64_t)gi * per + i];
    mean[gi] = sum / (double)per;
  }
  std::sort(mean.begin(), mean.end());
  *out = (groups & 1) ? mean[groups / 2] : 0.5 * (mean[groups / 2 - 1] + mean[groups / 2]);
  return BFC_OK;
}

int bfc_mom_sizes(double var1, double B, double epsilon, double delta, uint64_t *alpha, uint32_t *groups) {
  if (!alpha || !groups || !(var1 >= 0.0) || !(B > 0.0) || !(epsilon > 0.0) || !(delta > 0.0 && delta < 1.0))
    return BFC_EINVAL;
  const double a = std::ceil(32.0 * var1 / (epsilon * epsilon * B * B));
  if (!(a < 9.2e18)) return BFC_ERANGE;
  const double margin = 0.5 - 1.0 / 32.0;
  uint32_t g = (uint32_t)std::ceil(std::log(1.0 / delta) / (2.0 * margin * margin));
  if (g == 0) g = 1;
  if (!(g & 1)) g++;
  *alpha = a < 1.0 ? 1 : (uint64_t)a;
  *groups = g;
  return BFC_OK;
}

const char *bfc_strerror(int code) {
  switch (code) {
    case BFC_OK: return "ok";
    case BFC_EINVAL: return "invalid argument";
    case BFC_ERANGE: return "vertex id or size out of range";
    case BFC_EDUP: return "duplicate edge";
    case BFC_ENOMEM: return "out of memory";
    case BFC_ECUDA: return "CUDA runtime error";
    case BFC_ETIMEOUT: return "device wait timed out";
    case BFC_EOVERFLOW: return "integer overflow";
    case BFC_EINTERNAL: return "internal consistency check failed";
  }
  return "unknown error";
}

}  // extern "C"
