// Exact counts of many independent graphs in one pass.
//
// A butterfly never spans two connected components, so the count of a
// disjoint union is the sum of its parts, and every start vertex's pair sum
// (Lemma 1, Eq. (3)) belongs to exactly one graph.  The batch is laid out as
// one union graph in which each graph is oriented so that the side Algorithm 1
// would start from (L unless sum_L d^2 < sum_R d^2, computed per graph) is on
// the union's U side; one rank layout and one set of persistent class launches
// then count every graph, each start vertex adding its sum to its graph's slot.
#include <algorithm>
#include <vector>

#include "bfc_internal.cuh"

namespace bfc {
namespace {

unsigned bt_grid(uint64_t n, unsigned threads, unsigned cap = 152 * 16) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

// last index g with off[g] <= x (off ascending, off[0] = 0)
__device__ __forceinline__ uint32_t seg_of(const uint64_t *off, uint32_t G, uint64_t x) {
  uint32_t lo = 0, hi = G - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) / 2;
    if (off[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// per edge: validate ids against its graph's sizes and count degrees in the
// (unoriented) union numbering
__global__ void k_bt_degrees(const uint32_t *u, const uint32_t *v, uint64_t m, const uint64_t *eoff, uint32_t G,
                             const uint32_t *nU, const uint32_t *nV, const uint64_t *uoff, const uint64_t *voff,
                             uint32_t *dU, uint32_t *dV, uint32_t *err) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = seg_of(eoff, G, e);
    const uint32_t a = u[e], x = v[e];
    if (a >= nU[g] || x >= nV[g]) { atomicOr(err, DERR_RANGE); continue; }
    atomicAdd(&dU[uoff[g] + a], 1u);
    atomicAdd(&dV[voff[g] + x], 1u);
  }
}
// per vertex: sum of squared degrees of its graph's side
__global__ void k_bt_squares(const uint32_t *d, uint64_t n, const uint64_t *off, uint32_t G,
                             unsigned long long *sq) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t di = d[i];
    if (di) atomicAdd(&sq[seg_of(off, G, i)], (unsigned long long)(di * di));
  }
}
// per edge: oriented union ids (the start side of every graph on U)
__global__ void k_bt_orient(const uint32_t *u, const uint32_t *v, uint64_t m, const uint64_t *eoff, uint32_t G,
                            const uint8_t *flip, const uint64_t *uoff2, const uint64_t *voff2, uint32_t *uu,
                            uint32_t *vv) {
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t g = seg_of(eoff, G, e);
    const uint32_t a = u[e], x = v[e];
    uu[e] = (uint32_t)(uoff2[g] + (flip[g] ? x : a));
    vv[e] = (uint32_t)(voff2[g] + (flip[g] ? a : x));
  }
}
// graph of every union U vertex (its graph's start side is the range uoff2[g] .. uoff2[g+1])
__global__ void k_bt_group_of_vertex(uint32_t n, const uint64_t *uoff2, uint32_t G, uint32_t *grp) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    grp[i] = seg_of(uoff2, G, i);
}
__global__ void k_bt_group_of_rank(const uint32_t *vert_of, uint32_t nS, const uint64_t *uoff2, uint32_t G,
                                   uint32_t *grp) {
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nS; r += (uint64_t)gridDim.x * blockDim.x)
    grp[r] = seg_of(uoff2, G, vert_of[r]);
}

}  // namespace
}  // namespace bfc

using namespace bfc;

extern "C" int bfc_exact_batch(const uint32_t *u, const uint32_t *v, const uint64_t *edge_off, const uint32_t *nU,
                               const uint32_t *nV, uint32_t G, uint32_t flags, uint64_t *B_out, int *side_out,
                               void *stream) {
  if (G == 0 || !edge_off || !nU || !nV || !B_out || (flags & ~BFC_INPUT_DEVICE)) return BFC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // host-side layout of the union
  std::vector<uint64_t> uoff(G + 1, 0), voff(G + 1, 0), eoff(edge_off, edge_off + G + 1);
  for (uint32_t g = 0; g < G; g++) {
    if (nU[g] == 0 || nV[g] == 0 || eoff[g + 1] < eoff[g]) return BFC_EINVAL;
    uoff[g + 1] = uoff[g] + nU[g];
    voff[g + 1] = voff[g] + nV[g];
  }
  const uint64_t m = eoff[G], NU = uoff[G], NV = voff[G];
  if (eoff[0] != 0 || m >= (1ull << 32) || NU + NV >= (1ull << 32)) return BFC_ERANGE;
  if (m > 0 && (!u || !v)) return BFC_EINVAL;

  bfc_graph *ug = nullptr;
  DBuf du, dv, meta, dU, dV, sq, uu, vv, grp, gB;
  int rc = BFC_OK;
  auto cleanup = [&]() {
    DBuf *bs[] = {&du, &dv, &meta, &dU, &dV, &sq, &uu, &vv, &grp, &gB};
    for (DBuf *b : bs) dfree(*b, s);
    if (ug) bfc_graph_free(ug);
  };
#define BT_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
#define BT_CUDA(x) do { if ((x) != cudaSuccess) { cleanup(); return BFC_ECUDA; } } while (0)
  const uint64_t mm = std::max<uint64_t>(m, 1);
  const uint32_t *pu = u, *pv = v;
  if (!(flags & BFC_INPUT_DEVICE) && m > 0) {
    BT_TRY(dalloc(du, m * 4, s));
    BT_TRY(dalloc(dv, m * 4, s));
    BT_CUDA(cudaMemcpyAsync(du.p, u, m * 4, cudaMemcpyHostToDevice, s));
    BT_CUDA(cudaMemcpyAsync(dv.p, v, m * 4, cudaMemcpyHostToDevice, s));
    pu = ptr<uint32_t>(du);
    pv = ptr<uint32_t>(dv);
  }
  // metadata on the device: eoff, uoff, voff, uoff2, voff2 (G+1 u64 each),
  // nU, nV (G u32 each), flip (G u8), error word
  const uint64_t G1 = G + 1;
  BT_TRY(dalloc(meta, G1 * 8 * 5 + (uint64_t)G * 9 + 64, s));
  uint64_t *d_eoff = ptr<uint64_t>(meta), *d_uoff = d_eoff + G1, *d_voff = d_uoff + G1, *d_uoff2 = d_voff + G1,
           *d_voff2 = d_uoff2 + G1;
  uint32_t *d_nU = reinterpret_cast<uint32_t *>(d_voff2 + G1), *d_nV = d_nU + G;
  uint32_t *d_err = d_nV + G;
  uint8_t *d_flip = reinterpret_cast<uint8_t *>(d_err + 4);
  BT_CUDA(cudaMemcpyAsync(d_eoff, eoff.data(), G1 * 8, cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaMemcpyAsync(d_uoff, uoff.data(), G1 * 8, cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaMemcpyAsync(d_voff, voff.data(), G1 * 8, cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaMemcpyAsync(d_nU, nU, (uint64_t)G * 4, cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaMemcpyAsync(d_nV, nV, (uint64_t)G * 4, cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaMemsetAsync(d_err, 0, 16, s));
  // per-graph sums of squared degrees -> the start side of each graph
  BT_TRY(dalloc(dU, std::max<uint64_t>(NU, 1) * 4, s));
  BT_TRY(dalloc(dV, std::max<uint64_t>(NV, 1) * 4, s));
  BT_TRY(dalloc(sq, (uint64_t)G * 16, s));
  BT_CUDA(cudaMemsetAsync(dU.p, 0, NU * 4, s));
  BT_CUDA(cudaMemsetAsync(dV.p, 0, NV * 4, s));
  BT_CUDA(cudaMemsetAsync(sq.p, 0, (uint64_t)G * 16, s));
  if (m > 0) {
    k_bt_degrees<<<bt_grid(m, 256), 256, 0, s>>>(pu, pv, m, d_eoff, G, d_nU, d_nV, d_uoff, d_voff, ptr<uint32_t>(dU),
                                                ptr<uint32_t>(dV), d_err);
    count_launch();
  }
  unsigned long long *sqU = ptr<unsigned long long>(sq), *sqV = sqU + G;
  k_bt_squares<<<bt_grid(NU, 256), 256, 0, s>>>(ptr<uint32_t>(dU), NU, d_uoff, G, sqU);
  count_launch();
  k_bt_squares<<<bt_grid(NV, 256), 256, 0, s>>>(ptr<uint32_t>(dV), NV, d_voff, G, sqV);
  count_launch();
  std::vector<unsigned long long> hsq(2 * (size_t)G);
  uint32_t herr = 0;
  BT_CUDA(cudaMemcpyAsync(hsq.data(), sq.p, (uint64_t)G * 16, cudaMemcpyDeviceToHost, s));
  BT_CUDA(cudaMemcpyAsync(&herr, d_err, 4, cudaMemcpyDeviceToHost, s));
  BT_CUDA(cudaStreamSynchronize(s));
  if (herr) { cleanup(); return BFC_ERANGE; }
  std::vector<uint8_t> flip(G);
  std::vector<uint64_t> uoff2(G + 1, 0), voff2(G + 1, 0);
  for (uint32_t g = 0; g < G; g++) {
    flip[g] = hsq[g] < hsq[G + g] ? 1 : 0;  // Algorithm 1: start from R when sum_L d^2 < sum_R d^2
    uoff2[g + 1] = uoff2[g] + (flip[g] ? nV[g] : nU[g]);
    voff2[g + 1] = voff2[g] + (flip[g] ? nU[g] : nV[g]);
    if (side_out) side_out[g] = flip[g];
  }
  BT_CUDA(cudaMemcpyAsync(d_uoff2, uoff2.data(), G1 * 8, cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaMemcpyAsync(d_voff2, voff2.data(), G1 * 8, cudaMemcpyHostToDevice, s));
  BT_CUDA(cudaMemcpyAsync(d_flip, flip.data(), G, cudaMemcpyHostToDevice, s));
  // the oriented union
  BT_TRY(dalloc(uu, mm * 4, s));
  BT_TRY(dalloc(vv, mm * 4, s));
  if (m > 0) {
    k_bt_orient<<<bt_grid(m, 256), 256, 0, s>>>(pu, pv, m, d_eoff, G, d_flip, d_uoff2, d_voff2, ptr<uint32_t>(uu),
                                               ptr<uint32_t>(vv));
    count_launch();
  }
  BT_TRY(bfc_graph_from_edges(ptr<uint32_t>(uu), ptr<uint32_t>(vv), m, (uint32_t)uoff2[G], (uint32_t)voff2[G],
                              BFC_INPUT_DEVICE, stream, &ug));
  dfree(uu, s);
  dfree(vv, s);
  // rank the union's start vertices graph by graph (then by degree, id), so
  // that a start vertex's later-ranked targets, all in its own graph, lie in
  // one short rank range instead of being spread over the whole union
  const uint32_t NS2 = (uint32_t)uoff2[G];
  BT_TRY(dalloc(grp, (uint64_t)std::max<uint32_t>(NS2, 1) * 4, s));
  k_bt_group_of_vertex<<<bt_grid(NS2, 256), 256, 0, s>>>(NS2, d_uoff2, G, ptr<uint32_t>(grp));
  count_launch();
  ug->rank_group = ptr<uint32_t>(grp);
  ug->rank_group_max = G - 1;
  BT_TRY(plan_build(ug, 0, s));
  ug->rank_group = nullptr;
  Plan &p = ug->plan[0];
  BT_TRY(dalloc(gB, (uint64_t)G * 8, s));
  BT_CUDA(cudaMemsetAsync(gB.p, 0, (uint64_t)G * 8, s));
  k_bt_group_of_rank<<<bt_grid(p.nS, 256), 256, 0, s>>>(ptr<uint32_t>(p.vert_of), p.nS, d_uoff2, G,
                                                       ptr<uint32_t>(grp));
  count_launch();
  BT_CUDA(cudaMemsetAsync(ug->acc.p, 0, 8, s));
  BT_TRY(wedge_count_groups(ug, p, ptr<uint32_t>(grp), ptr<unsigned long long>(gB), ptr<unsigned long long>(ug->acc),
                            s));
  BT_CUDA(cudaMemcpyAsync(B_out, gB.p, (uint64_t)G * 8, cudaMemcpyDeviceToHost, s));
  BT_TRY(read_device_error(ug, s));
  cleanup();
#undef BT_TRY
#undef BT_CUDA
  return BFC_OK;
}
