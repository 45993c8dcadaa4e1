// Sparsification estimators (Section 6) and the sampled-subgraph plumbing.
//
// ESpar (Algorithm 8): keep every edge independently with probability p,
// count the kept subgraph exactly, scale by p^-4.
// ClrSpar (Algorithm 9): colour every vertex uniformly from N colours, keep
// the monochromatic edges, count exactly, scale by N^3.
//
// Random draws: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), counter based:
// output k >= 1 of the sequence seeded by s is mix(s + k * 0x9E3779B97F4A7C15);
// trial t uses the sequence seeded by output t + 1 of the caller's seed.
//
// The kept subgraph is counted with Algorithm 1 using the full graph's start
// side and rank order: B of any graph does not depend on either (Lemma 1 and
// Eq. (4)), only the cost does.  The subgraph layout is obtained by filtering
// the full graph's layout (prefix sums + compaction), so no sort runs per trial,
// and every step of a trial stays on the device: one trial is recorded into a
// CUDA graph and the graph is replayed for the others.
#include <algorithm>
#include <vector>

#include "bfc_internal.cuh"

namespace bfc {

__device__ __forceinline__ uint64_t sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t sm64(uint64_t s, uint64_t k) { return sm64_mix(s + k * 0x9E3779B97F4A7C15ull); }

static unsigned grid_for(uint64_t n, unsigned threads, unsigned cap = 152 * 16) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

// ---------------------------------------------------------------------------
// keep predicates (over canonical edge ids); the trial index is read from the
// device so that one recorded trial can be replayed for every trial
// ---------------------------------------------------------------------------
__global__ void k_keep_espar(uint64_t m, uint64_t seed, const uint32_t *trial, uint32_t T, uint32_t *keep) {
  const uint64_t ts = sm64(seed, (uint64_t)*trial + 1);
  for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (uint64_t)gridDim.x * blockDim.x)
    keep[e] = ((uint32_t)(sm64(ts, e + 1) >> 32) < T) ? 1u : 0u;
}

__device__ __forceinline__ uint32_t colour_of(uint64_t ts, uint64_t k, uint32_t N) {
  return (uint32_t)(((sm64(ts, k) >> 32) * (uint64_t)N) >> 32);
}
// one warp per U row: the row's colour once, each neighbour's colour per edge
__global__ void k_keep_clrspar(const uint64_t *offU, const uint32_t *nbrU, uint32_t nU, uint64_t seed,
                               const uint32_t *trial, uint32_t N, uint32_t *keep) {
  const uint64_t ts = sm64(seed, (uint64_t)*trial + 1);
  const int lane = threadIdx.x & 31;
  uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t u = warp; u < nU; u += nw) {
    uint32_t cu = colour_of(ts, u + 1, N);
    for (uint64_t e = offU[u] + lane; e < offU[u + 1]; e += 32)
      keep[e] = (colour_of(ts, (uint64_t)nU + nbrU[e] + 1, N) == cu) ? 1u : 0u;
  }
}

// ---------------------------------------------------------------------------
// plan filtering
// ---------------------------------------------------------------------------
__global__ void k_gather_flags(const uint32_t *eid, uint64_t m, const uint32_t *keep, uint32_t *flag) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x)
    flag[i] = keep[eid[i]];
}
__global__ void k_remap_offsets(const uint64_t *off, uint64_t n1, const uint64_t *pos, uint64_t *out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1; i += (uint64_t)gridDim.x * blockDim.x)
    out[i] = pos[off[i]];
}
__global__ void k_compact_start(uint64_t m, const uint32_t *flagS, const uint64_t *posS, const uint64_t *posM,
                                const uint32_t *sX, const uint32_t *sEid, const uint32_t *sB, uint32_t *oX,
                                uint32_t *oEid, uint32_t *oB) {
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += (uint64_t)gridDim.x * blockDim.x) {
    if (!flagS[j]) continue;
    uint64_t d = posS[j];
    oX[d] = sX[j];
    oEid[d] = sEid[j];
    oB[d] = (uint32_t)(posM[sB[j] - 1] + 1);  // the edge itself is kept, so it keeps a slot in its mid row
  }
}
__global__ void k_compact_mid(uint64_t m, const uint32_t *flagM, const uint64_t *posM, const uint32_t *mR,
                              const uint32_t *mEid, uint32_t *oR, uint32_t *oEid) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (uint64_t)gridDim.x * blockDim.x) {
    if (!flagM[i]) continue;
    uint64_t d = posM[i];
    oR[d] = mR[i];
    oEid[d] = mEid[i];
  }
}
__global__ void k_work_f(const uint64_t *offR, uint32_t nS, const uint32_t *sX, const uint32_t *sB,
                         const uint64_t *offM, uint64_t *work) {
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
// beta of the trial: move the accumulator to its slot and advance the trial index
__global__ void k_trial_done(unsigned long long *acc, uint32_t *trial, unsigned long long *betas) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    betas[*trial] = *acc;
    *acc = 0;
    *trial += 1;
  }
}

void plan_free(Plan &p, cudaStream_t s) {
  DBuf *bufs[] = {&p.offR, &p.sX, &p.sEid, &p.sB, &p.mR, &p.mEid, &p.work, &p.cls, &p.offM_own};
  for (DBuf *b : bufs) dfree(*b, s);
  if (p.vert_of.bytes) dfree(p.vert_of, s);
  if (p.rank_of.bytes) dfree(p.rank_of, s);
  p.vert_of = DBuf{};
  p.rank_of = DBuf{};
  p.built = false;
}

// Buffers of a sparsification run, sized once from the parent layout so that
// every trial reuses them (nothing is allocated while trials run).
struct TrialPipe {
  Plan sub;
  DBuf keep, flags, pos, cls_of, dev, sums, acc, trial, betas;
  ~TrialPipe() {}
};

static void pipe_free(TrialPipe &tp, cudaStream_t s) {
  plan_free(tp.sub, s);
  DBuf *bs[] = {&tp.keep, &tp.flags, &tp.pos, &tp.cls_of, &tp.dev, &tp.sums, &tp.acc, &tp.trial, &tp.betas};
  for (DBuf *b : bs) dfree(*b, s);
}

static int pipe_init(bfc_graph *g, const Plan &parent, uint32_t trials, TrialPipe &tp, cudaStream_t s) {
  const uint64_t m = parent.m, mm = std::max<uint64_t>(m, 1);
  Plan &out = tp.sub;
  out.side = parent.side;
  out.nS = parent.nS;
  out.nM = parent.nM;
  out.m = m;
  out.max_deg_S = parent.max_deg_S;
  out.warp_max = parent.warp_max;
  out.small_max = parent.small_max;
  out.vert_of = DBuf{parent.vert_of.p, 0};  // borrowed: bytes = 0 marks "not owned"
  out.rank_of = DBuf{parent.rank_of.p, 0};
  BFC_TRY(dalloc(out.offR, ((uint64_t)out.nS + 1) * 8, s));
  BFC_TRY(dalloc(out.offM_own, ((uint64_t)out.nM + 1) * 8, s));
  out.offM = ptr<uint64_t>(out.offM_own);
  BFC_TRY(dalloc(out.sX, mm * 4, s));
  BFC_TRY(dalloc(out.sEid, mm * 4, s));
  BFC_TRY(dalloc(out.sB, mm * 4, s));
  BFC_TRY(dalloc(out.mR, mm * 4, s));
  BFC_TRY(dalloc(out.mEid, mm * 4, s));
  BFC_TRY(dalloc(out.work, (uint64_t)std::max<uint32_t>(out.nS, 1) * 8, s));
  BFC_TRY(dalloc(out.cls, (uint64_t)std::max<uint32_t>(out.nS, 1) * 4, s));
  BFC_TRY(dalloc(tp.keep, mm * 4, s));
  BFC_TRY(dalloc(tp.flags, mm * 4 * 2, s));
  BFC_TRY(dalloc(tp.pos, (mm + 1) * 8 * 2, s));
  BFC_TRY(dalloc(tp.cls_of, (uint64_t)std::max<uint32_t>(out.nS, 1) * 4, s));
  BFC_TRY(dalloc(tp.dev, 48 * 4, s));
  BFC_TRY(dalloc(tp.sums, (2 * Plan::NCLS + 1) * 8, s));
  BFC_TRY(dalloc(tp.acc, 8, s));
  BFC_TRY(dalloc(tp.trial, 8, s));
  BFC_TRY(dalloc(tp.betas, (uint64_t)trials * 8, s));
  BFC_CUDA_TRY(cudaMemsetAsync(tp.acc.p, 0, 8, s));
  BFC_CUDA_TRY(cudaMemsetAsync(tp.trial.p, 0, 8, s));
  // the scan partials and the big class's segment scratch are reserved before
  // any recording, at their largest sizes
  BFC_TRY(g->scr.reserve(((mm + 2047) / 2048 + 2) * 8, s));
  return BFC_OK;
}

// Enqueue the filtering and counting of one trial (the keep flags must be in
// tp.keep); no host round trip.
static int pipe_count(bfc_graph *g, const Plan &parent, TrialPipe &tp, cudaStream_t s) {
  const uint64_t m = parent.m, mm = std::max<uint64_t>(m, 1);
  Plan &out = tp.sub;
  uint32_t *flagS = ptr<uint32_t>(tp.flags), *flagM = flagS + mm;
  uint64_t *posS = ptr<uint64_t>(tp.pos), *posM = posS + mm + 1;
  if (m > 0) {
    k_gather_flags<<<grid_for(m, 256), 256, 0, s>>>(ptr<uint32_t>(parent.sEid), m, ptr<uint32_t>(tp.keep), flagS);
    count_launch();
    k_gather_flags<<<grid_for(m, 256), 256, 0, s>>>(ptr<uint32_t>(parent.mEid), m, ptr<uint32_t>(tp.keep), flagM);
    count_launch();
  }
  BFC_TRY(exclusive_scan_u32_to_u64(flagS, posS, m, g->scr, s));
  BFC_TRY(exclusive_scan_u32_to_u64(flagM, posM, m, g->scr, s));
  k_remap_offsets<<<grid_for((uint64_t)out.nS + 1, 256), 256, 0, s>>>(ptr<uint64_t>(parent.offR),
                                                                     (uint64_t)out.nS + 1, posS, ptr<uint64_t>(out.offR));
  count_launch();
  k_remap_offsets<<<grid_for((uint64_t)out.nM + 1, 256), 256, 0, s>>>(parent.offM, (uint64_t)out.nM + 1, posM,
                                                                     ptr<uint64_t>(out.offM_own));
  count_launch();
  if (m > 0) {
    k_compact_start<<<grid_for(m, 256), 256, 0, s>>>(m, flagS, posS, posM, ptr<uint32_t>(parent.sX),
                                                    ptr<uint32_t>(parent.sEid), ptr<uint32_t>(parent.sB),
                                                    ptr<uint32_t>(out.sX), ptr<uint32_t>(out.sEid),
                                                    ptr<uint32_t>(out.sB));
    count_launch();
    k_compact_mid<<<grid_for(m, 256), 256, 0, s>>>(m, flagM, posM, ptr<uint32_t>(parent.mR),
                                                  ptr<uint32_t>(parent.mEid), ptr<uint32_t>(out.mR),
                                                  ptr<uint32_t>(out.mEid));
    count_launch();
  }
  k_work_f<<<grid_for((uint64_t)out.nS * 32, 256), 256, 0, s>>>(ptr<uint64_t>(out.offR), out.nS,
                                                               ptr<uint32_t>(out.sX), ptr<uint32_t>(out.sB), out.offM,
                                                               ptr<uint64_t>(out.work));
  count_launch();
  BFC_TRY(plan_classify_device(out, ptr<uint32_t>(tp.cls_of), ptr<unsigned int>(tp.dev),
                               ptr<unsigned long long>(tp.sums), s));
  // trial-BIG vertices are parent-BIG vertices with fewer edges: the parent's
  // segment bound covers them
  BFC_TRY(wedge_count_device_lists(g, out, ptr<unsigned int>(tp.dev), parent.big_seg_cap,
                                   ptr<unsigned long long>(tp.acc), s));
  k_trial_done<<<1, 32, 0, s>>>(ptr<unsigned long long>(tp.acc), ptr<uint32_t>(tp.trial),
                                ptr<unsigned long long>(tp.betas));
  count_launch();
  BFC_CUDA_TRY(cudaGetLastError());
  return BFC_OK;
}

// Run all trials: one trial is enqueued once directly (warming every buffer
// and kernel attribute), then recorded into a CUDA graph and replayed for the
// remaining trials; if recording is not possible the trial is enqueued again
// each time.  The only host round trip is the final read of the betas.
template <class KeepFn>
static int sparsify_trials(bfc_graph *g, uint32_t trials, uint64_t *beta, cudaStream_t s, KeepFn enqueue_keep) {
  const int side = choose_side(g, 0);
  BFC_TRY(plan_build(g, side, s));
  Plan &parent = g->plan[side];
  TrialPipe tp;
  int rc = pipe_init(g, parent, trials, tp, s);
  auto one = [&]() -> int {
    int r = enqueue_keep(ptr<uint32_t>(tp.keep), ptr<uint32_t>(tp.trial));
    if (!r) r = pipe_count(g, parent, tp, s);
    return r;
  };
  if (!rc) rc = one();
  if (!rc && trials > 1) {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool recorded = false;
    if (s != nullptr && !profile_on() &&
        cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int r = one();
      const cudaError_t e = cudaStreamEndCapture(s, &graph);
      if (r == BFC_OK && e == cudaSuccess && graph &&
          cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
        recorded = true;
      cudaGetLastError();  // a failed recording leaves no sticky error
    }
    for (uint32_t t = 1; t < trials && !rc; t++) {
      if (recorded) rc = (cudaGraphLaunch(exec, s) == cudaSuccess) ? BFC_OK : BFC_ECUDA;
      else rc = one();
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
  if (!rc && cudaMemcpyAsync(beta, tp.betas.p, (uint64_t)trials * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = BFC_ECUDA;
  if (!rc) rc = read_device_error(g, s);
  pipe_free(tp, s);
  return rc;
}

}  // namespace bfc

using namespace bfc;

extern "C" {

int bfc_espar(bfc_graph *g, double p, uint32_t trials, uint64_t seed, double *est, uint64_t *beta, void *stream) {
  if (!g || trials == 0 || !(p > 0.0) || !(p < 1.0)) return BFC_EINVAL;
  const double Td = p * 4294967296.0;
  const uint32_t T = (uint32_t)Td;
  if (T == 0) return BFC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->last_stream = s;
  std::vector<uint64_t> b(trials);
  int rc = sparsify_trials(g, trials, b.data(), s, [&](uint32_t *keep, const uint32_t *trial) -> int {
    if (g->m == 0) return BFC_OK;
    k_keep_espar<<<grid_for(g->m, 256), 256, 0, s>>>(g->m, seed, trial, T, keep);
    BFC_LAUNCHED();
    return BFC_OK;
  });
  if (rc) return rc;
  const double inv_p = 4294967296.0 / (double)T;
  const double s2 = inv_p * inv_p;
  for (uint32_t t = 0; t < trials; t++) {
    if (beta) beta[t] = b[t];
    if (est) est[t] = (double)b[t] * (s2 * s2);
  }
  return BFC_OK;
}

int bfc_clrspar(bfc_graph *g, uint32_t colors, uint32_t trials, uint64_t seed, double *est, uint64_t *beta,
                void *stream) {
  if (!g || trials == 0 || colors == 0) return BFC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->last_stream = s;
  std::vector<uint64_t> b(trials);
  int rc = sparsify_trials(g, trials, b.data(), s, [&](uint32_t *keep, const uint32_t *trial) -> int {
    if (g->m == 0) return BFC_OK;
    unsigned grid = grid_for((uint64_t)g->nU * 32, 256);
    k_keep_clrspar<<<grid, 256, 0, s>>>(ptr<uint64_t>(g->offU), ptr<uint32_t>(g->nbrU), g->nU, seed, trial, colors,
                                        keep);
    BFC_LAUNCHED();
    return BFC_OK;
  });
  if (rc) return rc;
  const double n = (double)colors;
  for (uint32_t t = 0; t < trials; t++) {
    if (beta) beta[t] = b[t];
    if (est) est[t] = (double)b[t] * (n * n * n);
  }
  return BFC_OK;
}

// VSamp and proposals: see vsamp.cu (declared here so the ABI is complete)
}  // extern "C"
