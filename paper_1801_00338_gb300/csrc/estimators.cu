// Sparsification estimators (Section 6).
//
// ESpar (Algorithm 8): keep every edge independently with probability p,
// count the kept subgraph exactly, scale by p^-4.
// ClrSpar (Algorithm 9): colour every vertex uniformly from N colours, keep
// the monochromatic edges, count exactly, scale by N^3.
//
// Random draws: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), counter based:
// output k >= 1 of the sequence seeded by s is mix(s + k * 0x9E3779B97F4A7C15);
// trial t uses the sequence seeded by output t + 1 of the caller's seed; an
// edge e (canonical id) is kept by ESpar when the top 32 bits of output e + 1
// are below p 2^32, and vertex u of U gets colour floor(top32(output u + 1) N
// / 2^32), vertex v of V that of output nU + v + 1.
//
// Every trial is counted over the full graph's rank layout by the batched
// trial kernel (trials.cu): one persistent launch for all the trials, with
// the kept subgraph given by per-trial bit masks instead of a rebuilt layout.
// B of the kept subgraph does not depend on the start side or the rank order
// (Lemma 1 and Eq. (4)), so the full graph's are used.
#include <vector>

#include "bfc_internal.cuh"

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
  const int rc = run_trials(g, 0, seed, T, 0, trials, b.data(), s);
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
  const int rc = run_trials(g, 1, seed, 0, colors, trials, b.data(), s);
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
