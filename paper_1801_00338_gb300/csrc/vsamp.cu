// Vertex sampling (Section 5.1, Algorithm 4) -- batched vBFC on sampled vertices.
#include "bfc_internal.cuh"

struct bfc_proposal {
  bfc::DBuf weights;  // u32[n]
  bfc::DBuf prefix;   // u64[n]
  uint64_t n = 0, W = 0;
};

extern "C" {
int bfc_vsamp(bfc_graph *g, uint64_t k, const bfc_proposal *prop, uint32_t trials, uint64_t seed, double *est,
              uint64_t *drawn, uint64_t *bdraw, void *stream) {
  (void)g; (void)k; (void)prop; (void)trials; (void)seed; (void)est; (void)drawn; (void)bdraw; (void)stream;
  return BFC_EINVAL;
}
int bfc_proposal_from_weights(bfc_graph *g, const uint32_t *weights, uint32_t flags, void *stream,
                              bfc_proposal **out) {
  (void)g; (void)weights; (void)flags; (void)stream; (void)out;
  return BFC_EINVAL;
}
int bfc_proposal_free(bfc_proposal *p) {
  delete p;
  return BFC_OK;
}
}
