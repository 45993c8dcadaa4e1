// Vertex sampling (Section 5.1, Algorithm 4) with an optional importance
// proposal.
//
// A trial draws k vertices i.i.d. from the population V = U u V (n = nU + nV)
// and returns (1/k) sum_j b_{v_j} / (4 q(v_j)).  With q = 1/n every term is
// Algorithm 4's b_v * n / 4.  With a proposal, q is the mixture
// 1/(2n) + w_i/(2W) of a uniform draw and a draw proportional to integer
// weights; dividing by q keeps the estimator unbiased (Lemma 4's expectation
// argument with the uniform 1/n replaced by q).  b_v of every draw comes from
// Algorithm 2 run on the GPU for the batch of drawn vertices (vbfc_batch).
//
// Draw j of trial t uses outputs 2j+1 (r1) and 2j+2 (r2) of the SplitMix64
// sequence seeded by s_t = output t+1 of the caller's seed.
#include <algorithm>
#include <new>
#include <vector>

#include "bfc_internal.cuh"

struct bfc_proposal {
  bfc::DBuf weights;  // u32[n]
  bfc::DBuf excl;     // u64[n+1] exclusive prefix sums of the weights
  uint64_t n = 0, W = 0;
};

namespace bfc {

__device__ __forceinline__ uint64_t vs_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t vs_sm64(uint64_t s, uint64_t k) { return vs_mix(s + k * 0x9E3779B97F4A7C15ull); }

static unsigned vs_grid(uint64_t n, unsigned threads, unsigned cap = 152 * 16) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

// drawn[t*k + j] = population index of draw j of trial t
__global__ void k_vs_draw(uint64_t seed, uint32_t trials, uint64_t k, uint64_t n, const uint64_t *excl, uint64_t W,
                          uint64_t *drawn) {
  const uint64_t total = (uint64_t)trials * k;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t t = q / k, j = q % k;
    const uint64_t ts = vs_sm64(seed, t + 1);
    const uint64_t r1 = vs_sm64(ts, 2 * j + 1), r2 = vs_sm64(ts, 2 * j + 2);
    uint64_t i;
    if (!excl || (r1 >> 63) == 0) {
      i = __umul64hi(r2, n);
    } else {
      const uint64_t target = __umul64hi(r2, W);
      uint64_t lo = 0, hi = n - 1;  // first i with excl[i+1] > target
      while (lo < hi) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (excl[mid + 1] > target) hi = mid; else lo = mid + 1;
      }
      i = lo;
    }
    drawn[q] = i;
  }
}

// split the draws by side into rank lists (item order is arbitrary; results go back by draw id)
__global__ void k_vs_split(const uint64_t *drawn, uint64_t total, uint32_t nU, const uint32_t *rankU,
                           const uint32_t *rankV, unsigned int *cnt, uint32_t *rU, uint32_t *jU, uint32_t *rV,
                           uint32_t *jV) {
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = drawn[q];
    if (i < nU) {
      const uint32_t p = atomicAdd(&cnt[0], 1u);
      rU[p] = rankU[i];
      jU[p] = (uint32_t)q;
    } else {
      const uint32_t p = atomicAdd(&cnt[1], 1u);
      rV[p] = rankV[i - nU];
      jV[p] = (uint32_t)q;
    }
  }
}
__global__ void k_vs_scatter(const unsigned long long *b, const uint32_t *j, uint32_t n, uint64_t *bdraw) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x)
    bdraw[j[p]] = b[p];
}

// one block per trial: est[t] = (1/k) sum_j b_j / (4 q_j), summed in a fixed order
constexpr int VS_THREADS = 256;
__global__ void k_vs_estimate(const uint64_t *drawn, const uint64_t *bdraw, uint64_t k, uint64_t n,
                              const uint32_t *weights, uint64_t W, double *est) {
  __shared__ double part[VS_THREADS];
  const uint64_t t = blockIdx.x;
  double s = 0.0;
  for (uint64_t j = threadIdx.x; j < k; j += VS_THREADS) {
    const uint64_t q = t * k + j;
    const uint64_t i = drawn[q];
    const double prob = weights ? 0.5 / (double)n + 0.5 * (double)weights[i] / (double)W : 1.0 / (double)n;
    s += (double)bdraw[q] / (4.0 * prob);
  }
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = VS_THREADS / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) est[t] = k ? part[0] / (double)k : 0.0;
}

}  // namespace bfc

using namespace bfc;

extern "C" {

int bfc_proposal_from_weights(bfc_graph *g, const uint32_t *weights, uint32_t flags, void *stream,
                              bfc_proposal **out) {
  if (!g || !weights || !out || (flags & ~BFC_INPUT_DEVICE)) return BFC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  *out = nullptr;
  bfc_proposal *p = new (std::nothrow) bfc_proposal();
  if (!p) return BFC_ENOMEM;
  p->n = (uint64_t)g->nU + g->nV;
  int rc = dalloc(p->weights, p->n * 4, s);
  if (!rc) rc = dalloc(p->excl, (p->n + 1) * 8, s);
  if (!rc && cudaMemcpyAsync(p->weights.p, weights, p->n * 4,
                             (flags & BFC_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             s) != cudaSuccess)
    rc = BFC_ECUDA;
  if (!rc) rc = exclusive_scan_u32_to_u64(ptr<uint32_t>(p->weights), ptr<uint64_t>(p->excl), p->n, g->scr, s);
  if (!rc && cudaMemcpyAsync(&p->W, ptr<uint64_t>(p->excl) + p->n, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    rc = BFC_ECUDA;
  if (!rc && cudaStreamSynchronize(s) != cudaSuccess) rc = BFC_ECUDA;
  if (!rc && p->W == 0) rc = BFC_EINVAL;
  if (rc) {
    bfc_proposal_free(p);
    return rc;
  }
  *out = p;
  return BFC_OK;
}

int bfc_proposal_weights(const bfc_proposal *p, uint32_t *weights, uint64_t n, uint64_t *W) {
  if (!p || !weights || n != p->n) return BFC_EINVAL;
  if (cudaMemcpy(weights, p->weights.p, n * 4, cudaMemcpyDeviceToHost) != cudaSuccess) return BFC_ECUDA;
  if (W) *W = p->W;
  return BFC_OK;
}

int bfc_proposal_free(bfc_proposal *p) {
  if (!p) return BFC_EINVAL;
  cudaDeviceSynchronize();
  dfree(p->weights, nullptr);
  dfree(p->excl, nullptr);
  cudaDeviceSynchronize();
  delete p;
  return BFC_OK;
}

int bfc_vsamp(bfc_graph *g, uint64_t k, const bfc_proposal *prop, uint32_t trials, uint64_t seed, double *est,
              uint64_t *drawn, uint64_t *bdraw, void *stream) {
  if (!g || trials == 0 || !est) return BFC_EINVAL;
  if (prop && prop->n != (uint64_t)g->nU + g->nV) return BFC_EINVAL;
  const uint64_t total = (uint64_t)trials * k;
  if (total >= (1ull << 32)) return BFC_ERANGE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->last_stream = s;
  if (total == 0) {
    for (uint32_t t = 0; t < trials; t++) est[t] = 0.0;
    return BFC_OK;
  }
  BFC_TRY(plan_build(g, 0, s));
  BFC_TRY(plan_build(g, 1, s));
  const uint64_t n = (uint64_t)g->nU + g->nV;
  DBuf own_drawn, own_b, lists, outs, cnt, dest;
  auto cleanup = [&]() {
    dfree(own_drawn, s); dfree(own_b, s); dfree(lists, s); dfree(outs, s); dfree(cnt, s); dfree(dest, s);
  };
  int rc = BFC_OK;
#define VS_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
  if (!drawn) VS_TRY(dalloc(own_drawn, total * 8, s));
  if (!bdraw) VS_TRY(dalloc(own_b, total * 8, s));
  uint64_t *d_drawn = drawn ? drawn : ptr<uint64_t>(own_drawn);
  uint64_t *d_b = bdraw ? bdraw : ptr<uint64_t>(own_b);
  VS_TRY(dalloc(lists, total * 4 * 4, s));
  VS_TRY(dalloc(outs, total * 8, s));
  VS_TRY(dalloc(cnt, 64, s));
  VS_TRY(dalloc(dest, (uint64_t)trials * 8, s));
  k_vs_draw<<<vs_grid(total, 256), 256, 0, s>>>(seed, trials, k, n, prop ? ptr<uint64_t>(prop->excl) : nullptr,
                                               prop ? prop->W : 0, d_drawn);
  BFC_LAUNCHED();
  BFC_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, 64, s));
  uint32_t *rU = ptr<uint32_t>(lists), *jU = rU + total, *rV = jU + total, *jV = rV + total;
  k_vs_split<<<vs_grid(total, 256), 256, 0, s>>>(d_drawn, total, g->nU, ptr<uint32_t>(g->plan[0].rank_of),
                                                ptr<uint32_t>(g->plan[1].rank_of), ptr<unsigned int>(cnt), rU, jU,
                                                rV, jV);
  BFC_LAUNCHED();
  unsigned int hc[2];
  BFC_CUDA_TRY(cudaMemcpyAsync(hc, cnt.p, 8, cudaMemcpyDeviceToHost, s));
  BFC_CUDA_TRY(cudaStreamSynchronize(s));
  unsigned long long *ob = ptr<unsigned long long>(outs);
  if (hc[0]) {
    VS_TRY(vbfc_batch(g, g->plan[0], rU, hc[0], ob, s));
    k_vs_scatter<<<vs_grid(hc[0], 256), 256, 0, s>>>(ob, jU, hc[0], d_b);
    BFC_LAUNCHED();
  }
  if (hc[1]) {
    VS_TRY(vbfc_batch(g, g->plan[1], rV, hc[1], ob + hc[0], s));
    k_vs_scatter<<<vs_grid(hc[1], 256), 256, 0, s>>>(ob + hc[0], jV, hc[1], d_b);
    BFC_LAUNCHED();
  }
  k_vs_estimate<<<trials, VS_THREADS, 0, s>>>(d_drawn, d_b, k, n, prop ? ptr<uint32_t>(prop->weights) : nullptr,
                                             prop ? prop->W : 0, ptr<double>(dest));
  BFC_LAUNCHED();
  BFC_CUDA_TRY(cudaMemcpyAsync(est, dest.p, (uint64_t)trials * 8, cudaMemcpyDeviceToHost, s));
  rc = read_device_error(g, s);
  cleanup();
#undef VS_TRY
  return rc;
}

}  // extern "C"
