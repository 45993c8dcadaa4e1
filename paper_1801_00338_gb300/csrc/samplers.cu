// Edge sampling (Section 5.2, Algorithm 5), its fast per-edge estimate
// (Section 5.5, Algorithm 7) and wedge sampling (Section 5.3, Algorithm 6).
//
// Random draws (the same rule as the oracle): trial t has seed
// s_t = output t+1 of the SplitMix64 sequence seeded by the caller's seed, and
// draw j of trial t has its own seed ds = output j+1 of s_t's sequence.
//
// ESamp: the draw's edge is canonical edge e = mulhi64(output 1 of ds, m),
//   e = (a, x) with a in U.  A butterfly through e is a pair (a2, x2) with
//   a2 in Gamma_x \ {a}, x2 in Gamma_a \ {x} and (a2, x2) an edge, so
//   b_e = the number of edges between Gamma_x \ {a} and Gamma_a \ {x}
//   (Section 2's definition, the count eBFC returns).
//   - exact (reps = 0): the draw's value is b_e; term = b_e * m / 4.
//   - Algorithm 7 (reps > 0): repetition i picks a2 = row x's
//     mulhi64(output 2i+2 of ds, d_x)-th entry and x2 = row a's
//     mulhi64(output 2i+3 of ds, d_a)-th entry (full rows) and hits when
//     a2 != a, x2 != x and (a2, x2) is an edge; value = hits h,
//     term = h * d_a * d_x / reps * m / 4 (Lemma on Algorithm 7: E = b_e).
// WSamp: population index i < nU is U vertex i, else V vertex i - nU;
//   h = sum_i C(d_i, 2).  Centre c = first i with C(d_0,2)+...+C(d_i,2) >
//   mulhi64(output 1 of ds, h); p = mulhi64(output 2, d_c),
//   q = mulhi64(output 3, d_c - 1), q += (q >= p); the endpoints are the p-th
//   and q-th entries of c's row; beta = |Gamma_v ^ Gamma_w| - 1;
//   term = beta * h / 4.
// A trial's estimate is the mean of its k terms (summed per trial in a fixed
// order, so results repeat bit for bit).
#include <algorithm>

#include "bfc_internal.cuh"

namespace bfc {
namespace {

__device__ __forceinline__ uint64_t sp_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ uint64_t sp_sm64(uint64_t s, uint64_t k) { return sp_mix(s + k * 0x9E3779B97F4A7C15ull); }

__device__ __forceinline__ uint64_t draw_seed(uint64_t seed, uint64_t k, uint64_t q) {
  return sp_sm64(sp_sm64(seed, q / k + 1), q % k + 1);
}

unsigned sp_grid(uint64_t n, unsigned threads, unsigned cap = 152 * 16) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

int sp_sms() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 152;
}

// 1 iff key is in the ascending row[0, n)
__device__ __forceinline__ bool row_has(const uint32_t *row, uint64_t n, uint32_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (__ldg(&row[mid]) < key) lo = mid + 1; else hi = mid;
  }
  return lo < n && __ldg(&row[lo]) == key;
}

// (a, x) of canonical edge e: a = the last row whose offset is <= e
__device__ __forceinline__ void edge_ends(const uint64_t *offU, uint32_t nU, const uint32_t *nbrU, uint64_t e,
                                          uint32_t &a, uint32_t &x) {
  uint32_t lo = 0, hi = nU - 1;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo + 1) / 2;
    if (__ldg(&offU[mid]) <= e) lo = mid; else hi = mid - 1;
  }
  a = lo;
  x = __ldg(&nbrU[e]);
}

__device__ __forceinline__ uint64_t warp_sum(uint64_t v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct GraphArgs {
  const uint64_t *offU, *offV;
  const uint32_t *nbrU, *nbrV;
  uint32_t nU, nV;
  uint64_t m;
};

// ---------------------------------------------------------------------------
// ESamp with exact b_e: one CTA per draw (a queue over all draws)
// ---------------------------------------------------------------------------
constexpr int EX_THREADS = 256;
constexpr uint32_t EX_SLOTS = 8192;           // shared hash of the probe set (32 KB)
constexpr uint32_t EX_HASH_MAX = EX_SLOTS / 2; // load factor <= 1/2; larger sets use binary search
constexpr uint32_t EMPTY = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t hslot(uint32_t key) { return (key * 0x9E3779B1u) >> (32 - 13); }

__global__ void __launch_bounds__(EX_THREADS) k_es_exact(GraphArgs G, uint64_t seed, uint64_t k, uint64_t total,
                                                         unsigned int *queue, uint64_t *edges, uint64_t *vals) {
  __shared__ uint32_t table[EX_SLOTS];
  __shared__ unsigned long long red[2][EX_THREADS / 32];
  __shared__ unsigned int sh_q;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = EX_THREADS / 32;
  while (true) {
    if (threadIdx.x == 0) sh_q = atomicAdd(queue, 1u);
    __syncthreads();
    const uint64_t q = sh_q;
    if (q >= total) break;
    const uint64_t ds = draw_seed(seed, k, q);
    const uint64_t e = __umul64hi(sp_sm64(ds, 1), G.m);
    uint32_t a, x;
    edge_ends(G.offU, G.nU, G.nbrU, e, a, x);
    const uint64_t ab = G.offU[a], ae = G.offU[a + 1], xb = G.offV[x], xe = G.offV[x + 1];
    // cost of each orientation: walking the rows of Gamma_x's members (cA) or
    // of Gamma_a's members (cX)
    uint64_t cA = 0, cX = 0;
    for (uint64_t i = xb + threadIdx.x; i < xe; i += EX_THREADS) {
      const uint32_t a2 = G.nbrV[i];
      cA += G.offU[a2 + 1] - G.offU[a2];
    }
    for (uint64_t i = ab + threadIdx.x; i < ae; i += EX_THREADS) {
      const uint32_t x2 = G.nbrU[i];
      cX += G.offV[x2 + 1] - G.offV[x2];
    }
    cA = warp_sum(cA);
    cX = warp_sum(cX);
    if (lane == 0) { red[0][warp] = cA; red[1][warp] = cX; }
    __syncthreads();
    cA = 0; cX = 0;
    for (int w = 0; w < NW; w++) { cA += red[0][w]; cX += red[1][w]; }
    // orientation: probe set S (sorted row), outer rows, the excluded outer
    // member and the excluded element
    const bool fromX = cA <= cX;
    const uint32_t *S = fromX ? G.nbrU + ab : G.nbrV + xb;
    const uint64_t nS = fromX ? ae - ab : xe - xb;
    const uint32_t *outer = fromX ? G.nbrV + xb : G.nbrU + ab;
    const uint64_t nOut = fromX ? xe - xb : ae - ab;
    const uint64_t *rowOff = fromX ? G.offU : G.offV;
    const uint32_t *rowNbr = fromX ? G.nbrU : G.nbrV;
    const uint32_t skipOuter = fromX ? a : x, skipElem = fromX ? x : a;
    const bool hashed = nS <= EX_HASH_MAX;
    __syncthreads();  // red[] reads done
    if (hashed) {
      for (uint32_t i = threadIdx.x; i < EX_SLOTS; i += EX_THREADS) table[i] = EMPTY;
      __syncthreads();
      for (uint64_t i = threadIdx.x; i < nS; i += EX_THREADS) {
        const uint32_t key = S[i];
        uint32_t sl = hslot(key);
        while (atomicCAS(&table[sl], EMPTY, key) != EMPTY) sl = (sl + 1) & (EX_SLOTS - 1);
      }
      __syncthreads();
    }
    uint64_t cnt = 0;
    for (uint64_t o = warp; o < nOut; o += NW) {
      const uint32_t r = outer[o];
      if (r == skipOuter) continue;
      const uint64_t rb = rowOff[r], re = rowOff[r + 1];
      for (uint64_t i = rb + lane; i < re; i += 32) {
        const uint32_t y = __ldg(&rowNbr[i]);
        if (y == skipElem) continue;
        bool in;
        if (hashed) {
          uint32_t sl = hslot(y);
          while (true) {
            const uint32_t t = table[sl];
            if (t == y) { in = true; break; }
            if (t == EMPTY) { in = false; break; }
            sl = (sl + 1) & (EX_SLOTS - 1);
          }
        } else {
          in = row_has(S, nS, y);
        }
        cnt += in;
      }
    }
    cnt = warp_sum(cnt);
    if (lane == 0) red[0][warp] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t tot = 0;
      for (int w = 0; w < NW; w++) tot += red[0][w];
      vals[q] = tot;
      if (edges) edges[q] = e;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// ESamp with Algorithm 7: one warp per draw, lanes over the repetitions
// ---------------------------------------------------------------------------
__global__ void k_es_fast(GraphArgs G, uint64_t seed, uint64_t k, uint64_t total, uint32_t reps, uint64_t *edges,
                          uint64_t *vals, double *terms) {
  const int lane = threadIdx.x & 31;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t q = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < total; q += nw) {
    const uint64_t ds = draw_seed(seed, k, q);
    const uint64_t e = __umul64hi(sp_sm64(ds, 1), G.m);
    uint32_t a, x;
    edge_ends(G.offU, G.nU, G.nbrU, e, a, x);
    const uint64_t ab = G.offU[a], da = G.offU[a + 1] - ab, xb = G.offV[x], dx = G.offV[x + 1] - xb;
    uint64_t hits = 0;
    for (uint32_t i = lane; i < reps; i += 32) {
      const uint32_t a2 = __ldg(&G.nbrV[xb + __umul64hi(sp_sm64(ds, 2ull * i + 2), dx)]);
      const uint32_t x2 = __ldg(&G.nbrU[ab + __umul64hi(sp_sm64(ds, 2ull * i + 3), da)]);
      if (a2 == a || x2 == x) continue;
      // (a2, x2) is an edge: search the shorter of the two sorted rows
      const uint64_t r1 = G.offU[a2], n1 = G.offU[a2 + 1] - r1, r2 = G.offV[x2], n2 = G.offV[x2 + 1] - r2;
      hits += (n1 <= n2) ? row_has(G.nbrU + r1, n1, x2) : row_has(G.nbrV + r2, n2, a2);
    }
    hits = warp_sum(hits);
    if (lane == 0) {
      vals[q] = hits;
      if (edges) edges[q] = e;
      terms[q] = (double)hits * (double)da * (double)dx / (double)reps * ((double)G.m / 4.0);
    }
  }
}

// exact draws' terms: b_e * m / 4
__global__ void k_es_terms(const uint64_t *vals, uint64_t total, uint64_t m, double *terms) {
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (uint64_t)gridDim.x * blockDim.x)
    terms[q] = (double)vals[q] * ((double)m / 4.0);
}

// one block per trial: the mean of its k terms, summed in a fixed order
constexpr int RED_THREADS = 256;
__global__ void k_trial_mean(const double *terms, uint64_t k, double *est) {
  __shared__ double part[RED_THREADS];
  const uint64_t t = blockIdx.x;
  double s = 0.0;
  for (uint64_t j = threadIdx.x; j < k; j += RED_THREADS) s += terms[t * k + j];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) est[t] = k ? part[0] / (double)k : 0.0;
}

// ---------------------------------------------------------------------------
// WSamp: one warp per draw
// ---------------------------------------------------------------------------
__global__ void k_wedges_per_vertex(const uint64_t *offU, uint32_t nU, const uint64_t *offV, uint32_t nV,
                                    uint64_t *c2) {
  const uint64_t n = (uint64_t)nU + nV;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t d = (i < nU) ? offU[i + 1] - offU[i] : offV[i - nU + 1] - offV[i - nU];
    c2[i] = d * (d ? d - 1 : 0) / 2;
  }
}

__global__ void k_ws_draw(GraphArgs G, const uint64_t *excl, uint64_t h, uint64_t seed, uint64_t k, uint64_t total,
                          uint64_t *centres, uint64_t *betas, double *terms) {
  const int lane = threadIdx.x & 31;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t n = (uint64_t)G.nU + G.nV;
  for (uint64_t q = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < total; q += nw) {
    const uint64_t ds = draw_seed(seed, k, q);
    const uint64_t target = __umul64hi(sp_sm64(ds, 1), h);
    uint64_t lo = 0, hi = n - 1;  // first i with excl[i + 1] > target
    while (lo < hi) {
      const uint64_t mid = lo + (hi - lo) / 2;
      if (excl[mid + 1] > target) hi = mid; else lo = mid + 1;
    }
    const bool onU = lo < G.nU;
    const uint32_t c = (uint32_t)(onU ? lo : lo - G.nU);
    const uint64_t cb = onU ? G.offU[c] : G.offV[c];
    const uint64_t d = (onU ? G.offU[c + 1] : G.offV[c + 1]) - cb;
    const uint64_t p = __umul64hi(sp_sm64(ds, 2), d);
    uint64_t r = __umul64hi(sp_sm64(ds, 3), d - 1);
    r += (r >= p);
    const uint32_t *crow = onU ? G.nbrU : G.nbrV;
    const uint32_t v = crow[cb + p], w = crow[cb + r];
    // v, w lie on the other side: intersect their rows (the shorter one
    // searched in the longer one)
    const uint64_t *ooff = onU ? G.offV : G.offU;
    const uint32_t *onbr = onU ? G.nbrV : G.nbrU;
    uint64_t vb = ooff[v], vn = ooff[v + 1] - vb, wb = ooff[w], wn = ooff[w + 1] - wb;
    if (vn > wn) { uint64_t t = vb; vb = wb; wb = t; t = vn; vn = wn; wn = t; }
    uint64_t common = 0;
    for (uint64_t i = lane; i < vn; i += 32) common += row_has(onbr + wb, wn, __ldg(&onbr[vb + i]));
    common = warp_sum(common);
    if (lane == 0) {
      const uint64_t beta = common - 1;  // c itself is common to both
      if (centres) centres[q] = lo;
      betas[q] = beta;
      terms[q] = (double)beta * ((double)h / 4.0);
    }
  }
}

}  // namespace
}  // namespace bfc

using namespace bfc;

static GraphArgs graph_args(const bfc_graph *g) {
  GraphArgs G;
  G.offU = ptr<uint64_t>(g->offU);
  G.offV = ptr<uint64_t>(g->offV);
  G.nbrU = ptr<uint32_t>(g->nbrU);
  G.nbrV = ptr<uint32_t>(g->nbrV);
  G.nU = g->nU;
  G.nV = g->nV;
  G.m = g->m;
  return G;
}

extern "C" {

int bfc_esamp(bfc_graph *g, uint64_t k, uint32_t reps, uint32_t trials, uint64_t seed, double *est, uint64_t *edges,
              uint64_t *vals, void *stream) {
  if (!g || trials == 0 || !est) return BFC_EINVAL;
  if (g->m == 0) return BFC_EINVAL;
  const uint64_t total = (uint64_t)trials * k;
  if (total >= (1ull << 32)) return BFC_ERANGE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->last_stream = s;
  if (total == 0) {
    for (uint32_t t = 0; t < trials; t++) est[t] = 0.0;
    return BFC_OK;
  }
  DBuf own_vals, terms, dest, cnt;
  auto cleanup = [&]() { dfree(own_vals, s); dfree(terms, s); dfree(dest, s); dfree(cnt, s); };
  int rc = BFC_OK;
#define ES_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
#define ES_CUDA(x) do { if ((x) != cudaSuccess) { cleanup(); return BFC_ECUDA; } } while (0)
  if (!vals) ES_TRY(dalloc(own_vals, total * 8, s));
  uint64_t *d_vals = vals ? vals : ptr<uint64_t>(own_vals);
  ES_TRY(dalloc(terms, total * 8, s));
  ES_TRY(dalloc(dest, (uint64_t)trials * 8, s));
  const GraphArgs G = graph_args(g);
  if (reps == 0) {
    ES_TRY(dalloc(cnt, 4, s));
    ES_CUDA(cudaMemsetAsync(cnt.p, 0, 4, s));
    const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)sp_sms() * 4, total);
    profile_begin("esamp.exact", s);
    k_es_exact<<<grid, EX_THREADS, 0, s>>>(G, seed, k, total, ptr<unsigned int>(cnt), edges, d_vals);
    count_launch();
    profile_end("esamp.exact", s);
    k_es_terms<<<sp_grid(total, 256), 256, 0, s>>>(d_vals, total, g->m, ptr<double>(terms));
    count_launch();
  } else {
    profile_begin("esamp.fast", s);
    k_es_fast<<<sp_grid(total * 32, 256), 256, 0, s>>>(G, seed, k, total, reps, edges, d_vals, ptr<double>(terms));
    count_launch();
    profile_end("esamp.fast", s);
  }
  k_trial_mean<<<trials, RED_THREADS, 0, s>>>(ptr<double>(terms), k, ptr<double>(dest));
  count_launch();
  ES_CUDA(cudaGetLastError());
  ES_CUDA(cudaMemcpyAsync(est, dest.p, (uint64_t)trials * 8, cudaMemcpyDeviceToHost, s));
  ES_CUDA(cudaStreamSynchronize(s));
  cleanup();
#undef ES_TRY
#undef ES_CUDA
  return BFC_OK;
}

int bfc_wsamp(bfc_graph *g, uint64_t k, uint32_t trials, uint64_t seed, double *est, uint64_t *centres,
              uint64_t *betas, void *stream) {
  if (!g || trials == 0 || !est) return BFC_EINVAL;
  const uint64_t total = (uint64_t)trials * k;
  if (total >= (1ull << 32)) return BFC_ERANGE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  g->last_stream = s;
  const uint64_t h = g->wU + g->wV;  // wedges centred on U plus those centred on V
  if (h == 0) return BFC_EINVAL;
  if (total == 0) {
    for (uint32_t t = 0; t < trials; t++) est[t] = 0.0;
    return BFC_OK;
  }
  const uint64_t n = (uint64_t)g->nU + g->nV;
  DBuf c2, excl, own_b, terms, dest;
  auto cleanup = [&]() { dfree(c2, s); dfree(excl, s); dfree(own_b, s); dfree(terms, s); dfree(dest, s); };
  int rc = BFC_OK;
#define WS_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
#define WS_CUDA(x) do { if ((x) != cudaSuccess) { cleanup(); return BFC_ECUDA; } } while (0)
  WS_TRY(dalloc(c2, n * 8, s));
  WS_TRY(dalloc(excl, (n + 1) * 8, s));
  if (!betas) WS_TRY(dalloc(own_b, total * 8, s));
  WS_TRY(dalloc(terms, total * 8, s));
  WS_TRY(dalloc(dest, (uint64_t)trials * 8, s));
  const GraphArgs G = graph_args(g);
  k_wedges_per_vertex<<<sp_grid(n, 256), 256, 0, s>>>(G.offU, G.nU, G.offV, G.nV, ptr<uint64_t>(c2));
  count_launch();
  WS_TRY(exclusive_scan_u64(ptr<uint64_t>(c2), ptr<uint64_t>(excl), n, g->scr, s));
  profile_begin("wsamp", s);
  k_ws_draw<<<sp_grid(total * 32, 256), 256, 0, s>>>(G, ptr<uint64_t>(excl), h, seed, k, total, centres,
                                                     betas ? betas : ptr<uint64_t>(own_b), ptr<double>(terms));
  count_launch();
  profile_end("wsamp", s);
  k_trial_mean<<<trials, RED_THREADS, 0, s>>>(ptr<double>(terms), k, ptr<double>(dest));
  count_launch();
  WS_CUDA(cudaGetLastError());
  WS_CUDA(cudaMemcpyAsync(est, dest.p, (uint64_t)trials * 8, cudaMemcpyDeviceToHost, s));
  WS_CUDA(cudaStreamSynchronize(s));
  cleanup();
#undef WS_TRY
#undef WS_CUDA
  return BFC_OK;
}

}  // extern "C"
