// An ExactBFC entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need a count:
// services whose device memory is reserved up front by another allocator or
// held to a fixed budget, and latency-bound loops that must not block on the
// allocator.  For them,
// bfc_exact_csr_noalloc counts butterflies of a graph the caller already holds
// as device CSR arrays, using only a scratch array that is part of this
// library's image: a file-scope __device__ array of BFC_NOALLOC_SCRATCH_WORDS
// 32-bit words (64 MiB) that every GPU which loads the library keeps until the
// process exits.
//
// Counting: each CTA takes start vertices in turn and counts, for every later
// start vertex w (id order), c(v, w) = |Gamma_v ^ Gamma_w| in its own slice of
// the scratch array; an exchange pass adds C(c, 2) and resets the slice.  The
// start side follows the first three lines of Algorithm 1 unless the caller
// fixes it.  The result is written to a device word, in stream order.
#include <algorithm>
#include <mutex>

#include "bfc_internal.cuh"

namespace bfc {
namespace {

constexpr uint32_t NA_HEADER = 64;  // words before the counters: sums and the result
constexpr uint32_t NA_THREADS = 256;
constexpr uint32_t NA_MAX_CTAS = 152;

static __device__ __align__(256) uint32_t g_noalloc_scratch[BFC_NOALLOC_SCRATCH_WORDS];

// host-side device addresses of g_noalloc_scratch, one per device
std::mutex g_na_mu;
uint32_t *g_na_addr[64] = {};

int scratch_address(uint32_t **out) {
  int dev = 0;
  BFC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return BFC_EINVAL;
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_addr[dev]) {
    void *p = nullptr;
    BFC_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_na_addr[dev] = static_cast<uint32_t *>(p);
  }
  *out = g_na_addr[dev];
  return BFC_OK;
}

// header layout (u64 view): [0] sum_U d^2, [1] sum_V d^2, [2] B
__global__ void k_na_clear(uint32_t *scr, uint64_t words) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x)
    scr[i] = 0;
}

__global__ void k_na_square_sums(const uint64_t *offU, uint32_t nU, const uint64_t *offV, uint32_t nV,
                                 unsigned long long *hdr) {
  unsigned long long su = 0, sv = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nU; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t d = offU[i + 1] - offU[i];
    su += d * d;
  }
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nV; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t d = offV[i + 1] - offV[i];
    sv += d * d;
  }
  for (int o = 16; o > 0; o >>= 1) {
    su += __shfl_down_sync(0xffffffffu, su, o);
    sv += __shfl_down_sync(0xffffffffu, sv, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (su) atomicAdd(&hdr[0], su);
    if (sv) atomicAdd(&hdr[1], sv);
  }
}

// side: 0 = U starts, 1 = V starts, -1 = Algorithm 1's choice from hdr[0..1]
__global__ void __launch_bounds__(NA_THREADS) k_na_count(const uint64_t *offU, const uint32_t *nbrU, uint32_t nU,
                                                          const uint64_t *offV, const uint32_t *nbrV, uint32_t nV,
                                                          int side, uint32_t *scr) {
  unsigned long long *hdr = reinterpret_cast<unsigned long long *>(scr);
  const int s = side >= 0 ? side : (hdr[0] < hdr[1] ? 1 : 0);
  const uint64_t *offS = s ? offV : offU, *offM = s ? offU : offV;
  const uint32_t *nbrS = s ? nbrV : nbrU, *nbrM = s ? nbrU : nbrV;
  const uint32_t nS = s ? nV : nU, nM = s ? nU : nV;
  uint32_t *ctr = scr + NA_HEADER + (uint64_t)blockIdx.x * nS;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = NA_THREADS / 32;
  unsigned long long acc = 0;
  for (uint32_t v = blockIdx.x; v < nS; v += gridDim.x) {
    const uint64_t b = offS[v], e = offS[v + 1];
    if (e - b < 2) continue;  // every c(v, w) <= 1: no pair
    // count c(v, w) for w > v: one warp per midpoint
    for (uint64_t j = b + warp; j < e; j += NW) {
      const uint32_t x = nbrS[j];
      if (x >= nM) continue;  // ids outside the other side are ignored, never dereferenced
      for (uint64_t i = offM[x] + lane; i < offM[x + 1]; i += 32) {
        const uint32_t w = nbrM[i];
        if (w > v && w < nS) atomicAdd(&ctr[w], 1u);
      }
    }
    __syncthreads();
    // exchange: C(c, 2) once per distinct w, leaving zeros behind
    for (uint64_t j = b + warp; j < e; j += NW) {
      const uint32_t x = nbrS[j];
      if (x >= nM) continue;
      for (uint64_t i = offM[x] + lane; i < offM[x + 1]; i += 32) {
        const uint32_t w = nbrM[i];
        if (w > v && w < nS) {
          const uint64_t c = atomicExch(&ctr[w], 0u);
          acc += c * (c - (c > 0)) / 2;
        }
      }
    }
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0 && acc) atomicAdd(&hdr[2], acc);
}

__global__ void k_na_store(const uint32_t *scr, uint64_t *out_B) {
  *out_B = reinterpret_cast<const unsigned long long *>(scr)[2];
}

}  // namespace
}  // namespace bfc

using namespace bfc;

extern "C" int bfc_exact_csr_noalloc(const uint64_t *offU, const uint32_t *nbrU, uint32_t nU, const uint64_t *offV,
                                     const uint32_t *nbrV, uint32_t nV, uint32_t flags, uint64_t *out_B,
                                     void *stream) {
  if ((flags & ~(BFC_SIDE_U | BFC_SIDE_V)) || ((flags & BFC_SIDE_U) && (flags & BFC_SIDE_V))) return BFC_EINVAL;
  // the larger side bounds the counter slice whatever side starts
  const uint64_t nmax = nU > nV ? nU : nV;
  if (nmax == 0 || nmax > (uint64_t)BFC_NOALLOC_SCRATCH_WORDS - NA_HEADER) return BFC_ERANGE;
  if (!offU || !offV || !out_B || ((!nbrU || !nbrV) && nmax > 0)) return BFC_EINVAL;
  uint32_t *scr = nullptr;
  BFC_TRY(scratch_address(&scr));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // one counter slice of nmax words per CTA
  uint64_t ctas = ((uint64_t)BFC_NOALLOC_SCRATCH_WORDS - NA_HEADER) / nmax;
  if (ctas > NA_MAX_CTAS) ctas = NA_MAX_CTAS;
  const uint64_t used = NA_HEADER + ctas * nmax;
  k_na_clear<<<(unsigned)std::min<uint64_t>((used + 255) / 256, 152 * 8), 256, 0, s>>>(scr, used);
  BFC_LAUNCHED();
  const int side = (flags & BFC_SIDE_U) ? 0 : (flags & BFC_SIDE_V) ? 1 : -1;
  unsigned long long *hdr = reinterpret_cast<unsigned long long *>(scr);
  if (side < 0) {
    const uint64_t n = nmax + 1;
    k_na_square_sums<<<(unsigned)std::min<uint64_t>((n + 255) / 256, 152 * 4), 256, 0, s>>>(offU, nU, offV, nV,
                                                                                             hdr);
    BFC_LAUNCHED();
  }
  k_na_count<<<(unsigned)ctas, NA_THREADS, 0, s>>>(offU, nbrU, nU, offV, nbrV, nV, side, scr);
  BFC_LAUNCHED();
  k_na_store<<<1, 1, 0, s>>>(scr, out_B);
  BFC_LAUNCHED();
  return BFC_OK;
}
