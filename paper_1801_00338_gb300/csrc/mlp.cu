// Learned importance proposal for vertex sampling (an extension to Section
// 5.1: VSamp draws vertices uniformly; here a small network scores vertices
// from cheap features so that the mixture proposal leans towards vertices with
// many butterflies, and the importance weights keep the estimator unbiased).
//
// Features (per vertex v, both sides, O(m) in total):
//   0 log1p(d_v) / 8            1 log1p(sum_{u in Gamma_v} d_u) / 16
//   2 log1p(sum (d_u - 1)) / 16 (wedges with v as an end)
//   3 log1p(C(d_v, 2)) / 16     (wedges centred on v)
//   4 side (0 for U, 1 for V)   5 log1p(max_{u in Gamma_v} d_u) / 16
// (the fixed divisors keep the inputs near unit scale).
//
// Network: 6 -> 64 -> 64 -> 1, GELU (exact erf form) after both hidden
// layers, weights stored in bfloat16, activations and accumulation in fp32.
// Parameter vector (P = 4673 values): W1[6][64], b1[64], W2[64][64], b2[64],
// W3[64], b3.  Training minimises the mean squared error against
// t_v = log1p(b_v) with Adam (Kingma & Ba 2014).
#include <cuda_bf16.h>

#include <algorithm>
#include <new>

#include "bfc_internal.cuh"

namespace bfc {
namespace {

constexpr int F = BFC_MLP_FEATURES, H = 64;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + F * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H, NPARAM = OFF_B3 + 1;
static_assert(NPARAM == BFC_MLP_PARAMS, "parameter layout");

unsigned ml_grid(uint64_t n, unsigned threads, unsigned cap = 152 * 16) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  const float cdf = 0.5f * (1.0f + erff(z * 0.70710678118654752f));
  const float pdf = 0.39894228040143268f * expf(-0.5f * z * z);
  return cdf + z * pdf;
}

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
__global__ void k_features(const uint64_t *offA, const uint32_t *nbrA, const uint32_t *degB, uint32_t nA, float side,
                           float *feat) {
  const int lane = threadIdx.x & 31;
  uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t v = warp; v < nA; v += nw) {
    const uint64_t b = offA[v], e = offA[v + 1];
    uint64_t s1 = 0, mx = 0;
    for (uint64_t j = b + lane; j < e; j += 32) {
      const uint64_t du = degB[nbrA[j]];
      s1 += du;
      mx = du > mx ? du : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
      s1 += __shfl_down_sync(0xffffffffu, s1, o);
      const uint64_t other = __shfl_down_sync(0xffffffffu, mx, o);
      mx = other > mx ? other : mx;
    }
    if (lane == 0) {
      const uint64_t d = e - b;
      float *f = feat + v * F;
      f[0] = log1pf((float)d) * 0.125f;
      f[1] = log1pf((float)s1) * 0.0625f;
      f[2] = log1pf((float)(s1 - d)) * 0.0625f;
      f[3] = log1pf((float)(d * (d - (d > 0)) / 2)) * 0.0625f;
      f[4] = side;
      f[5] = log1pf((float)mx) * 0.0625f;
    }
  }
}

__global__ void k_targets(const uint64_t *b, uint64_t n, float *t) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    t[i] = log1pf((float)b[i]);
}

// ---------------------------------------------------------------------------
// forward: one thread per row, weights in shared memory as fp32
// ---------------------------------------------------------------------------
__device__ __forceinline__ void load_weights(const __nv_bfloat16 *w, float *sw) {
  for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) sw[i] = __bfloat162float(w[i]);
}

__global__ void __launch_bounds__(128) k_forward(const __nv_bfloat16 *w, const float *X, uint64_t n, float *y) {
  __shared__ float sw[NPARAM];
  load_weights(w, sw);
  __syncthreads();
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (uint64_t)gridDim.x * blockDim.x) {
    float x[F];
#pragma unroll
    for (int f = 0; f < F; f++) x[f] = X[r * F + f];
    float h1[H];
#pragma unroll
    for (int j = 0; j < H; j++) {
      float z = sw[OFF_B1 + j];
#pragma unroll
      for (int f = 0; f < F; f++) z = fmaf(x[f], sw[OFF_W1 + f * H + j], z);
      h1[j] = gelu(z);
    }
    float out = sw[OFF_B3];
    for (int j = 0; j < H; j++) {
      float z = sw[OFF_B2 + j];
#pragma unroll
      for (int i = 0; i < H; i++) z = fmaf(h1[i], sw[OFF_W2 + i * H + j], z);
      out = fmaf(gelu(z), sw[OFF_W3 + j], out);
    }
    y[r] = out;
  }
}

// ---------------------------------------------------------------------------
// gradient of the mean squared error over rows idx[0..n) (or 0..n when idx is
// null): tiles of 128 rows, activations staged in shared memory, weight
// gradients accumulated per CTA and added to grad once at the end.
// ---------------------------------------------------------------------------
constexpr int TILE = 128, GT = 256;

__global__ void __launch_bounds__(GT, 1) k_grad(const __nv_bfloat16 *w, const float *X, const float *T,
                                                const uint32_t *idx, uint64_t n, float inv_n, float *grad,
                                                float *loss) {
  extern __shared__ float sm[];
  float *sw = sm;                      // NPARAM
  float *sx = sw + NPARAM + 3;         // TILE * F   (aligned to 4 floats below)
  sx = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(sx) + 15) & ~uintptr_t(15));
  float *z1 = sx + TILE * F;           // TILE * H  (Z1, later dZ1)
  float *h1 = z1 + TILE * H;           // TILE * H
  float *z2 = h1 + TILE * H;           // TILE * H  (Z2, later dZ2)
  float *dy = z2 + TILE * H;           // TILE
  float *acc_b = dy + TILE;            // 2 H + 1 (db1, db2, db3) and W3 grads: H
  load_weights(w, sw);
  for (int i = threadIdx.x; i < 3 * H + 1; i += GT) acc_b[i] = 0.f;
  const int t = threadIdx.x;
  // register accumulators: dW2 (16 per thread), dW1 (<= 2 per thread)
  float gW2[16];
#pragma unroll
  for (int k = 0; k < 16; k++) gW2[k] = 0.f;
  float gW1[2] = {0.f, 0.f};
  float lsum = 0.f;
  __syncthreads();
  const uint64_t ntiles = (n + TILE - 1) / TILE;
  for (uint64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const uint64_t base = tile * TILE;
    const int rows = (n - base < (uint64_t)TILE) ? (int)(n - base) : TILE;
    // 1. inputs
    for (int i = t; i < TILE * F; i += GT) {
      const int r = i / F, f = i % F;
      float v = 0.f;
      if (r < rows) {
        const uint64_t row = idx ? idx[base + r] : base + r;
        v = X[row * F + f];
      }
      sx[i] = v;
    }
    __syncthreads();
    // 2. Z1, H1
    for (int i = t; i < TILE * H; i += GT) {
      const int r = i / H, j = i % H;
      float z = sw[OFF_B1 + j];
#pragma unroll
      for (int f = 0; f < F; f++) z = fmaf(sx[r * F + f], sw[OFF_W1 + f * H + j], z);
      z1[i] = z;
      h1[i] = gelu(z);
    }
    __syncthreads();
    // 3. Z2 = H1 W2 + b2
    for (int i = t; i < TILE * H; i += GT) {
      const int r = i / H, j = i % H;
      float z = sw[OFF_B2 + j];
#pragma unroll 8
      for (int k = 0; k < H; k++) z = fmaf(h1[r * H + k], sw[OFF_W2 + k * H + j], z);
      z2[i] = z;
    }
    __syncthreads();
    // 4. y, dy = 2 (y - t) / n (one warp per row)
    {
      const int lane = t & 31, wp = t >> 5;
      for (int r = wp; r < TILE; r += GT / 32) {
        float s = 0.f;
        for (int j = lane; j < H; j += 32) s = fmaf(gelu(z2[r * H + j]), sw[OFF_W3 + j], s);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) {
          float d = 0.f;
          if (r < rows) {
            const uint64_t row = idx ? idx[base + r] : base + r;
            const float e = s + sw[OFF_B3] - T[row];
            lsum += e * e;
            d = 2.f * e * inv_n;
          }
          dy[r] = d;
        }
      }
    }
    __syncthreads();
    // 5. W3, b3 gradients; dZ2 = dy W3 gelu'(Z2)
    if (t < H) {
      float g = 0.f;
      for (int r = 0; r < TILE; r++) g = fmaf(dy[r], gelu(z2[r * H + t]), g);
      acc_b[2 * H + 1 + t] += g;
    }
    if (t == H) {
      float g = 0.f;
      for (int r = 0; r < TILE; r++) g += dy[r];
      acc_b[2 * H] += g;
    }
    __syncthreads();
    for (int i = t; i < TILE * H; i += GT) {
      const int r = i / H, j = i % H;
      z2[i] = dy[r] * sw[OFF_W3 + j] * gelu_grad(z2[i]);
    }
    __syncthreads();
    // 6. W2, b2 gradients: thread t owns column j = t % 64 and rows k = (t / 64) * 16 .. +16 of W2
    {
      const int j = t % H, k0 = (t / H) * 16;
#pragma unroll
      for (int k = 0; k < 16; k++) {
        float g = 0.f;
        for (int r = 0; r < TILE; r++) g = fmaf(h1[r * H + k0 + k], z2[r * H + j], g);
        gW2[k] += g;
      }
      if (t < H) {
        float g = 0.f;
        for (int r = 0; r < TILE; r++) g += z2[r * H + t];
        acc_b[H + t] += g;
      }
    }
    __syncthreads();
    // 7. dZ1 = (dZ2 W2^T) gelu'(Z1)
    for (int i = t; i < TILE * H; i += GT) {
      const int r = i / H, k = i % H;
      float s = 0.f;
#pragma unroll 8
      for (int j = 0; j < H; j++) s = fmaf(z2[r * H + j], sw[OFF_W2 + k * H + j], s);
      z1[i] = s * gelu_grad(z1[i]);
    }
    __syncthreads();
    // 8. W1, b1 gradients
    for (int q = 0; q < 2; q++) {
      const int o = t + q * GT;
      if (o < F * H) {
        const int f = o / H, j = o % H;
        float g = 0.f;
        for (int r = 0; r < TILE; r++) g = fmaf(sx[r * F + f], z1[r * H + j], g);
        gW1[q] += g;
      }
    }
    if (t < H) {
      float g = 0.f;
      for (int r = 0; r < TILE; r++) g += z1[r * H + t];
      acc_b[t] += g;
    }
    __syncthreads();
  }
  // flush this CTA's gradients
  {
    const int j = t % H, k0 = (t / H) * 16;
#pragma unroll
    for (int k = 0; k < 16; k++) atomicAdd(&grad[OFF_W2 + (k0 + k) * H + j], gW2[k]);
    for (int q = 0; q < 2; q++) {
      const int o = t + q * GT;
      if (o < F * H) atomicAdd(&grad[OFF_W1 + o], gW1[q]);
    }
    if (t < H) {
      atomicAdd(&grad[OFF_B1 + t], acc_b[t]);
      atomicAdd(&grad[OFF_B2 + t], acc_b[H + t]);
      atomicAdd(&grad[OFF_W3 + t], acc_b[2 * H + 1 + t]);
    }
    if (t == 0) atomicAdd(&grad[OFF_B3], acc_b[2 * H]);
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xffffffffu, lsum, o);
    if ((t & 31) == 0 && loss) atomicAdd(loss, lsum * inv_n);
  }
}

__global__ void k_adam(float *w, __nv_bfloat16 *wb, float *m, float *v, const float *g, uint32_t P, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void k_to_bf16(const float *w, __nv_bfloat16 *wb, uint32_t P) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

// proposal weights: exp(s - max s) in units of 2^-24, at least 1
__global__ void k_max_score(const float *s, uint64_t n, unsigned int *mx) {
  float m = -INFINITY;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, s[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) {
    // order-preserving map of floats to unsigned ints
    unsigned int b = __float_as_uint(m);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
    atomicMax(mx, b);
  }
}
__global__ void k_score_weights(const float *s, uint64_t n, const unsigned int *mx, uint32_t *w) {
  unsigned int b = *mx;
  b = (b & 0x80000000u) ? (b & 0x7FFFFFFFu) : ~b;
  const float m = __uint_as_float(b);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const float e = expf(fminf(s[i] - m, 0.f)) * 16777216.0f;
    w[i] = e < 1.f ? 1u : (uint32_t)fminf(e, 16777216.0f);
  }
}

}  // namespace
}  // namespace bfc

using namespace bfc;

extern "C" {

int bfc_features(bfc_graph *g, float *feat, void *stream) {
  if (!g || !feat) return BFC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_features<<<ml_grid((uint64_t)g->nU * 32, 256), 256, 0, s>>>(ptr<uint64_t>(g->offU), ptr<uint32_t>(g->nbrU),
                                                                ptr<uint32_t>(g->degV), g->nU, 0.f, feat);
  BFC_LAUNCHED();
  k_features<<<ml_grid((uint64_t)g->nV * 32, 256), 256, 0, s>>>(ptr<uint64_t>(g->offV), ptr<uint32_t>(g->nbrV),
                                                                ptr<uint32_t>(g->degU), g->nV, 1.f,
                                                                feat + (uint64_t)g->nU * F);
  BFC_LAUNCHED();
  return BFC_OK;
}

int bfc_mlp_targets(const uint64_t *b, uint64_t n, float *t, void *stream) {
  if ((!b || !t) && n) return BFC_EINVAL;
  if (!n) return BFC_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_targets<<<ml_grid(n, 256), 256, 0, s>>>(b, n, t);
  BFC_LAUNCHED();
  return BFC_OK;
}

int bfc_mlp_forward(const uint16_t *w_bf16, const float *X, uint64_t n, float *y, void *stream) {
  if (!w_bf16 || ((!X || !y) && n)) return BFC_EINVAL;
  if (!n) return BFC_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_forward<<<ml_grid(n, 128, 152 * 8), 128, 0, s>>>(reinterpret_cast<const __nv_bfloat16 *>(w_bf16), X, n, y);
  BFC_LAUNCHED();
  return BFC_OK;
}

int bfc_mlp_grad(const uint16_t *w_bf16, const float *X, const float *T, const uint32_t *idx, uint64_t n,
                 float *grad, float *loss, void *stream) {
  if (!w_bf16 || !grad || ((!X || !T) && n)) return BFC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  BFC_CUDA_TRY(cudaMemsetAsync(grad, 0, NPARAM * sizeof(float), s));
  if (loss) BFC_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), s));
  if (!n) return BFC_OK;
  const size_t smem = (size_t)(NPARAM + 8 + TILE * F + 3 * TILE * H + TILE + 3 * H + 1) * sizeof(float) + 64;
  BFC_CUDA_TRY(cudaFuncSetAttribute(k_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const uint64_t tiles = (n + TILE - 1) / TILE;
  const unsigned grid = (unsigned)std::min<uint64_t>(tiles, 152);
  k_grad<<<grid, GT, smem, s>>>(reinterpret_cast<const __nv_bfloat16 *>(w_bf16), X, T, idx, n, 1.0f / (float)n,
                                grad, loss);
  BFC_LAUNCHED();
  return BFC_OK;
}

int bfc_mlp_adam(float *w, uint16_t *w_bf16, float *m, float *v, const float *grad, uint32_t P, float lr,
                 float beta1, float beta2, float eps, uint32_t step, void *stream) {
  if (!w || !w_bf16 || !m || !v || !grad || P != NPARAM || step == 0) return BFC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adam<<<ml_grid(P, 256), 256, 0, s>>>(w, reinterpret_cast<__nv_bfloat16 *>(w_bf16), m, v, grad, P, lr, beta1,
                                         beta2, eps, c1, c2);
  BFC_LAUNCHED();
  return BFC_OK;
}

int bfc_mlp_to_bf16(const float *w, uint16_t *w_bf16, uint32_t P, void *stream) {
  if (!w || !w_bf16 || P != NPARAM) return BFC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_to_bf16<<<ml_grid(P, 256), 256, 0, s>>>(w, reinterpret_cast<__nv_bfloat16 *>(w_bf16), P);
  BFC_LAUNCHED();
  return BFC_OK;
}

int bfc_proposal_from_scores(bfc_graph *g, const float *scores, void *stream, bfc_proposal **out) {
  if (!g || !scores || !out) return BFC_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const uint64_t n = (uint64_t)g->nU + g->nV;
  DBuf w, mx;
  int rc = dalloc(w, n * 4, s);
  if (!rc) rc = dalloc(mx, 16, s);
  if (!rc && cudaMemsetAsync(mx.p, 0, 4, s) != cudaSuccess) rc = BFC_ECUDA;
  if (!rc) {
    k_max_score<<<ml_grid(n, 256), 256, 0, s>>>(scores, n, ptr<unsigned int>(mx));
    count_launch();
    k_score_weights<<<ml_grid(n, 256), 256, 0, s>>>(scores, n, ptr<unsigned int>(mx), ptr<uint32_t>(w));
    count_launch();
    if (cudaGetLastError() != cudaSuccess) rc = BFC_ECUDA;
  }
  if (!rc) rc = bfc_proposal_from_weights(g, ptr<uint32_t>(w), BFC_INPUT_DEVICE, stream, out);
  dfree(w, s);
  dfree(mx, s);
  return rc;
}

}  // extern "C"
