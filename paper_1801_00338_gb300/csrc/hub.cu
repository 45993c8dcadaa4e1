// Hub-by-hub block of ExactBFC on the tensor cores (tcgen05).
//
// For start vertices v, w the multiplicity c(v, w) = |Gamma_v ^ Gamma_w| is
// the (v, w) entry of A A^T, A the 0/1 adjacency matrix of start rows against
// midpoint columns (Lemma 1, Eq. (2)-(3)).  Among the h highest-ranked start
// vertices ("hubs") this product is dense enough for a matrix engine:
//   - heavy columns (midpoints with >= tau hub neighbours) form a dense bf16
//     0/1 matrix A_H (h x K); the upper-triangle 128 x 128 tiles of
//     A_H A_H^T are computed by tcgen05.mma (kind::f16, fp32 accumulation in
//     tensor memory, exact because every entry is an integer below 2^24);
//   - light columns (2 <= hub neighbours < tau) add their hub pairs into an
//     int32 matrix C_L with atomics;
//   - the epilogue reads each accumulator tile, adds C_L and sums C(c, 2) over
//     the pairs i < j.
// A hub's later vertices (rank order) are all hubs, so the block counts every
// pair whose first vertex is a hub; the window kernels skip hub start vertices
// and count all other pairs as before.
#include <cuda.h>  // CUtensorMap and the tensor-map encoder's signature (reached through the runtime)

#include <algorithm>
#include <mutex>
#include <vector>

#include "bfc_internal.cuh"

namespace bfc {
namespace {

constexpr int TM = 128;          // tile rows / columns
constexpr int KC = 64;           // K elements per chunk (4 MMAs of K = 16)
constexpr int HB_THREADS = 128;  // one warpgroup
constexpr int SW = 4;            // tiles per strip at most: (ti, tj .. tj + 3) share the A_i chunk
constexpr int HB_PER_SM = 1;     // one CTA per SM: 4 x 128 TMEM columns, 2 x 80 KB of stages
constexpr uint64_t WAIT_NS = 1000000000ull;   // bounded waits give up after ~1 s
constexpr uint64_t DRAIN_NS = 2000000000ull;  // after giving up: the wait for work already issued
// the give-up limit of the next launches (bfc_set_wait_limit; 0: WAIT_NS)
static uint64_t g_wait_ns = 0;
constexpr uint32_t OP_BYTES = TM * KC * 2;                 // one 128 x 64 operand chunk, 16 KB
constexpr uint32_t STAGE_BYTES = (1 + SW) * OP_BYTES;      // A_i and up to four A_j chunks
constexpr size_t HB_SMEM = 2 * STAGE_BYTES + 1024;         // two stages, plus room to align them to 1 KB

unsigned hb_grid(uint64_t n, unsigned threads, unsigned cap = 152 * 16) {
  uint64_t g = (n + threads - 1) / threads;
  if (g > cap) g = cap;
  if (g == 0) g = 1;
  return (unsigned)g;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major operand layout with the 128-byte swizzle: a TMA box of 64 elements x
// 128 rows lands as 128 rows of 128 bytes, the 16-byte pieces of row r placed
// at piece ^ (r & 7); 8-row groups are 1,024 bytes apart (SBO), and the K step
// of 16 elements moves the descriptor's start by 32 bytes.  Operand bases are
// 1,024-byte aligned.
constexpr uint32_t LBO = 16, SBO = 1024;
constexpr uint32_t KSTEP_BYTES = 32;

// shared memory matrix descriptor (tcgen05): start, leading and stride byte
// offsets in 16-byte units, descriptor version 1, layout type 2 (128-byte swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// instruction descriptor: D fp32, A and B bf16, both K-major, M = N = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TM >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

// ---------------------------------------------------------------------------
// column split
// ---------------------------------------------------------------------------
// hub degree of every midpoint: its row (ascending ranks) ends with its hubs.
// The histogram of hub degrees >= 2 is gathered per block in shared memory
// (most columns have small hub degrees: one global bin would serialise).
constexpr uint32_t HIST = 4096;
__global__ void k_hub_degree(const uint64_t *offM, const uint32_t *mR, uint32_t nM, uint32_t hub0, uint32_t *hd,
                             unsigned int *hist) {
  __shared__ unsigned int sh[HIST];
  for (uint32_t i = threadIdx.x; i < HIST; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nM; x += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t lo = offM[x], hi = offM[x + 1];
    const uint64_t end = hi;
    while (lo < hi) {  // first entry with rank >= hub0
      const uint64_t mid = (lo + hi) / 2;
      if (mR[mid] < hub0) lo = mid + 1; else hi = mid;
    }
    const uint32_t d = (uint32_t)(end - lo);
    hd[x] = d;
    if (d >= 2) atomicAdd(&sh[d < HIST ? d : HIST - 1], 1u);
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < HIST; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

__global__ void k_heavy_list(const uint32_t *hd, uint32_t nM, uint32_t tau, unsigned int *count, uint32_t *cols) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nM; x += (uint64_t)gridDim.x * blockDim.x)
    if (hd[x] >= tau) cols[atomicAdd(count, 1u)] = (uint32_t)x;
}

// A_H[hub][k] = 1 for the hubs of heavy column k (one warp per column; the
// hubs are the suffix of the column's rank-sorted row)
__global__ void k_fill_dense(const uint64_t *offM, const uint32_t *mR, const uint32_t *hd, const uint32_t *cols,
                             uint32_t K, uint32_t Kp, uint32_t hub0, uint16_t *A) {
  const int lane = threadIdx.x & 31;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t k = warp; k < K; k += nw) {
    const uint32_t x = cols[k];
    const uint64_t e = offM[x + 1], b = e - hd[x];
    for (uint64_t i = b + lane; i < e; i += 32) A[(uint64_t)(mR[i] - hub0) * Kp + k] = 0x3F80;  // bf16 1.0
  }
}

// light columns: every hub pair (a < b) of the column adds one to C_L[b][a]
// (one warp per column: the first hub in turn, lanes over the second)
__global__ void k_light_pairs(const uint64_t *offM, const uint32_t *mR, const uint32_t *hd, uint32_t nM,
                              uint32_t tau, uint32_t hub0, uint32_t h, unsigned int *CL,
                              unsigned long long *npairs) {
  const int lane = threadIdx.x & 31;
  unsigned long long mine = 0;
  const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t x = warp; x < nM; x += nw) {
    const uint32_t d = hd[x];
    if (d < 2 || d >= tau) continue;
    const uint64_t e = offM[x + 1], b = e - d;  // the d hubs, ascending ranks
    mine += (uint64_t)d * (d - 1) / 2;
    for (uint32_t i = 0; i + 1 < d; i++) {
      const uint32_t a = mR[b + i] - hub0;
      for (uint32_t j = i + 1 + lane; j < d; j += 32) atomicAdd(&CL[(uint64_t)(mR[b + j] - hub0) * h + a], 1u);
    }
  }
  if (lane == 0 && mine) atomicAdd(npairs, mine);
}

// ---------------------------------------------------------------------------
// tensor-core tiles: C_ij = A_i A_j^T over upper-triangle tile pairs (ti <= tj)
// ---------------------------------------------------------------------------
// strip t: tile row ti and its first tile column tj0 (row ti has
// ceil((nt - ti) / sw) strips, tj0 = ti, ti + sw, ...)
__device__ __forceinline__ void strip_of(uint32_t t, uint32_t nt, uint32_t sw, uint32_t &ti, uint32_t &tj0) {
  uint32_t i = 0, rem = t;
  while (rem >= (nt - i + sw - 1) / sw) { rem -= (nt - i + sw - 1) / sw; i++; }
  ti = i;
  tj0 = i + rem * sw;
}

// Wait for phase `parity` of an mbarrier for at most limit_ns of global time;
// returns 1 when the phase completed.
__device__ __forceinline__ uint32_t mbar_wait_bounded(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
  uint64_t t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity));
    if (done) return 1;
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) return 0;
  }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// One CTA (one warpgroup) per SM, strips of up to four 128 x 128 tiles
// (ti, tj0 .. tj0 + 3) from a global queue; the four accumulators fill the
// SM's 512 TMEM columns.  Thread 0 runs the main loop: for each 64-wide K chunk
// it loads the A_i chunk and the strip's A_j chunks with TMA (one 64 x 128
// copy each) into one of two stages, issuing the next chunk's copies before
// the current chunk's MMAs so that loading and multiplying overlap; waits for
// them on the stage's `full` barrier; issues 4 x 4 MMAs of 128x128x16; and
// commits them to the stage's `empty` barrier, which frees the stage.  After
// the last chunk a commit to `done` releases the epilogue: the 4 warps read
// each accumulator (TMEM lane = tile row), add C_L and sum C(c, 2) over i < j.
// Every wait gives up after wait_ns: the CTA then stops issuing, sets
// DERR_TIMEOUT, waits (at most DRAIN_NS each) for the copies it issued and
// for its MMAs, and only then releases its tensor memory and exits.
__global__ void __launch_bounds__(HB_THREADS) k_hub_mma(const __grid_constant__ CUtensorMap amap, uint32_t Kp,
                                                        uint32_t h, const unsigned int *CL, unsigned int *queue,
                                                        unsigned long long *B, uint32_t *err, uint64_t wait_ns,
                                                        uint32_t sw) {
  extern __shared__ uint8_t hub_smem[];
  __shared__ __align__(8) uint64_t full[2], empty[2], done;
  __shared__ uint32_t tmem_holder, sh_item, sh_ok;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the stages start at the first 1 KB boundary of the dynamic buffer
  const uint32_t st0 = (smem_u32(hub_smem) + 1023u) & ~1023u;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                 "r"(sw * TM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int i = 0; i < 2; i++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[i])), "r"(1));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&done)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
    sh_ok = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t taddr = tmem_holder;
  const uint32_t nt = h / TM, nchunks = Kp / KC;
  uint32_t nitems = 0;
  for (uint32_t i = 0; i < nt; i++) nitems += (nt - i + sw - 1) / sw;
  uint32_t q = 0;      // chunks issued so far by this CTA (thread 0): stage q & 1, its use q >> 1
  uint32_t q_iss = 0;  // chunk copies issued (thread 0)
  uint32_t q_ful = 0;  // chunk copies waited for (thread 0): those in [q_ful, q_iss) may be in flight
  uint32_t nfin = 0;   // strips finished by this CTA
  unsigned long long acc = 0;
  // copy chunk c of the strip into the stage of chunk number qn
  auto issue = [&](uint32_t qn, uint32_t c, uint32_t ti, uint32_t tj0, uint32_t w) {
    const uint32_t stage = st0 + (qn & 1) * STAGE_BYTES, bar = smem_u32(&full[qn & 1]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((1 + w) * OP_BYTES));
    const int x = (int)(c * KC);
    tma_load_2d(stage, &amap, x, (int)(ti * TM), bar);
    for (uint32_t t = 0; t < w; t++) tma_load_2d(stage + (1 + t) * OP_BYTES, &amap, x, (int)((tj0 + t) * TM), bar);
  };
  while (true) {
    if (tid == 0) sh_item = sh_ok ? atomicAdd(queue, 1u) : nitems;
    __syncthreads();
    const uint32_t it = sh_item;
    if (it >= nitems) break;
    uint32_t ti, tj0;
    strip_of(it, nt, sw, ti, tj0);
    const uint32_t w = min(sw, nt - tj0);  // tiles in this strip
    if (tid == 0) {
      bool ok = true;
      if (q >= 2) ok = mbar_wait_bounded(smem_u32(&empty[q & 1]), ((q - 2) >> 1) & 1, wait_ns);
      if (ok) {
        issue(q, 0, ti, tj0, w);
        q_iss = q + 1;
      }
      for (uint32_t c = 0; c < nchunks && ok; c++) {
        const uint32_t qc = q + c;
        if (c + 1 < nchunks) {
          const uint32_t qn = qc + 1;  // its stage was last read by chunk qn - 2
          if (qn >= 2 && !mbar_wait_bounded(smem_u32(&empty[qn & 1]), ((qn - 2) >> 1) & 1, wait_ns)) {
            ok = false;
            break;
          }
          issue(qn, c + 1, ti, tj0, w);
          q_iss = qn + 1;
        }
        if (!mbar_wait_bounded(smem_u32(&full[qc & 1]), (qc >> 1) & 1, wait_ns)) { ok = false; break; }
        q_ful = qc + 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t stage = st0 + (qc & 1) * STAGE_BYTES;
#pragma unroll
        for (int k = 0; k < KC / 16; k++) {
          const uint64_t ad = smem_desc(stage + k * KSTEP_BYTES);
          const uint32_t accum = (c > 0 || k > 0) ? 1u : 0u;
          for (uint32_t t = 0; t < w; t++) {
            const uint64_t bd = smem_desc(stage + (1 + t) * OP_BYTES + k * KSTEP_BYTES);
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(taddr + t * TM),
                "l"(ad), "l"(bd), "r"(IDESC), "r"(accum));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(&empty[qc & 1])));
      }
      q += nchunks;
      // `done` completes when every MMA issued so far has finished
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&done)));
      if (!ok) {
        sh_ok = 0;
        atomicOr(err, DERR_TIMEOUT);
      }
    }
    const uint32_t fin = mbar_wait_bounded(smem_u32(&done), nfin & 1, wait_ns);
    nfin++;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (__syncthreads_and(fin) == 0 || !sh_ok) {
      if (tid == 0) {
        sh_ok = 0;
        atomicOr(err, DERR_TIMEOUT);
        // before the shared and tensor memory are released: the copies not
        // yet waited for (at most one per stage: a stage is refilled only
        // after its MMAs completed), then every MMA issued (the `done` phase
        // committed after them)
        for (uint32_t x = q_ful; x < q_iss; x++) mbar_wait_bounded(smem_u32(&full[x & 1]), (x >> 1) & 1, DRAIN_NS);
        mbar_wait_bounded(smem_u32(&done), (nfin - 1) & 1, DRAIN_NS);
        asm volatile("tcgen05.fence::after_thread_sync;");
      }
      __syncthreads();
      break;
    }
    // epilogue: row i of each tile is TMEM lane i; sum C(c, 2) over global i < j
    const uint32_t gi = ti * TM + 32 * warp + lane;
    for (uint32_t t = 0; t < w; t++) {
      const uint32_t tj = tj0 + t;
      for (int c0 = 0; c0 < TM; c0 += 8) {
        uint32_t r[8];
        const uint32_t ta = taddr + ((uint32_t)(32 * warp) << 16) + t * TM + (uint32_t)c0;
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
        for (int k = 0; k < 8; k++) {
          const uint32_t gj = tj * TM + c0 + k;
          if (gj <= gi) continue;
          // C_L is stored with the higher hub as the row: lanes (gi) read adjacent words
          const uint64_t c = (uint64_t)__uint_as_float(r[k]) + CL[(uint64_t)gj * h + gi];
          if (c > 1) acc += c * (c - 1) / 2;
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0 && acc) atomicAdd(B, acc);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(sw * TM));
}

__global__ void k_min_rank(const uint32_t *list, uint32_t n, unsigned int *out) {
  unsigned int mine = 0xFFFFFFFFu;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    mine = min(mine, list[i]);
  for (int o = 16; o > 0; o >>= 1) mine = min(mine, __shfl_down_sync(0xffffffffu, mine, o));
  if ((threadIdx.x & 31) == 0 && mine != 0xFFFFFFFFu) atomicMin(out, mine);
}

// cuTensorMapEncodeTiled, reached through the runtime's driver entry point
// (no link against the driver library)
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// tensor map of A_H (h rows of Kp bf16 values, row-major): boxes of 64
// elements x 128 rows, written to shared memory with the 128-byte swizzle
int hub_tensor_map(CUtensorMap *map, void *A, uint32_t h, uint32_t Kp) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return BFC_ECUDA;
  const cuuint64_t dims[2] = {Kp, h};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
  const cuuint32_t box[2] = {(cuuint32_t)KC, (cuuint32_t)TM};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A, dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? BFC_OK : BFC_ECUDA;
}

int sm_count_hub() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 152;
}

}  // namespace

// Automatic hub count: the smallest multiple of 128 whose top ranks hold every
// vertex of the big class (the start vertices whose wedge lists exceed the
// large windows' segment capacity: the walk's most expensive vertices), at
// most max_h; 0 when the class is empty.
int hub_auto_size(Plan &p, uint32_t max_h, uint32_t *h, cudaStream_t s) {
  constexpr int BIG = Plan::NCLS - 1;
  *h = 0;
  const uint32_t n = p.cls_count[BIG];
  if (n == 0 || p.nS < TM) return BFC_OK;
  DBuf out;
  BFC_TRY(dalloc(out, 4, s));
  unsigned int lo = 0xFFFFFFFFu;
  int rc = BFC_OK;
  if (cudaMemcpyAsync(out.p, &lo, 4, cudaMemcpyHostToDevice, s) != cudaSuccess) rc = BFC_ECUDA;
  if (!rc) {
    k_min_rank<<<hb_grid(n, 256, 152), 256, 0, s>>>(ptr<uint32_t>(p.cls) + p.cls_begin[BIG], n,
                                                     ptr<unsigned int>(out));
    count_launch();
    if (cudaMemcpyAsync(&lo, out.p, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = BFC_ECUDA;
  }
  dfree(out, s);
  if (rc) return rc;
  const uint64_t cover = (uint64_t)p.nS - lo;
  const uint64_t hh = std::min<uint64_t>((cover + TM - 1) / TM * TM, std::min<uint64_t>(max_h, p.nS) / TM * TM);
  *h = (uint32_t)hh;
  return BFC_OK;
}

// Count every pair of start vertices whose lower-ranked vertex is one of the
// top h ranks (both are then hubs), adding sum C(c, 2) to d_B.  h: a multiple
// of 128, <= nS.  tau: columns with >= tau hubs go to the dense product (0:
// chosen by a cost model).  stats (host, may be null, 4 entries): h, K (dense
// columns), tau, light pairs.
int hub_block_count(bfc_graph *g, Plan &p, uint32_t h, uint32_t tau, unsigned long long *d_B, uint64_t *stats,
                    cudaStream_t s) {
  if (h == 0 || h % TM || h > p.nS || tau == 1) return BFC_EINVAL;
  const uint32_t hub0 = p.nS - h, nM = p.nM;
  DBuf hd, hist, cnt, cols, A, CL;
  auto cleanup = [&]() { DBuf *bs[] = {&hd, &hist, &cnt, &cols, &A, &CL}; for (DBuf *b : bs) dfree(*b, s); };
  int rc = BFC_OK;
#define HB_TRY(x) do { rc = (x); if (rc) { cleanup(); return rc; } } while (0)
#define HB_CUDA(x) do { if ((x) != cudaSuccess) { cleanup(); return BFC_ECUDA; } } while (0)
  HB_TRY(dalloc(hd, (uint64_t)std::max<uint32_t>(nM, 1) * 4, s));
  HB_TRY(dalloc(cols, (uint64_t)std::max<uint32_t>(nM, 1) * 4, s));
  HB_TRY(dalloc(hist, HIST * 4, s));
  HB_TRY(dalloc(cnt, 32, s));
  HB_CUDA(cudaMemsetAsync(hist.p, 0, HIST * 4, s));
  HB_CUDA(cudaMemsetAsync(cnt.p, 0, 32, s));
  unsigned int *heavy_n = ptr<unsigned int>(cnt), *queue = heavy_n + 1;
  unsigned long long *light_n = reinterpret_cast<unsigned long long *>(ptr<unsigned int>(cnt) + 2);
  if (nM) {
    profile_begin("hub.degree", s);
    k_hub_degree<<<hb_grid(nM, 256, 152 * 4), 256, 0, s>>>(p.offM, ptr<uint32_t>(p.mR), nM, hub0, ptr<uint32_t>(hd),
                                                  ptr<unsigned int>(hist));
    count_launch();
    profile_end("hub.degree", s);
  }
  if (tau == 0) {
    // cost model: a dense column costs every tile its share of the tile
    // kernel (operand copies and MMAs, at the kernel's measured rate); a light
    // column costs C(d, 2) scattered atomics.  Columns lumped in the last bin
    // stay dense.
    std::vector<unsigned int> hh(HIST);
    HB_CUDA(cudaMemcpyAsync(hh.data(), hist.p, HIST * 4, cudaMemcpyDeviceToHost, s));
    HB_CUDA(cudaStreamSynchronize(s));
    const double tiles = (double)(h / TM) * (h / TM + 1) / 2;
    const double per_col = tiles * 4.0e-11;  // measured: 7.7 ms for 8,256 tiles x 22,974 columns
    const double per_pair = 1.0 / 1.1e11;    // measured: 1.07 ms for 1.19e8 light pairs
    std::vector<double> cols_ge(HIST + 1, 0.0), pairs_lt(HIST + 1, 0.0);
    for (int d = HIST - 1; d >= 0; d--) cols_ge[d] = cols_ge[d + 1] + hh[d];
    for (uint32_t d = 1; d <= HIST; d++) pairs_lt[d] = pairs_lt[d - 1] + (double)hh[d - 1] * (d - 1) * (d - 2) / 2.0;
    double best = 1e300;
    tau = HIST - 1;
    for (uint32_t t = 2; t < HIST; t++) {
      if (cols_ge[t] > 65536.0) continue;  // A_H stays within h x 65,536 x 2 bytes
      const double cost = cols_ge[t] * per_col + pairs_lt[t] * per_pair;
      if (cost < best) { best = cost; tau = t; }
    }
  }
  if (nM) {
    k_heavy_list<<<hb_grid(nM, 256), 256, 0, s>>>(ptr<uint32_t>(hd), nM, tau, heavy_n, ptr<uint32_t>(cols));
    count_launch();
  }
  unsigned int K = 0;
  HB_CUDA(cudaMemcpyAsync(&K, heavy_n, 4, cudaMemcpyDeviceToHost, s));
  HB_CUDA(cudaStreamSynchronize(s));
  const uint32_t Kp = std::max<uint32_t>(KC, (K + KC - 1) / KC * KC);
  HB_TRY(dalloc(A, (uint64_t)h * Kp * 2, s));
  HB_TRY(dalloc(CL, (uint64_t)h * h * 4, s));
  HB_CUDA(cudaMemsetAsync(A.p, 0, (uint64_t)h * Kp * 2, s));
  HB_CUDA(cudaMemsetAsync(CL.p, 0, (uint64_t)h * h * 4, s));
  if (K) {
    k_fill_dense<<<hb_grid((uint64_t)K * 32, 256), 256, 0, s>>>(p.offM, ptr<uint32_t>(p.mR), ptr<uint32_t>(hd),
                                                                ptr<uint32_t>(cols), K, Kp, hub0, ptr<uint16_t>(A));
    count_launch();
  }
  if (nM) {
    profile_begin("hub.light", s);
    k_light_pairs<<<hb_grid((uint64_t)nM * 32, 256), 256, 0, s>>>(p.offM, ptr<uint32_t>(p.mR), ptr<uint32_t>(hd),
                                                                  nM, tau, hub0, h, ptr<unsigned int>(CL), light_n);
    count_launch();
    profile_end("hub.light", s);
  }
  // strips of four tiles, or of two (or one) when four would leave more than
  // half of the SMs idle (narrower strips reload the shared A_i chunk more
  // often: at 3,840 hubs, 240 two-tile strips measured 0.65 ms against 0.39
  // for 128 four-tile strips)
  const uint64_t sms = (uint64_t)sm_count_hub() * HB_PER_SM;
  uint32_t sw = SW;
  uint64_t nitems = 0;
  for (;; sw >>= 1) {
    nitems = 0;
    for (uint32_t i = 0; i < h / TM; i++) nitems += (h / TM - i + sw - 1) / sw;
    if (2 * nitems >= sms || sw == 1) break;
  }
  const unsigned grid = (unsigned)std::min<uint64_t>(sms, nitems);
  CUtensorMap amap;
  HB_TRY(hub_tensor_map(&amap, A.p, h, Kp));
  HB_CUDA(cudaFuncSetAttribute(k_hub_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HB_SMEM));
  profile_begin("hub.total", s);
  k_hub_mma<<<grid, HB_THREADS, HB_SMEM, s>>>(amap, Kp, h, ptr<unsigned int>(CL), queue, d_B, ptr<uint32_t>(g->err),
                                              g_wait_ns ? g_wait_ns : WAIT_NS, sw);
  count_launch();
  profile_end("hub.total", s);
  HB_CUDA(cudaGetLastError());
  unsigned long long lp = 0;
  HB_CUDA(cudaMemcpyAsync(&lp, light_n, 8, cudaMemcpyDeviceToHost, s));
  HB_CUDA(cudaStreamSynchronize(s));  // the temporaries are freed below
  if (stats) {
    stats[0] = h;
    stats[1] = K;
    stats[2] = tau;
    stats[3] = lp;
  }
  cleanup();
#undef HB_TRY
#undef HB_CUDA
  return BFC_OK;
}

}  // namespace bfc

extern "C" int bfc_set_wait_limit(uint64_t ns) {
  bfc::g_wait_ns = ns;
  return BFC_OK;
}
