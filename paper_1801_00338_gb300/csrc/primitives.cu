// Device primitives: exclusive scan and a stable LSD radix sort.
// Written for sm_103a: 256-thread blocks, warp shuffles, __match_any_sync for
// stable in-warp ranking.  Used only for graph preparation.
#include <stdio.h>
#include <string.h>

#include <map>
#include <atomic>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "bfc_internal.cuh"

namespace bfc {

static __thread uint64_t g_launches_tls = 0;
static uint64_t g_launches = 0;

void note_cuda_error(cudaError_t e, const char *what, const char *file, int line) {
  if (getenv("BFC_DEBUG")) fprintf(stderr, "bfc: %s failed: %s (%s:%d)\n", what, cudaGetErrorString(e), file, line);
}
void count_launch(uint64_t n) {
  g_launches_tls += n;
  __atomic_add_fetch(&g_launches, n, __ATOMIC_RELAXED);
}
uint64_t launches_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

// ---------------------------------------------------------------------------
// kernel timing with CUDA events (enabled on request)
// ---------------------------------------------------------------------------
namespace {
struct ProfEntry {
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> done;
  cudaEvent_t open = nullptr;
};
std::mutex g_prof_mu;
std::map<std::string, ProfEntry> g_prof;
bool g_prof_on = false;
}  // namespace

bool profile_on() { return g_prof_on; }
void profile_begin(const char *tag, cudaStream_t s) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfEntry &e = g_prof[tag];
  if (cudaEventCreate(&e.open) != cudaSuccess) { e.open = nullptr; return; }
  cudaEventRecord(e.open, s);
}
void profile_end(const char *tag, cudaStream_t s) {
  if (!g_prof_on) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  ProfEntry &e = g_prof[tag];
  if (!e.open) return;
  cudaEvent_t end;
  if (cudaEventCreate(&end) != cudaSuccess) return;
  cudaEventRecord(end, s);
  e.done.emplace_back(e.open, end);
  e.open = nullptr;
}

// The library's own stream-ordered memory pool on each device, which keeps
// the memory it is given back (release threshold: unlimited) so that the
// next call's allocations reuse it instead of mapping new pages;
// bfc_trim_memory hands it back.
constexpr int MAX_DEVICES = 64;
static cudaMemPool_t g_pools[MAX_DEVICES];
static std::mutex g_pool_mu;
static int lib_pool(cudaMemPool_t *pool) {
  int dev = 0;
  BFC_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return BFC_EINTERNAL;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t p = nullptr;
    BFC_CUDA_TRY(cudaMemPoolCreate(&p, &props));
    uint64_t keep = ~0ull;
    BFC_CUDA_TRY(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
    g_pools[dev] = p;
  }
  *pool = g_pools[dev];
  return BFC_OK;
}

// Injected allocation failure (bfc_fail_alloc_after): the number of device
// allocations that still succeed before one fails; negative: none fails.
static std::atomic<long long> g_fail_after{-1};

int dalloc(DBuf &b, size_t bytes, cudaStream_t s) {
  if (b.p && b.bytes >= bytes) return BFC_OK;
  for (long long f = g_fail_after.load(); f >= 0;) {
    if (f == 0) {
      if (g_fail_after.compare_exchange_weak(f, -1)) return BFC_ENOMEM;
    } else if (g_fail_after.compare_exchange_weak(f, f - 1)) {
      break;
    }
  }
  dfree(b, s);
  if (bytes == 0) bytes = 16;
  cudaMemPool_t pool = nullptr;
  BFC_TRY(lib_pool(&pool));
  void *p = nullptr;  // b stays empty if the allocation fails
  BFC_CUDA_TRY(cudaMallocFromPoolAsync(&p, bytes, pool, s));
  b.p = p;
  b.bytes = bytes;
  return BFC_OK;
}
void dfree(DBuf &b, cudaStream_t s) {
  if (b.p) cudaFreeAsync(b.p, s);
  b.p = nullptr;
  b.bytes = 0;
}
int Scratch::reserve(size_t bytes, cudaStream_t s) {
  if (buf.bytes >= bytes) return BFC_OK;
  return dalloc(buf, bytes + bytes / 4, s);
}

int bits_for(uint64_t v) {
  int b = 0;
  while (v) { b++; v >>= 1; }
  return b;
}

static inline uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------------------
// scan
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <class In>
__global__ void k_scan_reduce(const In *in, uint64_t n, uint64_t *partial) {
  uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; i++) {
    uint64_t idx = base + (uint64_t)i * SCAN_THREADS + threadIdx.x;
    if (idx < n) s += (uint64_t)in[idx];
  }
  // block reduce
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  __shared__ uint64_t ws[SCAN_THREADS / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; w++) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

// single block: exclusive scan of partial[0..nb) in place; partial[nb] = total
__global__ void k_scan_partials(uint64_t *partial, uint64_t nb) {
  __shared__ uint64_t wsum[SCAN_THREADS / 32];
  __shared__ uint64_t carry_s;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_s = 0;
  __syncthreads();
  for (uint64_t base = 0; base < nb; base += SCAN_THREADS) {
    uint64_t idx = base + threadIdx.x;
    uint64_t x = idx < nb ? partial[idx] : 0;
    uint64_t inc = warp_inclusive_scan(x);
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t r = 0;
      for (int w = 0; w < SCAN_THREADS / 32; w++) { uint64_t t = wsum[w]; wsum[w] = r; r += t; }
    }
    __syncthreads();
    uint64_t c = carry_s;
    uint64_t ex = c + wsum[warp] + inc - x;
    if (idx < nb) partial[idx] = ex;
    __syncthreads();
    if (threadIdx.x == SCAN_THREADS - 1) carry_s = ex + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[nb] = carry_s;
}

template <class In>
__global__ void k_scan_down(const In *in, uint64_t *out, uint64_t n, const uint64_t *partial, uint64_t nb) {
  // each thread owns SCAN_ITEMS consecutive elements
  uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
  uint64_t v[SCAN_ITEMS];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; i++) {
    uint64_t idx = base + i;
    v[i] = idx < n ? (uint64_t)in[idx] : 0;
    s += v[i];
  }
  __shared__ uint64_t wsum[SCAN_THREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = warp_inclusive_scan(s);
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t r = 0;
    for (int w = 0; w < SCAN_THREADS / 32; w++) { uint64_t t = wsum[w]; wsum[w] = r; r += t; }
  }
  __syncthreads();
  uint64_t run = partial[blockIdx.x] + wsum[warp] + inc - s;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; i++) {
    uint64_t idx = base + i;
    if (idx < n) out[idx] = run;
    run += v[i];
  }
  if (blockIdx.x == nb - 1 && threadIdx.x == 0) out[n] = partial[nb];
}

template <class In>
static int scan_impl(const In *in, uint64_t *out, uint64_t n, Scratch &scr, cudaStream_t s) {
  uint64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nb == 0) {
    BFC_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
    return BFC_OK;
  }
  BFC_TRY(scr.reserve((nb + 1) * sizeof(uint64_t), s));
  uint64_t *partial = static_cast<uint64_t *>(scr.base());
  k_scan_reduce<In><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n, partial);
  BFC_LAUNCHED();
  k_scan_partials<<<1, SCAN_THREADS, 0, s>>>(partial, nb);
  BFC_LAUNCHED();
  k_scan_down<In><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, n, partial, nb);
  BFC_LAUNCHED();
  return BFC_OK;
}

int exclusive_scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n, Scratch &scr, cudaStream_t s) {
  return scan_impl<uint32_t>(in, out, n, scr, s);
}
int exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, Scratch &scr, cudaStream_t s) {
  return scan_impl<uint64_t>(in, out, n, scr, s);
}

// ---------------------------------------------------------------------------
// reduce
// ---------------------------------------------------------------------------
__global__ void k_reduce_add_u64(const uint64_t *in, uint64_t n, unsigned long long *out) {
  uint64_t s = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    s += in[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, (unsigned long long)s);
}
int reduce_add_u64(const uint64_t *in, uint64_t n, unsigned long long *out, cudaStream_t s) {
  if (n == 0) return BFC_OK;
  unsigned blocks = (unsigned)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_reduce_add_u64<<<blocks, 256, 0, s>>>(in, n, out);
  BFC_LAUNCHED();
  return BFC_OK;
}

// ---------------------------------------------------------------------------
// radix sort: 8-bit digits, 256 threads, 8 items per thread (2048 per block);
// warp w of a block owns the contiguous run [w*256, (w+1)*256) of the tile.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 8;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

template <class K>
__global__ void k_rs_hist(const K *keys, uint64_t n, int shift, uint32_t *hist, uint32_t nb) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  uint64_t base = (uint64_t)blockIdx.x * RS_TILE;
#pragma unroll
  for (int i = 0; i < RS_ITEMS; i++) {
    uint64_t idx = base + (uint64_t)i * RS_THREADS + threadIdx.x;
    if (idx < n) atomicAdd(&cnt[(uint32_t)(keys[idx] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(uint64_t)threadIdx.x * nb + blockIdx.x] = cnt[threadIdx.x];
}

// Scatter one tile: rank every element within its digit (warp match + per-warp
// digit counters), stage the tile in shared memory in digit order, then write
// each digit's run to its global position with consecutive threads writing
// consecutive addresses.
template <class K>
__global__ void k_rs_scatter(const K *keys, const uint32_t *vals, K *kout, uint32_t *vout, uint64_t n, int shift,
                             const uint64_t *offs, uint32_t nb) {
  __shared__ uint32_t wcnt[RS_WARPS][256];
  __shared__ uint64_t gbase[256];
  __shared__ uint32_t lstart[256];     // start of each digit's run in the staged tile
  __shared__ uint32_t wsum[RS_WARPS];
  __shared__ K sk[RS_TILE];
  __shared__ uint32_t sv[RS_TILE];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const uint64_t tile0 = (uint64_t)blockIdx.x * RS_TILE;
  const uint64_t base = tile0 + (uint64_t)warp * (32 * RS_ITEMS);
  K k[RS_ITEMS];
  uint32_t v[RS_ITEMS];
  uint32_t d[RS_ITEMS];
#pragma unroll
  for (int j = 0; j < RS_ITEMS; j++) {
    const uint64_t idx = base + (uint64_t)j * 32 + lane;
    const bool ok = idx < n;
    k[j] = ok ? keys[idx] : (K)0;
    v[j] = (ok && vals) ? vals[idx] : 0u;
    d[j] = ok ? ((uint32_t)(k[j] >> shift) & 255u) : 256u;
    if (ok) atomicAdd(&wcnt[warp][d[j]], 1u);
  }
  __syncthreads();
  {
    // thread t owns digit t: per-warp offsets within the digit, then the
    // digit's start in the tile (exclusive scan over digits)
    const uint32_t t = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; w++) {
      const uint32_t c = wcnt[w][t];
      wcnt[w][t] = run;
      run += c;
    }
    gbase[t] = offs[(uint64_t)t * nb + blockIdx.x];
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; w++) before += wsum[w];
    lstart[t] = before + incl - run;
  }
  __syncthreads();
  const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
  for (int j = 0; j < RS_ITEMS; j++) {
    const uint32_t peers = __match_any_sync(0xffffffffu, d[j]);
    const uint32_t rank = __popc(peers & lt);
    uint32_t lp = 0;
    if (d[j] < 256u) lp = lstart[d[j]] + wcnt[warp][d[j]] + rank;
    __syncwarp();
    if (d[j] < 256u && rank == 0) wcnt[warp][d[j]] += __popc(peers);
    __syncwarp();
    if (d[j] < 256u) {
      sk[lp] = k[j];
      sv[lp] = v[j];
    }
  }
  __syncthreads();
  const uint32_t cnt = (uint32_t)((n - tile0) < (uint64_t)RS_TILE ? (n - tile0) : (uint64_t)RS_TILE);
  for (uint32_t i = threadIdx.x; i < cnt; i += RS_THREADS) {
    const K key = sk[i];
    const uint32_t dg = (uint32_t)(key >> shift) & 255u;
    const uint64_t pos = gbase[dg] + (i - lstart[dg]);
    kout[pos] = key;
    if (vout) vout[pos] = sv[i];
  }
}

template <class K>
static int radix_sort_impl(const K *keys_in, K *keys_out, const uint32_t *vals_in, uint32_t *vals_out, uint64_t n,
                           int end_bit, Scratch &scr, cudaStream_t s) {
  if (n == 0) return BFC_OK;
  int passes = (end_bit + 7) / 8;
  if (passes == 0) {
    if (keys_out != keys_in) BFC_CUDA_TRY(cudaMemcpyAsync(keys_out, keys_in, n * sizeof(K), cudaMemcpyDeviceToDevice, s));
    if (vals_in && vals_out != vals_in)
      BFC_CUDA_TRY(cudaMemcpyAsync(vals_out, vals_in, n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    return BFC_OK;
  }
  uint32_t nb = (uint32_t)((n + RS_TILE - 1) / RS_TILE);
  uint64_t hist_n = (uint64_t)256 * nb;
  // scratch layout: hist u32[hist_n] | offs u64[hist_n+1] | scan partials | tmp keys | tmp vals
  uint64_t o_hist = 0;
  uint64_t o_offs = align_up(o_hist + hist_n * 4, 256);
  uint64_t o_part = align_up(o_offs + (hist_n + 1) * 8, 256);
  uint64_t part_bytes = ((hist_n + SCAN_TILE - 1) / SCAN_TILE + 1) * 8;
  uint64_t o_tk = align_up(o_part + part_bytes, 256);
  uint64_t o_tv = align_up(o_tk + n * sizeof(K), 256);
  uint64_t total = align_up(o_tv + (vals_in ? n * 4 : 0), 256);
  BFC_TRY(scr.reserve(total, s));
  char *sb = static_cast<char *>(scr.base());
  uint32_t *hist = reinterpret_cast<uint32_t *>(sb + o_hist);
  uint64_t *offs = reinterpret_cast<uint64_t *>(sb + o_offs);
  uint64_t *part = reinterpret_cast<uint64_t *>(sb + o_part);
  K *tk = reinterpret_cast<K *>(sb + o_tk);
  uint32_t *tv = vals_in ? reinterpret_cast<uint32_t *>(sb + o_tv) : nullptr;

  const K *src_k = keys_in;
  const uint32_t *src_v = vals_in;
  for (int p = 0; p < passes; p++) {
    bool to_out = ((passes - 1 - p) % 2) == 0;
    K *dst_k = to_out ? keys_out : tk;
    uint32_t *dst_v = vals_in ? (to_out ? vals_out : tv) : nullptr;
    int shift = 8 * p;
    k_rs_hist<K><<<nb, RS_THREADS, 0, s>>>(src_k, n, shift, hist, nb);
    BFC_LAUNCHED();
    // exclusive scan of the digit-major histogram (uses its own partial area)
    {
      uint64_t snb = (hist_n + SCAN_TILE - 1) / SCAN_TILE;
      k_scan_reduce<uint32_t><<<(unsigned)snb, SCAN_THREADS, 0, s>>>(hist, hist_n, part);
      BFC_LAUNCHED();
      k_scan_partials<<<1, SCAN_THREADS, 0, s>>>(part, snb);
      BFC_LAUNCHED();
      k_scan_down<uint32_t><<<(unsigned)snb, SCAN_THREADS, 0, s>>>(hist, offs, hist_n, part, snb);
      BFC_LAUNCHED();
    }
    k_rs_scatter<K><<<nb, RS_THREADS, 0, s>>>(src_k, src_v, dst_k, dst_v, n, shift, offs, nb);
    BFC_LAUNCHED();
    src_k = dst_k;
    src_v = dst_v;
  }
  return BFC_OK;
}

int radix_sort_u64(const uint64_t *keys_in, uint64_t *keys_out, const uint32_t *vals_in, uint32_t *vals_out,
                   uint64_t n, int end_bit, Scratch &scr, cudaStream_t s) {
  return radix_sort_impl<uint64_t>(keys_in, keys_out, vals_in, vals_out, n, end_bit, scr, s);
}
int radix_sort_u32(const uint32_t *keys_in, uint32_t *keys_out, const uint32_t *vals_in, uint32_t *vals_out,
                   uint64_t n, int end_bit, Scratch &scr, cudaStream_t s) {
  return radix_sort_impl<uint32_t>(keys_in, keys_out, vals_in, vals_out, n, end_bit, scr, s);
}

}  // namespace bfc

extern "C" {
uint64_t bfc_launch_count(void) { return bfc::launches_total(); }

int bfc_fail_alloc_after(int64_t n) {
  bfc::g_fail_after.store(n < 0 ? -1 : (long long)n);
  return BFC_OK;
}

int bfc_trim_memory(void) {
  std::lock_guard<std::mutex> lk(bfc::g_pool_mu);
  for (int d = 0; d < bfc::MAX_DEVICES; d++) {
    if (!bfc::g_pools[d]) continue;
    if (cudaDeviceSynchronize() != cudaSuccess) return BFC_ECUDA;
    if (cudaMemPoolTrimTo(bfc::g_pools[d], 0) != cudaSuccess) return BFC_ECUDA;
  }
  return BFC_OK;
}

int bfc_profile_enable(int on) {
  bfc::g_prof_on = on != 0;
  return BFC_OK;
}

int bfc_profile_reset(void) {
  std::lock_guard<std::mutex> lk(bfc::g_prof_mu);
  for (auto &kv : bfc::g_prof) {
    for (auto &pr : kv.second.done) {
      cudaEventSynchronize(pr.second);
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    if (kv.second.open) cudaEventDestroy(kv.second.open);
  }
  bfc::g_prof.clear();
  return BFC_OK;
}

int bfc_profile_read(const char *tag, uint64_t *launches, double *total_ms) {
  if (!tag) return BFC_EINVAL;
  std::lock_guard<std::mutex> lk(bfc::g_prof_mu);
  uint64_t n = 0;
  double ms = 0.0;
  auto it = bfc::g_prof.find(tag);
  if (it != bfc::g_prof.end()) {
    for (auto &pr : it->second.done) {
      if (cudaEventSynchronize(pr.second) != cudaSuccess) return BFC_ECUDA;
      float t = 0.f;
      if (cudaEventElapsedTime(&t, pr.first, pr.second) != cudaSuccess) return BFC_ECUDA;
      ms += t;
      n++;
    }
  }
  if (launches) *launches = n;
  if (total_ms) *total_ms = ms;
  return BFC_OK;
}
}  // extern "C"
