// Internal declarations of the butterfly-counting library (not installed).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/bfc.h"

namespace bfc {

// ---------------------------------------------------------------------------
// status handling
// ---------------------------------------------------------------------------
struct Status {
  int code = BFC_OK;
  bool ok() const { return code == BFC_OK; }
};

#define BFC_CUDA_TRY(expr)                                        \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) {                                      \
      bfc::note_cuda_error(_e, #expr, __FILE__, __LINE__);        \
      return (_e == cudaErrorMemoryAllocation) ? BFC_ENOMEM : BFC_ECUDA; \
    }                                                             \
  } while (0)

#define BFC_TRY(expr)          \
  do {                         \
    int _rc = (expr);          \
    if (_rc != BFC_OK) return _rc; \
  } while (0)

void note_cuda_error(cudaError_t e, const char *what, const char *file, int line);

// Optional event timing of kernel launches (see bfc_profile_* in bfc.h).
bool profile_on();
void profile_begin(const char *tag, cudaStream_t s);  // record the start event
void profile_end(const char *tag, cudaStream_t s);    // record the end event
void count_launch(uint64_t n = 1);

// Check the launch that was just made.
#define BFC_LAUNCHED()                     \
  do {                                     \
    bfc::count_launch();                   \
    BFC_CUDA_TRY(cudaGetLastError());      \
  } while (0)

// ---------------------------------------------------------------------------
// device-side error word: kernels set bits, the host reads it after a call
// ---------------------------------------------------------------------------
enum DeviceError : uint32_t {
  DERR_NONE = 0,
  DERR_RANGE = 1u << 0,      // an id out of range
  DERR_DUP = 1u << 1,        // a duplicate edge
  DERR_CAPACITY = 1u << 2,   // a table ran out of room (internal consistency)
  DERR_TIMEOUT = 1u << 3,    // a bounded wait gave up
  DERR_OVERFLOW = 1u << 4,   // a counter would have wrapped
  DERR_INVALID = 1u << 5,    // malformed input rows (order, offsets, edge ids)
};

// ---------------------------------------------------------------------------
// stream-ordered device buffers
// ---------------------------------------------------------------------------
struct DBuf {
  void *p = nullptr;
  size_t bytes = 0;
};
int dalloc(DBuf &b, size_t bytes, cudaStream_t s);
void dfree(DBuf &b, cudaStream_t s);
template <class T>
T *ptr(const DBuf &b) { return static_cast<T *>(b.p); }

// Scratch arena grown on demand (stream ordered), used by one call at a time.
struct Scratch {
  DBuf buf;
  int reserve(size_t bytes, cudaStream_t s);
  void *base() const { return buf.p; }
};

// ---------------------------------------------------------------------------
// primitives (primitives.cu)
// ---------------------------------------------------------------------------
// Exclusive scan of n values into out[0..n] (out[n] = total).  in may alias out
// only if it is not used afterwards.
int exclusive_scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n, Scratch &scr, cudaStream_t s);
int exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, Scratch &scr, cudaStream_t s);

// Stable LSD radix sort of (key, value) pairs over key bits [0, end_bit).
// Buffers: keys/vals are double buffers; the result ends in *_out after the
// call (the functions ping-pong internally and copy when needed).
int radix_sort_u64(const uint64_t *keys_in, uint64_t *keys_out, const uint32_t *vals_in, uint32_t *vals_out,
                   uint64_t n, int end_bit, Scratch &scr, cudaStream_t s);
int radix_sort_u32(const uint32_t *keys_in, uint32_t *keys_out, const uint32_t *vals_in, uint32_t *vals_out,
                   uint64_t n, int end_bit, Scratch &scr, cudaStream_t s);

int bits_for(uint64_t max_value);  // number of bits to represent max_value (0 -> 0)

// sum of a u64 array into one device word (added to *out)
int reduce_add_u64(const uint64_t *in, uint64_t n, unsigned long long *out, cudaStream_t s);

// ---------------------------------------------------------------------------
// graph (graph.cu)
// ---------------------------------------------------------------------------
// Per-start-side layout for wedge aggregation ("plan").  Start vertices are
// renumbered by rank: ascending degree, ties by id.  The total order "w after
// v" of Algorithm 1's coloured line is rank(w) > rank(v).
struct Plan {
  bool built = false;
  int side = 0;          // 0: U starts, 1: V starts
  uint32_t nS = 0, nM = 0;
  uint64_t m = 0;
  DBuf vert_of;          // u32[nS]  vertex id at rank r
  DBuf rank_of;          // u32[nS]  rank of vertex id
  DBuf offR;             // u64[nS+1] start rows in rank order
  DBuf sX;               // u32[m]   midpoint of each start-row entry
  DBuf sEid;             // u32[m]   canonical id of that edge
  DBuf sB;               // u32[m]   index in mR just after this edge (suffix begin)
  DBuf mR;               // u32[m]   midpoint rows (offsets offM): start ranks, ascending
  DBuf mEid;             // u32[m]   canonical id of each midpoint-row entry
  const uint64_t *offM = nullptr;  // midpoint row offsets (the graph's, or offM_own)
  DBuf offM_own;         // u64[nM+1] for a filtered (sparsified) plan
  DBuf work;             // u64[nS]  ordered wedges walked from each start rank
  // vertex classes (ranks), see wedge.cu
  DBuf cls;              // u32[nS]  ranks grouped by class
  static constexpr int NCLS = 13;     // skip, warp, 5 small windows, 5 large windows, big (wedge.cu)
  uint32_t cls_count[NCLS] = {};
  uint32_t cls_begin[NCLS] = {};
  uint64_t cls_work[NCLS] = {};       // wedges walked per class
  uint64_t cls_rows[NCLS] = {};       // start-row entries per class
  uint32_t big_seg_cap = 0;           // segment capacity of the big class
  // class limits the classification was made with (bfc_tuning's
  // warp_max_wedges and small_max_segs; wedge.cu caps them)
  uint32_t warp_max = 512, small_max = 128;
  uint64_t total_work = 0;     // sum of work = W of the midpoint side
  uint32_t max_deg_S = 0;
};

}  // namespace bfc

struct bfc_graph {
  uint32_t nU = 0, nV = 0;
  uint64_t m = 0;
  bfc::DBuf offU, nbrU;        // u64[nU+1], u32[m] (canonical order)
  bfc::DBuf offV, nbrV, eidV;  // u64[nV+1], u32[m], u32[m]
  bfc::DBuf degU, degV;        // u32
  uint64_t sqU = 0, sqV = 0, wU = 0, wV = 0;
  uint32_t maxU = 0, maxV = 0;
  bfc::Plan plan[2];
  bfc::Scratch scr;
  bfc::DBuf beM;               // u64[m]  per-edge partial sums in midpoint-row order
  bfc::DBuf err;               // u32 device error word
  bfc::DBuf acc;               // u64 accumulators (small)
  bfc_tuning tune = {};        // scheduling settings (bfc_set_tuning; 0 = default)
  // optional group of every U vertex (device, borrowed): the U-side plan then
  // ranks by (group, degree, id), so each group's start vertices hold
  // consecutive ranks and their wedge targets stay within them (a disjoint
  // union of graphs, one group per graph)
  const uint32_t *rank_group = nullptr;
  uint32_t rank_group_max = 0;
  cudaStream_t last_stream = nullptr;
};

namespace bfc {
int graph_build(bfc_graph *g, const uint32_t *u, const uint32_t *v, uint64_t m, uint32_t flags, cudaStream_t s);
// The same graph from caller-owned device rows (copied and checked); eidV may be null.
int graph_from_rows(bfc_graph *g, const uint64_t *offU, const uint32_t *nbrU, const uint64_t *offV,
                    const uint32_t *nbrV, const uint32_t *eidV, cudaStream_t s);
int plan_build(bfc_graph *g, int side, cudaStream_t s);
int choose_side(const bfc_graph *g, uint32_t flags);
int read_device_error(bfc_graph *g, cudaStream_t s);  // maps DERR_* bits to a status and clears

// wedge.cu
enum Mode { MODE_TOTAL = 0, MODE_EDGE = 1, MODE_SINGLE = 2, MODE_LOCAL = 3 };
// Counts with the start side of plan p (Algorithm 1's order, each pair once).
// d_B receives B (device u64).  MODE_EDGE also adds b_e to be (device,
// canonical ids, zeroed by the caller); MODE_TOTAL ignores be.
int wedge_count(bfc_graph *g, Plan &p, Mode mode, unsigned long long *d_B, uint64_t *be, cudaStream_t s);
// TOTAL mode on a disjoint union: also adds each start vertex's pair sum to
// gB[grp_of_rank[rank]].
int wedge_count_groups(bfc_graph *g, Plan &p, const uint32_t *grp_of_rank, unsigned long long *gB,
                       unsigned long long *d_B, cudaStream_t s);
int plan_classify(bfc_graph *g, Plan &p, cudaStream_t s);
// ESpar (kind 0, keep threshold thr) or ClrSpar (kind 1, colors) trials
// 0 .. trials - 1 of the sequence seeded by seed; beta: host (trials.cu)
int run_trials(bfc_graph *g, int kind, uint64_t seed, uint32_t thr, uint32_t colors, uint32_t trials, uint64_t *beta,
               cudaStream_t s);
// b_x = 1/2 sum of b_e over the rows off[x] .. off[x+1] (Lemma 1's identity
// for one vertex); eid: canonical id of each row entry, or null for identity.
int vertex_from_edges(const uint64_t *off, uint32_t n, const uint32_t *eid, const uint64_t *be, uint64_t *out,
                      cudaStream_t s);
// TOTAL mode over start ranks < rank_end only (ranks >= rank_end walk nothing).
int wedge_count_below(bfc_graph *g, Plan &p, uint32_t rank_end, unsigned long long *d_B, cudaStream_t s);

// hub.cu: the pairs among the top h start ranks on the tensor cores (h a
// multiple of 128; tau = 0 picks the dense-column threshold; stats: h, K,
// tau, light pairs, may be null).
int hub_block_count(bfc_graph *g, Plan &p, uint32_t h, uint32_t tau, unsigned long long *d_B, uint64_t *stats,
                    cudaStream_t s);
// The automatic hub count (top ranks covering the walk's big class, <= max_h).
int hub_auto_size(Plan &p, uint32_t max_h, uint32_t *h, cudaStream_t s);
// Algorithm 2 for a batch of start ranks of plan p: out[i] = b of the vertex
// at rank item_rank[i] (every other start vertex w != v, full midpoint rows).
int vbfc_batch(bfc_graph *g, Plan &p, const uint32_t *item_rank, uint32_t n_items, unsigned long long *out,
               cudaStream_t s);
// Local counts in one pass over whole midpoint rows (Algorithm 2 for every
// start vertex): bS[v] = b_v, be[e] = b_e (each optional), bM[x] = b_x of the
// midpoint side from be (needs be), and d_2B += 2B (Lemma 1, Eq. (1)).
int wedge_local(bfc_graph *g, Plan &p, unsigned long long *d_2B, uint64_t *bS, uint64_t *bM, uint64_t *be,
                cudaStream_t s);
}  // namespace bfc
