/*
 * bfc.h -- exact and sampled butterfly counting in bipartite graphs on one
 * GB300 (sm_103a).  C ABI: plain pointers and sizes, no C++ or framework types.
 *
 * Method: Sanei-Mehri, Sariyuce, Tirthapura, "Butterfly Counting in Bipartite
 * Networks" (arXiv 1801.00338).
 *
 * Graph model (Section 2): a simple bipartite graph G = (L u R, E), E a subset
 * of L x R.  This library calls L "U" (ids 0..nU-1) and R "V" (ids 0..nV-1);
 * an edge is a pair (u, v).  A butterfly is a 2x2 biclique {a, b} x {x, y};
 * B is their number, b_v the number that contain vertex v, b_e the number that
 * contain edge e.
 *
 * Canonical edge order: edge ids 0..m-1 number the DISTINCT edges in
 * lexicographic (u, v) order.  Per-edge outputs use this order.
 *
 * Conventions for every call:
 *   - Return value: BFC_OK (0) or a negative BFC_E* code; bfc_strerror() names it.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  Work is enqueued on it in order.
 *   - Host scalar outputs (uint64_t*, double* documented as host) are written
 *     before the call returns; the call synchronises `stream` for them.
 *   - Device array outputs are caller-owned device memory, written in stream
 *     order; the caller synchronises before reading them.
 *   - The library owns only bfc_graph and bfc_proposal handles and the device
 *     memory they hold; inputs are borrowed for the duration of the call.
 *   - All counts are exact unsigned 64-bit integers.
 *   - A handle may be used by one stream at a time.
 */
#ifndef BFC_H
#define BFC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define BFC_OK          0
#define BFC_EINVAL     -1   /* null pointer, bad flag, bad size or parameter   */
#define BFC_ERANGE     -2   /* a vertex id >= nU or >= nV, or m >= 2^32         */
#define BFC_EDUP       -3   /* duplicate edge and BFC_DEDUP not set             */
#define BFC_ENOMEM     -4   /* device or host allocation failed                 */
#define BFC_ECUDA      -5   /* a CUDA runtime call failed                       */
#define BFC_ETIMEOUT   -6   /* a device wait hit its iteration limit            */
#define BFC_EOVERFLOW  -7   /* a count exceeded its integer range               */
#define BFC_EINTERNAL  -8   /* a device-side consistency check failed           */

/* ---- flags ------------------------------------------------------------ */
/* bfc_graph_from_edges */
#define BFC_INPUT_DEVICE  0x1u  /* u, v are device pointers (else host)        */
#define BFC_DEDUP         0x2u  /* drop repeated edges instead of BFC_EDUP      */
/* counting calls: which side holds the start vertices (Algorithm 1).
 * AUTO follows Algorithm 1: start from L (= U) unless
 * sum_{L} d^2 < sum_{R} d^2, then from R. */
#define BFC_SIDE_AUTO     0x0u
#define BFC_SIDE_U        0x10u
#define BFC_SIDE_V        0x20u
/* bfc_per_vertex / bfc_per_edge / bfc_local_counts: count with whole-row
 * sweeps (Algorithm 2 for every start vertex: every pair seen from both ends,
 * every output written by its owner) instead of the default one-sided ordered
 * sweep of Algorithm 1 (each pair once, the far endpoint's outputs updated
 * with scattered atomics).  Same results; the cost differs with the degree
 * skew. */
#define BFC_WHOLE_ROWS    0x100u

/* bfc_exact: count the pairs among the highest-ranked start vertices with the
 * tensor-core hub block (bfc_exact_hub with its automatic hub set).  Same B. */
#define BFC_HUB_MMA       0x200u
#define BFC_HUB_MAX       16384u

typedef struct bfc_graph bfc_graph;
typedef struct bfc_proposal bfc_proposal;

/* ---- graph ------------------------------------------------------------- */

/* Build a graph from an edge list (Section 2: simple bipartite graph; input
 * cleaning as in "Networks and Experimental Setup").
 *   u[i], v[i]  : endpoints of edge i, u in [0, nU), v in [0, nV); host or
 *                 device memory per BFC_INPUT_DEVICE; length m (m < 2^32).
 *   flags       : BFC_INPUT_DEVICE | BFC_DEDUP.
 *   out         : receives the handle (free with bfc_graph_free).
 * The handle keeps both adjacency structures (rows of U and rows of V, each
 * sorted) on the device.  Vertices of degree 0 are kept: they count in n for
 * vertex sampling and get b_v = 0.
 * Errors: BFC_EINVAL (null pointers, nU or nV == 0), BFC_ERANGE (an id out of
 * range), BFC_EDUP (a repeated edge without BFC_DEDUP), BFC_ENOMEM, BFC_ECUDA. */
int bfc_graph_from_edges(const uint32_t *u, const uint32_t *v, uint64_t m, uint32_t nU, uint32_t nV,
                         uint32_t flags, void *stream, bfc_graph **out);

/* Build a graph from compressed rows already on the device (the caller keeps
 * its arrays; the library copies and checks them).  Same graph as
 * bfc_graph_from_edges on the same edge set.
 *   offU (nU + 1 u64), nbrU (m u32): U rows, V ids strictly ascending in each
 *     row; the canonical id of an edge is its position in nbrU.
 *   offV (nV + 1 u64), nbrV (m u32): V rows, U ids strictly ascending.
 *   eidV (m u32, may be NULL): canonical id of each V-row entry (computed,
 *     or checked when given).
 * m = offU[nU] = offV[nV].
 * Errors: BFC_EINVAL (null pointers, nU or nV == 0, offsets that do not start
 * at 0, decrease or disagree on m, a row not strictly ascending, the two
 * sides not holding the same edges, eidV inconsistent with the rows),
 * BFC_ERANGE (an id out of range, m >= 2^32), BFC_ENOMEM, BFC_ECUDA. */
int bfc_graph_from_csr(const uint64_t *offU, const uint32_t *nbrU, uint32_t nU, const uint64_t *offV,
                       const uint32_t *nbrV, const uint32_t *eidV, uint32_t nV, void *stream, bfc_graph **out);

/* Release a graph and its device memory (after work on its stream is done). */
int bfc_graph_free(bfc_graph *g);

/* Sizes and degree statistics (host outputs, any may be NULL):
 *   m, sum_{U} d^2, sum_{V} d^2 (the Table 1 columns), and the wedge count
 *   W_U = sum_{u in U} C(d_u, 2), W_V = sum_{v in V} C(d_v, 2) (Lemma 2: the
 *   work of Algorithm 1 is the wedge count of the side that does NOT start). */
int bfc_graph_stats(const bfc_graph *g, uint64_t *m, uint64_t *sq_u, uint64_t *sq_v, uint64_t *wedges_u,
                    uint64_t *wedges_v);

/* Copy the canonical edge list out (device outputs, each of length m):
 * edge e of the canonical order is (u_out[e], v_out[e]).  Either may be NULL. */
int bfc_graph_edges(const bfc_graph *g, uint32_t *u_out, uint32_t *v_out, void *stream);

/* ---- exact counting (Section 4) --------------------------------------- */

/* ExactBFC (Algorithm 1; Lemma 1 Eq. (3)): B(G) into *out_B (host).
 * flags: one of BFC_SIDE_AUTO / BFC_SIDE_U / BFC_SIDE_V selects the start
 * side; the count does not depend on it, the work does (Lemma 2).
 * *out_side (host, may be NULL) receives 0 if U started, 1 if V.
 * Each unordered pair of start vertices is counted once (the ordering of
 * Algorithm 1's coloured line), so no halving is needed.
 * Errors: BFC_EINVAL, BFC_ECUDA, BFC_ETIMEOUT, BFC_EOVERFLOW. */
int bfc_exact(bfc_graph *g, uint32_t flags, uint64_t *out_B, int *out_side, void *stream);

/* ExactBFC with the hub-by-hub block on the tensor cores (Lemma 1 Eq. (2)-(3):
 * c(v, w) = |Gamma_v ^ Gamma_w| is entry (v, w) of A A^T, A the 0/1 matrix of
 * start rows against midpoint columns).  The `hubs` highest-ranked start
 * vertices (rank: degree ascending, ties by id) form the hub set H; every
 * pair whose lower-ranked end is in H has both ends in H, and those pairs are
 * counted as follows:
 *   - midpoint columns with >= tau hubs form a dense bf16 0/1 matrix A_H
 *     (|H| x K) and the upper-triangle 128 x 128 tiles of A_H A_H^T run on
 *     tcgen05.mma with fp32 accumulation in tensor memory (exact: every
 *     entry is an integer <= K <= 65,536 < 2^24);
 *   - the other columns add their hub pairs into an int32 |H| x |H| matrix;
 *   - the tile epilogue sums C(c, 2) over v < w.
 * The other start vertices run Algorithm 1's walk as in bfc_exact.
 *   hubs : a multiple of 128, <= the start side's vertex count; 0 selects
 *          it: the fewest top ranks (a multiple of 128, at most BFC_HUB_MAX)
 *          that hold every start vertex whose wedge lists exceed the walk's
 *          largest shared-memory window, i.e. the vertices the walk serves
 *          from global-memory cursors; none such: no hubs (plain bfc_exact).
 *   tau  : dense-column threshold (>= 2); 0 picks it by a cost model (with
 *          K <= 65,536).  An explicit tau may give K > 65,536, which stays
 *          exact while K < 2^24 and costs |H| x K x 2 bytes.
 *   out_stats (host, may be NULL, 4 entries): |H|, K, tau, light pairs.
 * Device memory for the call: |H|^2 x 4 + |H| x K x 2 bytes plus 8 bytes per
 * midpoint vertex (1.1 GB at |H| = 16,384, K = 2,048).
 * Errors: as bfc_exact; BFC_EINVAL for a bad hubs or tau = 1. */
int bfc_exact_hub(bfc_graph *g, uint32_t flags, uint32_t hubs, uint32_t tau, uint64_t *out_B, int *out_side,
                  uint64_t *out_stats, void *stream);

/* vBFC for every vertex (Algorithm 2; Lemma 1 Eq. (2)).
 *   bU : device, nU entries, b_u for u in U
 *   bV : device, nV entries, b_v for v in V
 *   out_B (host, may be NULL): B.
 * Either array may be NULL to skip it (its side's work is still done). */
int bfc_per_vertex(bfc_graph *g, uint32_t flags, uint64_t *bU, uint64_t *bV, uint64_t *out_B, void *stream);

/* eBFC for every edge: be[e] (device, m entries, canonical order) = number of
 * butterflies containing edge e (Section 2 definition; computed as
 * b_(a,x) = sum over the other endpoint w of x of (|Gamma_a ^ Gamma_w| - 1)).
 * out_B (host, may be NULL): B. */
int bfc_per_edge(bfc_graph *g, uint32_t flags, uint64_t *be, uint64_t *out_B, void *stream);

/* vBFC and eBFC together in one sweep (Algorithm 2's counts for every vertex
 * and the per-edge counts of Section 2).  Default: the ordered sweep of
 * Algorithm 1, where each wedge v - x - w of a pair {v, w} of start vertices
 * with c = |Gamma_v ^ Gamma_w| adds c - 1 to b_(v,x) and b_(w,x); every
 * vertex count then follows from b_y = 1/2 sum of b_e over y's edges (each
 * butterfly through y holds two of y's edges).  bfc_per_vertex and
 * bfc_per_edge run the same sweep.  BFC_WHOLE_ROWS: Algorithm 2 for every start
 * vertex v gives b_v and the row sums b_(v,x) = sum over w in Gamma_x \ {v}
 * of (c(v, w) - 1), and the midpoint side gets b_x = 1/2 sum of b_e over x's
 * edges.
 *   bU, bV : device, nU / nV entries (either may be NULL)
 *   be     : device, m entries, canonical order (may be NULL)
 *   out_B  : host, B (may be NULL).
 * Errors as bfc_exact. */
int bfc_local_counts(bfc_graph *g, uint32_t flags, uint64_t *bU, uint64_t *bV, uint64_t *be, uint64_t *out_B,
                     void *stream);

/* ExactBFC (Algorithm 1) of G independent graphs in one pass.
 *   u, v     : the graphs' edge lists one after another (host or device per
 *              BFC_INPUT_DEVICE); graph g owns edges edge_off[g] .. edge_off[g+1]
 *              and its ids are local: u < nU[g], v < nV[g]; no repeated edges.
 *   edge_off : host, G + 1 entries, edge_off[0] = 0
 *   nU, nV   : host, G entries each (all > 0)
 *   B_out    : host, G entries: B of each graph
 *   side_out : host, G entries (may be NULL): 0 if graph g started from U,
 *              1 if from V (each graph gets Algorithm 1's own choice)
 * A butterfly never spans two components, so the batch is counted as one
 * disjoint union in which each graph's start side is placed on the union's U
 * side; every start vertex's pair sum goes to its graph.
 * Errors: BFC_EINVAL, BFC_ERANGE (an id outside its graph, or the union has
 * 2^32 edges or vertices or more), BFC_EDUP, BFC_ENOMEM, BFC_ECUDA. */
int bfc_exact_batch(const uint32_t *u, const uint32_t *v, const uint64_t *edge_off, const uint32_t *nU,
                    const uint32_t *nV, uint32_t G, uint32_t flags, uint64_t *B_out, int *side_out, void *stream);

/* ---- sparsification (Section 6) --------------------------------------- */

/* ESpar (Algorithm 8), `trials` independent trials.  Trial t keeps canonical
 * edge e iff hi32(SplitMix64 output e+1 of the sequence seeded by s_t) < T,
 * T = floor(p * 2^32), s_t = output t+1 of the sequence seeded by `seed`
 * (SplitMix64: Steele, Lea, Flood, OOPSLA 2014).  beta_t = ExactBFC(E'_t);
 * est_t = beta_t * (2^32 / T)^4, which is unbiased for the rounded p.
 *   est  : host, trials doubles (may be NULL)
 *   beta : host, trials uint64 (may be NULL)
 * Errors: BFC_EINVAL (p <= 0, p >= 1 or T == 0, trials == 0). */
int bfc_espar(bfc_graph *g, double p, uint32_t trials, uint64_t seed, double *est, uint64_t *beta,
              void *stream);

/* ClrSpar (Algorithm 9): colour c_t(x) in [0, N) of a vertex is
 * (hi32(output k of s_t's sequence) * N) >> 32, with k = u + 1 for u in U and
 * k = nU + v + 1 for v in V; keep the edges whose ends share a colour;
 * est_t = beta_t * N^3.  Outputs as bfc_espar.  Errors: BFC_EINVAL (N == 0). */
int bfc_clrspar(bfc_graph *g, uint32_t colors, uint32_t trials, uint64_t seed, double *est, uint64_t *beta,
                void *stream);

/* ---- vertex sampling (Section 5.1) ------------------------------------- */

/* VSamp (Algorithm 4), `trials` trials of k draws each over the population
 * V = U u V (n = nU + nV; population index i < nU is U vertex i, else V vertex
 * i - nU).  Draw j of trial t uses outputs 2j+1 (r1) and 2j+2 (r2) of s_t's
 * sequence.
 *   prop == NULL : uniform, index = mulhi64(r2, n), q = 1/n; the draw's term is
 *                  b * n / 4 (Algorithm 4's return value).
 *   prop != NULL : the mixture q(i) = 1/(2n) + w_i / (2 W) over the proposal's
 *                  integer weights w (W = sum w); top bit of r1 = 0 -> uniform
 *                  index as above, 1 -> first i with w_0+..+w_i > mulhi64(r2, W).
 *                  The draw's term is b / (4 q) (importance weighting, so the
 *                  estimator stays unbiased).
 *   est : host, trials doubles: the mean of the k terms of each trial.
 *   drawn : device, trials*k uint64 population indices (may be NULL).
 *   bdraw : device, trials*k uint64 counts b of the draws (may be NULL). */
int bfc_vsamp(bfc_graph *g, uint64_t k, const bfc_proposal *prop, uint32_t trials, uint64_t seed,
              double *est, uint64_t *drawn, uint64_t *bdraw, void *stream);

/* ESamp (Algorithm 5): `trials` independent trials of k uniform edge draws.
 * Draw j of trial t has seed ds = output j+1 of the SplitMix64 sequence
 * seeded by s_t (s_t = output t+1 of `seed`'s sequence); its edge is
 * canonical edge e = mulhi64(output 1 of ds, m) = (a, x), a in U.
 *   reps == 0: the draw's value is b_e, computed exactly (Section 2's
 *     definition: the edges between Gamma_x \ {a} and Gamma_a \ {x}), and its
 *     term is b_e * m / 4.
 *   reps > 0: Algorithm 7 in place of the exact count, repeated reps times:
 *     repetition i takes the mulhi64(output 2i+2 of ds, d_x)-th entry a2 of x's
 *     row and the mulhi64(output 2i+3 of ds, d_a)-th entry x2 of a's row (rows
 *     ascending; full lists) and hits when a2 != a, x2 != x and (a2, x2) is an
 *     edge.  Value = hits h; term = h * d_a * d_x / reps * m / 4.
 *   est   (host, trials): the mean of each trial's k terms.
 *   edges (device, trials * k, may be NULL): canonical edge of each draw.
 *   vals  (device, trials * k, may be NULL): the draw's value.
 * trials * k < 2^32.  Errors: BFC_EINVAL (m == 0, trials == 0, null est),
 * BFC_ERANGE, BFC_ENOMEM, BFC_ECUDA. */
int bfc_esamp(bfc_graph *g, uint64_t k, uint32_t reps, uint32_t trials, uint64_t seed, double *est,
              uint64_t *edges, uint64_t *vals, void *stream);

/* WSamp (Algorithm 6): `trials` trials of k wedge draws.  Population as in
 * bfc_vsamp (index i < nU: U vertex i, else V vertex i - nU); h = sum_i
 * C(d_i, 2), the number of wedges.  Draw j of trial t (seed ds as in
 * bfc_esamp): the centre is the first i with C(d_0,2) + ... + C(d_i,2) >
 * mulhi64(output 1 of ds, h) (the prefix-sum search of Section 5.3); with
 * p = mulhi64(output 2, d_c) and q = mulhi64(output 3, d_c - 1), q += (q >= p),
 * the endpoints are the p-th and q-th entries of the centre's row, and
 * beta = |Gamma_v ^ Gamma_w| - 1; term = beta * h / 4.
 *   est     (host, trials): the mean of each trial's k terms.
 *   centres (device, trials * k, may be NULL): population index of each centre.
 *   betas   (device, trials * k, may be NULL): beta of each draw.
 * Errors: BFC_EINVAL (no wedge, trials == 0, null est), BFC_ERANGE,
 * BFC_ENOMEM, BFC_ECUDA. */
int bfc_wsamp(bfc_graph *g, uint64_t k, uint32_t trials, uint64_t seed, double *est, uint64_t *centres,
              uint64_t *betas, void *stream);

/* ---- (epsilon, delta) amplification of the sampling estimators ------------ */

/* Median of means (Section 5.1: averages of independent instances, made an
 * (epsilon, delta) estimator by the median of O(log 1/delta) of them).
 *   y      (host, n values): estimator instances, e.g. single-draw terms or
 *          per-trial estimates; split into `groups` consecutive groups of
 *          n / groups values (n must be a positive multiple of groups).
 *   out    (host): the median of the group means (the mean of the two middle
 *          ones when groups is even).
 * Errors: BFC_EINVAL (null pointers, groups == 0, n % groups != 0, n == 0). */
int bfc_median_of_means(const double *y, uint64_t n, uint32_t groups, double *out);

/* Sizes for an (epsilon, delta) estimate from the variance var1 of one
 * instance and the count B (or estimates of both):
 *   alpha  = ceil(32 var1 / (epsilon^2 B^2)) instances per group, so that by
 *            Chebyshev a group mean misses B by epsilon B with probability
 *            <= 1/32 (the choice of alpha in Section 5.1);
 *   groups = ceil(ln(1/delta) / (2 (1/2 - 1/32)^2)), odd, so that by
 *            Hoeffding's inequality at least half of the groups miss with
 *            probability <= delta.
 * Errors: BFC_EINVAL (var1 < 0, B <= 0, epsilon <= 0, delta not in (0, 1),
 * null outputs), BFC_ERANGE (alpha beyond 2^63). */
int bfc_mom_sizes(double var1, double B, double epsilon, double delta, uint64_t *alpha, uint32_t *groups);

/* A sampling proposal from integer weights (device or host per flags
 * BFC_INPUT_DEVICE), one per population index (nU + nV entries, U first).
 * The weights are copied; W = sum must be > 0. */
int bfc_proposal_from_weights(bfc_graph *g, const uint32_t *weights, uint32_t flags, void *stream,
                              bfc_proposal **out);
int bfc_proposal_free(bfc_proposal *p);
/* Read a proposal's integer weights back: weights (host, n = nU + nV entries,
 * caller-owned) receives them in population order, *W (optional) their sum.
 * Synchronous: waits for the device.  Errors: BFC_EINVAL (null pointers, n not
 * the proposal's population size), BFC_ECUDA. */
int bfc_proposal_weights(const bfc_proposal *p, uint32_t *weights, uint64_t n, uint64_t *W);

/* ---- instrumentation (no counterpart in the paper) --------------------- */

/* Work split of the start side `side` (0 = U, 1 = V) after its layout is
 * built (any counting call builds it; this call builds it if needed).
 * out (host, 41 entries): out[0] = nS; then for the 13 kernel classes
 * skip, warp, small windows with 2/4/8/16/32-bit counters, large windows
 * with 2/4/8/16/32-bit counters, big: vertex counts out[1..13], wedges walked
 * out[14..26], start-row entries out[27..39]; out[40] = total wedges W of
 * the midpoint side (Lemma 2). */
int bfc_plan_stats(bfc_graph *g, int side, uint64_t *out, void *stream);

/* Device memory: every call allocates its temporaries from the library's own
 * stream-ordered pool on the current device, which keeps freed memory for the
 * next call instead of returning it (so repeated calls do not map new pages).
 * bfc_trim_memory waits for the device and releases the pools' unused
 * memory.  Errors: BFC_ECUDA. */
int bfc_trim_memory(void);

/* Fault injection for tests of the error paths: after n more device
 * allocations by the library succeed, the next one fails and its call
 * returns BFC_ENOMEM, as a real out-of-memory would; the injection then
 * switches itself off.  n < 0 switches it off.  Process-wide; an allocation
 * that reuses a buffer already large enough does not count.  Every call is
 * expected to leave its handles usable after such a failure. */
int bfc_fail_alloc_after(int64_t n);

/* Wait limit for tests of the timeout path: the device-side waits of the
 * tensor-core hub kernel (bfc_exact_hub, bfc_exact with BFC_HUB_MMA) give up
 * after ns nanoseconds of GPU global time instead of the built-in one second
 * (ns = 0 restores it).  A kernel that gives up stops issuing work, waits for
 * the copies and tensor-core operations it already issued, releases its
 * tensor memory and exits, and its call returns BFC_ETIMEOUT; the handle
 * stays usable.  Process-wide; applies to launches made after the call. */
int bfc_set_wait_limit(uint64_t ns);

/* Device timing of the library's counting kernels: when enabled, every
 * wedge-kernel launch is bracketed by CUDA events on the launch stream.
 * bfc_profile_read synchronises on the recorded events and returns, for the
 * kernel tag (e.g. "win.total", "warp.edge", "big.edge"), the number of
 * launches and their summed device time in milliseconds.  Tags:
 * {warp,win,big}.{total,edge,single,local}, for bfc_exact_hub
 * hub.total (the tensor-core tile kernel), hub.degree and hub.light, and
 * esamp.exact, esamp.fast and wsamp for the samplers. */
int bfc_profile_enable(int on);
int bfc_profile_reset(void);
int bfc_profile_read(const char *tag, uint64_t *launches, double *total_ms);

/* ---- scheduling settings (no counterpart in the paper) ------------------- */

/* How one graph's counting work is scheduled on the GPU.  The settings never
 * change a count, only its speed; they are picked per graph by the
 * autotuner of the Python package (paper_1801_00338_gb300/autotune.py),
 * which times the candidates and checks that their counts agree.  A field
 * left 0 keeps the built-in default.
 *   warp_max_wedges : start vertices that walk at most this many wedges
 *                     (Lemma 3's per-vertex work) get one warp and a
 *                     shared-memory hash table; 1..512, default 512 (the
 *                     table's capacity at load factor 1/2).
 *   small_max_segs  : the others whose wedge lists hold at most this many
 *                     segments of 512 wedges (plus one per row), or who have
 *                     at most half this many rows (their segments are then
 *                     lengthened), run in the 128-thread window CTAs (eleven
 *                     per SM, 16 KB counter windows); the rest, up to 1,280
 *                     segments or 640 rows, in the 512-thread CTAs (three per
 *                     SM, 48 KB windows), and beyond that in the big-class
 *                     kernel; 1..128, default 128.
 *   hubs            : hub count of bfc_exact with BFC_HUB_MMA: 0 the automatic
 *                     choice (bfc_exact_hub with hubs = 0), BFC_TUNE_NO_HUBS
 *                     none (the walk counts every pair), else a multiple of
 *                     128 <= BFC_HUB_MAX (capped at the start side's size).
 *   tau             : that hub block's dense-column threshold (0: the cost
 *                     model; else >= 2).
 *   local_sweep     : the sweep of bfc_local_counts, bfc_per_vertex and
 *                     bfc_per_edge when BFC_WHOLE_ROWS is not given: 0 the
 *                     ordered sweep, 1 whole rows.
 *   flat_max_avg    : a window-class start vertex whose later ranks all fit in
 *                     one counter window skips the window walk and expands its
 *                     wedge lists 32 targets at a time when they hold at most
 *                     this many targets per start-row entry on average;
 *                     default 64, BFC_TUNE_NO_FLAT never.
 *   hl_max_light    : a window-class start vertex of the ordered sweeps
 *                     (bfc_exact, and the per-edge and per-vertex counts
 *                     without BFC_WHOLE_ROWS) whose wedge lists other than its
 *                     longest hold at most this many wedges is counted without
 *                     windows: those lists in a shared-memory hash table, the
 *                     longest one streamed once against it.  Default 0: as
 *                     many as the table holds at three-quarter load (768 in
 *                     the 128-thread CTAs, 1,536 in the 512-thread ones);
 *                     BFC_TUNE_NO_HL never.
 * A changed class limit redoes the cached classification of the start
 * vertices on the next counting call (the rank layout is kept).
 * Errors: BFC_EINVAL (null handle, a value out of range). */
typedef struct bfc_tuning {
  uint32_t warp_max_wedges;
  uint32_t small_max_segs;
  uint32_t hubs;
  uint32_t tau;
  uint32_t local_sweep;
  uint32_t flat_max_avg;
  uint32_t hl_max_light;
} bfc_tuning;
#define BFC_TUNE_NO_HUBS 0xFFFFFFFFu
#define BFC_TUNE_NO_FLAT 0xFFFFFFFFu
#define BFC_TUNE_NO_HL   0xFFFFFFFFu
/* t == NULL restores every default. */
int bfc_set_tuning(bfc_graph *g, const bfc_tuning *t);
/* The settings in effect, with the class-limit defaults filled in. */
int bfc_get_tuning(const bfc_graph *g, bfc_tuning *t);

/* ---- allocation-free exact count (the paper has no counterpart) --------- */

/* Size of the library-resident scratch array used by bfc_exact_csr_noalloc:
 * 16,777,216 32-bit words (64 MiB), held by every GPU that loads the library
 * until the process exits. */
#define BFC_NOALLOC_SCRATCH_WORDS (16u * 1024u * 1024u)

/* B(G) of a graph given as device CSR arrays, without allocating anything.
 * For callers that cannot allocate device memory when they need the count:
 * services whose device memory is reserved up front by another allocator or
 * held to a fixed budget (an allocation could fail or take memory they do not
 * own), and latency-bound loops that must not wait on the allocator.
 *   offU : device, nU + 1 row offsets of the U rows;  nbrU : device, V ids
 *   offV : device, nV + 1 row offsets of the V rows;  nbrV : device, U ids
 *          (both sides describe the same simple graph; rows need not be sorted)
 *   flags: BFC_SIDE_AUTO (start from V when sum over U of d^2 < sum over V of
 *          d^2, else from U) / BFC_SIDE_U / BFC_SIDE_V
 *   out_B: device, one uint64, written in stream order (no host sync)
 * The only working memory is a __device__ array of BFC_NOALLOC_SCRATCH_WORDS
 * words inside this library; its device address is looked up (with
 * cudaGetSymbolAddress) on the first call on each device, so make that first
 * call before any stream capture.  Every call shares the array and clears the
 * part it uses; calls that overlap on the GPU (different streams, no ordering
 * between them) race on it and must be serialised by the caller.
 * Errors: BFC_ERANGE if max(nU, nV) > BFC_NOALLOC_SCRATCH_WORDS - 64 or both
 * are 0 (checked before any pointer is touched), BFC_EINVAL for bad flags or
 * null pointers, BFC_ECUDA for a failed launch or symbol lookup. */
int bfc_exact_csr_noalloc(const uint64_t *offU, const uint32_t *nbrU, uint32_t nU, const uint64_t *offV,
                          const uint32_t *nbrV, uint32_t nV, uint32_t flags, uint64_t *out_B, void *stream);

/* ---- learned sampling proposal (an extension, not in the paper) --------- */
/* A small network scores every vertex from cheap features; the scores become
 * the weights of bfc_vsamp's mixture proposal.  Unbiasedness rests on the
 * importance weights b / (4 q) of bfc_vsamp, not on the network.
 * Layout of the parameter vector (BFC_MLP_PARAMS values): W1[6][64], b1[64],
 * W2[64][64], b2[64], W3[64], b3; GELU (erf form) after each hidden layer;
 * weights in bfloat16 (stored as uint16_t bits), fp32 accumulation. */
#define BFC_MLP_FEATURES 6
#define BFC_MLP_PARAMS 4673

/* Per-vertex features, row-major float[nU + nV][6] (device), U rows first:
 * log1p(d)/8, log1p(sum of neighbour degrees)/16, log1p(wedges ending at v)/16,
 * log1p(wedges centred on v)/16, side (0 = U, 1 = V), log1p(max neighbour
 * degree)/16.  O(m) work. */
int bfc_features(bfc_graph *g, float *feat, void *stream);
/* t[i] = log1p(b[i]) (device arrays of n), the regression target. */
int bfc_mlp_targets(const uint64_t *b, uint64_t n, float *t, void *stream);
/* y[i] = network(X[i]) for n rows (device). */
int bfc_mlp_forward(const uint16_t *w_bf16, const float *X, uint64_t n, float *y, void *stream);
/* grad (device, BFC_MLP_PARAMS floats, overwritten) = gradient of
 * (1/n) sum_i (network(X[r_i]) - T[r_i])^2 over rows r_i = idx[i] (or i when
 * idx is NULL); *loss (device, may be NULL) receives that mean. */
int bfc_mlp_grad(const uint16_t *w_bf16, const float *X, const float *T, const uint32_t *idx, uint64_t n,
                 float *grad, float *loss, void *stream);
/* One Adam step (Kingma & Ba 2014) on the fp32 master weights w, refreshing
 * their bfloat16 copy; step counts from 1. */
int bfc_mlp_adam(float *w, uint16_t *w_bf16, float *m, float *v, const float *grad, uint32_t P, float lr,
                 float beta1, float beta2, float eps, uint32_t step, void *stream);
/* w_bf16[i] = round-to-nearest-even bfloat16 of w[i]. */
int bfc_mlp_to_bf16(const float *w, uint16_t *w_bf16, uint32_t P, void *stream);
/* A vsamp proposal from scores s (device, nU + nV floats): integer weights
 * max(1, floor(2^24 exp(s_i - max s))), i.e. proportional to exp(s). */
int bfc_proposal_from_scores(bfc_graph *g, const float *scores, void *stream, bfc_proposal **out);

/* ---- misc -------------------------------------------------------------- */
const char *bfc_strerror(int code);
/* Number of kernel launches this library has made on the calling thread's
 * behalf since load (for launch accounting in benchmarks). */
uint64_t bfc_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* BFC_H */
