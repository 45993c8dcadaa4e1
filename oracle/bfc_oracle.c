/*
 * Butterfly-counting oracle: plain, slow, single-threaded C.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path: it builds its own adjacency lists from the edge list and
 * follows the paper's definitions and algorithms step by step.
 *
 * Paper: Sanei-Mehri, Sariyuce, Tirthapura, "Butterfly Counting in Bipartite
 * Networks" (arXiv 1801.00338).
 *   - butterfly, b_v, b_e: Section 2 (Preliminaries)
 *   - B = 1/2 sum_{v in L} b_v and b_v = sum_{w in Gamma^2_v} C(|Gamma_v ^ Gamma_w|, 2):
 *     Lemma 1, Eq. (1)-(3)
 *   - ExactBFC with the side choice: Algorithm 1 (its first three lines choose
 *     the start set), run without the optional w < v ordering
 *   - vBFC: Algorithm 2;  eBFC: the definition of b_e (Section 2), see orc_per_edge
 *   - ESpar: Algorithm 8;  ClrSpar: Algorithm 9;  VSamp: Algorithm 4
 *   - ESamp: Algorithm 5 (exact b_e per draw) and with Algorithm 7 (fast
 *     per-edge estimate);  WSamp: Algorithm 6
 *
 * Conventions shared with the library interface (these are not arithmetic of
 * the method):
 *   - L = U with ids [0, nU), R = V with ids [0, nV); an edge is a pair (u, v).
 *   - The canonical id of an edge is its position in the lexicographic (u, v)
 *     order of the edge set.
 *   - Random draws use SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), written
 *     here from its published definition: output k >= 1 of the sequence seeded
 *     by s is mix(s + k * 0x9E3779B97F4A7C15).
 *
 * Every function returns 0 on success and a negative number on bad input
 * (-1 allocation, -2 id out of range, -3 duplicate edge, -4 odd ordered sum).
 * Counts are exact unsigned integers; sums that could pass 64 bits are carried
 * in unsigned __int128 and range-checked before they are returned.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* graph: both adjacency structures, rows sorted by neighbour id             */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t nU, nV;
    uint64_t m;
    uint64_t *offU;  /* nU + 1 */
    uint32_t *nbrU;  /* V ids, canonical order: entry e is canonical edge e */
    uint64_t *offV;  /* nV + 1 */
    uint32_t *nbrV;  /* U ids, ascending within a row */
    uint64_t *eidV;  /* canonical edge id of each V-side entry */
    uint64_t *canon; /* canonical id of each input edge */
} graph;

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

static void graph_free(graph *g) {
    free(g->offU); free(g->nbrU); free(g->offV); free(g->nbrV); free(g->eidV); free(g->canon);
    memset(g, 0, sizeof(*g));
}

/* Sort the edges by (u, v), reject ids out of range and duplicates, then
 * lay out the U rows in that order and the V rows by a stable counting sort
 * over it (so V rows come out ascending in u). */
static int graph_build(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, graph *g) {
    memset(g, 0, sizeof(*g));
    g->nU = nU; g->nV = nV; g->m = m;
    for (uint64_t e = 0; e < m; e++)
        if (u[e] >= nU || v[e] >= nV) return -2;
    uint64_t *key = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
    uint64_t *idx = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t) * 2);
    g->offU = (uint64_t *)calloc((size_t)nU + 1, sizeof(uint64_t));
    g->nbrU = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    g->offV = (uint64_t *)calloc((size_t)nV + 1, sizeof(uint64_t));
    g->nbrV = (uint32_t *)malloc((m ? m : 1) * sizeof(uint32_t));
    g->eidV = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
    g->canon = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
    if (!key || !idx || !g->offU || !g->nbrU || !g->offV || !g->nbrV || !g->eidV || !g->canon) {
        free(key); free(idx); graph_free(g); return -1;
    }
    /* pairs (key, input index) sorted by key; keys are distinct iff the graph is simple */
    for (uint64_t e = 0; e < m; e++) { idx[2 * e] = ((uint64_t)u[e] << 32) | v[e]; idx[2 * e + 1] = e; }
    qsort(idx, m, 2 * sizeof(uint64_t), cmp_u64);
    for (uint64_t e = 0; e < m; e++) {
        key[e] = idx[2 * e];
        g->canon[idx[2 * e + 1]] = e;
        if (e > 0 && key[e] == key[e - 1]) { free(key); free(idx); graph_free(g); return -3; }
    }
    free(idx);
    for (uint64_t e = 0; e < m; e++) {
        uint32_t a = (uint32_t)(key[e] >> 32), x = (uint32_t)key[e];
        g->nbrU[e] = x;
        g->offU[a + 1]++;
        g->offV[x + 1]++;
    }
    for (uint32_t i = 0; i < nU; i++) g->offU[i + 1] += g->offU[i];
    for (uint32_t i = 0; i < nV; i++) g->offV[i + 1] += g->offV[i];
    uint64_t *cur = (uint64_t *)malloc(((size_t)nV + 1) * sizeof(uint64_t));
    if (!cur) { free(key); graph_free(g); return -1; }
    memcpy(cur, g->offV, ((size_t)nV + 1) * sizeof(uint64_t));
    for (uint64_t e = 0; e < m; e++) {
        uint32_t a = (uint32_t)(key[e] >> 32), x = (uint32_t)key[e];
        uint64_t p = cur[x]++;
        g->nbrV[p] = a;
        g->eidV[p] = e;
    }
    free(cur);
    free(key);
    return 0;
}

/* side 0 = L (= U), side 1 = R (= V) */
static uint32_t side_n(const graph *g, int s) { return s ? g->nV : g->nU; }
static const uint64_t *side_off(const graph *g, int s) { return s ? g->offV : g->offU; }
static const uint32_t *side_nbr(const graph *g, int s) { return s ? g->nbrV : g->nbrU; }

/* ------------------------------------------------------------------------ */
/* the "hash map C" of Algorithms 1-2: a zeroed counter per vertex of the     */
/* start side plus the list of keys that became non-zero                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t *count;
    uint32_t *keys;
    uint64_t nkeys;
} counter_map;

static int cmap_init(counter_map *c, uint32_t n) {
    c->count = (uint32_t *)calloc((size_t)n + 1, sizeof(uint32_t));
    c->keys = (uint32_t *)malloc(((size_t)n + 1) * sizeof(uint32_t));
    c->nkeys = 0;
    return (c->count && c->keys) ? 0 : -1;
}
static void cmap_free(counter_map *c) { free(c->count); free(c->keys); }
static void cmap_inc(counter_map *c, uint32_t w) {
    if (c->count[w]++ == 0) c->keys[c->nkeys++] = w;
}
/* sum over keys of C(count, 2); clears the map */
static u128 cmap_sum_pairs_and_clear(counter_map *c) {
    u128 s = 0;
    for (uint64_t i = 0; i < c->nkeys; i++) {
        uint64_t k = c->count[c->keys[i]];
        s += (u128)(k * (k - 1) / 2);
        c->count[c->keys[i]] = 0;
    }
    c->nkeys = 0;
    return s;
}

/* b_v by Algorithm 2: for u in Gamma_v, for w in Gamma_u with w != v, C[w]++;
 * then sum C(C[w], 2).  v lives on side s. */
static u128 vbfc(const graph *g, int s, uint32_t v, counter_map *c) {
    const uint64_t *off = side_off(g, s), *moff = side_off(g, !s);
    const uint32_t *nbr = side_nbr(g, s), *mnbr = side_nbr(g, !s);
    for (uint64_t i = off[v]; i < off[v + 1]; i++) {
        uint32_t u = nbr[i];
        for (uint64_t j = moff[u]; j < moff[u + 1]; j++) {
            uint32_t w = mnbr[j];
            if (w != v) cmap_inc(c, w);
        }
    }
    return cmap_sum_pairs_and_clear(c);
}

/* ------------------------------------------------------------------------ */
/* public functions                                                          */
/* ------------------------------------------------------------------------ */

/* out[0] = sum_{v in L} d_v^2, out[1] = sum_{v in R} d_v^2 (Table 1 columns). */
int orc_degree_square_sums(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v,
                           uint64_t *out) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    for (int s = 0; s < 2; s++) {
        u128 t = 0;
        const uint64_t *off = side_off(&g, s);
        for (uint32_t i = 0; i < side_n(&g, s); i++) {
            uint64_t d = off[i + 1] - off[i];
            t += (u128)d * d;
        }
        out[s] = (uint64_t)t;
    }
    graph_free(&g);
    return 0;
}

/* ExactBFC, Algorithm 1 without the optional ordering.
 * side_req: -1 = choose as Algorithm 1 does (start from L unless
 * sum_L d^2 < sum_R d^2, then start from R), 0 = start from L, 1 = from R.
 * For every start vertex v the inner loops count 2-paths v -> u -> w (w != v,
 * Eq. (2)) in the map C, then add C(C[w], 2); the total counts every butterfly
 * twice (once from each of its two start-side vertices, Eq. (3)), so it must be
 * even and is halved. */
int orc_exact(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, int side_req,
              uint64_t *out_B, int *out_side) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    int s = 0;
    if (side_req < 0) {
        u128 sq[2] = {0, 0};
        for (int t = 0; t < 2; t++) {
            const uint64_t *off = side_off(&g, t);
            for (uint32_t i = 0; i < side_n(&g, t); i++) {
                uint64_t d = off[i + 1] - off[i];
                sq[t] += (u128)d * d;
            }
        }
        s = (sq[0] < sq[1]) ? 1 : 0;
    } else {
        s = side_req ? 1 : 0;
    }
    counter_map c;
    if (cmap_init(&c, side_n(&g, s))) { graph_free(&g); return -1; }
    u128 beta = 0;
    for (uint32_t x = 0; x < side_n(&g, s); x++) beta += vbfc(&g, s, x, &c);
    cmap_free(&c);
    graph_free(&g);
    if (beta & 1) return -4;
    beta >>= 1;
    if (beta >> 64) return -5;
    *out_B = (uint64_t)beta;
    if (out_side) *out_side = s;
    return 0;
}

/* vBFC (Algorithm 2) for every vertex of both sides. */
int orc_per_vertex(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, uint64_t *bU,
                   uint64_t *bV) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    counter_map c;
    if (cmap_init(&c, nU > nV ? nU : nV)) { graph_free(&g); return -1; }
    for (uint32_t x = 0; x < nU; x++) bU[x] = (uint64_t)vbfc(&g, 0, x, &c);
    for (uint32_t x = 0; x < nV; x++) bV[x] = (uint64_t)vbfc(&g, 1, x, &c);
    cmap_free(&c);
    graph_free(&g);
    return 0;
}

/* vBFC for a list of vertices of one side (side 0 = L, 1 = R). */
int orc_per_vertex_list(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, int side,
                        uint64_t count, const uint32_t *ids, uint64_t *out) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    int s = side ? 1 : 0;
    for (uint64_t i = 0; i < count; i++)
        if (ids[i] >= side_n(&g, s)) { graph_free(&g); return -2; }
    counter_map c;
    if (cmap_init(&c, side_n(&g, s))) { graph_free(&g); return -1; }
    for (uint64_t i = 0; i < count; i++) out[i] = (uint64_t)vbfc(&g, s, ids[i], &c);
    cmap_free(&c);
    graph_free(&g);
    return 0;
}

/* b_e for edge e = (a, x), a in L, x in R, from the definition (Section 2: the
 * number of butterflies that contain e).  A butterfly through (a, x) is fixed by
 * a second R vertex y in Gamma_a \ {x} and a second L vertex b != a adjacent to
 * both x and y, so b_e = sum_{y in Gamma_a \ {x}} (|Gamma_x ^ Gamma_y| - 1),
 * the -1 removing a itself, which lies in both sets.  (Algorithm 3 as printed
 * sums C(C[x], 2) over the common-neighbour counts instead; that counts
 * butterflies through a pair of vertices, not through the edge, so the
 * definition is followed here.)  `mark` is a zeroed array over L. */
static uint64_t ebfc(const graph *g, uint32_t a, uint32_t x, uint8_t *mark) {
    for (uint64_t j = g->offV[x]; j < g->offV[x + 1]; j++) mark[g->nbrV[j]] = 1;
    uint64_t total = 0;
    for (uint64_t i = g->offU[a]; i < g->offU[a + 1]; i++) {
        uint32_t y = g->nbrU[i];
        if (y == x) continue;
        uint64_t common = 0;
        for (uint64_t j = g->offV[y]; j < g->offV[y + 1]; j++) common += mark[g->nbrV[j]];
        total += common - 1;
    }
    for (uint64_t j = g->offV[x]; j < g->offV[x + 1]; j++) mark[g->nbrV[j]] = 0;
    return total;
}

/* b_e for every edge, written at the edge's INPUT index. */
int orc_per_edge(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, uint64_t *be) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    uint8_t *mark = (uint8_t *)calloc((size_t)nU + 1, 1);
    if (!mark) { graph_free(&g); return -1; }
    for (uint64_t e = 0; e < m; e++) be[e] = ebfc(&g, u[e], v[e], mark);
    free(mark);
    graph_free(&g);
    return 0;
}

/* b_e for a list of input edge indices. */
int orc_per_edge_list(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, uint64_t count,
                      const uint64_t *edge_idx, uint64_t *out) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    uint8_t *mark = (uint8_t *)calloc((size_t)nU + 1, 1);
    if (!mark) { graph_free(&g); return -1; }
    for (uint64_t i = 0; i < count; i++) {
        if (edge_idx[i] >= m) { free(mark); graph_free(&g); return -2; }
        out[i] = ebfc(&g, u[edge_idx[i]], v[edge_idx[i]], mark);
    }
    free(mark);
    graph_free(&g);
    return 0;
}

/* Canonical id of every input edge (its rank in (u, v) order). */
int orc_canonical_ids(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, uint64_t *out) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    for (uint64_t e = 0; e < m; e++) out[e] = g.canon[e];
    graph_free(&g);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood 2014)                                      */
/* ------------------------------------------------------------------------ */

static uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
/* output k (k >= 1) of the sequence seeded by s */
uint64_t orc_splitmix64(uint64_t s, uint64_t k) { return sm64_mix(s + k * 0x9E3779B97F4A7C15ULL); }

/* seed of trial t: output t + 1 of the sequence seeded by the caller's seed */
static uint64_t trial_seed(uint64_t seed, uint32_t t) { return orc_splitmix64(seed, (uint64_t)t + 1); }

/* ------------------------------------------------------------------------ */
/* sparsification (Section 6)                                                */
/* ------------------------------------------------------------------------ */

/* count butterflies of the subgraph made of the kept canonical edges, with
 * Algorithm 1 (start side chosen on the subgraph's own degrees) */
static int exact_on_subset(const graph *g, const uint8_t *keep, uint64_t *out) {
    uint64_t k = 0;
    for (uint64_t e = 0; e < g->m; e++) k += keep[e];
    uint32_t *su = (uint32_t *)malloc((k ? k : 1) * sizeof(uint32_t));
    uint32_t *sv = (uint32_t *)malloc((k ? k : 1) * sizeof(uint32_t));
    if (!su || !sv) { free(su); free(sv); return -1; }
    uint64_t p = 0;
    for (uint32_t a = 0; a < g->nU; a++)
        for (uint64_t i = g->offU[a]; i < g->offU[a + 1]; i++)
            if (keep[i]) { su[p] = a; sv[p] = g->nbrU[i]; p++; }
    int rc = orc_exact(g->nU, g->nV, k, su, sv, -1, out, NULL);
    free(su); free(sv);
    return rc;
}

/* ESpar (Algorithm 8), one trial.  Edge with canonical id e is kept in trial t
 * iff the high 32 bits of output e + 1 of the trial's sequence are below
 * threshold (so the keep probability is p = threshold / 2^32).  Returns the
 * count beta of the kept subgraph and the estimate beta * p^-4. */
int orc_espar_trial(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, uint32_t threshold,
                    uint64_t seed, uint32_t t, uint64_t *beta, double *est) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    if (threshold == 0) { graph_free(&g); return -2; }
    uint8_t *keep = (uint8_t *)malloc(m ? m : 1);
    if (!keep) { graph_free(&g); return -1; }
    uint64_t ts = trial_seed(seed, t);
    for (uint64_t e = 0; e < m; e++) keep[e] = (orc_splitmix64(ts, e + 1) >> 32) < threshold;
    rc = exact_on_subset(&g, keep, beta);
    free(keep);
    graph_free(&g);
    if (rc) return rc;
    double inv_p = 4294967296.0 / (double)threshold;
    double s2 = inv_p * inv_p;
    *est = (double)*beta * (s2 * s2);
    return 0;
}

/* colour in [0, N) of a vertex: multiply-high of the output's top 32 bits.
 * L vertex a uses output a + 1, R vertex x uses output nU + x + 1. */
static uint32_t colour(uint64_t ts, uint64_t counter, uint32_t N) {
    return (uint32_t)(((orc_splitmix64(ts, counter) >> 32) * (uint64_t)N) >> 32);
}

/* ClrSpar (Algorithm 9), one trial: keep the edges whose two ends have the
 * same colour; estimate beta * N^3 (p = 1/N). */
int orc_clrspar_trial(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, uint32_t N,
                      uint64_t seed, uint32_t t, uint64_t *beta, double *est) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    if (N == 0) { graph_free(&g); return -2; }
    uint8_t *keep = (uint8_t *)malloc(m ? m : 1);
    if (!keep) { graph_free(&g); return -1; }
    uint64_t ts = trial_seed(seed, t);
    for (uint32_t a = 0; a < nU; a++) {
        uint32_t ca = colour(ts, (uint64_t)a + 1, N);
        for (uint64_t i = g.offU[a]; i < g.offU[a + 1]; i++)
            keep[i] = (colour(ts, (uint64_t)nU + g.nbrU[i] + 1, N) == ca);
    }
    rc = exact_on_subset(&g, keep, beta);
    free(keep);
    graph_free(&g);
    if (rc) return rc;
    double n = (double)N;
    *est = (double)*beta * (n * n * n);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* vertex sampling (Algorithm 4)                                             */
/* ------------------------------------------------------------------------ */

static uint64_t mulhi64(uint64_t a, uint64_t b) { return (uint64_t)(((u128)a * b) >> 64); }

/* Vertex population V = L u R, n = nU + nV; index i < nU is L vertex i, else
 * R vertex i - nU.  Draw j of trial t uses outputs 2j + 1 and 2j + 2 of the
 * trial's sequence, r1 and r2.
 *   weights == NULL (uniform, Algorithm 4): vertex = mulhi64(r2, n), q = 1/n.
 *   weights != NULL: a mixture q(i) = 1/(2n) + w_i / (2 W), W = sum w_i.  The
 *   top bit of r1 picks the part: 0 -> uniform as above, 1 -> the first i with
 *   w_0 + ... + w_i > mulhi64(r2, W).
 * The estimate of the trial is (1/k) sum_j b_{v_j} / (4 q(v_j)); with q = 1/n
 * each term is b_v * n / 4, Algorithm 4's return value.
 * drawn[j] (optional) receives the population index of draw j and bdraw[j]
 * (optional) its count b_v. */
int orc_vsamp_trial(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, uint64_t k,
                    const uint32_t *weights, uint64_t seed, uint32_t t, double *est, uint64_t *drawn,
                    uint64_t *bdraw) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    uint64_t n = (uint64_t)nU + nV;
    uint64_t W = 0;
    uint64_t *prefix = NULL;
    if (weights) {
        prefix = (uint64_t *)malloc(n * sizeof(uint64_t));
        if (!prefix) { graph_free(&g); return -1; }
        for (uint64_t i = 0; i < n; i++) { W += weights[i]; prefix[i] = W; }
        if (W == 0) { free(prefix); graph_free(&g); return -2; }
    }
    counter_map c;
    if (cmap_init(&c, nU > nV ? nU : nV)) { free(prefix); graph_free(&g); return -1; }
    uint64_t ts = trial_seed(seed, t);
    double acc = 0.0;
    for (uint64_t j = 0; j < k; j++) {
        uint64_t r1 = orc_splitmix64(ts, 2 * j + 1), r2 = orc_splitmix64(ts, 2 * j + 2);
        uint64_t i;
        if (!weights || (r1 >> 63) == 0) {
            i = mulhi64(r2, n);
        } else {
            uint64_t target = mulhi64(r2, W);
            uint64_t lo = 0, hi = n - 1;      /* first i with prefix[i] > target */
            while (lo < hi) {
                uint64_t mid = lo + (hi - lo) / 2;
                if (prefix[mid] > target) hi = mid; else lo = mid + 1;
            }
            i = lo;
        }
        uint64_t b = (i < nU) ? (uint64_t)vbfc(&g, 0, (uint32_t)i, &c) : (uint64_t)vbfc(&g, 1, (uint32_t)(i - nU), &c);
        double q = weights ? 0.5 / (double)n + 0.5 * (double)weights[i] / (double)W : 1.0 / (double)n;
        acc += (double)b / (4.0 * q);
        if (drawn) drawn[j] = i;
        if (bdraw) bdraw[j] = b;
    }
    cmap_free(&c);
    free(prefix);
    graph_free(&g);
    *est = k ? acc / (double)k : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* edge sampling (Algorithm 5) with exact per-edge counts or with the fast    */
/* per-edge estimate of Algorithm 7                                          */
/* ------------------------------------------------------------------------ */

/* 1 iff (a, x) is an edge: binary search in U row a (ascending V ids). */
static int has_edge(const graph *g, uint32_t a, uint32_t x) {
    uint64_t lo = g->offU[a], hi = g->offU[a + 1];
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (g->nbrU[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < g->offU[a + 1] && g->nbrU[lo] == x;
}

/* Draw j of trial t has its own seed ds = output j + 1 of the trial's
 * sequence, and its edge is the canonical edge mulhi64(output 1 of ds, m),
 * (a, x) with a in L.
 *   reps == 0 (Algorithm 5 with exact counts): the draw's value is b_e
 *     (Section 2 definition, ebfc) and its term b_e * m / 4.
 *   reps > 0 (Algorithm 5 with Algorithm 7 in place of the exact count):
 *     repetition i picks a2 = the mulhi64(output 2i + 2 of ds, d_x)-th L
 *     neighbour of x and x2 = the mulhi64(output 2i + 3 of ds, d_a)-th R
 *     neighbour of a, both from the full neighbour lists (rows ascending);
 *     it is a hit when a2 != a, x2 != x and (a2, x2) is an edge, i.e. when
 *     a, x, a2, x2 form a butterfly.  The draw's value is the hit count h,
 *     its estimate of b_e is h * d_a * d_x / reps, and its term that times m / 4.
 * The trial estimate is the mean of the k terms.  edges[j] / vals[j]
 * (optional) receive the canonical edge id and the draw's value. */
int orc_esamp_trial(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, uint64_t k,
                    uint32_t reps, uint64_t seed, uint32_t t, double *est, uint64_t *edges, uint64_t *vals) {
    if (m == 0) return -2;
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    uint8_t *mark = (uint8_t *)calloc((size_t)nU + 1, 1);
    if (!mark) { graph_free(&g); return -1; }
    uint64_t ts = trial_seed(seed, t);
    double acc = 0.0;
    for (uint64_t j = 0; j < k; j++) {
        uint64_t ds = orc_splitmix64(ts, j + 1);
        uint64_t e = mulhi64(orc_splitmix64(ds, 1), m);
        /* the L end of canonical edge e: the row that holds position e */
        uint32_t lo = 0, hi = nU - 1;
        while (lo < hi) {
            uint32_t mid = lo + (hi - lo + 1) / 2;
            if (g.offU[mid] <= e) lo = mid; else hi = mid - 1;
        }
        uint32_t a = lo, x = g.nbrU[e];
        uint64_t val;
        double term;
        if (reps == 0) {
            val = ebfc(&g, a, x, mark);
            term = (double)val * (double)m / 4.0;
        } else {
            uint64_t da = g.offU[a + 1] - g.offU[a], dx = g.offV[x + 1] - g.offV[x];
            uint64_t hits = 0;
            for (uint32_t i = 0; i < reps; i++) {
                uint32_t a2 = g.nbrV[g.offV[x] + mulhi64(orc_splitmix64(ds, 2 * (uint64_t)i + 2), dx)];
                uint32_t x2 = g.nbrU[g.offU[a] + mulhi64(orc_splitmix64(ds, 2 * (uint64_t)i + 3), da)];
                if (a2 != a && x2 != x && has_edge(&g, a2, x2)) hits++;
            }
            val = hits;
            term = (double)hits * (double)da * (double)dx / (double)reps * (double)m / 4.0;
        }
        acc += term;
        if (edges) edges[j] = e;
        if (vals) vals[j] = val;
    }
    free(mark);
    graph_free(&g);
    *est = k ? acc / (double)k : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* wedge sampling (Algorithm 6)                                              */
/* ------------------------------------------------------------------------ */

/* Population as in VSamp: index i < nU is L vertex i, else R vertex i - nU;
 * h = sum_i C(d_i, 2), the number of wedges.  Draw j of trial t, with
 * ds = output j + 1 of the trial's sequence:
 *   centre c = the first i with C(d_0, 2) + ... + C(d_i, 2) > mulhi64(output 1 of ds, h)
 *     (probability C(d_c, 2) / h);
 *   endpoints: p = mulhi64(output 2 of ds, d_c), q = mulhi64(output 3 of ds, d_c - 1),
 *     q' = q + (q >= p); v, w = the p-th and q'-th neighbours of c (rows
 *     ascending), two distinct neighbours with every unordered pair equally likely;
 *   beta = |Gamma_v ^ Gamma_w| - 1, the butterflies that contain the wedge;
 *   term = beta * h / 4.
 * The trial estimate is the mean of the k terms.  centres[j] / betas[j]
 * (optional) receive the centre's population index and beta. */
int orc_wsamp_trial(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, uint64_t k,
                    uint64_t seed, uint32_t t, double *est, uint64_t *centres, uint64_t *betas) {
    graph g;
    int rc = graph_build(nU, nV, m, u, v, &g);
    if (rc) return rc;
    uint64_t n = (uint64_t)nU + nV;
    uint64_t *prefix = (uint64_t *)malloc((n ? n : 1) * sizeof(uint64_t));
    uint8_t *mark = (uint8_t *)calloc((size_t)(nU > nV ? nU : nV) + 1, 1);
    if (!prefix || !mark) { free(prefix); free(mark); graph_free(&g); return -1; }
    u128 h = 0;
    for (uint64_t i = 0; i < n; i++) {
        int s = i < nU ? 0 : 1;
        uint32_t id = (uint32_t)(s ? i - nU : i);
        const uint64_t *off = side_off(&g, s);
        uint64_t d = off[id + 1] - off[id];
        h += (u128)d * (d ? d - 1 : 0) / 2;
        if (h >> 64) { free(prefix); free(mark); graph_free(&g); return -5; }
        prefix[i] = (uint64_t)h;
    }
    if (h == 0) { free(prefix); free(mark); graph_free(&g); return -2; }
    uint64_t ts = trial_seed(seed, t);
    double acc = 0.0;
    for (uint64_t j = 0; j < k; j++) {
        uint64_t ds = orc_splitmix64(ts, j + 1);
        uint64_t target = mulhi64(orc_splitmix64(ds, 1), (uint64_t)h);
        uint64_t lo = 0, hi = n - 1;       /* first i with prefix[i] > target */
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (prefix[mid] > target) hi = mid; else lo = mid + 1;
        }
        int s = lo < nU ? 0 : 1;
        uint32_t c = (uint32_t)(s ? lo - nU : lo);
        const uint64_t *off = side_off(&g, s);
        const uint32_t *nbr = side_nbr(&g, s);
        uint64_t d = off[c + 1] - off[c];
        uint64_t p = mulhi64(orc_splitmix64(ds, 2), d);
        uint64_t q = mulhi64(orc_splitmix64(ds, 3), d - 1);
        if (q >= p) q++;
        uint32_t a = nbr[off[c] + p], b = nbr[off[c] + q];
        /* a and b are on the other side: intersect their rows */
        int o = 1 - s;
        const uint64_t *ooff = side_off(&g, o);
        const uint32_t *onbr = side_nbr(&g, o);
        for (uint64_t i = ooff[a]; i < ooff[a + 1]; i++) mark[onbr[i]] = 1;
        uint64_t common = 0;
        for (uint64_t i = ooff[b]; i < ooff[b + 1]; i++) common += mark[onbr[i]];
        for (uint64_t i = ooff[a]; i < ooff[a + 1]; i++) mark[onbr[i]] = 0;
        uint64_t beta = common - 1;        /* c itself is common to both */
        acc += (double)beta * (double)(uint64_t)h / 4.0;
        if (centres) centres[j] = lo;
        if (betas) betas[j] = beta;
    }
    free(prefix);
    free(mark);
    graph_free(&g);
    *est = k ? acc / (double)k : 0.0;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* CPU baseline: Algorithm 1's per-start-vertex loops over a chosen list of   */
/* start vertices, on a graph prepared once, returning the partial ordered    */
/* sum and the number of 2-paths v -> u -> w (w != v) walked.                 */
/* ------------------------------------------------------------------------ */
/* Separate entry that times only the counting (the graph is prepared once). */
typedef struct { graph g; counter_map c; int s; } orc_prepared;

void *orc_prepare(uint32_t nU, uint32_t nV, uint64_t m, const uint32_t *u, const uint32_t *v, int side) {
    orc_prepared *p = (orc_prepared *)calloc(1, sizeof(orc_prepared));
    if (!p) return NULL;
    if (graph_build(nU, nV, m, u, v, &p->g)) { free(p); return NULL; }
    p->s = side ? 1 : 0;
    if (cmap_init(&p->c, side_n(&p->g, p->s))) { graph_free(&p->g); free(p); return NULL; }
    return p;
}

int orc_prepared_count(void *h, uint64_t count, const uint32_t *ids, uint64_t *out_sum, uint64_t *out_paths) {
    orc_prepared *p = (orc_prepared *)h;
    u128 beta = 0;
    uint64_t paths = 0;
    const uint64_t *off = side_off(&p->g, p->s), *moff = side_off(&p->g, !p->s);
    const uint32_t *nbr = side_nbr(&p->g, p->s);
    for (uint64_t i = 0; i < count; i++) {
        uint32_t x = ids[i];
        if (x >= side_n(&p->g, p->s)) return -2;
        for (uint64_t j = off[x]; j < off[x + 1]; j++) paths += moff[nbr[j] + 1] - moff[nbr[j]] - 1;
        beta += vbfc(&p->g, p->s, x, &p->c);
    }
    *out_sum = (uint64_t)beta;
    *out_paths = paths;
    return 0;
}

void orc_prepared_free(void *h) {
    orc_prepared *p = (orc_prepared *)h;
    if (!p) return;
    cmap_free(&p->c);
    graph_free(&p->g);
    free(p);
}
