/*
 * CPU oracle for single-source 2-RPQ (TEST INFRASTRUCTURE, not product code).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library.  It shares no code with the GPU library.
 *
 * What it computes (paper section 2, definition of single-source
 * reachability, and section 4, Algorithm 1 with its correctness theorem):
 * the set of pairs (q, v) such that some 2-path from the source v_s to v and
 * some automaton path from a start state to q read a common word, and from
 * it the answer {v : (q, v) visited for some final q}.
 *
 * It is written as a plain breadth-first search over (state, vertex) pairs
 * with adjacency lists, one level at a time, so that level k holds exactly
 * the pairs first reached by words of length k (the invariant (**) of the
 * appendix proof):
 *   - level 0 is Q_S x {v_s} (zero-length paths, section 2 definition of a
 *     path; Algorithm 2 also starts from it);
 *   - from a pair (q, v), a forward edge v -a-> w leads to (q', w) for every
 *     transition q -a-> q', and a backward traversal of an edge u -a-> v
 *     (label a^-, section 2: inverse symbols, and G^{a^-} = (G^a)^T,
 *     section 3) leads to (q', u) for every transition q -a^-> q';
 *   - a pair already visited is not visited again (the mask <not P> of
 *     Algorithm 1);
 *   - the search stops when a level is empty (the loop condition M != 0) or
 *     after `max_levels` levels (then the visited set is P_k of section 4:
 *     pairs reached by words of length <= k).
 *
 * Labels: a in [0, L) is a forward label, a + L stands for a^-.
 *
 * Two more outputs, from the same search:
 *   - a set of sources V_s (the 2-RPQ of section 2 takes a set of starting
 *     vertices): level 0 is then Q_S x V_s, and the answer is the set of
 *     vertices reached from some source, i.e. the union of the answers of
 *     the single sources;
 *   - the level of first reach of every answer vertex v: the smallest k such
 *     that (q_f, v) is in level k for some final q_f.  By the invariant (**)
 *     this is the length of the shortest accepted word that labels a 2-path
 *     from a source to v (a shortest-path output in the sense of the
 *     semiring variants the paper's conclusion lists).
 *
 * Parity pins: brute-force path enumeration, closed forms and metamorphic
 * identities in tests/test_oracle.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define EXPORT __attribute__((visibility("default")))

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOMEM = 3 };

/* counters[] layout */
enum {
    ORC_C_LEVELS = 0,        /* number of non-empty levels after level 0 */
    ORC_C_VISITED = 1,       /* |P| */
    ORC_C_PRODUCT_EDGES = 2, /* sum over expanded pairs of |delta(q,a)| * deg_a(v) */
    ORC_C_PUSH_BYTES = 3,    /* sum over expanded pairs and labels a with delta(q,a) != {} of 8 + 4 deg_a(v) */
    ORC_C_EXPANDED = 4,      /* number of pairs expanded */
    ORC_C_ANSWER = 5,        /* |answer| */
    ORC_NCOUNTERS = 6
};

typedef struct {
    int64_t *off; /* n+1 */
    int32_t *lab; /* label of each entry, in [0, 2L) */
    int32_t *nbr; /* neighbour vertex */
} adjlist_t;

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Adjacency lists: entry (a, w) in row v for every edge v -a-> w, and entry
 * (a + L, u) in row v for every edge u -a-> v.  A repeated (u, v, a) triple
 * is kept once: the edge set E is a set (section 2) and G^a is a Boolean
 * matrix (section 3), so degrees count distinct neighbours per label. */
static int build_adjacency(int32_t n, int32_t L, int64_t m, const int32_t *src,
                           const int32_t *dst, const int32_t *lab, adjlist_t *g) {
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    uint64_t *key = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * m + 1));
    g->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    g->lab = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    g->nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(2 * m + 1));
    if (!off || !key || !g->off || !g->lab || !g->nbr) { free(off); free(key); return ORC_ENOMEM; }
    for (int64_t i = 0; i < m; i++) { off[src[i] + 1]++; off[dst[i] + 1]++; }
    for (int32_t v = 0; v < n; v++) off[v + 1] += off[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!fill) { free(off); free(key); return ORC_ENOMEM; }
    memcpy(fill, off, sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t i = 0; i < m; i++) {
        key[fill[src[i]]++] = ((uint64_t)(uint32_t)lab[i] << 32) | (uint32_t)dst[i];
        key[fill[dst[i]]++] = ((uint64_t)(uint32_t)(lab[i] + L) << 32) | (uint32_t)src[i];
    }
    free(fill);
    int64_t out = 0;
    for (int32_t v = 0; v < n; v++) {
        const int64_t b = off[v], e = off[v + 1];
        qsort(key + b, (size_t)(e - b), sizeof(uint64_t), cmp_u64);
        g->off[v] = out;
        for (int64_t k = b; k < e; k++) {
            if (k > b && key[k] == key[k - 1]) continue;
            g->lab[out] = (int32_t)(key[k] >> 32);
            g->nbr[out] = (int32_t)(key[k] & 0xffffffffu);
            out++;
        }
    }
    g->off[n] = out;
    free(off);
    free(key);
    return ORC_OK;
}

static void free_adjacency(adjlist_t *g) { free(g->off); free(g->lab); free(g->nbr); }

/* A graph held between queries, so that its adjacency lists are built once
 * (the paper also loads the data before timing, section 5.3). */
typedef struct { int32_t n, L; int64_t m; adjlist_t g; } oracle_graph_t;

EXPORT void *oracle_graph_new(int32_t n, int32_t L, int64_t m, const int32_t *src,
                              const int32_t *dst, const int32_t *lab) {
    if (n <= 0 || L <= 0 || m < 0) return NULL;
    for (int64_t i = 0; i < m; i++)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n || lab[i] < 0 || lab[i] >= L)
            return NULL;
    oracle_graph_t *h = (oracle_graph_t *)calloc(1, sizeof(oracle_graph_t));
    if (!h) return NULL;
    h->n = n; h->L = L; h->m = m;
    if (build_adjacency(n, L, m, src, dst, lab, &h->g) != ORC_OK) {
        free_adjacency(&h->g); free(h); return NULL;
    }
    return h;
}

EXPORT void oracle_graph_free(void *hp) {
    oracle_graph_t *h = (oracle_graph_t *)hp;
    if (!h) return;
    free_adjacency(&h->g); free(h);
}

/*
 * 2-RPQ from a set of sources by pair BFS on a graph from oracle_graph_new.
 *   automaton: S states, T transitions (t_from, t_label, t_to), t_label in [0, 2L);
 *          start and final states as lists.
 *   sources: n_sources vertex ids (repeats allowed), the set V_s.
 *   max_levels: 0 = until the frontier is empty.
 *   out_answer: n bytes, 1 where v is in the answer.
 *   out_visited: S*n bytes (row q, column v) or NULL.
 *   out_level_sizes: number of pairs in each level 0,1,2,... (up to level_cap entries) or NULL.
 *   counters: ORC_NCOUNTERS int64 or NULL.
 *   out_first_level: n int32 or NULL: level of first reach of each answer
 *          vertex (see above), -1 for vertices outside the answer.
 */
EXPORT int oracle_query_graph(const void *hp, int32_t S, int32_t T, const int32_t *t_from,
                              const int32_t *t_label, const int32_t *t_to, int32_t n_start,
                              const int32_t *starts, int32_t n_final, const int32_t *finals,
                              int32_t n_sources, const int32_t *sources, int32_t max_levels,
                              uint8_t *out_answer, uint8_t *out_visited,
                              int64_t *out_level_sizes, int32_t level_cap, int64_t *counters,
                              int32_t *out_first_level) {
    const oracle_graph_t *h = (const oracle_graph_t *)hp;
    if (!h) return ORC_EINVAL;
    const int32_t n = h->n, L = h->L;
    if (S <= 0 || T < 0 || n_sources < 0 || (n_sources > 0 && !sources) || max_levels < 0)
        return ORC_EINVAL;
    for (int32_t i = 0; i < n_sources; i++)
        if (sources[i] < 0 || sources[i] >= n) return ORC_EINVAL;
    for (int32_t t = 0; t < T; t++)
        if (t_from[t] < 0 || t_from[t] >= S || t_to[t] < 0 || t_to[t] >= S || t_label[t] < 0 ||
            t_label[t] >= 2 * L)
            return ORC_EINVAL;
    for (int32_t i = 0; i < n_final; i++)
        if (finals[i] < 0 || finals[i] >= S) return ORC_EINVAL;

    int rc = ORC_OK;
    const adjlist_t g = h->g;
    int64_t *d_off = NULL;   /* delta(q, a) as lists: index q*2L + a */
    int32_t *d_to = NULL;
    uint8_t *vis = NULL;
    uint8_t *is_final = NULL;
    int32_t *first = NULL;   /* level of first reach in a final state, per vertex */
    int32_t *cur = NULL, *nxt = NULL; /* frontier pairs, (q, v) interleaved */
    int64_t *deg = NULL;      /* deg_a(v) per (v, a) is computed on the fly */
    int64_t cnt[ORC_NCOUNTERS] = {0};

    /* delta(q, a) lists */
    int64_t nqa = (int64_t)S * 2 * L;
    d_off = (int64_t *)calloc((size_t)nqa + 1, sizeof(int64_t));
    d_to = (int32_t *)malloc(sizeof(int32_t) * (size_t)(T + 1));
    if (!d_off || !d_to) { rc = ORC_ENOMEM; goto done; }
    for (int32_t t = 0; t < T; t++) d_off[(int64_t)t_from[t] * 2 * L + t_label[t] + 1]++;
    for (int64_t i = 0; i < nqa; i++) d_off[i + 1] += d_off[i];
    {
        int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nqa + 1));
        if (!fill) { rc = ORC_ENOMEM; goto done; }
        memcpy(fill, d_off, sizeof(int64_t) * (size_t)(nqa + 1));
        for (int32_t t = 0; t < T; t++) d_to[fill[(int64_t)t_from[t] * 2 * L + t_label[t]]++] = t_to[t];
        free(fill);
    }

    int64_t npairs = (int64_t)S * n;
    vis = (uint8_t *)calloc((size_t)npairs, 1);
    is_final = (uint8_t *)calloc((size_t)S, 1);
    first = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    cur = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)npairs);
    nxt = (int32_t *)malloc(sizeof(int32_t) * 2 * (size_t)npairs);
    deg = (int64_t *)calloc((size_t)2 * L, sizeof(int64_t));
    if (!vis || !is_final || !first || !cur || !nxt || !deg) { rc = ORC_ENOMEM; goto done; }
    for (int32_t i = 0; i < n_final; i++) is_final[finals[i]] = 1;
    for (int32_t v = 0; v < n; v++) first[v] = -1;

    /* level 0: Q_S x V_s */
    int64_t ncur = 0;
    for (int32_t k = 0; k < n_sources; k++) {
        const int32_t v = sources[k];
        for (int32_t i = 0; i < n_start; i++) {
            int32_t q = starts[i];
            if (q < 0 || q >= S) { rc = ORC_EINVAL; goto done; }
            if (!vis[(int64_t)q * n + v]) {
                vis[(int64_t)q * n + v] = 1;
                cur[2 * ncur] = q; cur[2 * ncur + 1] = v; ncur++;
                if (is_final[q] && first[v] < 0) first[v] = 0;
            }
        }
    }
    cnt[ORC_C_VISITED] = ncur;
    if (out_level_sizes && level_cap > 0) out_level_sizes[0] = ncur;

    int32_t level = 0;
    while (ncur > 0 && (max_levels == 0 || level < max_levels)) {
        int64_t nnext = 0;
        for (int64_t i = 0; i < ncur; i++) {
            int32_t q = cur[2 * i], v = cur[2 * i + 1];
            cnt[ORC_C_EXPANDED]++;
            for (int32_t a = 0; a < 2 * L; a++) deg[a] = 0;
            for (int64_t e = g.off[v]; e < g.off[v + 1]; e++) {
                int32_t a = g.lab[e], w = g.nbr[e];
                deg[a]++;
                const int64_t base = (int64_t)q * 2 * L + a;
                for (int64_t k = d_off[base]; k < d_off[base + 1]; k++) {
                    int32_t q2 = d_to[k];
                    cnt[ORC_C_PRODUCT_EDGES]++;
                    int64_t idx = (int64_t)q2 * n + w;
                    if (!vis[idx]) {
                        vis[idx] = 1;
                        nxt[2 * nnext] = q2; nxt[2 * nnext + 1] = w; nnext++;
                        /* levels are visited in increasing order: the first
                         * final pair of w found is at its smallest level */
                        if (is_final[q2] && first[w] < 0) first[w] = level + 1;
                    }
                }
            }
            for (int32_t a = 0; a < 2 * L; a++) {
                const int64_t base = (int64_t)q * 2 * L + a;
                if (d_off[base + 1] > d_off[base]) cnt[ORC_C_PUSH_BYTES] += 8 + 4 * deg[a];
            }
        }
        level++;
        if (out_level_sizes && level < level_cap) out_level_sizes[level] = nnext;
        if (nnext > 0) cnt[ORC_C_LEVELS] = level;
        cnt[ORC_C_VISITED] += nnext;
        int32_t *t = cur; cur = nxt; nxt = t;
        ncur = nnext;
    }

    memset(out_answer, 0, (size_t)n);
    for (int32_t i = 0; i < n_final; i++) {
        int32_t q = finals[i];
        for (int32_t v = 0; v < n; v++)
            if (vis[(int64_t)q * n + v]) out_answer[v] = 1;
    }
    for (int32_t v = 0; v < n; v++) cnt[ORC_C_ANSWER] += out_answer[v];
    if (out_visited) memcpy(out_visited, vis, (size_t)npairs);
    if (counters) memcpy(counters, cnt, sizeof(cnt));
    if (out_first_level) memcpy(out_first_level, first, sizeof(int32_t) * (size_t)n);

done:
    free(d_off); free(d_to); free(vis); free(is_final); free(first); free(cur); free(nxt);
    free(deg);
    return rc;
}

/* The single-source form: V_s = {source}. */
EXPORT int oracle_ssr_graph(const void *hp, int32_t S, int32_t T, const int32_t *t_from,
                            const int32_t *t_label, const int32_t *t_to, int32_t n_start,
                            const int32_t *starts, int32_t n_final, const int32_t *finals,
                            int32_t source, int32_t max_levels, uint8_t *out_answer,
                            uint8_t *out_visited, int64_t *out_level_sizes, int32_t level_cap,
                            int64_t *counters) {
    return oracle_query_graph(hp, S, T, t_from, t_label, t_to, n_start, starts, n_final, finals,
                              1, &source, max_levels, out_answer, out_visited, out_level_sizes,
                              level_cap, counters, NULL);
}

/* One-shot form: builds the adjacency lists, runs one query, frees them. */
EXPORT int oracle_ssr(int32_t n, int32_t L, int64_t m, const int32_t *src, const int32_t *dst,
                      const int32_t *lab, int32_t S, int32_t T, const int32_t *t_from,
                      const int32_t *t_label, const int32_t *t_to, int32_t n_start,
                      const int32_t *starts, int32_t n_final, const int32_t *finals,
                      int32_t source, int32_t max_levels, uint8_t *out_answer,
                      uint8_t *out_visited, int64_t *out_level_sizes, int32_t level_cap,
                      int64_t *counters) {
    void *h = oracle_graph_new(n, L, m, src, dst, lab);
    if (!h) return ORC_EINVAL;
    int rc = oracle_ssr_graph(h, S, T, t_from, t_label, t_to, n_start, starts, n_final, finals,
                              source, max_levels, out_answer, out_visited, out_level_sizes,
                              level_cap, counters);
    oracle_graph_free(h);
    return rc;
}

EXPORT int oracle_ncounters(void) { return ORC_NCOUNTERS; }
