/*
 * rpq.h -- C ABI of the GB300 single-source 2-RPQ library (librpq.so).
 *
 * Implements the method of "Single-Source Regular Path Querying in Terms of
 * Linear Algebra" (arXiv:2412.10287): a level-synchronous breadth-first
 * search over the product of an edge-labelled graph and a query automaton
 * (section 4, Algorithm 1).  Every level computes
 *     M <- ( OR_a (N^a)^T x M x G^a ) <not P>,   P <- P + M,
 * until M = 0, and the answer is F x P.  The traversal runs in hand-written
 * CUDA kernels for sm_103a; the host code only validates, builds the
 * automaton and moves data.
 *
 * Conventions for every call:
 *   - Every call returns an rpq_status; nothing throws across the ABI.
 *     rpq_last_error() gives a message for the last failure on this thread.
 *   - Vertex ids are 0-based int32 in [0, n) (the paper numbers them 1..|V|,
 *     section 2).  Label ids are int32 in [0, L); in automaton transitions a
 *     label a in [L, 2L) denotes the inverse label (a-L)^- of section 2.
 *   - Inputs are copied: the caller keeps ownership of every array it passes.
 *     Handles (rpq_graph, rpq_nfa, rpq_server) are owned by the library and
 *     released with the matching *_free / *_destroy call.  Output arrays are
 *     owned by the caller.
 *   - Output arrays may be host or device memory (detected per call).  When a
 *     result does not fit in `capacity`, the call returns RPQ_ERR_CAPACITY and
 *     sets the count to the full size, so the caller can retry with a larger
 *     buffer.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *     that return results synchronise that stream before returning.
 *   - Graphs and automata are immutable once created and may be shared
 *     between threads.  Queries on one graph from several threads are safe;
 *     each takes its own device workspace.
 */
#ifndef RPQ_H
#define RPQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rpq_status {
    RPQ_OK = 0,
    RPQ_ERR_INVALID = 1,  /* bad argument: id out of range, null pointer, > 64 states ... */
    RPQ_ERR_PARSE = 2,    /* regular expression syntax error */
    RPQ_ERR_OOM = 3,      /* device or host allocation failed */
    RPQ_ERR_CUDA = 4,     /* a CUDA call failed (message in rpq_last_error) */
    RPQ_ERR_TIMEOUT = 5,  /* a device-side wait exceeded its limit; the query was abandoned */
    RPQ_ERR_CAPACITY = 6, /* output buffer too small; the count holds the size needed */
    RPQ_ERR_BUSY = 7      /* server queue full / result not ready yet */
} rpq_status;

typedef struct rpq_graph rpq_graph;
typedef struct rpq_nfa rpq_nfa;
typedef struct rpq_server rpq_server;

/* Per-query counters.  The first six fields are properties of
 * (graph, automaton, source, max_levels) alone, identical for any correct
 * implementation of Algorithm 1. */
typedef struct rpq_stats {
    int64_t levels;          /* non-empty levels after level 0 (BFS depth) */
    int64_t visited_pairs;   /* |P|: (state, vertex) pairs reached */
    int64_t expanded_pairs;  /* pairs whose out-edges were traversed */
    int64_t product_edges;   /* sum over expanded (q,v) of |delta(q,a)| * deg_a(v) */
    int64_t push_bytes;      /* sum over expanded (q,v), labels a with delta(q,a) != {}: 8 + 4 deg_a(v) */
    int64_t answer_count;    /* |answer| */
    int64_t push_unit_levels;/* (level, unit) steps run as push (implementation detail) */
    int64_t pull_unit_levels;/* (level, unit) steps run as pull (implementation detail) */
    int64_t h2d_bytes;       /* bytes this call copied host -> device */
    int64_t d2h_bytes;       /* bytes this call copied device -> host */
    double device_ms;        /* device time of the traversal kernel, or -1 if not timed */
} rpq_stats;

/* ------------------------------------------------------------- memory -- */

/* Replace the device allocator used for graphs and workspaces (for example
 * with PyTorch's caching allocator).  alloc(size, ctx) returns device memory
 * or NULL (the library then fails the call with RPQ_ERR_OOM and keeps
 * working); free(ptr, ctx) releases it.  Pass NULLs to restore cudaMalloc /
 * cudaFree.  The change applies to later allocations; every buffer goes
 * back to the allocator that made it, so the allocator may be changed while
 * graphs exist.  The callbacks may be called from the library's worker
 * threads (batch and server slots). */
rpq_status rpq_set_allocator(void *(*alloc)(size_t size, void *ctx),
                             void (*free_fn)(void *ptr, void *ctx), void *ctx);

/* --------------------------------------------------------------- graph -- */

/* Builds the per-label Boolean decomposition {G^a} of section 3 on the
 * device: for each label a, a CSR (out-edges, G^a) and a CSC (in-edges,
 * (G^a)^T = G^{a^-}) with int32 ids, rows sorted, duplicate (u, v, a) triples
 * removed (the matrices are Boolean).  Both forms stay resident, as in the
 * paper's implementation (section 5).  Labels with few non-empty rows are
 * stored hypersparse (sorted row ids + offsets).
 *   src, dst, label: host arrays of n_edges entries; edge src[i] -label[i]-> dst[i].
 *   Errors: RPQ_ERR_INVALID if an id is out of range or a label holds 2^31 or
 *   more distinct edges; RPQ_ERR_OOM; RPQ_ERR_CUDA. */
rpq_status rpq_graph_load(int32_t n_vertices, int32_t n_labels, int64_t n_edges,
                          const int32_t *src, const int32_t *dst, const int32_t *label,
                          void *stream, rpq_graph **out);
void rpq_graph_free(rpq_graph *g);

/* Sizes of a loaded graph: distinct edges of label `label` (or of all labels
 * when label < 0). */
rpq_status rpq_graph_info(const rpq_graph *g, int32_t label, int32_t *n_vertices,
                          int32_t *n_labels, int64_t *n_edges);

/* Copies the CSR (inverse = 0) or CSC (inverse = 1) of one label to host
 * arrays in dense form: offsets[n+1] (int64) and neighbours[nnz] (int32).
 * Pass neighbours = NULL to get the offsets only. */
rpq_status rpq_graph_export(const rpq_graph *g, int32_t label, int32_t inverse,
                            int64_t *offsets, int32_t *neighbours, int64_t capacity);

/* Autotuner for single queries.  First the direction choice (push for
 * sparse frontiers, pull for dense ones; the paper's section 5.1 switches
 * between its two formulations at an empirically chosen nnz, here the
 * threshold is measured): runs the n sample queries (nfas[i] from
 * sources[i]) under every candidate setting -- pull when the frontier's edge
 * mass x alpha exceeds the in-adjacency's edges + rows, alpha in {0 (push
 * only), 1, 2, 4, 8, 16, 64}, and the frontier holds at least min_pull in
 * {64, 256, 2048} pairs.  Then, with that setting, the size below which a
 * level runs on one CTA with no grid barrier: push edge mass solo_mass in
 * {-1 (never), 512, 2048, 8192} (with solo_mass / 8 frontier items).  Keeps
 * the fastest by device time, stores it in the graph for later rpq_query
 * calls (the environment variables RPQ_PULL_ALPHA, RPQ_PULL_MIN,
 * RPQ_SOLO_MASS and RPQ_SOLO_ITEMS still override) and reports it; any out
 * pointer may be NULL.  Results never depend on the setting. */
rpq_status rpq_graph_autotune(rpq_graph *g, int32_t n, const rpq_nfa *const *nfas,
                              const int32_t *sources, float *alpha_out, int32_t *min_pull_out,
                              int32_t *solo_mass_out, void *stream);

/* The hybrid of section 5.1: Algorithm 2 (section 4: no traversal matrix;
 * every step expands the whole visited set P) while P holds fewer than
 * `switch_pairs` (state, vertex) pairs, then Algorithm 1 from the pairs the
 * last step found (the paper's constant is 100).  Algorithm 2 steps run on
 * one CTA of the persistent kernel, push only.  Answers, levels and visited
 * counts never change; the expanded-pair, product-edge and push-byte
 * counters then count the re-expanded pairs too.  0 (the default) runs
 * Algorithm 1 throughout.  Applies to later queries on g (RPQ_ALG2_SWITCH
 * overrides). */
rpq_status rpq_graph_set_hybrid(rpq_graph *g, int64_t switch_pairs);

/* Rare label first, an evaluation order (the paper finds its BFS slowest
 * where it does not exploit rare labels or evaluation order, sections
 * 5.4-5.5, and names rare labels as future work, section 6).  For rpq_query
 * calls whose automaton reads, on every accepting path, a label direction
 * with at most `max_edges` edges (the rarest such one that some transition
 * not leaving a start state reads is taken): (1) a
 * backward search, the reversed automaton without that label (section 4,
 * SSR of N^-) from the vertices with such an edge, finds the (state,
 * vertex) pairs that can still reach one; (2) the forward search of
 * Algorithm 1 on a two-copy automaton (before / after reading the label)
 * never enters a pair before the label that the backward search did not
 * find.  The answer never changes; the counters are the forward search's.
 * 0 (the default) turns it off; RPQ_RARE_MAX overrides.  Automata of more
 * than 32 states are run as usual. */
rpq_status rpq_graph_set_rare_plan(rpq_graph *g, int64_t max_edges);

/* Autotuner of the bit-lane engine of rpq_query_batch (the push/pull
 * threshold and tile shape of the batched form): runs the n sample queries
 * (nfas[i] from sources[i]) on the lane kernel, in groups of up to 256, under
 * every pair of (a) the inline row length, the edges of a (vertex, label
 * direction) row a warp pushes itself before the rest of the row is cut into
 * 128-edge chunks for other warps, in {32, 64, 128, 256}, and (b) the pull
 * divisor: a level pulls (every vertex ORs the frontier lanes of its
 * in-neighbours until the lanes it still misses are found) when the
 * frontier holds more than n / divisor vertices, divisor in {0 (never), 2,
 * 4, 8, 16}.  Keeps the fastest by device time for later batches on g
 * (RPQ_LANE_HUB and RPQ_LANE_PULL_DIV override) and reports it; out pointers
 * may be NULL.  Answers never depend on the setting. */
rpq_status rpq_graph_autotune_batch(rpq_graph *g, int32_t n, const rpq_nfa *const *nfas,
                                    const int32_t *sources, int32_t *lane_hub_out,
                                    int32_t *pull_div_out, void *stream);

/* ---------------------------------------------------------- automaton -- */

/* Compiles a regular expression over labels and inverse labels into a
 * minimised DFA (section 5.2: queries become minimised DFAs), dead state
 * dropped.  Syntax:
 *     alt  := seq ('|' seq)*
 *     seq  := post (['/' | '.' | U+00B7 | whitespace] post)*   (juxtaposition concatenates)
 *     post := atom ('*' | '+' | '?')*
 *     atom := LABEL | '^' atom | '(' alt ')'
 * LABEL is a decimal id in [0, n_labels); '^R' is the inverse language R^-
 * (words reversed, every label inverted; section 4).
 *   Errors: RPQ_ERR_PARSE (syntax), RPQ_ERR_INVALID (label out of range, or
 *   more than 64 states after minimisation). */
rpq_status rpq_nfa_compile(const char *regex, int32_t n_labels, rpq_nfa **out);

/* Uses a given automaton verbatim (section 2, 2-NFA): n_states <= 64,
 * transitions from[i] -label[i]-> to[i] with label in [0, 2 n_labels), start
 * and final state lists.  Several start states and non-determinism are
 * allowed. */
rpq_status rpq_nfa_from_transitions(int32_t n_states, int32_t n_labels, int32_t n_trans,
                                    const int32_t *from, const int32_t *to,
                                    const int32_t *label, int32_t n_start,
                                    const int32_t *starts, int32_t n_final,
                                    const int32_t *finals, rpq_nfa **out);
void rpq_nfa_free(rpq_nfa *nfa);

/* Number of states and transitions of an automaton. */
rpq_status rpq_nfa_info(const rpq_nfa *nfa, int32_t *n_states, int32_t *n_trans,
                        int32_t *n_labels);

/* Copies the transitions (capacity entries each) and the start/final masks
 * (bit q set = state q) of an automaton to host memory. */
rpq_status rpq_nfa_export(const rpq_nfa *nfa, int32_t *from, int32_t *to, int32_t *label,
                          int32_t capacity, uint64_t *start_mask, uint64_t *final_mask);

/* Whether the automaton accepts a word of symbols in [0, 2L) (host-side
 * simulation; for checking compiled automata). */
rpq_status rpq_nfa_accepts(const rpq_nfa *nfa, const int32_t *word, int32_t length,
                           int32_t *accepted);

/* Reversed automaton N^- of section 4 (transitions reversed with inverted
 * labels, start and final sets swapped): SSR with N^- from v answers the
 * single-destination query of N for v. */
rpq_status rpq_nfa_reverse(const rpq_nfa *nfa, rpq_nfa **out);

/* -------------------------------------------------------------- query -- */

/* Single-source 2-RPQ (section 2, single-source reachability): the vertices v
 * such that some 2-path from `source` to v spells a word accepted by `nfa`,
 * in ascending order.  Runs Algorithm 1 on the device in one persistent
 * kernel; each level expands the frontier by push (sparse frontier) or pull
 * (dense frontier) per (label, target state).
 *   max_levels: 0 = until the frontier is empty; k > 0 = pairs reached by
 *     words of length <= k only (P_k of section 4).
 *   out_vertices/capacity/out_count: the answer (see conventions).
 *   stats: may be NULL.
 *   Errors: RPQ_ERR_INVALID (source outside [0,n), labels of nfa beyond the
 *   graph's), RPQ_ERR_CAPACITY, RPQ_ERR_TIMEOUT, RPQ_ERR_CUDA, RPQ_ERR_OOM. */
rpq_status rpq_query(const rpq_graph *g, const rpq_nfa *nfa, int32_t source, int32_t max_levels,
                     int32_t *out_vertices, int64_t capacity, int64_t *out_count,
                     rpq_stats *stats, void *stream);

/* The answer of the calling thread's most recent rpq_query whose output was
 * not device memory -- also when out_vertices was NULL or too small, so that
 * a caller can size its buffer from *out_count and copy the answer from here
 * without a second traversal.  The paper has no counterpart (it is the
 * second half of the two-call pattern).  *answer: *count vertex ids in
 * ascending order, in library-owned pinned host memory that the kernel
 * wrote directly; valid until this thread's next rpq_query call.
 *   Errors: RPQ_ERR_INVALID (null argument, or the thread has no such
 *   answer: its last rpq_query wrote device memory or failed). */
rpq_status rpq_last_answer(const int32_t **answer, int64_t *count);

/* Single-source query that allocates no device memory.  The paper has no
 * counterpart: this is for callers that must not allocate on the GPU --
 * code running where every byte of device memory is owned by another
 * allocator (an inference server's memory pool, a real-time system that
 * fixes its footprint at start-up) or where an allocation would
 * synchronise or fail.  The traversal is the same as rpq_query; its
 * workspace is a fixed 64 MiB array in device memory that the library
 * reserves on every GPU that loads it, for as long as it stays loaded.
 *   out_vertices: DEVICE memory, capacity entries (the sorted answer).
 *   Errors as rpq_query, plus RPQ_ERR_INVALID when out_vertices is not device
 *   memory, when the graph's device is not the current one, or when the
 *   query needs more than the 64 MiB of scratch (about S x n x 12.5 bytes
 *   for an automaton of S states on n vertices; use rpq_query then).
 * The first call on a device looks up the array's device address and clears
 * its counters; make that first call before any stream capture.  All calls
 * share the one array: calls whose work overlaps on the GPU (other threads,
 * other streams) race and must be serialised by the caller. */
rpq_status rpq_query_noalloc(const rpq_graph *g, const rpq_nfa *nfa, int32_t source,
                             int32_t max_levels, int32_t *out_vertices, int64_t capacity,
                             int64_t *out_count, void *stream);

/* Same query; the answer is written as a bitset of ceil(n/64) uint64 words
 * (bit v of word v/64 set iff v answers).  `out_bits` host or device. */
rpq_status rpq_query_bitset(const rpq_graph *g, const rpq_nfa *nfa, int32_t source,
                            int32_t max_levels, uint64_t *out_bits, int64_t *out_count,
                            rpq_stats *stats, void *stream);

/* 2-RPQ from a set of sources (section 2: a 2-RPQ takes a set V_s of
 * starting vertices): the vertices v such that some 2-path from some vertex
 * of V_s to v spells a word accepted by `nfa`, in ascending order -- the
 * union of the single-source answers of the vertices of V_s.  One traversal:
 * level 0 of Algorithm 1 is Q_S x V_s.
 *   sources: host memory, n_sources vertex ids in [0, n) (repeats allowed);
 *     n_sources = 0 gives the empty answer.
 *   Other arguments, outputs (rpq_last_answer included) and errors as
 *   rpq_query. */
rpq_status rpq_query_multi(const rpq_graph *g, const rpq_nfa *nfa, int32_t n_sources,
                           const int32_t *sources, int32_t max_levels, int32_t *out_vertices,
                           int64_t capacity, int64_t *out_count, rpq_stats *stats, void *stream);

/* Single-destination reachability (section 2): the vertices u such that
 * some 2-path from u to `target` spells a word accepted by `nfa`, in
 * ascending order.  Computed as section 4 states, SDR(Q) = SSR(Q^-): the
 * single-source query of the reversed automaton N^- (transitions reversed
 * with inverted labels, start and final sets swapped) from `target`.
 *   max_levels: 0 = unbounded; k > 0 = paths of length <= k.
 *   Outputs (rpq_last_answer included) and errors as rpq_query. */
rpq_status rpq_query_sdr(const rpq_graph *g, const rpq_nfa *nfa, int32_t target,
                         int32_t max_levels, int32_t *out_vertices, int64_t capacity,
                         int64_t *out_count, rpq_stats *stats, void *stream);

/* The answer of the query from `sources` (as rpq_query_multi) with each
 * vertex's level of first reach: the smallest k such that a pair (q_f, v),
 * q_f final, is discovered at level k, which is the length of the shortest
 * accepted word that labels a 2-path from a source to v (section 4: level k
 * holds the pairs first reached by words of length k; one of the path
 * outputs the conclusion, section 6, lists).
 *   out_vertices, out_levels: capacity entries each, both host or both
 *     device memory; entry i of out_levels belongs to out_vertices[i].
 *   Errors as rpq_query_multi; RPQ_ERR_CAPACITY with *out_count set. */
rpq_status rpq_query_levels(const rpq_graph *g, const rpq_nfa *nfa, int32_t n_sources,
                            const int32_t *sources, int32_t max_levels, int32_t *out_vertices,
                            int32_t *out_levels, int64_t capacity, int64_t *out_count,
                            void *stream);

/* A shortest witness for `target` (single path output, section 6): a 2-path
 * from a vertex of `sources` to `target` whose word is accepted by `nfa` and
 * has the length of the target's level of first reach.  Built on the device
 * backwards from the target, one level at a time, through the discovery
 * level of every visited pair; where several predecessors qualify, the one
 * earliest in the automaton's transition order and then in the adjacency
 * row is taken.
 *   path_vertices: *out_length + 1 vertices, path_vertices[0] a source,
 *     the last one `target`; path_symbols: *out_length symbols, symbol i
 *     leads from path_vertices[i] to path_vertices[i+1]: a < L walks an edge
 *     of label a forwards, a >= L an edge of label a - L backwards.  Both
 *     host memory of `capacity` entries.
 *   *out_length = -1 (and RPQ_OK) when the target is not in the answer.
 *   Errors: RPQ_ERR_INVALID (empty source set, target or a source out of
 *   range), RPQ_ERR_CAPACITY (with *out_length set) when the path does not
 *   fit, and those of rpq_query. */
rpq_status rpq_query_witness(const rpq_graph *g, const rpq_nfa *nfa, int32_t n_sources,
                             const int32_t *sources, int32_t target, int32_t max_levels,
                             int32_t *path_vertices, int32_t *path_symbols, int32_t capacity,
                             int32_t *out_length, void *stream);

/* Many single-source queries in one call: query i is (nfas[i], sources[i]).
 * Two engines, chosen per call:
 *   - bit lanes, when every query shares one automaton and there are at
 *     least 16 of them: up to 256 queries packed as bits of uint64 lane
 *     words, so one pass over G^a per level serves all of them (multi-source
 *     BFS, named as future work in section 6);
 *   - otherwise concurrent query slots: the single-query kernel of rpq_query
 *     runs the queries in turn on several streams at once, each kernel on a
 *     share of the SMs.
 * The environment variable RPQ_BATCH_ENGINE (= "lanes" or "slots") overrides
 * the choice.  Answers never depend on the engine.  Results are
 * concatenated: query i's vertices (ascending) are
 * out_vertices[out_offsets[i] .. out_offsets[i+1]).  out_offsets (n+1 int64)
 * is always filled; RPQ_ERR_CAPACITY when the total exceeds `capacity`.
 * `stats` may be NULL or an array of n entries: on the slots engine each
 * query's own counters; on the bit lanes the level count, the answer size,
 * the group's kernel time, and in product_edges the edges the group's
 * shared pass read for all of its queries together (the same value for
 * every query of a group of up to 256; the other counters are -1).
 * Automata may have up to 64 states each. */
rpq_status rpq_query_batch(const rpq_graph *g, int32_t n, const rpq_nfa *const *nfas,
                           const int32_t *sources, int32_t max_levels, int64_t *out_offsets,
                           int32_t *out_vertices, int64_t capacity, rpq_stats *stats,
                           void *stream);

/* ------------------------------------------------------------- serving -- */

typedef struct rpq_serve_config {
    int32_t max_lanes;       /* queries in flight on the device: query slots for engine 0
                                (0 = 8, at most 64), bit lanes for engine 1 (0 = 256) */
    int32_t max_states;      /* state slots per lane, engine 1 (0 = 16) */
    int32_t queue_capacity;  /* submitted-but-not-admitted queries (0 = 65536) */
    int64_t memory_budget;   /* bytes of device state the admitted queries may hold at once
                                (0 = no limit); see rpq_serve_create */
    int32_t max_levels;      /* per-query level cap (0 = none) */
    int32_t engine;          /* 0: concurrent query slots -- each admitted query runs the
                                single-query kernel on its own stream and 1/slots of the SMs;
                                1: bit lanes -- every admitted query advances one level per
                                replay of a captured CUDA graph of the lane step */
} rpq_serve_config;

typedef struct rpq_serve_stats {
    int64_t submitted, admitted, completed, rejected;
    int64_t level_steps;     /* level expansions run on the device: engine 0, the levels each
                                completed query expanded; engine 1, lane steps (one level of
                                every active lane each) */
    double p50_ms, p99_ms;   /* submit -> completion latency over completed queries */
    double mean_ms;
    double elapsed_s;        /* since the first submission */
    double qps;              /* completed / elapsed_s */
    int64_t peak_in_flight;  /* most queries admitted at once */
    int64_t peak_bytes;      /* most device-state bytes of admitted queries at once */
    int64_t oom_retries;     /* engine 0: queries put back in the queue after a device
                                allocation failed beside other queries in flight */
} rpq_serve_stats_t;  /* (the struct tag, not a typedef, carries the name of the call below) */

/* A server keeps the graph and every admitted query's state on the device;
 * queries arriving while others run are admitted as soon as a slot or lane
 * frees up, and their work overlaps on the device (continuous batching).
 * Engine 0: `max_lanes` host workers each run one admitted query at a time
 * with the persistent query kernel on their own stream and a share of the
 * SMs.  Engine 1: a host thread (1) admits queued queries into free bit
 * lanes, (2) advances every active lane by one level per step (a captured
 * CUDA graph replay), (3) retires lanes whose frontier emptied and stores
 * their answers.  Each answer is the same as the query alone would give.
 * Memory-bounded admission: a queued query is admitted, in arrival order,
 * only when its device state fits `memory_budget` beside that of the queries
 * in flight -- engine 0: its workspace, the visited and three frontier
 * bitsets of S' x ceil(n/64) words plus visited lists of S' x n ids (S' =
 * its state count rounded up to a power of two, at least 4); engine 1: its
 * bits in the four lane arrays, 4 x S x n bits (the lane arrays themselves
 * are allocated whole at creation, sized by max_lanes and max_states).  A
 * query that could never fit is refused at submission with RPQ_ERR_OOM.
 * Engine 0 also sizes each query's share of the SMs by the queue at
 * admission: a query that finds k - 1 others waiting runs on 1/k of the grid
 * (at most 1/max_lanes), one that finds the queue empty on half of it
 * (RPQ_SERVE_IDLE_DIV changes that divisor).  When a
 * query's device allocation fails while other queries held memory during its
 * attempt (in flight when it was admitted, still, or finished meanwhile),
 * engine 0 puts it back at the head of the queue and admits fewer queries at
 * once (raised again as queries complete); a query that fails alone
 * completes with RPQ_ERR_OOM. */
rpq_status rpq_serve_create(const rpq_graph *g, const rpq_serve_config *cfg, rpq_server **out);

/* Non-blocking.  RPQ_ERR_BUSY when the queue is full.  The automaton must
 * stay alive until the ticket is polled complete. */
rpq_status rpq_serve_submit(rpq_server *s, const rpq_nfa *nfa, int32_t source, uint64_t *ticket);

/* RPQ_OK with the answer when done (the ticket is then released);
 * RPQ_ERR_BUSY while running; RPQ_ERR_CAPACITY with *out_count set (the
 * ticket is kept); RPQ_ERR_INVALID for an unknown ticket. */
rpq_status rpq_serve_poll(rpq_server *s, uint64_t ticket, int32_t *out_vertices,
                          int64_t capacity, int64_t *out_count);

/* Blocks until every submitted query has completed (or timeout_ms passes;
 * then RPQ_ERR_TIMEOUT). */
rpq_status rpq_serve_drain(rpq_server *s, int64_t timeout_ms);

/* Server statistics (the counters above and the latency percentiles). */
rpq_status rpq_serve_stats(rpq_server *s, struct rpq_serve_stats *out);
/* The same call under its earlier name. */
rpq_status rpq_serve_stats_get(rpq_server *s, struct rpq_serve_stats *out);
void rpq_serve_destroy(rpq_server *s);

/* ---------------------------------------------------------------- misc -- */

/* Message for the last failed call on the calling thread ("" if none). */
const char *rpq_last_error(void);

/* Library version, e.g. "0.1.0". */
const char *rpq_version(void);

/* Kernels this library has launched since the process loaded it, over every
 * thread, device and entry point (a replayed lane level step counts each of
 * its kernels).  Never fails; monotone.  Callers take the difference around
 * a region of interest. */
uint64_t rpq_kernel_launches(void);

#ifdef __cplusplus
}
#endif

#endif /* RPQ_H */
