// Single-source 2-RPQ on the device: Algorithm 1 of the paper (section 4)
//     M <- ( OR_a (N^a)^T x M x G^a ) <not P>,  P <- P + M,  until M = 0;
//     answer F x P
// run as ONE persistent cooperative kernel per query.  The Boolean matrices
// are bitsets with one row of |V| bits per automaton state (P: visited,
// F_j: the frontier M_j).  Every visited pair is also appended, in discovery
// order, to an append-only list per state, so that level j's frontier of
// state q is one contiguous range of q's list.  A level runs either on the
// whole grid (one grid-wide phase, then one grid barrier) or, while the
// frontier is small, on CTA 0 alone with no grid barrier at all, the other
// CTAs parked at a gate until CTA 0 needs them again:
//
//   expand j   for every (label direction d, target state q'):
//     push     for every frontier pair (q, v) with q -d-> q' and every w in
//              row v of G^d: atomicOr P[q'][w]; the lane that flips the bit
//              from 0 has discovered (q', w) in M_{j+1} (it was not in P_j,
//              the mask <not P> of Algorithm 1) and appends it;
//     pull     for every w not in P[q'] with in-edges of direction d: one
//              in-neighbour u with X_{d,q'}[u] = OR_{q: q -d-> q'} M_j[q][u]
//              suffices (early exit); then the same atomicOr discovery.
//   A discovered pair is appended to the visited list of q', its bit set in
//   F_{j+1} (on grid levels: only pull reads it), and the rows it will
//   expand are measured: their edge mass steers the next push/pull choice
//   (a direction-optimising BFS: the push-pull optimisation the paper's
//   conclusion names); rows of >= kWarpRow edges go to a chunk list that
//   every warp draws 128-edge chunks from; shorter rows are expanded by a
//   CTA-wide scan-based gather, from a list of them made at discovery
//   (where finding a row again is costly or mostly finds nothing) or from
//   the frontier list and the row offsets.
//   plan j+1 (every working CTA, same data): stop when M_{j+1} is empty or
//   the level cap is reached; else pick push or pull per (d, q') and
//   whether CTA 0 runs the level alone.
//
// The answer F x P is either swept from P by the grid or, when it is small,
// gathered from the final states' lists and sorted by CTA 0.  The kernel
// leaves P and the F bitsets all-zero when it ends (cleared through the
// lists, or densely where that is cheaper), so the next query on the same
// workspace starts without an O(S |V|) clear.
//
// Every wait on other CTAs (the grid barrier, the gate) is bounded by a
// wall-clock limit; on expiry the kernel records RPQ_ERR_TIMEOUT and returns.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <unistd.h>  // environ

#include "graph.h"

namespace rpq {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kR = 4;                 // edges per lane per round in the batched loops
constexpr int kWarpRow = rpq_graph::kLongRow;  // rows with at least this many edges are chunked
constexpr int kChunk = 32 * kR;       // edges per chunk: one warp round
static_assert(kChunk == rpq_graph::kLongChunk, "chunk size must match the graph's row statistics");
constexpr int kPullRows = 2;          // in-rows a pull thread tests together
constexpr int kPullBatch = 4;         // in-neighbours per row a pull lane tests per round trip
constexpr int kPullTile = kThreads * kPullRows;  // in-rows per pull tile claim
constexpr int kGather = 1024;         // gather buffer entries per CTA
constexpr int kMaxGroups = 512;
constexpr int kMaxUnits = 512;
constexpr int kMaxTargets = 2048;
constexpr uint64_t kBarrierTimeoutNs = 4000000000ull;  // default limit of every device wait

// (source state q, direction d) with the targets delta(q, d) as a mask.
struct QGroup {
    int32_t q, d;
    uint64_t tmask;
    int32_t t_first, t_count;  // slots in the target table: (unit, q') pairs
    int32_t listed;            // its short rows go to the level's short-row list
    int32_t pad;
};
// (direction d, target state q') with the source states {q : q -d-> q'}.
struct QUnit {
    int32_t d, q2, in_dir, g_first, g_count;
    int32_t pad;
    uint64_t smask;
    int64_t in_rows;   // rows of the in-adjacency to sweep when pulling
    int64_t in_nnz;
};

// A long row of a frontier pair: group g, vertex v, edges [b, e), and the
// index of its first chunk.
struct Row {
    int32_t g, v, b, e;
    long long chunk0;
};

// Device counters of one query.  Per-level fields rotate over 3 slots:
// slot j % 3 holds level j.
struct Counters {
    unsigned bar_count;
    int32_t pub_level;
    // (grid barrier generation << 32) | status (0, or the rpq_status that
    // stopped the query): the load that ends a CTA's barrier wait also tells
    // it whether the query failed
    unsigned long long gen_status;
    unsigned long long gate;  // (launch epoch << 32) | releases of the gate so far
    unsigned long long beat;  // CTA 0's progress while it runs levels alone
    unsigned long long parked;  // CTAs that have parked (cumulative over the launch)
    // level state CTA 0 publishes when it releases the gate into a level
    long long pub_vstart[kMaxStates], pub_vprev[kMaxStates], pub_flprev[kMaxStates];
    unsigned long long fl_count[3][kMaxStates];  // frontier pairs per state
    unsigned long long rows_packed[3];           // (rows << 40) | chunks
    unsigned long long lvl_bytes[3], lvl_edges[3];
    unsigned long long claim_chunk[3], claim_item[3], claim_pull[3];
    unsigned long long srows_count[3];  // short rows listed per level slot
    long long answer_count;
    long long vcount[kMaxStates];  // visited pairs per state when the query ended
};

// Where a level's counters live: device memory on grid levels or, while CTA
// 0 runs levels alone, its shared memory (no round trips).  Slot j % 3
// holds level j.
struct Ctrs {
    unsigned long long *fl;     // [3][kMaxStates] pairs per state
    unsigned long long *rows;   // [3] long rows << 40 | chunks
    unsigned long long *bytes;  // [3] push bytes of the level's rows
    unsigned long long *edges;  // [3] product edges of the level's rows
    unsigned long long *srows;  // [3] short rows listed
    unsigned long long *mf;     // [3][mstride] edge mass per group
    int32_t mstride, pad;
};

// Automaton tables of up to this many bytes travel inside the kernel's
// parameters (no host-to-device copy before the launch).
constexpr int kInlineTables = 2048;

// Query summary CTA 0 writes to host-mapped memory when the kernel ends, so
// the host reads it (after synchronising the stream) without a device-to-host
// copy.  A failed launch writes none: `epoch` then differs from the launch's.
// the query's statistics, kept by CTA 0 in shared memory
enum : int {
    kStLevels, kStVisited, kStExpanded, kStProductEdges, kStPushBytes, kStPushUnits, kStPullUnits,
    kStats
};

struct QueryResult {
    long long levels, visited, expanded, product_edges, push_bytes;
    long long push_units, pull_units, answer_count;
    uint32_t epoch;
    int32_t small;  // 1: the answer went to out_list_small
};

struct KParams {
    const DevAdj *adj;
    int32_t n, W, S;
    int32_t n_groups, n_units, n_targets, n_ugroups;
    int32_t source, max_levels;
    // level 0 is Q_S x V_s: the vertices sources[0..n_sources) when sources
    // is set (device memory; repeats allowed), else {source}
    const int32_t *sources;
    int32_t n_sources;
    uint64_t start_mask, final_mask;
    float alpha;       // pull when frontier edge mass * alpha > in-adjacency edges + rows
    int32_t min_pull;  // ... and the unit's source frontier holds at least this many pairs
    int32_t solo_mass;   // a level runs on CTA 0 alone when its push edge mass <= this,
    int32_t solo_items;  // its frontier items <= this and no unit pulls (solo_mass < 0: never)
    uint32_t epoch;      // distinct per launch on this workspace (tags the gate word)
    uint64_t wait_ns;    // limit of every wait on other CTAs (then RPQ_ERR_TIMEOUT)
    // failure test: the last CTA leaves at its first release from the gate,
    // so the grid's next barrier waits for it until the limit runs out
    int32_t test_leave;
    int32_t clear_first; // P and F hold garbage: clear them before the traversal
    int32_t disc_cap;    // a CTA measures its own discoveries when at most this many (<= kDisc)
    // automaton tables (device)
    const QGroup *groups;
    const QUnit *units;
    const int32_t *t_unit;   // per target slot: unit index
    const int32_t *t_state;  // per target slot: q'
    const int32_t *u_group;  // per unit group slot: group index
    // state (device)
    uint64_t *P;             // [S][W]
    uint64_t *F[3];          // [S][W] per level slot
    int32_t *VL;             // [S][n] visited vertices of each state, in discovery order
    Row *rows[3];            // long rows per level slot
    int32_t *cmap[3];        // chunk -> row index per level slot
    int4 *srl[3];            // short rows (group, begin, end, vertex) per level slot
    long long row_cap, chunk_cap, srow_cap;
    unsigned long long *mf;  // [3][kMaxGroups]: frontier edge mass per group
    long long *fin_sums;     // [gridDim]
    // a grid level that discovers at least sort_min pairs (0: never) has
    // each state's new list range rewritten in ascending vertex order from
    // its frontier bits, so that the rows of the next level are measured and
    // expanded in address order; sort_cnt [S][gridDim] holds per-CTA counts
    long long sort_min;
    uint32_t *sort_cnt;
    // Algorithm 2 (section 4, no traversal matrix) while the visited set
    // holds fewer than alg2_until pairs, then Algorithm 1 (the hybrid switch
    // of section 5.1); 0 = Algorithm 1 throughout
    long long alg2_until;
    // push levels with more edge mass than this read the visited word before
    // each atomicOr (most of their targets are already visited)
    long long precheck_mass;
    // states [0, dense_clear) entered the launch with visited bits that no
    // list holds (pairs excluded beforehand): their rows of P are cleared
    // densely at the end, and the one-CTA answer path is not taken
    int32_t dense_clear;
    Counters *c;
    // output
    int32_t *out_list;
    int64_t capacity;
    int32_t *out_list_small;  // small answers (CTA 0 alone) go here instead, if set
    uint64_t *out_bits;  // bitset output (or nullptr)
    // optional per-level trace (block 0's view)
    unsigned long long *trace;
    int32_t trace_cap;
    QueryResult *result;  // host-mapped summary, or null
    // when set ([S][n], -1 = not visited on entry): the level at which each
    // visited pair was discovered, for path outputs (first reach, witness)
    int32_t *pair_level;
    // tables inside the parameters: byte offsets into tab (when tab_inline)
    int32_t tab_inline, o_groups, o_units, o_tu, o_ts, o_ug;
    alignas(16) uint8_t tab[kInlineTables];
};

constexpr int kTraceFields = 16;  // t_plan, t_expand, t_barrier, pairs, push units, pull units,
                                  // grid, push bytes of the level's rows, block 0's chunks done,
                                  // its short rows done, ~(first CTA done), last CTA done, and on
                                  // grid levels: last CTA whose warps all ended the expansion,
                                  // last CTA done measuring its buffer, block 0 past the barrier,
                                  // block 0 done sorting the level (overflow only)
constexpr int kTraceLevels = 4096;

__device__ __forceinline__ void trace_put(const KParams &p, int j, int f, unsigned long long v) {
    if (p.trace && blockIdx.x == 0 && threadIdx.x == 0 && j < p.trace_cap)
        p.trace[(size_t)j * kTraceFields + f] = v;
}

// Field f of the launch's own trace row (block 0, thread 0): 0 start, 1
// level 0 measured, 2 loop end, 3 end; 4 tables loaded, 5 seeds set, 6
// level 0 advanced, 7 level 0 planned.
__device__ __forceinline__ void trace_launch(const KParams &p, int f) {
    if (p.trace && blockIdx.x == 0 && threadIdx.x == 0)
        p.trace[(size_t)(p.trace_cap) * kTraceFields + f] = global_timer_ns();
}

// The latest of every CTA's time for field f (thread 0 of each CTA).
__device__ __forceinline__ void trace_last(const KParams &p, int j, int f) {
    if (p.trace && threadIdx.x == 0 && j < p.trace_cap)
        atomicMax(&p.trace[(size_t)j * kTraceFields + f], global_timer_ns());
}

// ------------------------------------------------------------ barrier ----
constexpr unsigned long long kStatusMask = (1ull << 30) - 1;
// Set in the barrier word when some CTA discovered more pairs in a level
// than its shared-memory buffer holds (the level is then measured again
// from the visited lists): bit 30 + (g & 1) for the barrier that closes
// generation g, so that a CTA still leaving barrier g cannot mistake a
// flag raised for barrier g + 1 for its own.
__host__ __device__ __forceinline__ unsigned long long overflow_bit(unsigned gen) {
    return 1ull << (30 + (gen & 1u));
}
constexpr unsigned long long kOverflowBits = 3ull << 30;

__host__ __device__ __forceinline__ int32_t status_of(unsigned long long gen_status) {
    return (int32_t)(gen_status & kStatusMask);
}

__device__ __forceinline__ int load_status(const Counters *c) {
    return status_of(*(volatile const unsigned long long *)&c->gen_status);
}

// Records the first failure of the query (later ones are dropped).
__device__ __forceinline__ void set_status(Counters *c, int32_t err) {
    unsigned long long old = *(volatile unsigned long long *)&c->gen_status;
    while (status_of(old) == 0) {
        const unsigned long long seen =
            atomicCAS(&c->gen_status, old, (old & ~kStatusMask) | (uint32_t)err);
        if (seen == old) break;
        old = seen;  // a barrier moved the generation on: try again
    }
}

// Grid barrier: -1 when the query failed, else 1 when some CTA (this one
// with `overflow`) flagged a discovery-buffer overflow on arriving, else 0.
__device__ __forceinline__ int grid_sync(const KParams &p, bool overflow = false) {
    Counters *c = p.c;
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        // arrive with release semantics (this CTA's writes, ordered by the
        // __syncthreads above), leave with acquire semantics
        unsigned long long w = *(volatile unsigned long long *)&c->gen_status;
        const unsigned gen = (unsigned)(w >> 32);  // cannot move on before this CTA arrives
        if (overflow) atomicOr(&c->gen_status, overflow_bit(gen));
        unsigned arrived;
        asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(&c->bar_count) : "memory");
        if (arrived == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.u32 [%0], 0;" ::"l"(&c->bar_count) : "memory");
            asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], %2;"
                         : "=l"(w)
                         : "l"(&c->gen_status), "l"(1ull << 32)
                         : "memory");
        } else {
            const uint64_t t0 = global_timer_ns();
            for (unsigned it = 1;; it++) {
                asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(w) : "l"(&c->gen_status) : "memory");
                if ((unsigned)(w >> 32) != gen || status_of(w) != 0) break;
                if ((it & 255u) == 0 && global_timer_ns() - t0 > p.wait_ns) {
                    set_status(c, (int32_t)RPQ_ERR_TIMEOUT);
                    w = 1;
                    break;
                }
            }
        }
        s_ok = status_of(w) != 0 ? -1 : (w & overflow_bit(gen)) ? 1 : 0;
    }
    __syncthreads();
    return s_ok;
}

__device__ __forceinline__ bool grid_barrier(const KParams &p) { return grid_sync(p) >= 0; }

// ------------------------------------------------------- shared layout ---
// Per-query tables live in shared memory for the whole kernel, so that the
// per-level control work never waits on global memory.
struct Shared {
    uint64_t *tpush;    // push-mode targets of each group (decided per level)
    long long *nsrow;   // [2]: [0] short rows listed for the current level
    long long *dpref;   // [n_groups + 1] prefix of frontier items over dense push groups
    uint8_t *gdense;    // [n_groups] short rows found from the frontier list and dense offsets
                        // (else listed at discovery)
    const int32_t **gnbr;
    int32_t *gq, *gd, *gtpop;
    int32_t *gt_first, *gt_count;
    long long *upref;   // prefix of pull rows over pull units (n_units + 1)
    long long *urows, *unnz;
    int32_t *ug_first, *ug_count, *uq2, *uin;
    uint64_t *usmask;
    uint8_t *upull;
    int32_t *t_unit, *t_state, *u_group;
    unsigned long long *fl;       // [kMaxStates] pairs per state at the current level
    unsigned long long *fl_prev;  // [kMaxStates] at the previous level
    long long *vstart;            // [kMaxStates] current level's first list entry
    long long *vprev;             // [kMaxStates] previous level's first list entry
    long long *vnext;             // [kMaxStates] next level's first list entry
    unsigned long long *mfv;      // [n_groups]
    unsigned long long *s_mf;     // [n_groups] per-CTA edge mass of discoveries
    int32_t *gbuf_k;
    int16_t *gbuf_g;
    unsigned long long *lvl;      // [2] level's push bytes / product edges (CTA 0's statistics)
    long long *stats;             // [kStats] the query's statistics (CTA 0, thread 0)
    unsigned long long *sctr;     // CTA 0's level counters in shared memory (Ctrs layout)
    Ctrs *cv;                     // [2] counter views: device memory, shared memory
    int32_t *flags;               // [2] test P before the atomicOr (big levels); spare
};

template <class F>
__host__ __device__ size_t shared_layout(int ng, int nu, int nt, int nug, F take) {
    take(0, sizeof(uint64_t) * ng);
    take(1, sizeof(long long) * 2);
    take(2, sizeof(void *) * ng);
    take(3, sizeof(int32_t) * ng);
    take(4, sizeof(int32_t) * ng);
    take(5, sizeof(int32_t) * ng);
    take(6, sizeof(int32_t) * ng);
    take(7, sizeof(int32_t) * ng);
    take(8, sizeof(long long) * (nu + 1));
    take(9, sizeof(long long) * nu);
    take(10, sizeof(long long) * nu);
    take(11, sizeof(int32_t) * nu);
    take(12, sizeof(int32_t) * nu);
    take(13, sizeof(int32_t) * nu);
    take(14, sizeof(int32_t) * nu);
    take(15, sizeof(uint64_t) * nu);
    take(16, nu);
    take(17, sizeof(int32_t) * nt);
    take(18, sizeof(int32_t) * nt);
    take(19, sizeof(int32_t) * nug);
    take(20, sizeof(unsigned long long) * kMaxStates);
    take(21, sizeof(unsigned long long) * kMaxStates);
    take(22, sizeof(unsigned long long) * ng);
    take(23, sizeof(unsigned long long) * ng);
    take(24, sizeof(int32_t) * kGather);
    take(25, sizeof(int16_t) * kGather);
    take(26, sizeof(long long) * kMaxStates);
    take(27, sizeof(long long) * kMaxStates);
    take(28, sizeof(long long) * kMaxStates);
    take(29, sizeof(unsigned long long) * 2);
    take(30, sizeof(int32_t) * 2);
    take(31, sizeof(long long) * kStats);
    take(32, sizeof(unsigned long long) * (3 * kMaxStates + 12 + 3 * (size_t)ng));
    take(33, sizeof(Ctrs) * 2);
    take(34, sizeof(long long) * (ng + 1));
    return take(35, ng);
}

__host__ __device__ size_t shared_bytes(int ng, int nu, int nt, int nug) {
    size_t off = 0;
    return shared_layout(ng, nu, nt, nug, [&](int, size_t bytes) {
        off = (off + 15) & ~size_t(15);
        off += bytes;
        return off;
    }) + 16;
}

__device__ Shared carve(const KParams &p, uint8_t *base) {
    Shared s;
    uint8_t *ptr[36];
    size_t off = 0;
    shared_layout(p.n_groups, p.n_units, p.n_targets, p.n_ugroups, [&](int i, size_t bytes) {
        off = (off + 15) & ~size_t(15);
        ptr[i] = base + off;
        off += bytes;
        return off;
    });
    s.tpush = (uint64_t *)ptr[0];
    s.nsrow = (long long *)ptr[1];
    s.gnbr = (const int32_t **)ptr[2];
    s.gq = (int32_t *)ptr[3];
    s.gd = (int32_t *)ptr[4];
    s.gtpop = (int32_t *)ptr[5];
    s.gt_first = (int32_t *)ptr[6];
    s.gt_count = (int32_t *)ptr[7];
    s.upref = (long long *)ptr[8];
    s.urows = (long long *)ptr[9];
    s.unnz = (long long *)ptr[10];
    s.ug_first = (int32_t *)ptr[11];
    s.ug_count = (int32_t *)ptr[12];
    s.uq2 = (int32_t *)ptr[13];
    s.uin = (int32_t *)ptr[14];
    s.usmask = (uint64_t *)ptr[15];
    s.upull = (uint8_t *)ptr[16];
    s.t_unit = (int32_t *)ptr[17];
    s.t_state = (int32_t *)ptr[18];
    s.u_group = (int32_t *)ptr[19];
    s.fl = (unsigned long long *)ptr[20];
    s.fl_prev = (unsigned long long *)ptr[21];
    s.mfv = (unsigned long long *)ptr[22];
    s.s_mf = (unsigned long long *)ptr[23];
    s.gbuf_k = (int32_t *)ptr[24];
    s.gbuf_g = (int16_t *)ptr[25];
    s.vstart = (long long *)ptr[26];
    s.vprev = (long long *)ptr[27];
    s.vnext = (long long *)ptr[28];
    s.lvl = (unsigned long long *)ptr[29];
    s.flags = (int32_t *)ptr[30];
    s.stats = (long long *)ptr[31];
    s.sctr = (unsigned long long *)ptr[32];
    s.cv = (Ctrs *)ptr[33];
    s.dpref = (long long *)ptr[34];
    s.gdense = (uint8_t *)ptr[35];
    return s;
}

__device__ void load_tables(const KParams &p, const Shared &sh) {
    const QGroup *groups = p.groups;
    const QUnit *units = p.units;
    const int32_t *t_unit = p.t_unit, *t_state = p.t_state, *u_group = p.u_group;
    if (p.tab_inline) {  // the parameter block is grid-constant: its address is usable
        const uint8_t *b = p.tab;
        groups = reinterpret_cast<const QGroup *>(b + p.o_groups);
        units = reinterpret_cast<const QUnit *>(b + p.o_units);
        t_unit = reinterpret_cast<const int32_t *>(b + p.o_tu);
        t_state = reinterpret_cast<const int32_t *>(b + p.o_ts);
        u_group = reinterpret_cast<const int32_t *>(b + p.o_ug);
    }
    for (int g = threadIdx.x; g < p.n_groups; g += kThreads) {
        const QGroup G = groups[g];
        sh.gq[g] = G.q;
        sh.gd[g] = G.d;
        sh.gnbr[g] = p.adj[G.d].nbr;
        // only a dense adjacency has offsets to find a row by (an empty one
        // has none: its groups take the listed path, which lists nothing)
        sh.gdense[g] = (!G.listed && p.adj[G.d].fmt == ADJ_DENSE) ? 1 : 0;
        sh.gtpop[g] = __popcll(G.tmask);
        sh.gt_first[g] = G.t_first;
        sh.gt_count[g] = G.t_count;
        sh.tpush[g] = 0;
        sh.s_mf[g] = 0;
    }
    for (int u = threadIdx.x; u < p.n_units; u += kThreads) {
        const QUnit U = units[u];
        sh.urows[u] = U.in_rows;
        sh.unnz[u] = U.in_nnz;
        sh.ug_first[u] = U.g_first;
        sh.ug_count[u] = U.g_count;
        sh.uq2[u] = U.q2;
        sh.uin[u] = U.in_dir;
        sh.usmask[u] = U.smask;
        sh.upull[u] = 0;
    }
    for (int i = threadIdx.x; i < p.n_targets; i += kThreads) {
        sh.t_unit[i] = t_unit[i];
        sh.t_state[i] = t_state[i];
    }
    for (int i = threadIdx.x; i < p.n_ugroups; i += kThreads) sh.u_group[i] = u_group[i];
    for (int q = threadIdx.x; q < kMaxStates; q += kThreads) {
        sh.fl[q] = 0;
        sh.fl_prev[q] = 0;
        sh.vstart[q] = 0;
        sh.vprev[q] = 0;
        sh.vnext[q] = 0;
    }
    if (threadIdx.x < 2) {
        sh.lvl[threadIdx.x] = 0;
        sh.flags[threadIdx.x] = 0;
    }
    if (threadIdx.x < kStats) sh.stats[threadIdx.x] = 0;
    for (int i = threadIdx.x; i < 3 * kMaxStates + 12 + 3 * p.n_groups; i += kThreads) sh.sctr[i] = 0;
    if (threadIdx.x == 0) {
        sh.cv[0] = Ctrs{&p.c->fl_count[0][0], p.c->rows_packed, p.c->lvl_bytes, p.c->lvl_edges,
                        p.c->srows_count, p.mf, kMaxGroups, 0};
        unsigned long long *b = sh.sctr + 3 * kMaxStates;
        sh.cv[1] = Ctrs{sh.sctr, b, b + 3, b + 6, b + 9, b + 12, p.n_groups, 0};
    }
    __syncthreads();
}

// ------------------------------------------------------------ discovery --
struct LevelCtx {
    int slot;                     // slot of the level being discovered
    int level;                    // the level being discovered
    const Ctrs *C;                // where its counters go
    int32_t *VL;
    const long long *vnext;       // first list entry of the level being discovered
    uint64_t *F;                  // frontier bits of that level, or null (not kept)
    // its long-row list, chunk map and short-row list are p.rows / p.cmap /
    // p.srl[slot] (read from the parameters when used, not held in registers)
};

// Ids of a row before the 16-byte boundary at or below its start: chunks of
// a long row begin on such boundaries so that every lane loads its 4 ids
// with one 128-bit load.
__device__ __forceinline__ int32_t row_skew(const int32_t *nbr, int32_t rb) {
    return (int32_t)(((uintptr_t)(nbr + rb) >> 2) & 3);
}

// Pairs a CTA discovers in one level, kept in its shared memory as well as
// in the visited lists, so that the CTA measures them itself as soon as its
// expansion ends (no grid barrier, no list reads); more than this in one CTA
// sends the level to the grid-wide measure pass over the lists.
constexpr int kDisc = 4096;
__shared__ int32_t s_dw[kDisc];  // the vertices
__shared__ uint8_t s_dq[kDisc];  // their states
__shared__ int s_nd;             // pairs discovered by this CTA in the level

// Lanes with found[r] have discovered the new pair (q2, w[r]) of the next
// level: kept in the CTA's discovery buffer (a shared-memory counter gives
// the position: no global round trip) and, on grid levels, its frontier bit
// set.  The buffer goes to the visited lists when the CTA's expansion ends
// (flush_discoveries: one reservation per state and CTA); pairs past the
// buffer's end are appended to the list of q2 at once (one reservation for
// the warp).  The rows the pair will expand are measured after the level
// (measure_buffer), with many lookups in flight instead of one chain per
// discovery.  q2 warp-uniform; all 32 lanes call.
template <int kB>
__device__ __forceinline__ void warp_discover_batch(const KParams &p, const LevelCtx &L,
                                                    const bool (&found)[kB], int q2,
                                                    const int32_t (&w)[kB]) {
    unsigned m[kB];
    int total = 0;
#pragma unroll
    for (int r = 0; r < kB; r++) {
        m[r] = __ballot_sync(kFull, found[r]);
        total += __popc(m[r]);
    }
    if (!total) return;
    const unsigned lane = lane_id();
    int pos = 0;
    if (lane == 0) pos = atomicAdd(&s_nd, total);
    pos = __shfl_sync(kFull, pos, 0);
    // entries k >= fit do not fit the buffer: listed directly
    const int fit = max(0, min(total, kDisc - pos));
    unsigned long long base = 0;
    if (fit < total) {  // warp-uniform
        if (lane == 0)
            base = atomicAdd(&L.C->fl[L.slot * kMaxStates + q2], (unsigned long long)(total - fit));
        base = __shfl_sync(kFull, base, 0);
    }
    int32_t *lst = L.VL + (size_t)q2 * p.n + L.vnext[q2];
    uint64_t *Fq = L.F ? L.F + (size_t)q2 * p.W : nullptr;
    int run = 0;
#pragma unroll
    for (int r = 0; r < kB; r++) {
        if (found[r]) {
            const int k = run + __popc(m[r] & lanemask_lt());
            if (k < fit) {
                s_dw[pos + k] = w[r];
                s_dq[pos + k] = (uint8_t)q2;
            } else {
                lst[base + (k - fit)] = w[r];
            }
            if (Fq)
                atomicOr((unsigned long long *)(Fq + ((uint32_t)w[r] >> 6)), 1ull << (w[r] & 63));
            if (p.pair_level) p.pair_level[(size_t)q2 * p.n + w[r]] = L.level;
        }
        run += __popc(m[r]);
    }
}

__device__ __forceinline__ void warp_discover(const KParams &p, const LevelCtx &L, bool found,
                                              int q2, int32_t w) {
    const bool f[1] = {found};
    const int32_t x[1] = {w};
    warp_discover_batch<1>(p, L, f, q2, x);
}

// End of a CTA's expansion (all its threads): the buffered discoveries go to
// the visited lists of the level in counter slot `slot` of C, after one
// reservation per state.  The buffer stays as it is for measure_buffer.
__device__ void flush_discoveries(const KParams &p, const Shared &sh, const Ctrs &C, int slot) {
    __shared__ unsigned s_cnt[kMaxStates];
    __shared__ unsigned long long s_base[kMaxStates];
    __syncthreads();
    const int nd = min(s_nd, kDisc);
    if (nd == 0) return;  // CTA-uniform
    if (threadIdx.x < kMaxStates) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < nd; i += kThreads) atomicAdd(&s_cnt[s_dq[i]], 1u);
    __syncthreads();
    if (threadIdx.x < p.S) {
        const unsigned c = s_cnt[threadIdx.x];
        s_base[threadIdx.x] =
            c ? atomicAdd(&C.fl[slot * kMaxStates + threadIdx.x], (unsigned long long)c) : 0ull;
        s_cnt[threadIdx.x] = 0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nd; i += kThreads) {
        const int q = s_dq[i];
        const unsigned k = atomicAdd(&s_cnt[q], 1u);
        p.VL[(size_t)q * p.n + sh.vnext[q] + s_base[q] + k] = s_dw[i];
    }
    __syncthreads();
}

// Rows in group g of new pairs (q, w[r]) of the level in counter slot
// `slot` (q the group's source state): edge mass of the group (the next
// push/pull choice), rows of >= kWarpRow edges to the long-row list
// (128-edge chunks from a 16-byte boundary), short rows of a listed group to
// the short-row list, and the push bytes / product edges of the rows.
// g warp-uniform; all 32 lanes call.
template <int kB>
__device__ __forceinline__ void measure_rows(const KParams &p, const Shared &sh, const Ctrs &C,
                                             int slot, const bool (&found)[kB], int g,
                                             const int32_t (&w)[kB],
                                             unsigned long long &acc_b, unsigned long long &acc_e) {
    const unsigned lane = lane_id();
    const DevAdj A = p.adj[sh.gd[g]];
    int32_t rb[kB], re[kB];
#pragma unroll
    for (int r = 0; r < kB; r++) {
        rb[r] = re[r] = 0;
        if (found[r]) adj_row(A, w[r], rb[r], re[r]);
    }
    int nch[kB];
    int my_rows = 0, my_chunks = 0, my_short = 0;
    unsigned long long mass = 0;
#pragma unroll
    for (int r = 0; r < kB; r++) {
        const int32_t deg = re[r] - rb[r];
        if (found[r]) {
            mass += (unsigned long long)deg;
            acc_b += 8ull + 4ull * (unsigned long long)deg;
            acc_e += (unsigned long long)deg * (unsigned long long)sh.gtpop[g];
        }
        nch[r] = (found[r] && deg >= kWarpRow)
                     ? (deg + row_skew(sh.gnbr[g], rb[r]) + kChunk - 1) / kChunk
                     : 0;
        my_rows += nch[r] ? 1 : 0;
        my_chunks += nch[r];
        my_short += (found[r] && deg > 0 && deg < kWarpRow && !sh.gdense[g]) ? 1 : 0;
    }
    if (mass) atomicAdd(&sh.s_mf[g], mass);
    // warp prefix of (short rows | long rows << 16, chunks); one
    // reservation in each list, both in flight together
    int ipk = my_short | (my_rows << 16), ic = my_chunks;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int yp = __shfl_up_sync(kFull, ipk, o);
        const int yc = __shfl_up_sync(kFull, ic, o);
        if ((int)lane >= o) {
            ipk += yp;
            ic += yc;
        }
    }
    const int tpk = __shfl_sync(kFull, ipk, 31), tc = __shfl_sync(kFull, ic, 31);
    const int ts = tpk & 0xffff, tr = tpk >> 16;
    if (!ts && !tr) return;  // warp-uniform
    unsigned long long sb = 0, old = 0;
    if (lane == 31 && ts) sb = atomicAdd(&C.srows[slot], (unsigned long long)ts);
    if (lane == 0 && tr)
        old = atomicAdd(&C.rows[slot], ((unsigned long long)tr << 40) | (unsigned long long)tc);
    sb = __shfl_sync(kFull, sb, 31);
    old = __shfl_sync(kFull, old, 0);
    if (ts) {
        long long at = (long long)sb + ((ipk & 0xffff) - my_short);
#pragma unroll
        for (int r = 0; r < kB; r++) {
            const int32_t deg = re[r] - rb[r];
            if (found[r] && deg > 0 && deg < kWarpRow && !sh.gdense[g]) {
                if (at < p.srow_cap) p.srl[slot][at] = make_int4(g, rb[r], re[r], w[r]);
                else set_status(p.c, (int32_t)RPQ_ERR_OOM);
                at++;
            }
        }
    }
    if (!tr) return;  // warp-uniform
    const int ir = ipk >> 16;
    long long ri = (long long)(old >> 40) + (ir - my_rows);
    long long cb = (long long)(old & ((1ull << 40) - 1)) + (ic - my_chunks);
#pragma unroll
    for (int r = 0; r < kB; r++) {
        if (!nch[r]) continue;
        if (ri < p.row_cap && cb + nch[r] <= p.chunk_cap) {
            p.rows[slot][ri] = Row{g, w[r], rb[r], re[r], cb};
            for (int k = 0; k < nch[r]; k++) p.cmap[slot][cb + k] = (int32_t)ri;
        } else {
            set_status(p.c, (int32_t)RPQ_ERR_OOM);
        }
        ri++;
        cb += nch[r];
    }
}

// End of a measure pass on this CTA: its sums of push bytes / product edges
// (per lane in acc_b / acc_e) and of edge mass per group go to counter slot
// `slot` of C.
__device__ __forceinline__ void measure_flush(const KParams &p, const Shared &sh, const Ctrs &C,
                                              int slot, unsigned long long *s_acc,
                                              unsigned long long acc_b, unsigned long long acc_e) {
    const unsigned lane = lane_id();
    for (int o = 16; o > 0; o >>= 1) {
        acc_b += __shfl_down_sync(kFull, acc_b, o);
        acc_e += __shfl_down_sync(kFull, acc_e, o);
    }
    if (threadIdx.x < 2) s_acc[threadIdx.x] = 0;
    __syncthreads();
    if (lane == 0) {
        if (acc_b) atomicAdd(&s_acc[0], acc_b);
        if (acc_e) atomicAdd(&s_acc[1], acc_e);
    }
    __syncthreads();
    for (int g = threadIdx.x; g < p.n_groups; g += kThreads) {
        const unsigned long long v = sh.s_mf[g];
        if (v) {
            atomicAdd(&C.mf[slot * C.mstride + g], v);
            sh.s_mf[g] = 0;
        }
    }
    if (threadIdx.x == 0) {
        if (s_acc[0]) atomicAdd(&C.bytes[slot], s_acc[0]);
        if (s_acc[1]) atomicAdd(&C.edges[slot], s_acc[1]);
    }
}

// After level j: measures the rows of every pair it discovered (level j+1's
// frontier: VL[q][vnext[q], vnext[q] + n_q), n_q in counter slot `slot` of
// C), on CTA `cta` of `ncta`.  The work is (group, batch of 32 x kR pairs)
// units spread over every warp, so the groups leaving one state are measured
// side by side, each lane with its kR lookups in flight together; then this
// CTA's sums of edge mass and push bytes / product edges go to the slot's
// counters.
// With `all`, every visited pair is measured instead (the whole list of each
// state, VL[q][0, vnext[q] + n_q)): the frontier of an Algorithm 2 step.
__device__ void measure_level(const KParams &p, const Shared &sh, const Ctrs &C, int slot, int cta,
                              int ncta, unsigned long long *s_acc, bool all = false) {
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    __shared__ long long s_cnt[kMaxStates];  // pairs per state, read in one round trip
    __shared__ long long s_first[kMaxStates];  // their first list entry
    if (threadIdx.x < p.S) {
        const long long fresh =
            (long long)*(volatile unsigned long long *)&C.fl[slot * kMaxStates + threadIdx.x];
        s_cnt[threadIdx.x] = all ? sh.vnext[threadIdx.x] + fresh : fresh;
        s_first[threadIdx.x] = all ? 0 : sh.vnext[threadIdx.x];
    }
    __syncthreads();
    // bpre[g] = batches of the groups before g (kept in the gather buffer,
    // idle between expansions); batch b goes to warp b / ncta of CTA b % ncta
    static_assert(kMaxGroups < kGather, "batch prefix fits the gather buffer");
    int32_t *bpre = sh.gbuf_k;
    if (warp == 0) {
        int32_t run = 0;
        for (int g0 = 0; g0 < p.n_groups; g0 += 32) {
            const int g = g0 + (int)lane;
            int32_t v = g < p.n_groups ? (int32_t)((s_cnt[sh.gq[g]] + 32 * kR - 1) / (32 * kR)) : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, v, o);
                if ((int)lane >= o) v += y;
            }
            if (g < p.n_groups) bpre[g + 1] = run + v;
            run += __shfl_sync(kFull, v, 31);
        }
        if (lane == 0) bpre[0] = 0;
    }
    __syncthreads();
    unsigned long long acc_b = 0, acc_e = 0;
    const int32_t nbatch = bpre[p.n_groups];
    for (int32_t b = warp * ncta + cta; b < nbatch; b += ncta * kWarps) {
        int lo = 0, hi = p.n_groups;  // the last group whose batches start at or before b
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (bpre[mid] <= b) lo = mid; else hi = mid;
        }
        const int g = lo, q = sh.gq[g];
        const long long cnt = s_cnt[q];
        const long long b0 = (long long)(b - bpre[g]) * 32 * kR;
        const int32_t *lst = p.VL + (size_t)q * p.n + s_first[q];
        bool ok[kR];
        int32_t w[kR];
#pragma unroll
        for (int r = 0; r < kR; r++) {
            const long long i = b0 + r * 32 + lane;
            ok[r] = i < cnt;
            w[r] = ok[r] ? __ldcg(lst + i) : 0;
        }
        measure_rows<kR>(p, sh, C, slot, ok, g, w, acc_b, acc_e);
    }
    measure_flush(p, sh, C, slot, s_acc, acc_b, acc_e);
}

// Measures the pairs this CTA discovered in the level (its buffer, s_nd <=
// kDisc of them) into counter slot `slot` of C: (batch of 32 x kR buffered
// pairs, group) units dealt round-robin to the CTA's warps, each lane's
// pairs of the group's source state measured together.
__device__ bool measure_buffer(const KParams &p, const Shared &sh, const Ctrs &C, int slot,
                               unsigned long long *s_acc) {
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int nd = s_nd;    // read by every thread before anyone resets it
    if (nd > p.disc_cap) {  // CTA-uniform
        __syncthreads();
        if (threadIdx.x == 0) s_nd = 0;
        return false;
    }
    const int nunits = (nd + 32 * kR - 1) / (32 * kR) * p.n_groups;
    unsigned long long acc_b = 0, acc_e = 0;
    for (int u = warp; u < nunits; u += kWarps) {
        const int b = u / p.n_groups, g = u - b * p.n_groups;
        const int q = sh.gq[g];
        bool ok[kR];
        int32_t w[kR];
        bool any = false;
#pragma unroll
        for (int r = 0; r < kR; r++) {
            const int i = b * 32 * kR + r * 32 + (int)lane;
            ok[r] = i < nd && s_dq[i] == q;
            w[r] = ok[r] ? s_dw[i] : 0;
            any = any || ok[r];
        }
        if (!__any_sync(kFull, any)) continue;
        measure_rows<kR>(p, sh, C, slot, ok, g, w, acc_b, acc_e);
    }
    measure_flush(p, sh, C, slot, s_acc, acc_b, acc_e);
    if (threadIdx.x == 0) s_nd = 0;
    return true;
}

// CTA 0, when some CTA's buffer overflowed: counter slot `slot` forgets
// the partial measurements before the grid measures the level from the
// lists.
__device__ __forceinline__ void measure_reset(const KParams &p, const Shared &sh, int slot) {
    const Ctrs &C = sh.cv[0];
    for (int g = threadIdx.x; g < p.n_groups; g += kThreads) C.mf[slot * C.mstride + g] = 0;
    if (threadIdx.x == 0) C.rows[slot] = C.srows[slot] = C.bytes[slot] = C.edges[slot] = 0;
}

// General relaxation (any number of target states per lane): edge (., w)
// into every target in tmask.  All 32 lanes must call.
__device__ void relax_general(const KParams &p, const Shared &sh, const int32_t *gsf,
                              const LevelCtx &L, bool valid, uint64_t tmask, int32_t w) {
    const uint64_t todo = valid ? tmask : 0ull;
    const uint32_t lo = __reduce_or_sync(kFull, (uint32_t)todo);
    const uint32_t hi = __reduce_or_sync(kFull, (uint32_t)(todo >> 32));
    uint64_t all = ((uint64_t)hi << 32) | lo;
    const uint32_t wi = (uint32_t)w >> 6;
    const uint64_t bit = 1ull << (w & 63);
    while (all) {
        const int q2 = __ffsll((long long)all) - 1;
        all &= all - 1;
        bool found = false;
        if ((todo >> q2) & 1ull) {
            uint64_t *Pw = p.P + (size_t)q2 * p.W + wi;
            if (!(__ldca(Pw) & bit)) {
                const unsigned long long old = atomicOr((unsigned long long *)Pw, bit);
                found = !(old & bit);
            }
        }
        warp_discover(p, L, found, q2, w);
    }
}

// Batched relaxation: kR edges per lane, loads issued together.  Fast path
// when every active edge of the warp round has the same single target
// state (the common case for a DFA).  All 32 lanes must call.
__device__ __forceinline__ void relax_batch(const KParams &p, const Shared &sh, const int32_t *gsf,
                                            const LevelCtx &L, const bool (&valid)[kR],
                                            const uint64_t (&tm)[kR], const int32_t (&w)[kR]) {
    uint64_t any = 0;
#pragma unroll
    for (int r = 0; r < kR; r++) any |= valid[r] ? tm[r] : 0ull;
    const uint32_t lo = __reduce_or_sync(kFull, (uint32_t)any);
    const uint32_t hi = __reduce_or_sync(kFull, (uint32_t)(any >> 32));
    const uint64_t all = ((uint64_t)hi << 32) | lo;
    if (!all) return;
    if (all & (all - 1)) {
#pragma unroll
        for (int r = 0; r < kR; r++) relax_general(p, sh, gsf, L, valid[r], tm[r], w[r]);
        return;
    }
    const int q2 = __ffsll((long long)all) - 1;
    uint64_t *Pq = p.P + (size_t)q2 * p.W;
    bool act[kR];
    uint64_t pw[kR];
    // on big levels most targets are visited: test first.  The test may be
    // served from L1 (hub words are read by many warps): P only gains bits
    // during a launch, so a stale copy can only miss bits, and the atomicOr
    // decides
    const bool pre = sh.flags[0] != 0;
#pragma unroll
    for (int r = 0; r < kR; r++) {
        act[r] = valid[r] && ((tm[r] >> q2) & 1ull);
        pw[r] = (act[r] && pre) ? __ldca(Pq + ((uint32_t)w[r] >> 6)) : (act[r] ? 0ull : ~0ull);
    }
#pragma unroll
    for (int r = 0; r < kR; r++) {
        act[r] = act[r] && !((pw[r] >> (w[r] & 63)) & 1ull);
        if (act[r]) {
            const uint64_t bit = 1ull << (w[r] & 63);
            const unsigned long long old =
                atomicOr((unsigned long long *)(Pq + ((uint32_t)w[r] >> 6)), bit);
            act[r] = !(old & bit);
        }
    }
    warp_discover_batch<kR>(p, L, act, q2, w);
}

// ---------------------------------------------------------------- phases -
// Tile claims of CTA `cta` of `ncta` working CTAs: the first tile of every
// CTA is static, later ones come from a counter that therefore starts past
// the static ones; a CTA working alone just steps.  Thread 0 asks for the
// next tile as soon as the current one is known, so the counter's round
// trip overlaps the tile's work.  CTA-uniform results.
struct TileClaims {
    unsigned long long *ctr;
    long long tile;
    int cta, ncta;
    int k = 0;
    long long next = 0;  // thread 0: the tile claimed ahead
    __device__ TileClaims(unsigned long long *c, long long t, int a, int n)
        : ctr(c), tile(t), cta(a), ncta(n) {}
    __device__ __forceinline__ long long take(long long *s_claim, long long total) {
        long long t;
        if (k == 0) {
            t = (long long)cta * tile;
        } else if (ncta == 1) {
            t = (long long)k * tile;
        } else {
            if (threadIdx.x == 0) *s_claim = next;
            __syncthreads();
            t = *s_claim;
            __syncthreads();
        }
        k++;
        if (ncta > 1 && threadIdx.x == 0 && t < total)
            next = (long long)ncta * tile + (long long)atomicAdd(ctr, (unsigned long long)tile);
        return t;
    }
};

// Level j on CTA `cta` of `ncta` working CTAs (the whole grid, or CTA 0
// alone for a small level).  Frontier bits (read only by pull) are kept for
// the levels a grid level (`on_grid`) discovers; `clear_prev`: level j-1's
// bits exist and are cleared here.
__device__ void expand_phase(const KParams &p, int j, const Shared &sh, const int32_t *gsf,
                             long long *s_claim, unsigned long long *s_acc, int cta, int ncta,
                             bool on_grid, bool clear_prev, bool cur_smem) {
    const int cs = j % 3, ns = (j + 1) % 3, os = (j + 2) % 3;
    const uint64_t *F = p.F[cs];
    // level j's counters are where the level before left them; level j+1's
    // go to device memory on a grid level, to CTA 0's shared memory otherwise
    const Ctrs &Cc = sh.cv[cur_smem ? 1 : 0];
    const Ctrs &Cn = sh.cv[on_grid ? 0 : 1];
    (void)s_acc;
    LevelCtx L{ns, j + 1, &Cn, p.VL, sh.vnext, on_grid ? p.F[ns] : nullptr};
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x < 2) s_acc[threadIdx.x] = 0;

    // housekeeping: clear F of level j-1 (slot os) through its list range
    // and reset slot os's counters (nothing else touches slot os now)
    if (clear_prev) {
        for (int q = 0; q < p.S; q++) {
            const unsigned long long cnt = sh.fl_prev[q];
            const int32_t *lst = p.VL + (size_t)q * p.n + sh.vprev[q];
            uint64_t *Fo = p.F[os] + (size_t)q * p.W;
            for (unsigned long long i = (unsigned long long)cta * kThreads + threadIdx.x; i < cnt;
                 i += (unsigned long long)ncta * kThreads)
                Fo[(uint32_t)__ldcg(lst + i) >> 6] = 0;
        }
    }
    if (cta == 0) {
        // slot os serves level j+2, which may run in either mode: clear both
        for (int k = 0; k < 2; k++) {
            const Ctrs &C = sh.cv[k];
            for (int i = threadIdx.x; i < p.S; i += kThreads) C.fl[os * kMaxStates + i] = 0;
            for (int i = threadIdx.x; i < p.n_groups; i += kThreads) C.mf[os * C.mstride + i] = 0;
            if (threadIdx.x == 0) C.rows[os] = C.bytes[os] = C.edges[os] = C.srows[os] = 0;
        }
        if (threadIdx.x == 0) {
            p.c->claim_chunk[os] = 0;
            p.c->claim_item[os] = 0;
            p.c->claim_pull[os] = 0;
        }
    }
    __syncthreads();

    // (1) chunks of long rows: chunk c goes to CTA c % grid, warp
    //     (c / grid) % kWarps of it, so consecutive chunks (one long row)
    //     spread over all SMs; static, no claims
    {
        const unsigned long long packed = *(volatile unsigned long long *)&Cc.rows[cs];
        const long long nchunks = (long long)(packed & ((1ull << 40) - 1));
        const Row *R = p.rows[cs];
        const int32_t *CM = p.cmap[cs];
        const long long stride = (long long)ncta * kWarps;
        long long c = (long long)cta + (long long)warp * ncta;
        int ri_next = c < nchunks ? __ldcg(CM + c) : 0;
        for (; c < nchunks; c += stride) {
            // this chunk's row record and the next chunk's row index: one round trip
            const int ri = ri_next;
            const int2 gv = __ldcg(reinterpret_cast<const int2 *>(&R[ri].g));
            const int2 be = __ldcg(reinterpret_cast<const int2 *>(&R[ri].b));
            const long long c0r = __ldcg(&R[ri].chunk0);
            ri_next = c + stride < nchunks ? __ldcg(CM + c + stride) : 0;
            const int g = gv.x;
            const uint64_t tmv = sh.tpush[g];
            if (!tmv) continue;  // warp-uniform
            const int32_t rb = be.x, re = be.y;
            const int32_t *nbr = sh.gnbr[g];
            // the chunk's kChunk ids from a 16-byte boundary: lane i loads
            // its kR ids with kR / 4 128-bit loads (ids 4i.. of each 128-id
            // block); ids outside the row are masked
            const int32_t b = rb - row_skew(nbr, rb) + (int32_t)((c - c0r) * kChunk);
            const int32_t e = min(re, b + kChunk);
            static_assert(kR % 4 == 0, "whole 128-bit loads per lane and round");
            int32_t vv[kR];
#pragma unroll
            for (int h = 0; h < kR / 4; h++) {
                const int32_t k0 = b + h * 128 + 4 * (int32_t)lane;
                int4 v4 = make_int4(0, 0, 0, 0);
                if (k0 < e) v4 = __ldg(reinterpret_cast<const int4 *>(nbr + k0));
                vv[4 * h] = v4.x;
                vv[4 * h + 1] = v4.y;
                vv[4 * h + 2] = v4.z;
                vv[4 * h + 3] = v4.w;
            }
            bool valid[kR];
            uint64_t tm[kR];
            int32_t w[kR];
#pragma unroll
            for (int r = 0; r < kR; r++) {
                const int32_t k = b + (r / 4) * 128 + 4 * (int32_t)lane + (r & 3);
                valid[r] = k >= rb && k < e;
                w[r] = valid[r] ? vv[r] : 0;
                tm[r] = tmv;
            }
            relax_batch(p, sh, gsf, L, valid, tm, w);
        }
    }

    trace_put(p, j, 8, global_timer_ns());
    // (2) short rows of push groups: first the level's short-row list
    //     (hypersparse groups: only non-empty rows, ranges known), then the
    //     frontier items of dense groups (row found by its offsets).  Each
    //     warp takes batches of 32 items (batch b to warp b / ncta of CTA
    //     b % ncta, so a small level spreads over every CTA), scans their
    //     degrees (< kWarpRow each) with shuffles and walks the batch's edges
    //     32 x kR at a time; the row of an edge is found by a binary search
    //     over the lanes' inclusive sums.  No CTA barrier: every warp keeps
    //     its own loads in flight.
    {
        const long long n_listed = sh.nsrow[0];
        const long long total_items = n_listed + sh.dpref[p.n_groups];
        const int4 *SRL = p.srl[cs];
        const long long nbatch = (total_items + 31) / 32;
        const long long stride = (long long)ncta * kWarps;
        for (long long bt = (long long)cta + (long long)warp * ncta; bt < nbatch; bt += stride) {
            const long long i = bt * 32 + lane;
            int g = 0;
            int32_t rb = 0, re = 0;
            if (i < n_listed) {
                const int4 e = __ldcg(SRL + i);
                g = e.x;
                if (sh.tpush[g]) {  // rows of groups that pull this level are skipped
                    rb = e.y;
                    re = e.z;
                }
            } else if (i < total_items) {
                const long long k = i - n_listed;
                int lo = 0, hi = p.n_groups - 1;  // last group with dpref <= k
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sh.dpref[mid] <= k) lo = mid; else hi = mid - 1;
                }
                g = lo;
                const int q = sh.gq[g];
                const int32_t v = __ldcg(p.VL + (size_t)q * p.n + sh.vstart[q] + (k - sh.dpref[g]));
                const int32_t *off = p.adj[sh.gd[g]].off;
                rb = __ldg(off + v);
                re = __ldg(off + v + 1);
                if (re - rb >= kWarpRow) re = rb;  // expanded through the chunk list
            }
            const int32_t deg = re - rb;
            int32_t incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, incl, o);
                if ((int)lane >= o) incl += y;
            }
            const int32_t excl = incl - deg;
            const int32_t tot = __shfl_sync(kFull, incl, 31);
            for (int32_t base = 0; base < tot; base += 32 * kR) {
                bool valid[kR];
                uint64_t tm[kR];
                int32_t w[kR];
#pragma unroll
                for (int r = 0; r < kR; r++) {
                    const int32_t e = base + r * 32 + (int32_t)lane;
                    // owner: the first lane whose inclusive sum exceeds e
                    int own = 0;
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1) {
                        const int32_t x = __shfl_sync(kFull, incl, own + st - 1);
                        if (x <= e) own += st;
                    }
                    own = min(own, 31);
                    const int32_t orb = __shfl_sync(kFull, rb, own);
                    const int32_t oex = __shfl_sync(kFull, excl, own);
                    const int og = __shfl_sync(kFull, g, own);
                    valid[r] = e < tot;
                    w[r] = valid[r] ? __ldg(sh.gnbr[og] + orb + (e - oex)) : 0;
                    tm[r] = valid[r] ? sh.tpush[og] : 0ull;
                }
                relax_batch(p, sh, gsf, L, valid, tm, w);
            }
        }
    }

    trace_put(p, j, 9, global_timer_ns());
    // (3) pull units: sweep the rows of the in-adjacency, kPullRows rows per
    //     thread with their round trips overlapped
    const long long total_rows = sh.upref[p.n_units];
    TileClaims pull_claims(&p.c->claim_pull[cs], kPullTile, cta, ncta);
    while (total_rows > 0) {
        const long long t0 = pull_claims.take(s_claim, total_rows);
        if (t0 >= total_rows) break;
        int u = 0;
        {
            int lo = 0, hi = p.n_units - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sh.upref[mid] <= t0) lo = mid; else hi = mid - 1;
            }
            u = lo;
        }
        const DevAdj A = p.adj[sh.uin[u]];
        const int uq2 = sh.uq2[u];
        const uint64_t usm = sh.usmask[u];
        int32_t w[kPullRows], rb[kPullRows], re[kPullRows];
        bool cand[kPullRows], found[kPullRows], pending[kPullRows];
#pragma unroll
        for (int h = 0; h < kPullRows; h++) {
            const long long r = t0 + h * kThreads + threadIdx.x - sh.upref[u];
            w[h] = rb[h] = re[h] = 0;
            cand[h] = found[h] = pending[h] = false;
            if (r < sh.urows[u]) {
                if (A.fmt == ADJ_DENSE) {
                    w[h] = (int32_t)r;
                    rb[h] = __ldg(A.off + w[h]);
                    re[h] = __ldg(A.off + w[h] + 1);
                } else {
                    w[h] = __ldg(A.rows + r);
                    rb[h] = __ldg(A.off + r);
                    re[h] = __ldg(A.off + r + 1);
                }
                cand[h] = true;
            }
        }
#pragma unroll
        for (int h = 0; h < kPullRows; h++)
            cand[h] = cand[h] && re[h] > rb[h] &&
                      !((__ldca(p.P + (size_t)uq2 * p.W + ((uint32_t)w[h] >> 6)) >> (w[h] & 63)) &
                        1ull);
        // up to kWarpRow in-neighbours of each row, kPullBatch at a time:
        // their ids, then their frontier bits, every row's batch together
        for (int32_t step = 0; step < kWarpRow; step += kPullBatch) {
            bool more = false;
#pragma unroll
            for (int h = 0; h < kPullRows; h++)
                more |= cand[h] && !found[h] && rb[h] + step < min(re[h], rb[h] + kWarpRow);
            if (!more) break;
            int32_t x[kPullRows][kPullBatch];
#pragma unroll
            for (int h = 0; h < kPullRows; h++) {
                const int32_t lim = min(re[h], rb[h] + kWarpRow);
                const bool live = cand[h] && !found[h];
#pragma unroll
                for (int r = 0; r < kPullBatch; r++) {
                    const int32_t k = rb[h] + step + r;
                    x[h][r] = live && k < lim ? __ldg(A.nbr + k) : -1;
                }
            }
            uint64_t sm = usm;
            while (sm) {
                const int q = __ffsll((long long)sm) - 1;
                sm &= sm - 1;
                const uint64_t *Fq = F + (size_t)q * p.W;
                uint64_t fw[kPullRows][kPullBatch];
#pragma unroll
                for (int h = 0; h < kPullRows; h++)
#pragma unroll
                    for (int r = 0; r < kPullBatch; r++)
                        fw[h][r] = x[h][r] >= 0 ? __ldcg(Fq + ((uint32_t)x[h][r] >> 6)) : 0ull;
#pragma unroll
                for (int h = 0; h < kPullRows; h++)
#pragma unroll
                    for (int r = 0; r < kPullBatch; r++)
                        found[h] |= x[h][r] >= 0 && ((fw[h][r] >> (x[h][r] & 63)) & 1ull);
            }
        }
#pragma unroll
        for (int h = 0; h < kPullRows; h++)
            pending[h] = cand[h] && !found[h] && re[h] - rb[h] > kWarpRow;
        // rows of more than kWarpRow in-edges: the warp scans the rest of
        // each, 32 in-neighbours a round, one row after the other
#pragma unroll
        for (int h = 0; h < kPullRows; h++) {
            unsigned m;
            while ((m = __ballot_sync(kFull, pending[h])) != 0) {
                const int leader = __ffs(m) - 1;
                const int32_t b = __shfl_sync(kFull, rb[h], leader) + kWarpRow;
                const int32_t e = __shfl_sync(kFull, re[h], leader);
                bool hit = false;
                for (int32_t base = b; base < e; base += 32) {
                    const int32_t k = base + (int32_t)lane;
                    bool hk = false;
                    if (k < e) {
                        const int32_t x = __ldg(A.nbr + k);
                        uint64_t sm = usm;
                        while (sm) {
                            const int q = __ffsll((long long)sm) - 1;
                            sm &= sm - 1;
                            if ((__ldcg(F + (size_t)q * p.W + ((uint32_t)x >> 6)) >> (x & 63)) &
                                1ull) {
                                hk = true;
                                break;
                            }
                        }
                    }
                    if (__ballot_sync(kFull, hk)) {
                        hit = true;
                        break;
                    }
                }
                if ((int)lane == leader) {
                    pending[h] = false;
                    found[h] = hit;
                }
            }
        }
        bool disc[kPullRows];
#pragma unroll
        for (int h = 0; h < kPullRows; h++) {
            disc[h] = false;
            if (found[h]) {
                const uint64_t bit = 1ull << (w[h] & 63);
                const unsigned long long old = atomicOr(
                    (unsigned long long *)(p.P + (size_t)uq2 * p.W + ((uint32_t)w[h] >> 6)), bit);
                disc[h] = !(old & bit);
            }
        }
        warp_discover_batch<kPullRows>(p, L, disc, uq2, w);
    }

    if (threadIdx.x == 0) {
        if (p.trace && j < p.trace_cap) {  // spread of the CTAs' finishing times
            const unsigned long long t = global_timer_ns();
            atomicMax(&p.trace[(size_t)j * kTraceFields + 10], ~t);
            atomicMax(&p.trace[(size_t)j * kTraceFields + 11], t);
        }
    }
}

// Writes the set bits of words [w0, w1) of `bits` as ascending vertex ids to
// out[0..), skipping positions at or past `limit` (CTA-wide; all threads).
__device__ void compact_bits(const uint64_t *bits, int64_t w0, int64_t w1, int32_t *out,
                             long long limit) {
    __shared__ long long s_wsum[kWarps + 1];
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    long long run = 0;
    for (int64_t base = w0; base < w1; base += kThreads) {
        const int64_t wi = base + threadIdx.x;
        uint64_t r = wi < w1 ? __ldcg(bits + wi) : 0ull;
        const int32_t c = __popcll(r);
        int32_t incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[warp] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long acc = 0;
            for (int x = 0; x < kWarps; x++) {
                const long long t = s_wsum[x];
                s_wsum[x] = acc;
                acc += t;
            }
            s_wsum[kWarps] = acc;
        }
        __syncthreads();
        long long pos = run + s_wsum[warp] + incl - c;
        while (r) {
            const int b = __ffsll((long long)r) - 1;
            r &= r - 1;
            if (pos < limit) out[pos] = (int32_t)(wi * 64 + b);
            pos++;
        }
        run += s_wsum[kWarps];
        __syncthreads();
    }
}

// After grid level j (every CTA, after the barrier that closed it): when
// the level discovered at least p.sort_min pairs, each state's new list
// range VL[q][vnext[q], vnext[q] + n_q) is rewritten in ascending vertex
// order from the frontier bits F_{j+1}[q] (which hold exactly those pairs):
// per-CTA bit counts over contiguous word ranges, one barrier, then each CTA
// writes its range's ids after the counts of the CTAs before it, and one
// more barrier.  The range holds the same set, so nothing but the order
// changes.  Returns false when a barrier failed.
__device__ bool sort_level(const KParams &p, const Shared &sh, int j) {
    const int ns = (j + 1) % 3;
    __shared__ long long s_n[kMaxStates];
    __shared__ long long s_tot;
    if (threadIdx.x < p.S)
        s_n[threadIdx.x] =
            (long long)*(volatile unsigned long long *)&p.c->fl_count[ns][threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int q = 0; q < p.S; q++) t += s_n[q];
        s_tot = t;
    }
    __syncthreads();
    if (p.sort_min <= 0 || s_tot < p.sort_min) return true;  // uniform over the grid
    const int64_t W = p.W;
    const int64_t per = (W + gridDim.x - 1) / gridDim.x;
    const int64_t w0 = min((int64_t)W, (int64_t)blockIdx.x * per);
    const int64_t w1 = min((int64_t)W, w0 + per);
    __shared__ unsigned long long s_c;
    for (int q = 0; q < p.S; q++) {
        if (!s_n[q]) continue;
        const uint64_t *Fq = p.F[ns] + (size_t)q * W;
        unsigned long long c = 0;
        for (int64_t wi = w0 + threadIdx.x; wi < w1; wi += kThreads) c += __popcll(__ldcg(Fq + wi));
        for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFull, c, o);
        if (threadIdx.x == 0) s_c = 0;
        __syncthreads();
        if (lane_id() == 0 && c) atomicAdd(&s_c, c);
        __syncthreads();
        if (threadIdx.x == 0) p.sort_cnt[(size_t)q * gridDim.x + blockIdx.x] = (uint32_t)s_c;
    }
    if (!grid_barrier(p)) return false;
    __shared__ long long s_base;
    for (int q = 0; q < p.S; q++) {
        if (!s_n[q]) continue;
        long long b = 0;
        for (unsigned x = threadIdx.x; x < blockIdx.x; x += kThreads)
            b += __ldcg(p.sort_cnt + (size_t)q * gridDim.x + x);
        for (int o = 16; o > 0; o >>= 1) b += __shfl_down_sync(kFull, b, o);
        if (threadIdx.x == 0) s_base = 0;
        __syncthreads();
        if (lane_id() == 0 && b) atomicAdd((unsigned long long *)&s_base, (unsigned long long)b);
        __syncthreads();
        const long long base = s_base;
        __syncthreads();
        compact_bits(p.F[ns] + (size_t)q * W, w0, w1, p.VL + (size_t)q * p.n + sh.vnext[q] + base,
                     s_n[q] - base);
    }
    return grid_barrier(p);
}

// Level bookkeeping in shared memory, from the device counters of level j
// (stable while level j runs: its discoveries go to slot (j+1) % 3): the
// current level becomes the previous one, and level j's frontier of state q
// is the list range VL[q][vstart[q], vstart[q] + fl[q]).  All loads are
// issued before the first use (one memory round trip).
__device__ __forceinline__ void level_advance(const KParams &p, int j, const Shared &sh, bool account,
                                              bool in_smem) {
    static_assert(kMaxGroups <= 2 * kThreads && kMaxStates <= kThreads, "one pass of loads");
    const int cs = j % 3;
    const int t = threadIdx.x, g1 = t + kThreads;
    const Ctrs &C = sh.cv[in_smem ? 1 : 0];
    const volatile unsigned long long *fl = C.fl + cs * kMaxStates;
    const volatile unsigned long long *mf = C.mf + cs * C.mstride;
    const unsigned long long fv = t < p.S ? fl[t] : 0ull;
    const unsigned long long m0 = t < p.n_groups ? mf[t] : 0ull;
    const unsigned long long m1 = g1 < p.n_groups ? mf[g1] : 0ull;
    unsigned long long lb = 0, le = 0;
    const unsigned long long nsr = t == 0 ? *(volatile unsigned long long *)&C.srows[cs] : 0ull;
    if (account && t == 0) {
        lb = *(volatile unsigned long long *)&C.bytes[cs];
        le = *(volatile unsigned long long *)&C.edges[cs];
    }
    const bool a2 = sh.flags[1] != 0;
    __syncthreads();
    if (t < kMaxStates) {
        if (a2) {
            // an Algorithm 2 step expands every visited pair: the whole list
            // of each state; fl_prev / vprev hold the last step's new pairs
            const long long all = sh.vnext[t] + (long long)fv;
            sh.fl_prev[t] = fv;
            sh.vprev[t] = sh.vnext[t];
            sh.vstart[t] = 0;
            sh.fl[t] = (unsigned long long)all;
            sh.vnext[t] = all;
        } else {
            sh.fl_prev[t] = sh.fl[t];
            sh.vprev[t] = sh.vstart[t];
            sh.vstart[t] += (long long)sh.fl[t];
            sh.fl[t] = fv;
            sh.vnext[t] = sh.vstart[t] + (long long)fv;
        }
    }
    if (t < p.n_groups) sh.mfv[t] = m0;
    if (g1 < p.n_groups) sh.mfv[g1] = m1;
    if (t == 0) {
        sh.lvl[0] = lb;
        sh.lvl[1] = le;
        sh.nsrow[0] = (long long)nsr;
    }
    __syncthreads();
}

// The same state for a CTA joining at level j from the gate, from what CTA 0
// published when it released the gate.
__device__ __forceinline__ void level_join(const KParams &p, int j, const Shared &sh) {
    const int cs = j % 3;
    const int t = threadIdx.x, g1 = t + kThreads;
    const bool in = t < p.S;
    const unsigned long long fv = in ? *(volatile unsigned long long *)&p.c->fl_count[cs][t] : 0ull;
    const long long fp = in ? __ldcg(&p.c->pub_flprev[t]) : 0;
    const long long vp = in ? __ldcg(&p.c->pub_vprev[t]) : 0;
    const long long vs = in ? __ldcg(&p.c->pub_vstart[t]) : 0;
    const unsigned long long m0 = t < p.n_groups ? __ldcg(p.mf + cs * kMaxGroups + t) : 0ull;
    const unsigned long long m1 = g1 < p.n_groups ? __ldcg(p.mf + cs * kMaxGroups + g1) : 0ull;
    const unsigned long long nsr =
        t == 0 ? *(volatile unsigned long long *)&p.c->srows_count[cs] : 0ull;
    __syncthreads();
    if (t == 0) sh.nsrow[0] = (long long)nsr;
    if (t < kMaxStates) {
        sh.fl_prev[t] = (unsigned long long)fp;
        sh.vprev[t] = vp;
        sh.vstart[t] = vs;
        sh.fl[t] = fv;
        sh.vnext[t] = vs + (long long)fv;
    }
    if (t < p.n_groups) sh.mfv[t] = m0;
    if (g1 < p.n_groups) sh.mfv[g1] = m1;
    __syncthreads();
}

constexpr int kPlanStop = 0, kPlanGrid = 1, kPlanSolo = 2;
// push levels with more edges than this test P before each atomicOr (most
// of their targets are already visited); smaller ones go straight to it
constexpr unsigned long long kPrecheckMass = 4096;

// Plans level j from the shared state (every working CTA computes the same):
// stop when M_j is empty or the level cap is reached; else push or pull per
// unit (d, q'), and whether the level is small enough for CTA 0 alone.
// CTA 0 also accumulates the query's statistics (`account`).
__device__ __forceinline__ int level_plan(const KParams &p, int j, const Shared &sh, bool account) {
    __shared__ int s_plan;
    const bool a2 = sh.flags[1] != 0;  // an Algorithm 2 step (CTA 0 alone)
    long long total = 0, fresh = 0;
    for (int q = 0; q < p.S; q++) {
        total += (long long)sh.fl[q];
        fresh += (long long)(a2 ? sh.fl_prev[q] : sh.fl[q]);
    }
    // Algorithm 1 stops when M = 0, Algorithm 2 when P stops changing: both
    // when the last step found no new pair
    const bool expand = fresh > 0 && (p.max_levels == 0 || j < p.max_levels);
    if (account && threadIdx.x == 0) {
        sh.stats[kStVisited] += fresh;
        if (fresh > 0 && j > 0) sh.stats[kStLevels] = j;
        if (expand) {
            sh.stats[kStExpanded] += total;
            sh.stats[kStPushBytes] += (long long)sh.lvl[0];
            sh.stats[kStProductEdges] += (long long)sh.lvl[1];
        }
    }
    if (!expand) return kPlanStop;
    for (int u = threadIdx.x; u < p.n_units; u += kThreads) {
        unsigned long long mass = 0, pairs = 0;
        for (int k = 0; k < sh.ug_count[u]; k++) {
            const int g = sh.u_group[sh.ug_first[u] + k];
            mass += sh.mfv[g];
            pairs += sh.fl[sh.gq[g]];
        }
        const bool pull = !a2 &&
                          (double)mass * (double)p.alpha >
                              (double)sh.unnz[u] + (double)sh.urows[u] &&
                          (long long)pairs >= p.min_pull;
        sh.upull[u] = pull ? 1 : 0;
    }
    __syncthreads();
    for (int g = threadIdx.x; g < p.n_groups; g += kThreads) {
        uint64_t tm = 0;
        for (int k = 0; k < sh.gt_count[g]; k++) {
            const int t = sh.gt_first[g] + k;
            if (!sh.upull[sh.t_unit[t]]) tm |= 1ull << sh.t_state[t];
        }
        sh.tpush[g] = tm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;  // frontier items of dense push groups
        unsigned long long mass = 0;
        for (int g = 0; g < p.n_groups; g++) {
            sh.dpref[g] = acc;
            if (sh.tpush[g]) {
                mass += sh.mfv[g];
                if (sh.gdense[g]) acc += (long long)sh.fl[sh.gq[g]];
            }
        }
        sh.dpref[p.n_groups] = acc;
        acc += sh.nsrow[0];  // plus the listed short rows: the items to gather
        long long ra = 0, npush = 0, npull = 0;
        for (int u = 0; u < p.n_units; u++) {
            sh.upref[u] = ra;
            if (sh.upull[u]) {
                ra += (sh.urows[u] + kPullTile - 1) / kPullTile * kPullTile;
                npull++;
            } else {
                npush++;
            }
        }
        sh.upref[p.n_units] = ra;
        if (account) {
            sh.stats[kStPushUnits] += npush;
            sh.stats[kStPullUnits] += npull;
        }
        const bool solo = a2 || (p.solo_mass >= 0 && npull == 0 &&
                                 mass <= (unsigned long long)p.solo_mass && acc <= p.solo_items);
        s_plan = solo ? kPlanSolo : kPlanGrid;
        sh.flags[0] = (long long)mass > p.precheck_mass ? 1 : 0;
    }
    __syncthreads();
    const int plan = s_plan;
    __syncthreads();
    return plan;
}

// ---------------------------------------------------------------- gate ---
// While CTA 0 runs levels alone the other CTAs wait at the gate: a word
// holding (launch epoch << 32) | (command << 24) | releases so far.  Every
// CTA counts the releases it has seen, so a CTA that arrives late still
// finds its release; the epoch tells this launch's releases from a previous
// launch's.
constexpr int kGateLevel = 1;   // join the published level
constexpr int kGateFinal = 2;   // join the grid-wide answer sweep after the published level
constexpr int kGateDone = 3;    // the query is finished: exit
constexpr int kGateError = -1;  // the query failed, or CTA 0 stalled past the limit

// Waits for release number seen + 1 and returns its command; kGateError when
// the query failed or CTA 0 made no progress (its heartbeat did not change)
// for the timeout.
__device__ __forceinline__ int gate_wait(const KParams &p, unsigned &seen) {
    __shared__ int s_cmd;
    if (threadIdx.x == 0) {
        volatile unsigned long long *gp = &p.c->gate;
        volatile unsigned long long *bp = &p.c->beat;
        unsigned long long beat = *bp;
        uint64_t t0 = global_timer_ns();
        int cmd = kGateError;
        for (unsigned it = 1;; it++) {
            const unsigned long long gv = *gp;
            if ((uint32_t)(gv >> 32) == p.epoch && ((uint32_t)gv & 0xffffffu) > seen) {
                cmd = (int)((gv >> 24) & 0xffu);
                if (cmd != kGateDone) __threadfence();  // before reading what CTA 0 published
                break;
            }
            if ((it & 31u) == 0) {
                if (load_status(p.c) != 0) break;
                const unsigned long long b = *bp;
                const uint64_t now = global_timer_ns();
                if (b != beat) {
                    beat = b;
                    t0 = now;
                } else if (now - t0 > p.wait_ns) {
                    set_status(p.c, (int32_t)RPQ_ERR_TIMEOUT);
                    break;
                }
            }
            __nanosleep(128);
        }
        s_cmd = cmd;
    }
    __syncthreads();
    const int cmd = s_cmd;
    __syncthreads();
    seen++;
    return cmd;
}

// CTA 0 (all its threads): publish the state of level j, then release the
// gate with `cmd`.
__device__ __forceinline__ void gate_release(const KParams &p, const Shared &sh, unsigned &seen, int cmd,
                                             int j) {
    const unsigned long long word = ((unsigned long long)p.epoch << 32) |
                                    ((unsigned long long)cmd << 24) | (unsigned long long)(seen + 1);
    seen++;
    if (cmd == kGateDone) {  // nothing to publish: the parked CTAs just exit
        if (threadIdx.x == 0) *(volatile unsigned long long *)&p.c->gate = word;
        return;
    }
    for (int q = threadIdx.x; q < p.S; q += kThreads) {
        p.c->pub_vstart[q] = sh.vstart[q];
        p.c->pub_vprev[q] = sh.vprev[q];
        p.c->pub_flprev[q] = (long long)sh.fl_prev[q];
    }
    if (threadIdx.x == 0) *(volatile int32_t *)&p.c->pub_level = j;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) *(volatile unsigned long long *)&p.c->gate = word;
    __syncthreads();
}

__device__ __forceinline__ void heartbeat(const KParams &p) {
    if (threadIdx.x == 0) atomicAdd(&p.c->beat, 1ull);
}

// A CTA leaving the grid for the gate has finished with the level it
// leaves (its counters read, its frontier bits cleared): it says so here.
__device__ __forceinline__ void park_arrive(const KParams &p) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(&p.c->parked, 1ull);
    }
}

// CTA 0 (all threads): waits until `expected` parkings have arrived, before
// it reuses what the parking CTAs were still reading or clearing.  Bounded;
// false on timeout or a failed query.
__device__ __forceinline__ bool park_wait(const KParams &p, unsigned long long expected) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        volatile unsigned long long *pk = &p.c->parked;
        int ok = 1;
        if (*pk < expected) {
            const uint64_t t0 = global_timer_ns();
            for (unsigned it = 1; *pk < expected; it++) {
                if ((it & 63u) == 0) {
                    if (load_status(p.c) != 0) {
                        ok = 0;
                        break;
                    }
                    if (global_timer_ns() - t0 > p.wait_ns) {
                        set_status(p.c, (int32_t)RPQ_ERR_TIMEOUT);
                        ok = 0;
                        break;
                    }
                }
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    const int ok = s_ok;
    __syncthreads();
    return ok != 0;
}

// F x P with ordered compaction (two phases around one barrier).
__device__ void final_phase(const KParams &p, long long *s_tmp) {
    const int64_t W = p.W;
    const int64_t per = (W + gridDim.x - 1) / gridDim.x;
    const int64_t w0 = (int64_t)min((long long)W, (long long)blockIdx.x * per);
    const int64_t w1 = (int64_t)min((long long)W, (long long)(w0 + per));
    long long cnt = 0;
    for (int64_t wi = w0 + threadIdx.x; wi < w1; wi += kThreads) {
        uint64_t r = 0;
        uint64_t fm = p.final_mask;
        while (fm) {
            const int q = __ffsll((long long)fm) - 1;
            fm &= fm - 1;
            r |= __ldcg(p.P + (size_t)q * W + wi);
        }
        if (p.out_bits) p.out_bits[wi] = r;
        cnt += __popcll(r);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kFull, cnt, o);
    if (threadIdx.x == 0) *s_tmp = 0;
    __syncthreads();
    if (lane_id() == 0) atomicAdd((unsigned long long *)s_tmp, (unsigned long long)cnt);
    __syncthreads();
    if (threadIdx.x == 0) p.fin_sums[blockIdx.x] = *s_tmp;
}

// Second pass: each CTA writes its range's answer vertices after the counts
// of the CTAs before it, and clears the final states' P words it read.
__device__ void final_write(const KParams &p, long long *s_tmp) {
    const int64_t W = p.W;
    const int64_t per = (W + gridDim.x - 1) / gridDim.x;
    const int64_t w0 = (int64_t)min((long long)W, (long long)blockIdx.x * per);
    const int64_t w1 = (int64_t)min((long long)W, (long long)(w0 + per));
    __shared__ long long wsum[kWarps + 1];
    __shared__ long long s_pre[kWarps], s_tot[kWarps];
    {
        long long pre = 0, tot = 0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += kThreads) {
            const long long v = __ldcg(p.fin_sums + b);
            if (b < blockIdx.x) pre += v;
            tot += v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            pre += __shfl_down_sync(kFull, pre, o);
            tot += __shfl_down_sync(kFull, tot, o);
        }
        if (lane_id() == 0) {
            s_pre[threadIdx.x >> 5] = pre;
            s_tot[threadIdx.x >> 5] = tot;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long a = 0, t = 0;
            for (int w = 0; w < kWarps; w++) {
                a += s_pre[w];
                t += s_tot[w];
            }
            *s_tmp = a;
            if (blockIdx.x == 0) p.c->answer_count = t;
        }
    }
    __syncthreads();
    long long run = *s_tmp;
    __syncthreads();
    const unsigned lane = lane_id();
    for (int64_t base = w0; base < w1; base += kThreads) {
        const int64_t wi = base + threadIdx.x;
        uint64_t r = 0;
        if (wi < w1) {
            uint64_t fm = p.final_mask;
            while (fm) {
                const int q = __ffsll((long long)fm) - 1;
                fm &= fm - 1;
                uint64_t *Pw = p.P + (size_t)q * W + wi;
                const uint64_t v = __ldcg(Pw);
                if (v) *Pw = 0;
                r |= v;
            }
        }
        if (!p.out_list) continue;  // CTA-uniform
        const int32_t c = __popcll(r);
        int32_t incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += y;
        }
        if (lane == 31) wsum[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long acc = 0;
            for (int w = 0; w < kWarps; w++) {
                const long long s = wsum[w];
                wsum[w] = acc;
                acc += s;
            }
            wsum[kWarps] = acc;
        }
        __syncthreads();
        long long pos = run + wsum[threadIdx.x >> 5] + incl - c;
        while (r) {
            const int b = __ffsll((long long)r) - 1;
            r &= r - 1;
            if (pos < p.capacity) p.out_list[pos] = (int32_t)(wi * 64 + b);
            pos++;
        }
        run += wsum[kWarps];
        __syncthreads();
    }
}

// Frontier bits of levels j-1 and j cleared on CTA `cta` of `ncta`: the
// list ranges [vprev, vstart) in slot (j-1) % 3 and [vstart, vnext) in slot
// j % 3.  Loads go in batches of four ahead of their stores.
__device__ __forceinline__ void clear_frontier_bits(const KParams &p, const Shared &sh, int j, int cta, int ncta) {
    const long long first = (long long)cta * kThreads + threadIdx.x;
    const long long stride = (long long)ncta * kThreads;
    for (int q = 0; q < p.S; q++) {
        const int32_t *lst = p.VL + (size_t)q * p.n;
        const long long b = sh.vprev[q], m = sh.vstart[q], e = sh.vnext[q];
        uint64_t *Fa = p.F[(j + 2) % 3] + (size_t)q * p.W;
        uint64_t *Fb = p.F[j % 3] + (size_t)q * p.W;
        for (long long i0 = b + first; i0 < e; i0 += 4 * stride) {
            int32_t v[4];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const long long i = i0 + r * stride;
                v[r] = i < e ? __ldcg(lst + i) : -1;
            }
#pragma unroll
            for (int r = 0; r < 4; r++)
                if (v[r] >= 0) (i0 + r * stride < m ? Fa : Fb)[(uint32_t)v[r] >> 6] = 0;
        }
    }
}

// CTA 0: copies level j's counters from its shared memory to device memory,
// where the CTAs it is about to wake read them.
__device__ __forceinline__ void publish_counters(const KParams &p, const Shared &sh, int j) {
    const int cs = j % 3;
    const Ctrs &G = sh.cv[0], &S = sh.cv[1];
    for (int q = threadIdx.x; q < p.S; q += kThreads)
        G.fl[cs * kMaxStates + q] = S.fl[cs * kMaxStates + q];
    for (int g = threadIdx.x; g < p.n_groups; g += kThreads)
        G.mf[cs * G.mstride + g] = S.mf[cs * S.mstride + g];
    if (threadIdx.x == 0) {
        G.rows[cs] = S.rows[cs];
        G.srows[cs] = S.srows[cs];
    }
}

// CTA 0: sets the frontier bits of level j (list range [vstart, vnext)) in
// slot j % 3, for a level that the whole grid is about to run.
__device__ __forceinline__ void set_frontier_bits(const KParams &p, const Shared &sh, int j) {
    for (int q = 0; q < p.S; q++) {
        const int32_t *lst = p.VL + (size_t)q * p.n;
        uint64_t *Fq = p.F[j % 3] + (size_t)q * p.W;
        for (long long i = sh.vstart[q] + threadIdx.x; i < sh.vnext[q]; i += kThreads) {
            const int32_t v = __ldcg(lst + i);
            atomicOr((unsigned long long *)(Fq + ((uint32_t)v >> 6)), 1ull << (v & 63));
        }
    }
}

// Restores the all-zero P and F on CTA `cta` of `ncta` after a query whose
// last level is j: P rows (all states, or only the non-final ones when the
// answer sweep cleared the final rows), through the lists when they are
// short, densely over this CTA's word range otherwise; and, when the last
// levels kept frontier bits (`f_live`), those bits.
__device__ void clear_state(const KParams &p, const Shared &sh, bool finals_too, bool f_live,
                            int j, int cta, int ncta) {
    const int64_t W = p.W;
    const int64_t per = (W + ncta - 1) / ncta;
    const int64_t w0 = (int64_t)min((long long)W, (long long)cta * per);
    const int64_t w1 = (int64_t)min((long long)W, (long long)(w0 + per));
    const long long first = (long long)cta * kThreads + threadIdx.x;
    const long long stride = (long long)ncta * kThreads;
    for (int q = 0; q < p.S; q++) {
        if (!finals_too && ((p.final_mask >> q) & 1ull)) continue;
        const long long vend = sh.vstart[q] + (long long)sh.fl[q];
        const int32_t *lst = p.VL + (size_t)q * p.n;
        uint64_t *Pq = p.P + (size_t)q * W;
        if (vend * 8 < W && q >= p.dense_clear) {
            for (long long i0 = first; i0 < vend; i0 += 4 * stride) {
                int32_t v[4];
#pragma unroll
                for (int r = 0; r < 4; r++) {
                    const long long i = i0 + r * stride;
                    v[r] = i < vend ? __ldcg(lst + i) : -1;
                }
#pragma unroll
                for (int r = 0; r < 4; r++)
                    if (v[r] >= 0) Pq[(uint32_t)v[r] >> 6] = 0;
            }
        } else {
            for (int64_t wi = w0 + threadIdx.x; wi < w1; wi += kThreads) Pq[wi] = 0;
        }
    }
    if (f_live) clear_frontier_bits(p, sh, j, cta, ncta);
}

constexpr int kSoloAnswer = kGather;    // answer entries CTA 0 sorts in shared memory
constexpr long long kSoloClear = 4096;  // visited pairs CTA 0 clears through the lists

// Whether CTA 0 alone finishes the query: a list answer of at most
// kSoloAnswer entries (before removing duplicates across final states) and
// at most kSoloClear visited pairs.  Same result on every CTA.
__device__ bool solo_finish(const KParams &p, const Shared &sh) {
    if (p.out_bits || p.dense_clear > 0) return false;
    long long t = 0, v = 0;
    for (int q = 0; q < p.S; q++) {
        const long long e = sh.vstart[q] + (long long)sh.fl[q];
        v += e;
        if ((p.final_mask >> q) & 1ull) t += e;
    }
    return t <= kSoloAnswer && v <= kSoloClear;
}

// CTA 0 alone, after a query whose last level is j: one pass over every
// visited list clears P (and the kept frontier bits) and gathers the final
// states' vertices; the answer is their union, sorted by a bitonic network
// in shared memory with duplicates dropped.
__device__ void solo_answer(const KParams &p, const Shared &sh, bool f_live, int j) {
    int32_t *buf = sh.gbuf_k;
    __shared__ long long s_off[kMaxStates + 1];  // list prefix over all states
    __shared__ long long s_fo[kMaxStates + 1];   // list prefix over final states
    __shared__ int s_wc[kWarps];
    if (threadIdx.x == 0) {
        long long t = 0, f = 0;
        for (int q = 0; q < p.S; q++) {
            s_off[q] = t;
            s_fo[q] = f;
            const long long e = sh.vstart[q] + (long long)sh.fl[q];
            t += e;
            if ((p.final_mask >> q) & 1ull) f += e;
        }
        s_off[p.S] = t;
        s_fo[p.S] = f;
    }
    __syncthreads();
    const long long V = s_off[p.S];
    const int T = (int)s_fo[p.S];
    uint64_t *Fa = p.F[(j + 2) % 3], *Fb = p.F[j % 3];
    for (long long base = 0; base < V; base += 4 * kThreads) {
        int32_t v[4];
        int qq[4];
        long long ii[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const long long idx = base + r * kThreads + threadIdx.x;
            qq[r] = -1;
            ii[r] = 0;
            v[r] = 0;
            if (idx < V) {
                int q = 0;
                while (q + 1 < p.S && s_off[q + 1] <= idx) q++;
                qq[r] = q;
                ii[r] = idx - s_off[q];
                v[r] = __ldcg(p.VL + (size_t)q * p.n + ii[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int q = qq[r];
            if (q < 0) continue;
            const uint32_t wi = (uint32_t)v[r] >> 6;
            p.P[(size_t)q * p.W + wi] = 0;
            if (f_live && ii[r] >= sh.vprev[q])
                (ii[r] < sh.vstart[q] ? Fa : Fb)[(size_t)q * p.W + wi] = 0;
            if ((p.final_mask >> q) & 1ull) buf[s_fo[q] + ii[r]] = v[r];
        }
    }
    int n2 = 32;
    while (n2 < T) n2 <<= 1;
    for (int i = T + threadIdx.x; i < n2; i += kThreads) buf[i] = INT32_MAX;
    __syncthreads();
    const unsigned lane = lane_id();
    const int warp = threadIdx.x >> 5;
    if (T <= 32) {
        // one warp: a bitonic network over the lanes' registers
        if (warp == 0) {
            int32_t v = buf[lane];
#pragma unroll
            for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
                for (int jj = k >> 1; jj > 0; jj >>= 1) {
                    const int32_t o = __shfl_xor_sync(kFull, v, jj);
                    const bool lower = (lane & jj) == 0, ascending = (lane & k) == 0;
                    v = lower == ascending ? min(v, o) : max(v, o);
                }
            }
            const int32_t prev = __shfl_up_sync(kFull, v, 1);
            const bool keep = v != INT32_MAX && (lane == 0 || prev != v);
            const unsigned bm = __ballot_sync(kFull, keep);
            const long long pos = __popc(bm & lanemask_lt());
            int32_t *dst = p.out_list_small ? p.out_list_small : p.out_list;
            if (keep && dst && pos < p.capacity) dst[pos] = v;
            if (lane == 0) p.c->answer_count = __popc(bm);
        }
        return;
    }
    for (int k = 2; k <= n2; k <<= 1) {
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < n2; i += kThreads) {
                const int x = i ^ jj;
                if (x > i) {
                    const int32_t a = buf[i], b = buf[x];
                    if ((a > b) == ((i & k) == 0)) {
                        buf[i] = b;
                        buf[x] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    long long run = 0;
    for (int base = 0; base < n2; base += kThreads) {
        const int i = base + threadIdx.x;
        const int32_t v = i < n2 ? buf[i] : INT32_MAX;
        const bool keep = i < n2 && v != INT32_MAX && (i == 0 || buf[i - 1] != v);
        const unsigned bm = __ballot_sync(kFull, keep);
        if (lane == 0) s_wc[warp] = __popc(bm);
        __syncthreads();
        int before = 0, tot = 0;
        for (int w = 0; w < kWarps; w++) {
            const int c = s_wc[w];
            if (w < warp) before += c;
            tot += c;
        }
        const long long pos = run + before + __popc(bm & lanemask_lt());
        int32_t *dst = p.out_list_small ? p.out_list_small : p.out_list;
        if (keep && dst && pos < p.capacity) dst[pos] = v;
        run += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) p.c->answer_count = run;
}

// CTA 0, thread 0, at the end of a successful query: the summary to the
// host-mapped result (the answer count is thread 0's own earlier write).
__device__ __forceinline__ void write_result(const KParams &p, const Shared &sh, bool small) {
    if (!p.result || threadIdx.x != 0) return;
    QueryResult *r = p.result;
    r->small = small ? 1 : 0;
    r->levels = sh.stats[kStLevels];
    r->visited = sh.stats[kStVisited];
    r->expanded = sh.stats[kStExpanded];
    r->product_edges = sh.stats[kStProductEdges];
    r->push_bytes = sh.stats[kStPushBytes];
    r->push_units = sh.stats[kStPushUnits];
    r->pull_units = sh.stats[kStPullUnits];
    r->answer_count = *(volatile long long *)&p.c->answer_count;
    r->epoch = p.epoch;  // the host reads the summary after the stream has synchronised
}

__global__ void __launch_bounds__(kThreads, 3) rpq_query_kernel(const __grid_constant__ KParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int32_t s_gsf[kMaxStates + 1];
    __shared__ long long s_claim;
    __shared__ unsigned long long s_acc[2];
    const bool lead = blockIdx.x == 0;
    trace_launch(p, 0);
    // the layout's pointers live in shared memory, not in 30 registers
    __shared__ Shared s_layout;
    if (threadIdx.x == 0) s_layout = carve(p, smem);
    __syncthreads();
    const Shared &sh = s_layout;
    load_tables(p, sh);
    if (threadIdx.x <= p.S) {
        int lo = 0, hi = p.n_groups;  // groups are sorted by source state
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (sh.gq[mid] < (int)threadIdx.x) lo = mid + 1; else hi = mid;
        }
        s_gsf[threadIdx.x] = lo;
    }
    if (threadIdx.x < 2) s_acc[threadIdx.x] = 0;
    if (threadIdx.x == 0) s_nd = 0;
    __syncthreads();
    trace_launch(p, 4);
    if (p.clear_first) {
        const size_t words = (size_t)p.S * p.W;
        for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < words;
             i += (size_t)gridDim.x * kThreads) {
            p.P[i] = 0;
            p.F[0][i] = 0;
            p.F[1][i] = 0;
            p.F[2][i] = 0;
        }
        if (!grid_barrier(p)) return;
    }
    unsigned seen = 0;   // gate releases seen (the same count on every CTA)
    bool grid = false;   // the current level runs on the whole grid
    bool from_gate_final = false;
    int j = 0, plan = kPlanStop;
    if (lead) {
        // prologue on CTA 0: the device-memory counters of all slots cleared
        // (its shared-memory ones were cleared with the tables); P = F_0 =
        // Q_S x {v_s} with the level-0 lists, edge mass and long rows of every
        // start state, counted in shared memory (CTA 0 starts alone)
        Counters *c = p.c;
        for (int i = threadIdx.x; i < 3 * kMaxGroups; i += kThreads) p.mf[i] = 0;
        for (int i = threadIdx.x; i < 3 * kMaxStates; i += kThreads) (&c->fl_count[0][0])[i] = 0;
        if (threadIdx.x < 3) {
            const int k = threadIdx.x;
            c->rows_packed[k] = c->lvl_bytes[k] = c->lvl_edges[k] = c->srows_count[k] = 0;
            c->claim_chunk[k] = c->claim_item[k] = c->claim_pull[k] = 0;
        }
        if (threadIdx.x == 0) {
            c->answer_count = 0;
            c->parked = 0;
        }
        {
            // like every solo level, no frontier bits.  Each warp takes 32
            // sources at a time; the lane whose atomicOr sets the bit of a
            // start pair appends it (repeated sources are appended once)
            LevelCtx L0{0, 0, &sh.cv[1], p.VL, sh.vnext, nullptr};
            const int warp = threadIdx.x >> 5;
            for (int base = warp * 32; base < p.n_sources; base += kThreads) {
                const int i = base + (int)lane_id();
                const bool have = i < p.n_sources;
                const int32_t v = !have ? 0 : p.sources ? __ldg(p.sources + i) : p.source;
                const uint32_t swi = (uint32_t)v >> 6;
                const uint64_t sbit = 1ull << (v & 63);
                uint64_t sm = p.start_mask;
                while (sm) {
                    const int q = __ffsll((long long)sm) - 1;
                    sm &= sm - 1;
                    bool found = false;
                    if (have) {
                        const unsigned long long old =
                            atomicOr((unsigned long long *)(p.P + (size_t)q * p.W + swi), sbit);
                        found = !(old & sbit);
                    }
                    warp_discover(p, L0, found, q, v);
                }
            }
        }
        trace_launch(p, 5);
        flush_discoveries(p, sh, sh.cv[1], 0);
        if (!measure_buffer(p, sh, sh.cv[1], 0, s_acc))
            measure_level(p, sh, sh.cv[1], 0, 0, 1, s_acc);
        __syncthreads();
        trace_launch(p, 1);
        level_advance(p, 0, sh, true, true);
        trace_launch(p, 6);
        plan = level_plan(p, 0, sh, true);
        trace_launch(p, 7);
    }
    bool cur_smem = lead;  // level j's counters are in CTA 0's shared memory
    bool prev_grid = false;  // level j-1 ran on the grid (its frontier bits exist)
    unsigned long long parked_expected = 0;  // CTA 0: parkings so far
    bool park_pending = false;               // CTA 0: the last parking may be incomplete
    for (;;) {
        if (!lead && !grid) {
            // parked while CTA 0 runs levels alone
            const int cmd = gate_wait(p, seen);
            if (cmd != kGateLevel && cmd != kGateFinal) return;
            if (p.test_leave && blockIdx.x == gridDim.x - 1) return;  // failure test only
            j = *(volatile int32_t *)&p.c->pub_level;
            level_join(p, j, sh);
            grid = true;
            prev_grid = false;
            cur_smem = false;
            if (cmd == kGateFinal) {
                from_gate_final = true;
                break;
            }
            plan = level_plan(p, j, sh, false);
        }
        if (plan == kPlanStop) break;
        if (grid && plan == kPlanSolo) {
            // solo levels neither set nor clear frontier bits: the grid clears
            // those of levels j-1 and j now.  Each other CTA then parks;
            // CTA 0 runs level j at once and waits for the parkings only
            // before it recycles level j's counter slot or wakes the grid
            clear_frontier_bits(p, sh, j, (int)blockIdx.x, (int)gridDim.x);
            grid = false;
            prev_grid = false;
            if (!lead) {
                park_arrive(p);
                continue;  // park
            }
            parked_expected += gridDim.x - 1;
            park_pending = true;
        } else if (!grid && plan == kPlanGrid) {
            if (park_pending && !park_wait(p, parked_expected)) return;
            park_pending = false;
            set_frontier_bits(p, sh, j);  // level j may pull: its frontier needs its bits
            publish_counters(p, sh, j);
            cur_smem = false;
            gate_release(p, sh, seen, kGateLevel, j);
            grid = true;
        } else if (!grid && park_pending) {
            // the second solo level after a parking recycles the counter slot
            // of the level the parking CTAs last read
            if (!park_wait(p, parked_expected)) return;
            park_pending = false;
        }
        trace_put(p, j, 0, global_timer_ns());
        if (p.trace && lead && threadIdx.x == 0 && j < p.trace_cap) {
            unsigned long long tot = 0, npull = 0;
            for (int q = 0; q < p.S; q++) tot += sh.fl[q];
            for (int u = 0; u < p.n_units; u++) npull += sh.upull[u];
            p.trace[(size_t)j * kTraceFields + 3] = tot;
            p.trace[(size_t)j * kTraceFields + 4] = (unsigned long long)p.n_units - npull;
            p.trace[(size_t)j * kTraceFields + 5] = npull;
            p.trace[(size_t)j * kTraceFields + 6] = grid ? 1 : 0;
            p.trace[(size_t)j * kTraceFields + 7] = sh.lvl[0];
        }
        expand_phase(p, j, sh, s_gsf, &s_claim, s_acc, grid ? (int)blockIdx.x : 0,
                     grid ? (int)gridDim.x : 1, grid, grid && prev_grid, cur_smem);
        prev_grid = grid;
        cur_smem = !grid;
        trace_put(p, j, 1, global_timer_ns());
        // level j+1 is complete: measure the rows of its pairs, then plan it
        if (grid) {
            // every CTA measures what it discovered, from its buffer; if a
            // buffer overflowed, the grid measures the level again from the
            // lists
            if (p.trace) {
                __syncthreads();
                trace_last(p, j, 12);
            }
            flush_discoveries(p, sh, sh.cv[0], (j + 1) % 3);
            const bool fits = measure_buffer(p, sh, sh.cv[0], (j + 1) % 3, s_acc);
            trace_last(p, j, 13);
            const int r = grid_sync(p, !fits);
            if (r < 0) return;
            trace_put(p, j, 14, global_timer_ns());
            if (r > 0) {
                if (lead) measure_reset(p, sh, (j + 1) % 3);
                if (!grid_barrier(p)) return;
                // every CTA has left the barrier that saw the flag: clear it
                // now (earlier, a CTA still waiting there could miss it); the
                // other parity's bit is clear, the barrier just passed takes
                // no flags
                if (lead && threadIdx.x == 0) atomicAnd(&p.c->gen_status, ~kOverflowBits);
                if (!sort_level(p, sh, j)) return;
                trace_put(p, j, 15, global_timer_ns());
                measure_level(p, sh, sh.cv[0], (j + 1) % 3, (int)blockIdx.x, (int)gridDim.x,
                              s_acc);
                if (!grid_barrier(p)) return;
            }
        } else {
            flush_discoveries(p, sh, sh.cv[1], (j + 1) % 3);
            // the hybrid: level j+1 is an Algorithm 2 step while the visited
            // set (after level j) holds fewer than alg2_until pairs
            __shared__ int s_a2;
            if (threadIdx.x == 0) {
                bool a2 = false;
                if (p.alg2_until > 0) {
                    long long vis = 0;
                    const Ctrs &C1 = sh.cv[1];
                    for (int q = 0; q < p.S; q++)
                        vis += sh.vnext[q] + (long long)C1.fl[((j + 1) % 3) * kMaxStates + q];
                    a2 = vis < p.alg2_until;
                }
                s_a2 = a2 ? 1 : 0;
            }
            __syncthreads();
            if (s_a2) {
                __syncthreads();
                if (threadIdx.x == 0) s_nd = 0;  // the buffer holds only the new pairs: unused
                measure_level(p, sh, sh.cv[1], (j + 1) % 3, 0, 1, s_acc, true);
            } else if (!measure_buffer(p, sh, sh.cv[1], (j + 1) % 3, s_acc)) {
                measure_level(p, sh, sh.cv[1], (j + 1) % 3, 0, 1, s_acc);
            }
            __syncthreads();
            if (threadIdx.x == 0) sh.flags[1] = s_a2;
            heartbeat(p);
            if (load_status(p.c) != 0) return;
        }
        trace_put(p, j, 2, global_timer_ns());
        j++;
        level_advance(p, j, sh, lead, cur_smem);
        plan = level_plan(p, j, sh, lead);
    }
    trace_launch(p, 2);
    // frontier bits exist only when the last levels ran on the grid
    const bool f_live = grid && !from_gate_final;
    bool solo_end = false;
    if (!from_gate_final && solo_finish(p, sh)) {
        if (!lead) return;
        if (!grid) gate_release(p, sh, seen, kGateDone, j);
        solo_answer(p, sh, f_live, j);
        __syncthreads();
        solo_end = true;
    } else if (!grid) {
        // the grid joins the answer sweep: it needs level j's counters too
        if (park_pending && !park_wait(p, parked_expected)) return;
        publish_counters(p, sh, j);
        gate_release(p, sh, seen, kGateFinal, j);
        grid = true;
    }
    if (!solo_end) {
        final_phase(p, &s_claim);
        if (!grid_barrier(p)) return;
        final_write(p, &s_claim);
        clear_state(p, sh, false, f_live, j, (int)blockIdx.x, (int)gridDim.x);
    }
    if (lead) {
        for (int q = threadIdx.x; q < p.S; q += kThreads)
            p.c->vcount[q] = sh.vstart[q] + (long long)sh.fl[q];
        write_result(p, sh, solo_end);
    }
    trace_launch(p, 3);
}

// ------------------------------------------------- path outputs (kernels) --
// Level of first reach of every answer vertex: the smallest discovery level
// over the final states' pairs of v (section 4: level k holds the pairs first
// reached by words of length k, so this is the length of the shortest
// accepted word labelling a 2-path from a source to v).
__global__ void first_level_kernel(const int32_t *pair_level, int32_t n, uint64_t final_mask,
                                   const int32_t *answer, int64_t count, int32_t *out_levels) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = answer[i];
        int32_t best = INT32_MAX;
        uint64_t fm = final_mask;
        while (fm) {
            const int q = __ffsll((long long)fm) - 1;
            fm &= fm - 1;
            const int32_t x = __ldg(pair_level + (size_t)q * n + v);
            if (x >= 0 && x < best) best = x;
        }
        out_levels[i] = best;
    }
}

// The pair levels of the query's visited pairs back to -1, through the
// visited lists (their lengths per state are in the counters).
__global__ void reset_levels_kernel(int32_t *pair_level, const int32_t *VL, int32_t n, int32_t S,
                                    const Counters *c) {
    for (int q = 0; q < S; q++) {
        const long long cnt = c->vcount[q];
        const int32_t *lst = VL + (size_t)q * n;
        for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
             i += (long long)gridDim.x * blockDim.x)
            pair_level[(size_t)q * n + __ldg(lst + i)] = -1;
    }
}

// Before a pruned launch: rows q < S0 of P become the complement of
// `allowed` (those pairs count as visited, so the traversal never enters
// them).  Bits past vertex n - 1 are set too; nothing reads them.
__global__ void premask_kernel(uint64_t *P, const uint64_t *allowed, int64_t words) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x)
        P[i] = ~__ldg(allowed + i);
}

// After a query with pair levels: bit v of row q is set iff (q, v) was
// visited (one thread per output word).
__global__ void reach_bits_kernel(const int32_t *pair_level, int32_t n, int32_t S, int64_t W,
                                  uint64_t *out) {
    const int64_t words = (int64_t)S * W;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = i / W, w0 = (i - q * W) * 64;
        uint64_t b = 0;
        for (int k = 0; k < 64 && w0 + k < n; k++)
            if (__ldg(pair_level + q * n + w0 + k) >= 0) b |= 1ull << k;
        out[i] = b;
    }
}

// One transition q -d-> q' of the automaton, d a label direction of the graph.
struct WTrans {
    int32_t from, d, to;
};

// A shortest witness of `target` (one CTA): the final pair of the target with
// the smallest level k, then, for k, k-1, ..., 1, a predecessor pair one
// level lower: (q, u) with q -d-> q' and u a neighbour of v in the direction
// inverse to d (the rows of G^d's transpose), i.e. the forward step walks
// u -d-> v.  Among the candidates of a step the smallest (transition, row
// position) is taken, so the result is deterministic.  Writes k + 1
// vertices and k symbols (d, in [0, 2L)) when they fit in `cap` entries,
// and the length k (-1: the target is not in the answer) to out[0].
__global__ void witness_kernel(const DevAdj *adj, int32_t L, const int32_t *pair_level,
                               int32_t n, uint64_t final_mask, const WTrans *tr, int32_t T,
                               int32_t target, int32_t *path_v, int32_t *path_s, int32_t cap,
                               int32_t *out) {
    __shared__ int s_q, s_v, s_k;
    __shared__ unsigned long long s_best;
    if (threadIdx.x == 0) {
        int best = INT32_MAX, bq = -1;
        uint64_t fm = final_mask;
        while (fm) {
            const int q = __ffsll((long long)fm) - 1;
            fm &= fm - 1;
            const int32_t x = pair_level[(size_t)q * n + target];
            if (x >= 0 && x < best) {
                best = x;
                bq = q;
            }
        }
        s_k = bq < 0 ? -1 : best;
        s_q = bq;
        s_v = target;
        out[0] = s_k;
        if (s_k >= 0 && s_k < cap) path_v[s_k] = target;
    }
    __syncthreads();
    const int k = s_k;
    if (k < 0) return;
    for (int step = k; step >= 1; step--) {
        const int q2 = s_q;
        const int32_t v = s_v;
        if (threadIdx.x == 0) s_best = ~0ull;
        __syncthreads();
        for (int t = 0; t < T; t++) {
            if (tr[t].to != q2) continue;  // uniform
            const int q = tr[t].from, d = tr[t].d;
            const DevAdj A = adj[d < L ? d + L : d - L];
            int32_t b, e;
            adj_row(A, v, b, e);
            for (int32_t i = b + (int32_t)threadIdx.x; i < e; i += blockDim.x) {
                const int32_t u = __ldg(A.nbr + i);
                if (__ldg(pair_level + (size_t)q * n + u) == step - 1) {
                    atomicMin(&s_best, ((unsigned long long)t << 32) | (uint32_t)i);
                    break;
                }
            }
            __syncthreads();
            const bool found = s_best != ~0ull;
            __syncthreads();  // every thread has read s_best before later atomics
            if (found) break;
        }
        if (threadIdx.x == 0) {
            const unsigned long long b = s_best;
            if (b == ~0ull) {  // no predecessor: cannot happen for a visited pair
                out[0] = -2;
                s_v = -1;
            } else {
                const int t = (int)(b >> 32);
                const int32_t u = __ldg(adj[tr[t].d < L ? tr[t].d + L : tr[t].d - L].nbr +
                                        (int32_t)(b & 0xffffffffu));
                if (k < cap) {
                    path_v[step - 1] = u;
                    path_s[step - 1] = tr[t].d;
                }
                s_q = tr[t].from;
                s_v = u;
            }
        }
        __syncthreads();
        if (s_v < 0) return;
    }
}

// ------------------------------------------------------------ host side --

struct QueryWorkspace : WorkspaceBase {
    int S_cap = 0;
    long long row_cap = 0, chunk_cap = 0, srow_cap = 0;
    int32_t n = 0, W = 0;
    DevBuf P, F[3], VL, rows[3], cmap[3], srl[3], mf, fin, ctr, tables, out_list, trace;
    DevBuf sortc;         // [S_cap][max grid] per-CTA counts of the sorted list rebuild
    DevBuf srcs;          // the source set of the query (n_sources int32), grown on demand
    DevBuf plevel;        // [S_cap][n] int32 pair levels, -1 between queries (path outputs)
    DevBuf wtab, wout;    // witness: automaton transitions; path vertices, symbols, length
    bool plevel_dirty = false;  // a failed query may have left pair levels set
    void *staging = nullptr;  // pinned host: tables upload + counters download
    size_t staging_bytes = 0;
    QueryResult *result_dev = nullptr;  // device address of the summary slot of staging
    uint32_t epoch = 0;   // launches so far (tags the kernel's gate word and the summary)
    bool dirty = false;   // a failed launch may have left P / F non-zero
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    ~QueryWorkspace() override {
        if (staging) cudaFreeHost(staging);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

constexpr size_t kTablesBytes = 256 * 1024;

// Per host thread: pinned host memory, mapped into the device, that the
// kernel writes host answers to, and the last such answer.
struct HostAnswer {
    int32_t *h = nullptr, *d = nullptr;
    size_t cap = 0;
    int64_t count = 0;
    bool valid = false;
    ~HostAnswer() {
        if (h) cudaFreeHost(h);
    }
    bool reserve(size_t n) {
        if (cap >= n) return true;
        if (h) cudaFreeHost(h);
        h = d = nullptr;
        cap = 0;
        void *hp = nullptr, *dp = nullptr;
        if (cudaHostAlloc(&hp, sizeof(int32_t) * n, cudaHostAllocMapped | cudaHostAllocPortable) !=
                cudaSuccess ||
            cudaHostGetDevicePointer(&dp, hp, 0) != cudaSuccess) {
            if (hp) cudaFreeHost(hp);
            return false;
        }
        h = static_cast<int32_t *>(hp);
        d = static_cast<int32_t *>(dp);
        cap = n;
        return true;
    }
};
thread_local HostAnswer tl_answer;
// staging: tables | counters (read back after a failure) | summary
constexpr size_t kResultOffset = (kTablesBytes + sizeof(Counters) + 63) & ~size_t(63);

// Grid of the persistent kernel: every SM holds the same number of CTAs
// (cooperative launch requires all of them resident).  Computed per device
// and per shared-memory size (rounded up to 4 KiB) and cached.
struct GridKey {
    int device;
    size_t smem;
    bool operator<(const GridKey &o) const {
        return device != o.device ? device < o.device : smem < o.smem;
    }
};
std::map<GridKey, int> g_grid;
std::mutex g_grid_mu;
constexpr size_t kMaxDynSmem = 160 * 1024;
constexpr int kMaxGrid = 152 * 64;  // CTAs of the persistent grid at most (per-CTA scratch)

rpq_status get_launch_shape(int device, size_t smem, int *grid) {
    std::lock_guard<std::mutex> lk(g_grid_mu);
    smem = (smem + 4095) & ~size_t(4095);
    if (smem > kMaxDynSmem)
        return fail(RPQ_ERR_INVALID, "automaton tables need %zu bytes of shared memory", smem);
    auto it = g_grid.find({device, smem});
    if (it != g_grid.end()) {
        *grid = it->second;
        return RPQ_OK;
    }
    int coop = 0, sms = 0;
    RPQ_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    RPQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    if (!coop) return fail(RPQ_ERR_CUDA, "device lacks cooperative launch");
    RPQ_CUDA_TRY(cudaFuncSetAttribute(rpq_query_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kMaxDynSmem));
    int per_sm = 0;
    RPQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rpq_query_kernel, kThreads,
                                                               smem));
    if (per_sm <= 0) return fail(RPQ_ERR_CUDA, "query kernel does not fit on an SM");
    const char *cap = getenv("RPQ_CTAS_PER_SM");
    per_sm = std::min(per_sm, cap ? std::max(1, atoi(cap)) : 4);
    g_grid[{device, smem}] = sms * per_sm;
    *grid = sms * per_sm;
    return RPQ_OK;
}

rpq_status ws_alloc(QueryWorkspace *ws, const rpq_graph *g, int S_cap, long long row_cap,
                    long long chunk_cap, long long srow_cap, cudaStream_t st) {
    const int64_t W = ((int64_t)g->n + 63) / 64;
    const size_t bits = sizeof(uint64_t) * (size_t)S_cap * W;
    const size_t fl = sizeof(int32_t) * (size_t)S_cap * g->n;
    ws->S_cap = S_cap;
    ws->row_cap = row_cap;
    ws->chunk_cap = chunk_cap;
    ws->srow_cap = srow_cap;
    ws->n = g->n;
    ws->W = (int32_t)W;
    bool ok = ws->P.alloc(bits) && ws->mf.alloc(sizeof(unsigned long long) * 3 * kMaxGroups) &&
              ws->fin.alloc(sizeof(long long) * kMaxGrid) && ws->ctr.alloc(sizeof(Counters)) &&
              ws->sortc.alloc(sizeof(uint32_t) * (size_t)S_cap * kMaxGrid) &&
              ws->tables.alloc(kTablesBytes) && ws->VL.alloc(fl) &&
              ws->out_list.alloc(sizeof(int32_t) * (size_t)g->n);
    for (int k = 0; k < 3 && ok; k++)
        ok = ws->F[k].alloc(bits) && ws->rows[k].alloc(sizeof(Row) * (size_t)row_cap) &&
             ws->cmap[k].alloc(sizeof(int32_t) * (size_t)chunk_cap) &&
             ws->srl[k].alloc(sizeof(int4) * (size_t)srow_cap);
    if (!ok) return fail(RPQ_ERR_OOM, "query workspace (%d states)", S_cap);
    // the kernel expects P and F all-zero on entry and leaves them so.  The
    // clears go on the query's stream and complete before the workspace is
    // used: a plain cudaMemset would be ordered only on the legacy default
    // stream, which the non-blocking streams of the slot engines do not wait
    // for (a kernel there could see the memory's earlier contents)
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->ctr.p, 0, sizeof(Counters), st));
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->P.p, 0, bits, st));
    for (int k = 0; k < 3; k++) RPQ_CUDA_TRY(cudaMemsetAsync(ws->F[k].p, 0, bits, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    ws->staging_bytes = kResultOffset + sizeof(QueryResult);
    RPQ_CUDA_TRY(cudaHostAlloc(&ws->staging, ws->staging_bytes, cudaHostAllocMapped));
    memset(ws->staging, 0, ws->staging_bytes);
    void *rd = nullptr;
    RPQ_CUDA_TRY(cudaHostGetDevicePointer(&rd, static_cast<uint8_t *>(ws->staging) + kResultOffset, 0));
    ws->result_dev = static_cast<QueryResult *>(rd);
    RPQ_CUDA_TRY(cudaEventCreate(&ws->ev0));
    RPQ_CUDA_TRY(cudaEventCreate(&ws->ev1));
    return RPQ_OK;
}

std::unique_ptr<QueryWorkspace> ws_acquire(rpq_graph *g, int S, long long row_need,
                                           long long chunk_need, long long srow_need,
                                           rpq_status *st, cudaStream_t stream) {
    {
        std::lock_guard<std::mutex> lk(g->ws_mu);
        for (size_t i = 0; i < g->ws_free.size(); i++) {
            auto *w = dynamic_cast<QueryWorkspace *>(g->ws_free[i].get());
            if (w && w->S_cap >= S && w->row_cap >= row_need && w->chunk_cap >= chunk_need &&
                w->srow_cap >= srow_need) {
                std::unique_ptr<QueryWorkspace> r(static_cast<QueryWorkspace *>(g->ws_free[i].release()));
                g->ws_free.erase(g->ws_free.begin() + i);
                *st = RPQ_OK;
                return r;
            }
        }
    }
    std::unique_ptr<QueryWorkspace> w(new QueryWorkspace());
    int S_cap = 4;
    while (S_cap < S) S_cap *= 2;
    long long rc = 1024, cc = 4096, sc = 4096;
    while (rc < row_need) rc *= 2;
    while (cc < chunk_need) cc *= 2;
    while (sc < srow_need) sc *= 2;
    *st = ws_alloc(w.get(), g, S_cap, rc, cc, sc, stream);
    if (*st == RPQ_ERR_OOM) {
        // memory is short: the graph's idle cached workspaces (of other
        // shapes) go back to the allocator, then one more try
        std::vector<std::unique_ptr<WorkspaceBase>> idle;
        {
            std::lock_guard<std::mutex> lk(g->ws_mu);
            idle.swap(g->ws_free);
        }
        idle.clear();
        w.reset(new QueryWorkspace());
        *st = ws_alloc(w.get(), g, S_cap, rc, cc, sc, stream);
    }
    if (*st != RPQ_OK) return nullptr;
    return w;
}

void ws_release(rpq_graph *g, std::unique_ptr<QueryWorkspace> w) {
    std::lock_guard<std::mutex> lk(g->ws_mu);
    g->ws_free.emplace_back(std::move(w));
}

// Host-side automaton tables for the kernel.
struct Tables {
    std::vector<QGroup> groups;
    std::vector<QUnit> units;
    std::vector<int32_t> t_unit, t_state, u_group;
    long long row_need = 0, chunk_need = 0, srow_need = 0;
    void clear() {
        groups.clear();
        units.clear();
        t_unit.clear();
        t_state.clear();
        u_group.clear();
        row_need = chunk_need = srow_need = 0;
    }
};

// A (key, mask) list sorted by key with the masks of equal keys OR-ed.
struct KeyMask {
    int64_t key;
    uint64_t mask;
};
void merge_keys(std::vector<KeyMask> &v) {
    std::sort(v.begin(), v.end(), [](const KeyMask &x, const KeyMask &y) { return x.key < y.key; });
    size_t o = 0;
    for (size_t i = 0; i < v.size(); i++) {
        if (o > 0 && v[o - 1].key == v[i].key) v[o - 1].mask |= v[i].mask;
        else v[o++] = v[i];
    }
    v.resize(o);
}

// t must be empty (Tables::clear).  Allocation-free once this thread's
// scratch lists and t have grown to the automaton's size.
rpq_status build_tables(const rpq_graph *g, const Automaton &a, Tables *t) {
    // group (q, d) -> targets, ordered by q then d; unit (d, q') -> sources,
    // ordered by d then q'
    thread_local std::vector<KeyMask> gk, uk;
    gk.clear();
    uk.clear();
    const int64_t D = 2 * (int64_t)g->L;
    for (size_t i = 0; i < a.from.size(); i++) {
        const int s = a.sym[i];
        const int lab = s < a.L ? s : s - a.L;
        const bool inv = s >= a.L;
        if (lab >= g->L)
            return fail(RPQ_ERR_INVALID, "automaton label %d is not a label of the graph (L=%d)",
                        lab, g->L);
        const int d = inv ? g->L + lab : lab;
        gk.push_back({(int64_t)a.from[i] * D + d, 1ull << a.to[i]});
        uk.push_back({(int64_t)d * kMaxStates + a.to[i], 1ull << a.from[i]});
    }
    merge_keys(gk);
    merge_keys(uk);
    if ((int)gk.size() > kMaxGroups || (int)uk.size() > kMaxUnits)
        return fail(RPQ_ERR_INVALID, "automaton has too many (state, label) pairs");
    for (const KeyMask &km : uk) {
        QUnit u{};
        u.d = (int32_t)(km.key / kMaxStates);
        u.q2 = (int32_t)(km.key % kMaxStates);
        u.smask = km.mask;
        u.in_dir = g->inverse_dir(u.d);
        const DevAdj &A = g->adj[u.in_dir];
        u.in_rows = A.fmt == ADJ_EMPTY ? 0 : A.nrows;
        u.in_nnz = A.nnz;
        t->units.push_back(u);
    }
    auto unit_of = [&](int d, int q2) {
        const int64_t key = (int64_t)d * kMaxStates + q2;
        const auto it = std::lower_bound(uk.begin(), uk.end(), key,
                                         [](const KeyMask &x, int64_t k) { return x.key < k; });
        return (int32_t)(it - uk.begin());
    };
    for (const KeyMask &km : gk) {
        QGroup G{};
        G.q = (int32_t)(km.key / D);
        G.d = (int32_t)(km.key % D);
        G.tmask = km.mask;
        G.t_first = (int32_t)t->t_unit.size();
        uint64_t m = G.tmask;
        while (m) {
            const int q2 = __builtin_ctzll(m);
            m &= m - 1;
            t->t_unit.push_back(unit_of(G.d, q2));
            t->t_state.push_back(q2);
        }
        G.t_count = (int32_t)t->t_unit.size() - G.t_first;
        // Short rows are listed at discovery where looking them up again
        // costs several round trips: every adjacency but a dense one (whose
        // offsets find a row in one; an empty adjacency lists nothing).
        // Listing costs a reservation per discovery batch, which dense
        // adjacencies, even mostly empty ones, do not repay.
        G.listed = g->adj[G.d].fmt != ADJ_DENSE;
        t->groups.push_back(G);
        // a level holds each (state, vertex) pair at most once, so the long
        // (listed short) rows of one group are at most the long (short) rows
        // of its adjacency
        t->row_need += g->long_rows[G.d] + 1;
        t->chunk_need += g->long_chunks[G.d] + 1;
        t->srow_need += (G.listed ? g->short_rows[G.d] : 0) + 1;
    }
    for (size_t u = 0; u < t->units.size(); u++) {
        QUnit &U = t->units[u];
        U.g_first = (int32_t)t->u_group.size();
        for (size_t gi = 0; gi < t->groups.size(); gi++) {
            const QGroup &G = t->groups[gi];
            if (G.d == U.d && ((G.tmask >> U.q2) & 1)) t->u_group.push_back((int32_t)gi);
        }
        U.g_count = (int32_t)t->u_group.size() - U.g_first;
    }
    if ((int)t->t_unit.size() > kMaxTargets || (int)t->u_group.size() > kMaxTargets)
        return fail(RPQ_ERR_INVALID, "automaton has too many transitions");
    return RPQ_OK;
}

// Appends one JSON line per query: the kernel's phase times (`kernel`, and
// within the prologue `prologue`: tables loaded, seeds set, level 0 advanced
// and planned) and, per level,
// block 0's timestamps (ns, relative to the kernel start) with the frontier
// size, the number of push / pull units, whether the level ran on the
// whole grid (1) or on CTA 0 alone (0), the push-model bytes of its rows,
// block 0's end of the long-row and short-row phases, the first and last
// CTA's end of the expansion (thread 0), and on grid levels the last CTA
// whose warps all ended the expansion, the last CTA done measuring its
// discovery buffer, block 0 past the barrier that follows, and block 0 done
// sorting the level (levels re-measured from the lists only).
void write_trace(const char *path, QueryWorkspace *ws, int S, int source, int levels,
                 cudaStream_t st) {
    std::vector<unsigned long long> h((size_t)kTraceFields * levels), gs(kTraceFields);
    if (cudaMemcpyAsync(h.data(), ws->trace.p, h.size() * 8, cudaMemcpyDeviceToHost, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(gs.data(),
                        ws->trace.as<unsigned long long>() + (size_t)kTraceLevels * kTraceFields,
                        kTraceFields * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    FILE *f = fopen(path, "a");
    if (!f) return;
    auto rel = [&](unsigned long long t) { return t && gs[0] ? (long long)(t - gs[0]) : -1LL; };
    fprintf(f,
            "{\"source\": %d, \"states\": %d, \"kernel\": [%lld, %lld, %lld, %lld], "
            "\"prologue\": [%lld, %lld, %lld, %lld], \"levels\": [",
            source, S, rel(gs[0]), rel(gs[1]), rel(gs[2]), rel(gs[3]), rel(gs[4]), rel(gs[5]),
            rel(gs[6]), rel(gs[7]));
    for (int j = 0; j < levels; j++) {
        const unsigned long long *r = &h[(size_t)j * kTraceFields];
        if (r[0] == 0) break;
        fprintf(f,
                "%s[%lld, %lld, %lld, %llu, %llu, %llu, %llu, %llu, %lld, %lld, %lld, %lld, %lld, "
                "%lld, %lld, %lld]",
                j ? ", " : "", rel(r[0]), rel(r[1]), rel(r[2]), r[3], r[4], r[5], r[6], r[7],
                rel(r[8]), rel(r[9]), rel(r[10] ? ~r[10] : 0), rel(r[11]), rel(r[12]), rel(r[13]),
                rel(r[14]), rel(r[15]));
    }
    fprintf(f, "]}\n");
    fclose(f);
}

// Packs the tables at 16-byte aligned offsets into dst (cap bytes), writing
// the five offsets; returns the packed size, which may exceed cap (then
// nothing past cap is written).
size_t pack_tables(const Tables &t, uint8_t *dst, size_t cap, int32_t off[5]) {
    size_t o = 0;
    int k = 0;
    auto put = [&](const void *src, size_t bytes) {
        o = (o + 15) & ~size_t(15);
        off[k++] = (int32_t)o;
        if (bytes && o + bytes <= cap) memcpy(dst + o, src, bytes);
        o += bytes;
    };
    put(t.groups.data(), sizeof(QGroup) * t.groups.size());
    put(t.units.data(), sizeof(QUnit) * t.units.size());
    put(t.t_unit.data(), sizeof(int32_t) * t.t_unit.size());
    put(t.t_state.data(), sizeof(int32_t) * t.t_state.size());
    put(t.u_group.data(), sizeof(int32_t) * t.u_group.size());
    return (o + 15) & ~size_t(15);
}

// Tables into the launch parameters when they fit, else into `dev` (a
// device buffer of cap bytes) through `staging` (pinned host) on `st`.
rpq_status place_tables(const Tables &t, KParams &p, uint8_t *staging, uint8_t *dev, size_t cap,
                        cudaStream_t st, size_t *bytes) {
    int32_t off[5];
    size_t n = pack_tables(t, p.tab, kInlineTables, off);
    *bytes = n;
    if (n <= (size_t)kInlineTables) {
        p.tab_inline = 1;
        p.o_groups = off[0];
        p.o_units = off[1];
        p.o_tu = off[2];
        p.o_ts = off[3];
        p.o_ug = off[4];
        return RPQ_OK;
    }
    if (n > cap) return fail(RPQ_ERR_INVALID, "automaton tables too large (%zu bytes)", n);
    pack_tables(t, staging, cap, off);
    RPQ_CUDA_TRY(cudaMemcpyAsync(dev, staging, n, cudaMemcpyHostToDevice, st));
    p.tab_inline = 0;
    p.groups = reinterpret_cast<const QGroup *>(dev + off[0]);
    p.units = reinterpret_cast<const QUnit *>(dev + off[1]);
    p.t_unit = reinterpret_cast<const int32_t *>(dev + off[2]);
    p.t_state = reinterpret_cast<const int32_t *>(dev + off[3]);
    p.u_group = reinterpret_cast<const int32_t *>(dev + off[4]);
    return RPQ_OK;
}

// The RPQ_ variables of the environment (tuning overrides), taken by one
// pass over it at the start of each launch's set-up instead of one lookup
// per setting; env_float reads the taking of its own thread.
struct EnvSnapshot {
    int n = 0;
    const char *kv[64];
};
thread_local EnvSnapshot tl_env;

void env_snapshot() {
    tl_env.n = 0;
    for (char **e = environ; e && *e && tl_env.n < 64; e++)
        if (strncmp(*e, "RPQ_", 4) == 0) tl_env.kv[tl_env.n++] = *e;
}

float env_float(const char *name, float dflt) {
    const size_t len = strlen(name);
    for (int i = 0; i < tl_env.n; i++)
        if (strncmp(tl_env.kv[i], name, len) == 0 && tl_env.kv[i][len] == '=')
            return (float)atof(tl_env.kv[i] + len + 1);
    return dflt;
}

// Big levels on big graphs: when the row offsets of a label no longer fit
// the L2 cache (n >= 2^22 vertices: 16 MiB per label), a level's rows are
// measured and expanded in vertex order after a level of at least
// kSortPairs discoveries (sort_level); the discovery buffers then hand such
// levels to the list pass early (kSortBuffer pairs per CTA).  Smaller graphs
// keep discovery order.  RPQ_SORT_MIN (pairs, 0 = never) and
// RPQ_DISCOVERY_BUFFER override.
constexpr long long kSortPairs = 131072;
constexpr int kSortBuffer = 1024;
constexpr int32_t kSortVertices = 1 << 22;

// Limit of the device waits (RPQ_WAIT_LIMIT_MS, default 4 s) and the
// failure test's early exit of one CTA (RPQ_TEST_LEAVE_CTA=1).
// The Algorithm 2 -> Algorithm 1 switch: the graph's setting
// (rpq_graph_set_hybrid), RPQ_ALG2_SWITCH overrides.
void hybrid_policy(const rpq_graph *g, KParams &p) {
    p.alg2_until = std::max(0LL, (long long)env_float("RPQ_ALG2_SWITCH", (float)g->alg2_until));
}

void precheck_policy(KParams &p) {
    p.precheck_mass = (long long)env_float("RPQ_PRECHECK_MASS", (float)kPrecheckMass);
}

void wait_policy(KParams &p) {
    const float ms = env_float("RPQ_WAIT_LIMIT_MS", (float)(kBarrierTimeoutNs / 1000000ull));
    p.wait_ns = (uint64_t)(std::max(1.0f, ms) * 1e6f);
    p.test_leave = env_float("RPQ_TEST_LEAVE_CTA", 0.0f) != 0.0f ? 1 : 0;
}

void sort_policy(const rpq_graph *g, KParams &p) {
    const bool big = g->n >= kSortVertices;
    p.sort_min = (long long)env_float("RPQ_SORT_MIN", big ? (float)kSortPairs : 0.0f);
    const int dflt = p.sort_min > 0 ? kSortBuffer : kDisc;
    // a smaller limit (tests) sends more levels down the grid-wide measure pass
    p.disc_cap = std::min(kDisc, std::max(0, (int)env_float("RPQ_DISCOVERY_BUFFER", (float)dflt)));
}

// After a successful query with pair levels: the first-reach levels of the
// answer (device list of `n_ans` entries), the witness path, then the pair
// levels back to -1.  Stream-ordered after the traversal kernel.
rpq_status path_outputs(const rpq_graph *g, const Automaton &a, QueryWorkspace *ws, QueryExtras *x,
                        const int32_t *answer_dev, int64_t n_ans, cudaStream_t st) {
    int dev_sms = 0;
    RPQ_CUDA_TRY(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, g->device));
    if (x->out_levels_dev && n_ans > 0) {
        const int blocks = (int)std::min<int64_t>((int64_t)dev_sms * 8, (n_ans + 255) / 256);
        first_level_kernel<<<blocks, 256, 0, st>>>(ws->plevel.as<int32_t>(), g->n, a.final_mask,
                                                    answer_dev, n_ans, x->out_levels_dev);
        RPQ_CUDA_TRY(cudaGetLastError());
        note_launch();
    }
    if (x->witness) {
        std::vector<WTrans> tr;
        for (size_t t = 0; t < a.from.size(); t++) {
            const int s = a.sym[t];
            const int lab = s < a.L ? s : s - a.L;
            tr.push_back(WTrans{a.from[t], s < a.L ? lab : g->L + lab, a.to[t]});
        }
        const size_t tb = sizeof(WTrans) * std::max<size_t>(tr.size(), 1);
        const int32_t cap = std::max(0, x->path_cap);
        const size_t ob = sizeof(int32_t) * (2 * (size_t)cap + 1);
        if ((ws->wtab.bytes < tb && !ws->wtab.alloc(tb)) || (ws->wout.bytes < ob && !ws->wout.alloc(ob)))
            return fail(RPQ_ERR_OOM, "witness buffers");
        if (!tr.empty())
            RPQ_CUDA_TRY(cudaMemcpyAsync(ws->wtab.p, tr.data(), sizeof(WTrans) * tr.size(),
                                         cudaMemcpyHostToDevice, st));
        int32_t *wo = ws->wout.as<int32_t>();
        witness_kernel<<<1, 256, 0, st>>>(g->d_adj.as<DevAdj>(), g->L, ws->plevel.as<int32_t>(),
                                          g->n, a.final_mask, ws->wtab.as<WTrans>(),
                                          (int32_t)tr.size(), x->target, wo + 1, wo + 1 + cap, cap,
                                          wo);
        RPQ_CUDA_TRY(cudaGetLastError());
        note_launch();
        int32_t len = -1;
        RPQ_CUDA_TRY(cudaMemcpyAsync(&len, wo, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        RPQ_CUDA_TRY(cudaStreamSynchronize(st));
        if (len < -1) return fail(RPQ_ERR_CUDA, "witness: a visited pair has no predecessor");
        x->path_len = len;
        if (len >= 0 && len < cap) {
            RPQ_CUDA_TRY(cudaMemcpyAsync(x->path_v, wo + 1, sizeof(int32_t) * (size_t)(len + 1),
                                         cudaMemcpyDeviceToHost, st));
            if (len > 0)
                RPQ_CUDA_TRY(cudaMemcpyAsync(x->path_s, wo + 1 + cap, sizeof(int32_t) * (size_t)len,
                                             cudaMemcpyDeviceToHost, st));
        }
    }
    if (x->reach_bits_out) {
        const int64_t W = ((int64_t)g->n + 63) / 64;
        const int blocks = (int)std::min<int64_t>((int64_t)dev_sms * 8, ((int64_t)a.S * W + 255) / 256);
        reach_bits_kernel<<<blocks, 256, 0, st>>>(ws->plevel.as<int32_t>(), g->n, a.S, W,
                                                   x->reach_bits_out);
        RPQ_CUDA_TRY(cudaGetLastError());
        note_launch();
    }
    {
        const int blocks = dev_sms * 4;
        reset_levels_kernel<<<blocks, 256, 0, st>>>(ws->plevel.as<int32_t>(), ws->VL.as<int32_t>(),
                                                     g->n, a.S, ws->ctr.as<Counters>());
        RPQ_CUDA_TRY(cudaGetLastError());
        note_launch();
    }
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    return RPQ_OK;
}

}  // namespace

// Runs one query.  The answer goes to out_list_dev (device, `capacity`
// entries) or, when that is null, to out_host_list (host, copied when it
// fits in `capacity`); out_bits_dev receives the answer bitset if non-null.
rpq_status run_query(rpq_graph *g, const Automaton &a, int32_t source, int32_t max_levels,
                     int32_t *out_list_dev, int64_t capacity, uint64_t *out_bits_dev,
                     int32_t *out_host_list, rpq_stats *stats, int64_t *count, void *stream,
                     bool host_list) {
    return run_query_slot(g, a, source, max_levels, out_list_dev, capacity, out_bits_dev,
                          out_host_list, stats, count, stream, 1, host_list);
}

rpq_status last_host_answer(const int32_t **answer, int64_t *count) {
    if (!answer || !count) return fail(RPQ_ERR_INVALID, "null argument");
    if (!tl_answer.valid) return fail(RPQ_ERR_INVALID, "this thread has no host answer");
    *answer = tl_answer.h;
    *count = tl_answer.count;
    return RPQ_OK;
}

// As run_query, on 1/grid_div of the persistent grid, so that grid_div
// queries can run concurrently on separate streams.
rpq_status run_query_slot(rpq_graph *g, const Automaton &a, int32_t source, int32_t max_levels,
                          int32_t *out_list_dev, int64_t capacity, uint64_t *out_bits_dev,
                          int32_t *out_host_list, rpq_stats *stats, int64_t *count, void *stream,
                          int grid_div, bool host_list) {
    return run_query_ex(g, a, nullptr, source, max_levels, out_list_dev, capacity, out_bits_dev,
                        out_host_list, stats, count, stream, grid_div, host_list);
}

// The query with its optional parts (x may be null): a source set instead of
// the single source, first-reach levels of the answer, a witness path.
rpq_status run_query_ex(rpq_graph *g, const Automaton &a, QueryExtras *x, int32_t source,
                        int32_t max_levels, int32_t *out_list_dev, int64_t capacity,
                        uint64_t *out_bits_dev, int32_t *out_host_list, rpq_stats *stats,
                        int64_t *count, void *stream, int grid_div, bool host_list) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool want_host = !out_list_dev && (host_list || out_host_list);
    tl_answer.valid = false;  // a host answer lives until this thread's next query
    const bool multi = x && x->sources;
    const bool levels = x && (x->out_levels_dev || x->witness || x->reach_bits_out);
    if (multi) {
        if (x->n_sources <= 0) return fail(RPQ_ERR_INVALID, "empty source set");
        for (int32_t i = 0; i < x->n_sources; i++)
            if (x->sources[i] < 0 || x->sources[i] >= g->n)
                return fail(RPQ_ERR_INVALID, "source %d (entry %d) outside [0, %d)", x->sources[i],
                            i, g->n);
    } else if (source < 0 || source >= g->n) {
        return fail(RPQ_ERR_INVALID, "source %d outside [0, %d)", source, g->n);
    }
    if (x && x->out_levels_dev && !out_list_dev)
        return fail(RPQ_ERR_INVALID, "first-reach levels need the answer in device memory");
    if (max_levels < 0) return fail(RPQ_ERR_INVALID, "max_levels must be >= 0");
    if (a.S <= 0 || a.S > kMaxStates) return fail(RPQ_ERR_INVALID, "automaton has %d states", a.S);
    env_snapshot();
    thread_local Tables t;  // reused: no host allocation once grown
    t.clear();
    rpq_status s = build_tables(g, a, &t);
    if (s != RPQ_OK) return s;
    std::unique_ptr<QueryWorkspace> ws =
        ws_acquire(g, a.S, t.row_need, t.chunk_need, t.srow_need, &s, st);
    if (!ws) return s;
    uint8_t *hs = static_cast<uint8_t *>(ws->staging);
    KParams p{};
    size_t tab_bytes = 0;
    s = place_tables(t, p, hs, ws->tables.as<uint8_t>(), kTablesBytes, st, &tab_bytes);
    if (s != RPQ_OK) {
        ws_release(g, std::move(ws));
        return s;
    }
    p.adj = g->d_adj.as<DevAdj>();
    p.n = g->n;
    p.W = ws->W;
    p.S = a.S;
    p.n_groups = (int32_t)t.groups.size();
    p.n_units = (int32_t)t.units.size();
    p.n_targets = (int32_t)t.t_unit.size();
    p.n_ugroups = (int32_t)t.u_group.size();
    p.source = multi ? 0 : source;
    p.n_sources = 1;
    p.max_levels = max_levels;
    p.start_mask = a.start_mask;
    p.final_mask = a.final_mask;
    size_t src_bytes = 0;
    if (multi) {
        src_bytes = sizeof(int32_t) * (size_t)x->n_sources;
        if (ws->srcs.bytes < src_bytes && !ws->srcs.alloc(src_bytes)) {
            ws_release(g, std::move(ws));
            return fail(RPQ_ERR_OOM, "source set (%d entries)", x->n_sources);
        }
        RPQ_CUDA_TRY(cudaMemcpyAsync(ws->srcs.p, x->sources, src_bytes, cudaMemcpyHostToDevice, st));
        p.sources = ws->srcs.as<int32_t>();
        p.n_sources = x->n_sources;
    }
    if (levels) {
        const size_t pl_bytes = sizeof(int32_t) * (size_t)ws->S_cap * g->n;
        if (ws->plevel.bytes < pl_bytes) {
            if (!ws->plevel.alloc(pl_bytes)) {
                ws_release(g, std::move(ws));
                return fail(RPQ_ERR_OOM, "pair levels (%zu bytes)", pl_bytes);
            }
            ws->plevel_dirty = true;
        }
        if (ws->plevel_dirty) RPQ_CUDA_TRY(cudaMemsetAsync(ws->plevel.p, 0xff, pl_bytes, st));
        ws->plevel_dirty = false;
        p.pair_level = ws->plevel.as<int32_t>();
    }
    p.alpha = env_float("RPQ_PULL_ALPHA", g->pull_alpha);
    p.min_pull = (int32_t)env_float("RPQ_PULL_MIN", (float)g->pull_min);
    p.solo_mass = (int32_t)env_float("RPQ_SOLO_MASS", (float)g->solo_mass);
    p.solo_items = (int32_t)env_float("RPQ_SOLO_ITEMS", (float)g->solo_items);
    sort_policy(g, p);
    wait_policy(p);
    hybrid_policy(g, p);
    precheck_policy(p);
    p.sort_cnt = ws->sortc.as<uint32_t>();
    p.epoch = ++ws->epoch;
    p.clear_first = ws->dirty ? 1 : 0;
    if (x && x->premask_bits) {
        // the kernel must not clear P after the rows are pre-set: a dirty
        // workspace is cleared here first
        const size_t bits_bytes = sizeof(uint64_t) * (size_t)a.S * ws->W;
        if (ws->dirty) {
            RPQ_CUDA_TRY(cudaMemsetAsync(ws->P.p, 0, bits_bytes, st));
            for (int k = 0; k < 3; k++) RPQ_CUDA_TRY(cudaMemsetAsync(ws->F[k].p, 0, bits_bytes, st));
            p.clear_first = 0;
        }
        const int64_t words = (int64_t)x->premask_states * ws->W;
        int sms = 0;
        RPQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
        premask_kernel<<<(int)std::min<int64_t>((int64_t)sms * 8, (words + 255) / 256), 256, 0, st>>>(
            ws->P.as<uint64_t>(), x->premask_bits, words);
        RPQ_CUDA_TRY(cudaGetLastError());
        note_launch();
        p.dense_clear = x->premask_states;
    }
    QueryResult *hr = reinterpret_cast<QueryResult *>(hs + kResultOffset);
    p.result = ws->result_dev;
    p.P = ws->P.as<uint64_t>();
    p.VL = ws->VL.as<int32_t>();
    for (int k = 0; k < 3; k++) {
        p.F[k] = ws->F[k].as<uint64_t>();
        p.rows[k] = ws->rows[k].as<Row>();
        p.cmap[k] = ws->cmap[k].as<int32_t>();
        p.srl[k] = ws->srl[k].as<int4>();
    }
    p.row_cap = ws->row_cap;
    p.chunk_cap = ws->chunk_cap;
    p.srow_cap = ws->srow_cap;
    p.mf = ws->mf.as<unsigned long long>();
    p.fin_sums = ws->fin.as<long long>();
    p.c = ws->ctr.as<Counters>();
    p.out_bits = out_bits_dev;
    static const char *trace_path = getenv("RPQ_TRACE_FILE");
    if (trace_path) {
        if (!ws->trace.p &&
            !ws->trace.alloc(sizeof(unsigned long long) * kTraceFields * (kTraceLevels + 1))) {
            ws_release(g, std::move(ws));
            return fail(RPQ_ERR_OOM, "trace buffer");
        }
        RPQ_CUDA_TRY(cudaMemsetAsync(ws->trace.p, 0, ws->trace.bytes, st));
        p.trace = ws->trace.as<unsigned long long>();
        p.trace_cap = kTraceLevels;
    }
    if (out_list_dev) {
        p.out_list = out_list_dev;
        p.capacity = capacity;
    } else if (want_host) {
        // a small answer is written by the kernel straight to this thread's
        // pinned host buffer (over the host link); a large one goes to device
        // memory and comes over by one copy after the kernel
        if (!tl_answer.reserve((size_t)g->n)) {
            ws_release(g, std::move(ws));
            return fail(RPQ_ERR_OOM, "pinned answer buffer (%d entries)", g->n);
        }
        p.out_list = ws->out_list.as<int32_t>();
        p.out_list_small = tl_answer.d;
        p.capacity = g->n;
    } else {
        p.out_list = nullptr;
        p.capacity = 0;
    }
    const size_t smem = shared_bytes(p.n_groups, p.n_units, p.n_targets, p.n_ugroups);
    int grid = 0;
    s = get_launch_shape(g->device, smem, &grid);
    if (s != RPQ_OK) {
        ws_release(g, std::move(ws));
        return s;
    }
    if (grid > kMaxGrid) grid = kMaxGrid;
    if (grid_div > 1) grid = std::max(1, grid / grid_div);
    const bool timed = stats != nullptr;
    if (timed) RPQ_CUDA_TRY(cudaEventRecord(ws->ev0, st));
    void *args[] = {&p};
    RPQ_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)rpq_query_kernel, dim3(grid),
                                             dim3(kThreads), args, smem, st));
    note_launch();
    if (timed) RPQ_CUDA_TRY(cudaEventRecord(ws->ev1, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (*(volatile uint32_t *)&hr->epoch != p.epoch) {
        // no summary: the traversal gave up.  It leaves the barrier counters
        // mid-way and P / F not cleared: read the status, reset the
        // counters, clear P / F on next use
        Counters *hc = reinterpret_cast<Counters *>(hs + kTablesBytes);
        RPQ_CUDA_TRY(cudaMemcpyAsync(hc, ws->ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, st));
        cudaMemsetAsync(ws->ctr.p, 0, sizeof(Counters), st);
        RPQ_CUDA_TRY(cudaStreamSynchronize(st));
        ws->dirty = true;
        if (levels) ws->plevel_dirty = true;
        const int32_t hs_status = status_of(hc->gen_status);
        const rpq_status e = hs_status != 0 ? (rpq_status)hs_status : RPQ_ERR_CUDA;
        ws_release(g, std::move(ws));
        return fail(e, "device traversal failed (status %d)", (int)e);
    }
    ws->dirty = false;
    *count = hr->answer_count;
    const bool copy_list = out_host_list && !out_list_dev && *count <= capacity && *count > 0;
    const int64_t host_bytes = want_host ? 4 * *count : 0;
    if (levels) {
        rpq_status e = path_outputs(g, a, ws.get(), x, out_list_dev, std::min<int64_t>(*count, capacity), st);
        if (e != RPQ_OK) {
            ws->plevel_dirty = true;
            ws_release(g, std::move(ws));
            return e;
        }
    }
    if (stats) {
        stats->h2d_bytes = (int64_t)(tab_bytes + src_bytes);
        stats->d2h_bytes = (int64_t)sizeof(QueryResult) + host_bytes;
        stats->levels = hr->levels;
        stats->visited_pairs = hr->visited;
        stats->expanded_pairs = hr->expanded;
        stats->product_edges = hr->product_edges;
        stats->push_bytes = hr->push_bytes;
        stats->answer_count = hr->answer_count;
        stats->push_unit_levels = hr->push_units;
        stats->pull_unit_levels = hr->pull_units;
        float ms = -1.0f;
        if (cudaEventElapsedTime(&ms, ws->ev0, ws->ev1) != cudaSuccess) ms = -1.0f;
        stats->device_ms = ms;
    }
    if (want_host) {
        if (!hr->small && *count > 0) {
            RPQ_CUDA_TRY(cudaMemcpyAsync(tl_answer.h, ws->out_list.p, sizeof(int32_t) * (*count),
                                         cudaMemcpyDeviceToHost, st));
            RPQ_CUDA_TRY(cudaStreamSynchronize(st));
        }
        tl_answer.count = *count;
        tl_answer.valid = true;
    }
    if (copy_list) memcpy(out_host_list, tl_answer.h, sizeof(int32_t) * (size_t)(*count));
    if (trace_path)
        write_trace(trace_path, ws.get(), a.S, source,
                    (int)std::min<long long>(hr->levels + 2, kTraceLevels), st);
    ws_release(g, std::move(ws));
    return RPQ_OK;
}

}  // namespace rpq

// ------------------------------------------------------------- autotune --
namespace rpq {
rpq_status autotune(rpq_graph *g, int32_t n, const rpq_nfa *const *nfas, const int32_t *sources,
                    float *alpha_out, int32_t *min_out, int32_t *solo_out, void *stream) {
    static const float kAlphas[] = {0.0f, 1.0f, 2.0f, 4.0f, 8.0f, 16.0f, 64.0f};
    static const int32_t kMins[] = {64, 256, 2048};
    const float keep_a = g->pull_alpha;
    const int32_t keep_m = g->pull_min;
    double best = -1;
    float best_a = keep_a;
    int32_t best_m = keep_m;
    for (float a : kAlphas) {
        for (int32_t m : kMins) {
            if (a == 0.0f && m != kMins[0]) continue;  // push only: min_pull is moot
            g->pull_alpha = a;
            g->pull_min = m;
            double total = 0;
            for (int rep = 0; rep < 2; rep++) {  // first pass warms the workspace
                total = 0;
                for (int32_t i = 0; i < n; i++) {
                    rpq_stats st{};
                    int64_t cnt = 0;
                    rpq_status s = run_query(g, nfas[i]->a, sources[i], 0, nullptr, 0, nullptr,
                                             nullptr, &st, &cnt, stream);
                    if (s != RPQ_OK) {
                        g->pull_alpha = keep_a;
                        g->pull_min = keep_m;
                        return s;
                    }
                    total += st.device_ms;
                }
            }
            if (best < 0 || total < best) {
                best = total;
                best_a = a;
                best_m = m;
            }
        }
    }
    g->pull_alpha = best_a;
    g->pull_min = best_m;
    // then the one-CTA level threshold, under the chosen direction setting
    static const int32_t kSolo[] = {-1, 512, 2048, 8192};
    const int32_t keep_s = g->solo_mass, keep_i = g->solo_items;
    double best_solo = -1;
    int32_t best_s = keep_s, best_i = keep_i;
    for (int32_t sm : kSolo) {
        g->solo_mass = sm;
        g->solo_items = sm < 0 ? 0 : sm / 8;
        double total = 0;
        for (int rep = 0; rep < 2; rep++) {
            total = 0;
            for (int32_t i = 0; i < n; i++) {
                rpq_stats st{};
                int64_t cnt = 0;
                rpq_status s = run_query(g, nfas[i]->a, sources[i], 0, nullptr, 0, nullptr,
                                         nullptr, &st, &cnt, stream);
                if (s != RPQ_OK) {
                    g->solo_mass = keep_s;
                    g->solo_items = keep_i;
                    return s;
                }
                total += st.device_ms;
            }
        }
        if (best_solo < 0 || total < best_solo) {
            best_solo = total;
            best_s = g->solo_mass;
            best_i = g->solo_items;
        }
    }
    g->solo_mass = best_s;
    g->solo_items = best_i;
    if (alpha_out) *alpha_out = best_a;
    if (min_out) *min_out = best_m;
    if (solo_out) *solo_out = best_s;
    return RPQ_OK;
}
}  // namespace rpq

extern "C" rpq_status rpq_graph_set_hybrid(rpq_graph *g, int64_t switch_pairs) {
    rpq::clear_error();
    if (!g || switch_pairs < 0) return rpq::fail(RPQ_ERR_INVALID, "bad argument");
    g->alg2_until = switch_pairs;
    return RPQ_OK;
}

extern "C" rpq_status rpq_graph_autotune(rpq_graph *g, int32_t n, const rpq_nfa *const *nfas,
                                         const int32_t *sources, float *alpha_out,
                                         int32_t *min_pull_out, int32_t *solo_mass_out,
                                         void *stream) {
    rpq::clear_error();
    if (!g || n <= 0 || !nfas || !sources) return rpq::fail(RPQ_ERR_INVALID, "bad argument");
    for (int32_t i = 0; i < n; i++)
        if (!nfas[i]) return rpq::fail(RPQ_ERR_INVALID, "automaton %d is null", i);
    return rpq::autotune(g, n, nfas, sources, alpha_out, min_pull_out, solo_mass_out, stream);
}

// --------------------------------------------------- no-allocation entry --
// Scratch for rpq_query_noalloc: a fixed device array that exists for as
// long as the library is loaded, so a query needs no device allocation.
#define RPQ_NOALLOC_SCRATCH_BYTES (64ull << 20)
static __device__ __align__(256) unsigned char rpq_noalloc_scratch[RPQ_NOALLOC_SCRATCH_BYTES];

namespace rpq {
namespace {
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[64];      // device address of the scratch, per device
uint32_t g_noalloc_epoch[64]; // launches on the scratch, per device

// Device address of the scratch on `device` (which must be current), looked
// up once per device; the barrier counters are cleared on that first call.
// Also hands out the launch's epoch.
rpq_status noalloc_scratch(int device, void **out, uint32_t *epoch, cudaStream_t st) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (device < 0 || device >= 64) return fail(RPQ_ERR_CUDA, "device id %d", device);
    if (!g_noalloc_ptr[device]) {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, rpq_noalloc_scratch);
        if (e != cudaSuccess || !ptr)
            return fail(RPQ_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        // on the caller's stream, ordered before the launch that follows
        RPQ_CUDA_TRY(cudaMemsetAsync(ptr, 0, sizeof(Counters), st));
        RPQ_CUDA_TRY(cudaStreamSynchronize(st));
        g_noalloc_ptr[device] = ptr;
    }
    *out = g_noalloc_ptr[device];
    *epoch = ++g_noalloc_epoch[device];
    return RPQ_OK;
}
}  // namespace
}  // namespace rpq

using namespace rpq;

extern "C" rpq_status rpq_query_noalloc(const rpq_graph *g, const rpq_nfa *nfa, int32_t source,
                                        int32_t max_levels, int32_t *out_vertices,
                                        int64_t capacity, int64_t *out_count, void *stream) {
    clear_error();
    if (!g || !nfa || !out_count) return fail(RPQ_ERR_INVALID, "null argument");
    if (capacity < 0 || (capacity > 0 && !out_vertices))
        return fail(RPQ_ERR_INVALID, "bad output buffer");
    if (out_vertices && !is_device_pointer(out_vertices))
        return fail(RPQ_ERR_INVALID, "rpq_query_noalloc writes device memory only");
    *out_count = 0;
    const Automaton &a = nfa->a;
    if (source < 0 || source >= g->n)
        return fail(RPQ_ERR_INVALID, "source %d outside [0, %d)", source, g->n);
    if (max_levels < 0) return fail(RPQ_ERR_INVALID, "max_levels must be >= 0");
    if (a.S <= 0 || a.S > kMaxStates) return fail(RPQ_ERR_INVALID, "automaton has %d states", a.S);
    int dev = -1;
    RPQ_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != g->device)
        return fail(RPQ_ERR_INVALID, "make the graph's device (%d) current first", g->device);
    env_snapshot();
    thread_local Tables t;  // reused: no host allocation once grown
    t.clear();
    rpq_status s = build_tables(g, a, &t);
    if (s != RPQ_OK) return s;

    // scratch layout: counters | mf | per-CTA sums | tables | P | F[3] | VL | rows[3] | cmap[3]
    const int64_t W = ((int64_t)g->n + 63) / 64;
    std::vector<uint8_t> host_tables;
    size_t toff = 0;
    auto put = [&](const void *src, size_t bytes) {
        toff = (toff + 15) & ~size_t(15);
        const size_t at = toff;
        host_tables.resize(toff + bytes);
        if (bytes) memcpy(host_tables.data() + at, src, bytes);
        toff += bytes;
        return at;
    };
    const size_t o_groups = put(t.groups.data(), sizeof(QGroup) * t.groups.size());
    const size_t o_units = put(t.units.data(), sizeof(QUnit) * t.units.size());
    const size_t o_tu = put(t.t_unit.data(), sizeof(int32_t) * t.t_unit.size());
    const size_t o_ts = put(t.t_state.data(), sizeof(int32_t) * t.t_state.size());
    const size_t o_ug = put(t.u_group.data(), sizeof(int32_t) * t.u_group.size());
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~size_t(255);
        const size_t at = off;
        off += bytes;
        return at;
    };
    const size_t x_ctr = take(sizeof(Counters));
    const size_t x_mf = take(sizeof(unsigned long long) * 3 * kMaxGroups);
    const size_t x_fin = take(sizeof(long long) * kMaxGrid);
    const size_t x_sort = take(sizeof(uint32_t) * (size_t)a.S * kMaxGrid);
    const size_t x_tab = take(std::max<size_t>(toff, 16));
    const size_t bits = sizeof(uint64_t) * (size_t)a.S * W;
    const size_t fl = sizeof(int32_t) * (size_t)a.S * g->n;
    const size_t x_P = take(bits);
    size_t x_F[3], x_rows[3], x_cmap[3], x_srl[3];
    for (int k = 0; k < 3; k++) x_F[k] = take(bits);
    const size_t x_VL = take(fl);
    for (int k = 0; k < 3; k++) x_rows[k] = take(sizeof(Row) * (size_t)t.row_need);
    for (int k = 0; k < 3; k++) x_cmap[k] = take(sizeof(int32_t) * (size_t)t.chunk_need);
    for (int k = 0; k < 3; k++) x_srl[k] = take(sizeof(int4) * (size_t)t.srow_need);
    if (off > RPQ_NOALLOC_SCRATCH_BYTES)
        return fail(RPQ_ERR_INVALID,
                    "query needs %zu bytes of scratch; rpq_query_noalloc holds %llu "
                    "(use rpq_query)",
                    off, (unsigned long long)RPQ_NOALLOC_SCRATCH_BYTES);
    void *base_v = nullptr;
    uint32_t epoch = 0;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    s = noalloc_scratch(dev, &base_v, &epoch, st);
    if (s != RPQ_OK) return s;
    uint8_t *base = static_cast<uint8_t *>(base_v);
    RPQ_CUDA_TRY(cudaMemcpyAsync(base + x_tab, host_tables.data(), std::max<size_t>(toff, 1),
                                 cudaMemcpyHostToDevice, st));

    KParams p{};
    p.adj = g->d_adj.as<DevAdj>();
    p.n = g->n;
    p.W = (int32_t)W;
    p.S = a.S;
    p.n_groups = (int32_t)t.groups.size();
    p.n_units = (int32_t)t.units.size();
    p.n_targets = (int32_t)t.t_unit.size();
    p.n_ugroups = (int32_t)t.u_group.size();
    p.source = source;
    p.n_sources = 1;
    p.max_levels = max_levels;
    p.start_mask = a.start_mask;
    p.final_mask = a.final_mask;
    p.alpha = env_float("RPQ_PULL_ALPHA", g->pull_alpha);
    p.min_pull = (int32_t)env_float("RPQ_PULL_MIN", (float)g->pull_min);
    p.solo_mass = g->solo_mass;
    p.solo_items = g->solo_items;
    sort_policy(g, p);
    wait_policy(p);
    hybrid_policy(g, p);
    precheck_policy(p);
    p.sort_cnt = reinterpret_cast<uint32_t *>(base + x_sort);
    // the scratch layout moves with the automaton's size: clear P / F first
    p.clear_first = 1;
    p.groups = reinterpret_cast<const QGroup *>(base + x_tab + o_groups);
    p.units = reinterpret_cast<const QUnit *>(base + x_tab + o_units);
    p.t_unit = reinterpret_cast<const int32_t *>(base + x_tab + o_tu);
    p.t_state = reinterpret_cast<const int32_t *>(base + x_tab + o_ts);
    p.u_group = reinterpret_cast<const int32_t *>(base + x_tab + o_ug);
    p.P = reinterpret_cast<uint64_t *>(base + x_P);
    p.VL = reinterpret_cast<int32_t *>(base + x_VL);
    for (int k = 0; k < 3; k++) {
        p.F[k] = reinterpret_cast<uint64_t *>(base + x_F[k]);
        p.rows[k] = reinterpret_cast<Row *>(base + x_rows[k]);
        p.cmap[k] = reinterpret_cast<int32_t *>(base + x_cmap[k]);
        p.srl[k] = reinterpret_cast<int4 *>(base + x_srl[k]);
    }
    p.row_cap = t.row_need;
    p.chunk_cap = t.chunk_need;
    p.srow_cap = t.srow_need;
    p.mf = reinterpret_cast<unsigned long long *>(base + x_mf);
    p.fin_sums = reinterpret_cast<long long *>(base + x_fin);
    p.c = reinterpret_cast<Counters *>(base + x_ctr);
    p.out_list = out_vertices;
    p.capacity = out_vertices ? capacity : 0;
    p.out_bits = nullptr;
    p.epoch = epoch;
    const size_t smem = shared_bytes(p.n_groups, p.n_units, p.n_targets, p.n_ugroups);
    int grid = 0;
    s = get_launch_shape(dev, smem, &grid);
    if (s != RPQ_OK) return s;
    void *args[] = {&p};
    RPQ_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)rpq_query_kernel, dim3(grid),
                                             dim3(kThreads), args, smem, st));
    note_launch();
    Counters hc;
    RPQ_CUDA_TRY(cudaMemcpyAsync(&hc, p.c, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (const int32_t hs_status = status_of(hc.gen_status)) {
        // a traversal that gave up leaves the barrier counters mid-way: reset them
        cudaMemsetAsync(p.c, 0, sizeof(Counters), st);
        cudaStreamSynchronize(st);
        return fail((rpq_status)hs_status, "device traversal failed (status %d)", hs_status);
    }
    *out_count = hc.answer_count;
    if (hc.answer_count > capacity)
        return fail(RPQ_ERR_CAPACITY, "answer has %lld vertices, capacity %lld",
                    (long long)hc.answer_count, (long long)capacity);
    return RPQ_OK;
}
