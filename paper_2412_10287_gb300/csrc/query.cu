// Single-source 2-RPQ on the device: Algorithm 1 of the paper (section 4)
//     M <- ( OR_a (N^a)^T x M x G^a ) <not P>,  P <- P + M,  until M = 0;
//     answer F x P
// run as ONE persistent cooperative kernel per query.  The Boolean matrices
// are kept as bitsets (one row of |V| bits per automaton state) plus, for the
// frontier M, per-state vertex lists.  Each level is two grid-wide phases:
//
//   expand  for every (label direction d, target state q'):
//             push  -- for every frontier pair (q, v) with q -d-> q' and every
//                      w in row v of G^d: if w not in P[q'], set NX[q'][w]
//                      (atomicOr); rows are spread over a CTA by a scan-based
//                      gather, hub rows over many CTAs in fixed chunks;
//             pull  -- for every w not in P[q'] with in-edges of direction d:
//                      NX[q'][w] = OR over in-neighbours u of
//                      X_{d,q'}[u] = OR_{q: q -d-> q'} M[q][u]  (early exit);
//           the chosen direction per (d, q') follows the edge mass of the
//           frontier (a direction-optimising BFS: push-pull is the
//           optimisation the paper's conclusion names).
//   commit  for every word first set this level (a touched-word list):
//             M[q'] = NX word (already masked by not P), P |= M, NX = 0; the
//             new frontier pairs become vertex lists with their row lengths
//             (edge mass for the next direction choice, hub rows split off).
//
// Every wait on other CTAs (the grid barrier) is bounded by a wall-clock
// limit; on expiry the kernel records RPQ_ERR_TIMEOUT and returns.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>

#include "graph.h"

namespace rpq {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kHubDeg = 4096;    // rows at least this long are split across CTAs
constexpr int kHubChunk = 2048;  // edges per hub chunk
constexpr int kGather = 1024;    // gather buffer entries per CTA
constexpr int kWarpRow = 32;     // rows at least this long are expanded by a whole warp
constexpr int kMaxGroups = 512;
constexpr int kMaxUnits = 512;
constexpr int kMaxTargets = 4096;
constexpr uint64_t kBarrierTimeoutNs = 4000000000ull;

// (source state q, direction d) with the targets delta(q, d) as a mask.
struct QGroup {
    int32_t q, d;
    uint64_t tmask;
    int32_t t_first, t_count;  // slots in the target table: (unit, q') pairs
};
// (direction d, target state q') with the source states {q : q -d-> q'}.
struct QUnit {
    int32_t d, q2, in_dir, g_first, g_count;
    int32_t pad;
    uint64_t smask;
    int64_t in_rows;   // rows of the in-adjacency to sweep when pulling
    int64_t in_nnz;
};

struct Hub {
    int32_t g, v, b, e;
    int64_t chunk_base;
};

// Device counters of one query (zeroed by the kernel prologue except the
// barrier fields, which the host zeroes at workspace creation).
struct Counters {
    unsigned bar_count, bar_gen;
    int32_t status, where;
    unsigned long long touched[3];
    unsigned long long fl_count[2][kMaxStates];
    unsigned long long lvl_bytes[2], lvl_edges[2];
    unsigned long long hub_packed[2];  // (entries << 40) | chunks
    unsigned long long claim_hub[2], claim_item[2], claim_pull[2];
    long long levels, visited, expanded, product_edges, push_bytes;
    long long push_units, pull_units, answer_count;
    long long final_flag;
};

struct KParams {
    // graph
    const DevAdj *adj;
    int32_t n, W, S;
    int32_t n_groups, n_units, n_targets;
    int32_t source, max_levels;
    uint64_t start_mask, final_mask;
    float alpha;       // pull when frontier edge mass * alpha > in-adjacency edges
    int32_t min_pull;  // ... and the unit's source frontier has at least this many pairs
    // automaton tables (device)
    const QGroup *groups;
    const QUnit *units;
    const int32_t *t_unit;   // per target slot: unit index
    const int32_t *t_state;  // per target slot: q'
    const int32_t *u_group;  // per unit group slot: group index
    // state (device)
    uint64_t *P, *NX, *F0, *F1;
    uint32_t *T0, *T1, *T2;
    int32_t *FL0, *FL1;    // [S][n]
    Hub *H0, *H1;
    int64_t hub_cap;
    unsigned long long *mf;  // [2][kMaxGroups]
    long long *fin_sums;     // [gridDim]
    Counters *c;
    // output
    int32_t *out_list;
    int64_t capacity;
    uint64_t *out_bits;  // bitset output (or nullptr)
};

// ------------------------------------------------------------ barrier ----
__device__ __forceinline__ int load_status(const Counters *c) {
    return *(volatile const int32_t *)&c->status;
}

__device__ bool grid_barrier(Counters *c) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *genp = &c->bar_gen;
        const unsigned gen = *genp;
        __threadfence();
        const unsigned arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            const uint64_t t0 = global_timer_ns();
            unsigned it = 0;
            while (*genp == gen) {
                __nanosleep(32);
                if ((++it & 255u) == 0) {
                    if (load_status(c) != 0) break;
                    if (global_timer_ns() - t0 > kBarrierTimeoutNs) {
                        atomicCAS(&c->status, 0, (int32_t)RPQ_ERR_TIMEOUT);
                        break;
                    }
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return load_status(c) == 0;
}

// ------------------------------------------------------- warp helpers ----
// Appends `code` for every lane with `need`; all 32 lanes must call.
__device__ __forceinline__ void warp_append(bool need, uint32_t code, uint32_t *list,
                                            unsigned long long *count) {
    const unsigned m = __ballot_sync(kFull, need);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (need) list[base + __popc(m & lanemask_lt())] = code;
}

// Relaxation of edge (., w) into every target state in `tmask` (already
// restricted to push-mode targets).  All 32 lanes must call; lanes with
// valid = false take part in the collectives only.
__device__ __forceinline__ void relax(const KParams &p, bool valid, uint64_t tmask, int32_t w,
                                      uint32_t *tl, unsigned long long *tcount) {
    uint64_t todo = valid ? tmask : 0ull;
    // iterate over the union of target bits across the warp
    uint32_t lo = __reduce_or_sync(kFull, (uint32_t)todo);
    uint32_t hi = __reduce_or_sync(kFull, (uint32_t)(todo >> 32));
    uint64_t all = ((uint64_t)hi << 32) | lo;
    const uint32_t wi = (uint32_t)w >> 6;
    const uint64_t bit = 1ull << (w & 63);
    while (all) {
        const int q2 = __ffsll((long long)all) - 1;
        all &= all - 1;
        bool need = false;
        if ((todo >> q2) & 1ull) {
            const size_t idx = (size_t)q2 * p.W + wi;
            if (!(__ldcg(p.P + idx) & bit) && !(__ldcg(p.NX + idx) & bit)) {
                const unsigned long long old =
                    atomicOr((unsigned long long *)(p.NX + idx), (unsigned long long)bit);
                need = (old == 0ull);
            }
        }
        warp_append(need, (uint32_t)q2 * (uint32_t)p.W + wi, tl, tcount);
    }
}

// ------------------------------------------------------- shared layout ---
struct Shared {
    // per group (dynamic arrays carved from extern shared memory)
    uint64_t *tpush;    // push-mode targets of each group
    long long *gpref;   // prefix of frontier items over push groups (n_groups + 1)
    const int32_t **gnbr;
    int32_t *gq, *gd;
    // per unit
    long long *upref;   // prefix of pull rows over pull units (n_units + 1)
    uint8_t *upull;
    // gather buffer
    int32_t *gbuf_k;
    int16_t *gbuf_g;
};

__device__ Shared carve(const KParams &p, uint8_t *base) {
    Shared s;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        uint8_t *r = base + off;
        off += bytes;
        return r;
    };
    s.tpush = (uint64_t *)take(sizeof(uint64_t) * p.n_groups);
    s.gpref = (long long *)take(sizeof(long long) * (p.n_groups + 1));
    s.gnbr = (const int32_t **)take(sizeof(void *) * p.n_groups);
    s.gq = (int32_t *)take(sizeof(int32_t) * p.n_groups);
    s.gd = (int32_t *)take(sizeof(int32_t) * p.n_groups);
    s.upref = (long long *)take(sizeof(long long) * (p.n_units + 1));
    s.upull = (uint8_t *)take(p.n_units);
    s.gbuf_k = (int32_t *)take(sizeof(int32_t) * kGather);
    s.gbuf_g = (int16_t *)take(sizeof(int16_t) * kGather);
    return s;
}

__host__ __device__ size_t shared_bytes(int n_groups, int n_units) {
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 15) & ~size_t(15);
        off += bytes;
    };
    take(sizeof(uint64_t) * n_groups);
    take(sizeof(long long) * (n_groups + 1));
    take(sizeof(void *) * n_groups);
    take(sizeof(int32_t) * n_groups);
    take(sizeof(int32_t) * n_groups);
    take(sizeof(long long) * (n_units + 1));
    take(n_units);
    take(sizeof(int32_t) * kGather);
    take(sizeof(int16_t) * kGather);
    return off + 64;
}

// ---------------------------------------------------------------- phases -
// Commit of level j: consume the touched list TL_j.
__device__ void commit_phase(const KParams &p, int j, const Shared &sh, unsigned long long *s_cnt,
                             unsigned long long *s_base, unsigned long long *s_mf,
                             unsigned long long *s_acc) {
    const uint32_t *tl = (j % 3 == 0) ? p.T0 : (j % 3 == 1) ? p.T1 : p.T2;
    const unsigned long long nt = *(volatile unsigned long long *)&p.c->touched[j % 3];
    uint64_t *F = (j & 1) ? p.F1 : p.F0;
    int32_t *FL = (j & 1) ? p.FL1 : p.FL0;
    Hub *H = (j & 1) ? p.H1 : p.H0;
    const int par = j & 1;
    // zero the count of the list that the next expansion fills: TL_{j+1}
    if (blockIdx.x == 0 && threadIdx.x == 0) p.c->touched[(j + 1) % 3] = 0;
    for (int i = threadIdx.x; i < p.n_groups; i += kThreads) s_mf[i] = 0;
    if (threadIdx.x < 2) s_acc[threadIdx.x] = 0;
    for (int i = threadIdx.x; i < p.S; i += kThreads) s_cnt[i] = 0;
    __syncthreads();
    for (unsigned long long tile = (unsigned long long)blockIdx.x * kThreads; tile < nt;
         tile += (unsigned long long)gridDim.x * kThreads) {
        const unsigned long long e = tile + threadIdx.x;
        int q2 = 0;
        uint32_t wi = 0;
        uint64_t word = 0;
        unsigned long long loc = 0;
        if (e < nt) {
            const uint32_t code = __ldcg(tl + e);
            q2 = (int)(code / (uint32_t)p.W);
            wi = code - (uint32_t)q2 * (uint32_t)p.W;
            const size_t idx = (size_t)q2 * p.W + wi;
            word = __ldcg(p.NX + idx);
            p.NX[idx] = 0;
            p.P[idx] = __ldcg(p.P + idx) | word;
            F[idx] = word;
            loc = atomicAdd(&s_cnt[q2], (unsigned long long)__popcll(word));
        }
        __syncthreads();
        if (threadIdx.x < p.S) {
            const unsigned long long c = s_cnt[threadIdx.x];
            s_base[threadIdx.x] = c ? atomicAdd(&p.c->fl_count[par][threadIdx.x], c) : 0ull;
            s_cnt[threadIdx.x] = 0;
        }
        __syncthreads();
        if (word) {
            unsigned long long pos = s_base[q2] + loc;
            int32_t *list = FL + (size_t)q2 * p.n;
            uint64_t wd = word;
            while (wd) {
                const int b = __ffsll((long long)wd) - 1;
                wd &= wd - 1;
                const int32_t v = (int32_t)(wi * 64u + (uint32_t)b);
                list[pos++] = v;
                // edge mass of every group leaving state q2, hubs split off
                for (int g = 0; g < p.n_groups; g++) {
                    if (sh.gq[g] != q2) continue;
                    int32_t rb, re;
                    adj_row(p.adj[sh.gd[g]], v, rb, re);
                    const int32_t deg = re - rb;
                    atomicAdd(&s_mf[g], (unsigned long long)deg);
                    atomicAdd(&s_acc[0], 8ull + 4ull * (unsigned long long)deg);
                    const uint64_t tm = p.groups[g].tmask;
                    atomicAdd(&s_acc[1], (unsigned long long)deg * (unsigned long long)__popcll(tm));
                    if (deg >= kHubDeg) {
                        const unsigned long long nch = (deg + kHubChunk - 1) / kHubChunk;
                        const unsigned long long old =
                            atomicAdd(&p.c->hub_packed[par], (1ull << 40) | nch);
                        const unsigned long long hi = old >> 40;
                        if ((long long)hi < p.hub_cap) {
                            Hub h;
                            h.g = g; h.v = v; h.b = rb; h.e = re;
                            h.chunk_base = (long long)(old & ((1ull << 40) - 1));
                            H[hi] = h;
                        } else {
                            atomicCAS(&p.c->status, 0, (int32_t)RPQ_ERR_OOM);
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p.n_groups; i += kThreads)
        if (s_mf[i]) atomicAdd(&p.mf[par * kMaxGroups + i], s_mf[i]);
    if (threadIdx.x == 0) {
        if (s_acc[0]) atomicAdd(&p.c->lvl_bytes[par], s_acc[0]);
        if (s_acc[1]) atomicAdd(&p.c->lvl_edges[par], s_acc[1]);
    }
}

// Process push edges k in [kb, ke) of group g's neighbour array, one per thread
// per round; whole-block uniform loop.
__device__ __forceinline__ void push_range_block(const KParams &p, const Shared &sh, int g,
                                                 int64_t kb, int64_t ke, uint32_t *tl,
                                                 unsigned long long *tcount) {
    const int32_t *nbr = sh.gnbr[g];
    const uint64_t tm = sh.tpush[g];
    for (int64_t base = kb; base < ke; base += kThreads) {
        const int64_t k = base + threadIdx.x;
        const bool valid = k < ke;
        const int32_t w = valid ? __ldg(nbr + k) : 0;
        relax(p, valid, tm, w, tl, tcount);
    }
}

__device__ void expand_phase(const KParams &p, int j, const Shared &sh, long long *s_claim) {
    // this expansion reads level j (written by commit j) and fills TL_{j+1}
    const int par = j & 1;
    const uint64_t *F = par ? p.F1 : p.F0;
    const int32_t *FL = par ? p.FL1 : p.FL0;
    const Hub *H = par ? p.H1 : p.H0;
    uint32_t *tl = ((j + 1) % 3 == 0) ? p.T0 : ((j + 1) % 3 == 1) ? p.T1 : p.T2;
    unsigned long long *tcount = &p.c->touched[(j + 1) % 3];
    const unsigned lane = lane_id();

    // housekeeping for commit j+1 (nothing reads these now)
    {
        uint64_t *Fn = par ? p.F0 : p.F1;  // held level j-1: clear its words
        if (j >= 1) {
            const uint32_t *old = ((j - 1) % 3 == 0) ? p.T0 : ((j - 1) % 3 == 1) ? p.T1 : p.T2;
            const unsigned long long no = *(volatile unsigned long long *)&p.c->touched[(j - 1) % 3];
            for (unsigned long long i = (unsigned long long)blockIdx.x * kThreads + threadIdx.x;
                 i < no; i += (unsigned long long)gridDim.x * kThreads)
                Fn[__ldcg(old + i)] = 0;  // code = q * W + wi indexes the bitset directly
        }
        if (blockIdx.x == 0) {
            const int np = par ^ 1;
            for (int i = threadIdx.x; i < p.S; i += kThreads) p.c->fl_count[np][i] = 0;
            for (int i = threadIdx.x; i < p.n_groups; i += kThreads) p.mf[np * kMaxGroups + i] = 0;
            if (threadIdx.x == 0) {
                p.c->lvl_bytes[np] = 0;
                p.c->lvl_edges[np] = 0;
                p.c->hub_packed[np] = 0;
                p.c->claim_hub[np] = 0;
                p.c->claim_item[np] = 0;
                p.c->claim_pull[np] = 0;
            }
        }
    }

    // (1) hub rows, chunked across all CTAs
    {
        const unsigned long long packed = *(volatile unsigned long long *)&p.c->hub_packed[par];
        const long long nh = (long long)(packed >> 40);
        const long long nchunks = (long long)(packed & ((1ull << 40) - 1));
        for (;;) {
            if (threadIdx.x == 0) *s_claim = (long long)atomicAdd(&p.c->claim_hub[par], 1ull);
            __syncthreads();
            const long long c = *s_claim;
            __syncthreads();
            if (c >= nchunks) break;
            // hub whose chunk range holds c: last entry with chunk_base <= c
            long long lo = 0, hi = nh - 1;
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if (__ldcg(&H[mid].chunk_base) <= c) lo = mid; else hi = mid - 1;
            }
            const int g = __ldcg(&H[lo].g);
            if (sh.tpush[g] == 0) continue;
            const int64_t b = __ldcg(&H[lo].b), e = __ldcg(&H[lo].e);
            const int64_t kb = b + (c - __ldcg(&H[lo].chunk_base)) * kHubChunk;
            const int64_t ke = min(e, kb + kHubChunk);
            push_range_block(p, sh, g, kb, ke, tl, tcount);
        }
    }

    // (2) frontier items of push groups, tiles of kThreads items
    const long long total_items = sh.gpref[p.n_groups];
    for (;;) {
        if (threadIdx.x == 0)
            *s_claim = (long long)atomicAdd(&p.c->claim_item[par], (unsigned long long)kThreads);
        __syncthreads();
        const long long t0 = *s_claim;
        __syncthreads();
        if (t0 >= total_items) break;
        const long long i = t0 + threadIdx.x;
        int g = -1;
        int32_t rb = 0, re = 0;
        if (i < total_items) {
            int lo = 0, hi = p.n_groups - 1;  // last group with gpref <= i
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sh.gpref[mid] <= i) lo = mid; else hi = mid - 1;
            }
            g = lo;
            const int32_t v = __ldcg(FL + (size_t)sh.gq[g] * p.n + (i - sh.gpref[g]));
            adj_row(p.adj[sh.gd[g]], v, rb, re);
            if (re - rb >= kHubDeg) re = rb;  // handled as a hub
        }
        int32_t deg = re - rb;
        // (a) rows of at least kWarpRow edges: one warp per row
        {
            bool pending = deg >= kWarpRow;
            unsigned m;
            while ((m = __ballot_sync(kFull, pending)) != 0) {
                const int leader = __ffs(m) - 1;
                const int gg = __shfl_sync(kFull, g, leader);
                const int32_t b = __shfl_sync(kFull, rb, leader);
                const int32_t e = __shfl_sync(kFull, re, leader);
                if ((int)lane == leader) pending = false;
                const int32_t *nbr = sh.gnbr[gg];
                const uint64_t tm = sh.tpush[gg];
                for (int32_t base = b; base < e; base += 32) {
                    const int32_t k = base + (int32_t)lane;
                    const bool valid = k < e;
                    const int32_t w = valid ? __ldg(nbr + k) : 0;
                    relax(p, valid, tm, w, tl, tcount);
                }
            }
            if (deg >= kWarpRow) deg = 0;
        }
        // (b) short rows: CTA-wide scan-based gather
        {
            long long tot = 0;
            // block exclusive scan of deg
            __shared__ int32_t wsum[kWarps + 1];
            int32_t incl = deg;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, incl, o);
                if ((int)lane >= o) incl += y;
            }
            if (lane == 31) wsum[threadIdx.x >> 5] = incl;
            __syncthreads();
            if (threadIdx.x == 0) {
                int32_t run = 0;
                for (int w = 0; w < kWarps; w++) {
                    const int32_t s = wsum[w];
                    wsum[w] = run;
                    run += s;
                }
                wsum[kWarps] = run;
            }
            __syncthreads();
            const int32_t excl = wsum[threadIdx.x >> 5] + incl - deg;
            tot = wsum[kWarps];
            __syncthreads();
            for (long long rbase = 0; rbase < tot; rbase += kGather) {
                // scatter my edges that fall in [rbase, rbase + kGather)
                const long long lo = max((long long)excl, rbase);
                const long long hi = min((long long)excl + deg, rbase + kGather);
                for (long long r = lo; r < hi; r++) {
                    sh.gbuf_k[r - rbase] = rb + (int32_t)(r - excl);
                    sh.gbuf_g[r - rbase] = (int16_t)g;
                }
                __syncthreads();
                const long long cnt = min((long long)kGather, tot - rbase);
                for (long long base = 0; base < cnt; base += kThreads) {
                    const long long idx = base + threadIdx.x;
                    const bool valid = idx < cnt;
                    int gg = 0;
                    int32_t w = 0;
                    uint64_t tm = 0;
                    if (valid) {
                        gg = sh.gbuf_g[idx];
                        w = __ldg(sh.gnbr[gg] + sh.gbuf_k[idx]);
                        tm = sh.tpush[gg];
                    }
                    relax(p, valid, tm, w, tl, tcount);
                }
                __syncthreads();
            }
        }
    }

    // (3) pull units: sweep the rows of the in-adjacency
    const long long total_rows = sh.upref[p.n_units];
    for (;;) {
        if (threadIdx.x == 0)
            *s_claim = (long long)atomicAdd(&p.c->claim_pull[par], (unsigned long long)kThreads);
        __syncthreads();
        const long long t0 = *s_claim;
        __syncthreads();
        if (t0 >= total_rows) break;
        const long long i = t0 + threadIdx.x;
        // unit of this tile: tiles never straddle units (prefixes are padded to kThreads)
        int u = 0;
        {
            int lo = 0, hi = p.n_units - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (sh.upref[mid] <= t0) lo = mid; else hi = mid - 1;
            }
            u = lo;
        }
        const QUnit U = p.units[u];
        const DevAdj A = p.adj[U.in_dir];
        const long long r = i - sh.upref[u];
        const bool in_range = r < U.in_rows;
        int32_t w = 0;
        int32_t rb = 0, re = 0;
        bool cand = false;
        if (in_range) {
            if (A.fmt == ADJ_DENSE) {
                w = (int32_t)r;
                rb = __ldg(A.off + w);
                re = __ldg(A.off + w + 1);
            } else {
                w = __ldg(A.rows + r);
                rb = __ldg(A.off + r);
                re = __ldg(A.off + r + 1);
            }
            const size_t idx = (size_t)U.q2 * p.W + ((uint32_t)w >> 6);
            const uint64_t bit = 1ull << (w & 63);
            cand = (re > rb) && !(__ldcg(p.P + idx) & bit) && !(__ldcg(p.NX + idx) & bit);
        }
        // serial scan of up to kWarpRow in-neighbours
        bool found = false;
        bool pending = false;
        if (cand) {
            const int32_t lim = min(re, rb + kWarpRow);
            for (int32_t k = rb; k < lim && !found; k++) {
                const int32_t x = __ldg(A.nbr + k);
                uint64_t sm = U.smask;
                while (sm) {
                    const int q = __ffsll((long long)sm) - 1;
                    sm &= sm - 1;
                    if ((__ldcg(F + (size_t)q * p.W + ((uint32_t)x >> 6)) >> (x & 63)) & 1ull) {
                        found = true;
                        break;
                    }
                }
            }
            pending = !found && re - rb > kWarpRow;
        }
        // long rows: the whole warp scans, ballot for a hit, early exit
        {
            unsigned m;
            while ((m = __ballot_sync(kFull, pending)) != 0) {
                const int leader = __ffs(m) - 1;
                const int32_t b = __shfl_sync(kFull, rb, leader) + kWarpRow;
                const int32_t e = __shfl_sync(kFull, re, leader);
                bool hit = false;
                for (int32_t base = b; base < e; base += 32) {
                    const int32_t k = base + (int32_t)lane;
                    bool h = false;
                    if (k < e) {
                        const int32_t x = __ldg(A.nbr + k);
                        uint64_t sm = U.smask;
                        while (sm) {
                            const int q = __ffsll((long long)sm) - 1;
                            sm &= sm - 1;
                            if ((__ldcg(F + (size_t)q * p.W + ((uint32_t)x >> 6)) >> (x & 63)) &
                                1ull) {
                                h = true;
                                break;
                            }
                        }
                    }
                    if (__ballot_sync(kFull, h)) {
                        hit = true;
                        break;
                    }
                }
                if ((int)lane == leader) {
                    pending = false;
                    found = hit;
                }
            }
        }
        // set the found bits
        {
            bool need = false;
            uint32_t code = 0;
            if (found) {
                const uint32_t wi = (uint32_t)w >> 6;
                const size_t idx = (size_t)U.q2 * p.W + wi;
                const unsigned long long old =
                    atomicOr((unsigned long long *)(p.NX + idx), 1ull << (w & 63));
                need = old == 0ull;
                code = (uint32_t)U.q2 * (uint32_t)p.W + wi;
            }
            warp_append(need, code, tl, tcount);
        }
    }
}

// Decide for level j (all CTAs compute the same from the same counters).
// Returns false when the traversal is over.
__device__ bool decide_phase(const KParams &p, int j, const Shared &sh) {
    const int par = j & 1;
    volatile Counters *c = p.c;
    long long total = 0;
    for (int q = 0; q < p.S; q++) total += (long long)c->fl_count[par][q];
    const bool expand = total > 0 && (p.max_levels == 0 || j < p.max_levels);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        p.c->visited += total;
        if (total > 0 && j > 0) p.c->levels = j;
        if (expand) {
            p.c->expanded += total;
            p.c->push_bytes += (long long)c->lvl_bytes[par];
            p.c->product_edges += (long long)c->lvl_edges[par];
        }
    }
    if (!expand) return false;
    // direction per unit
    for (int u = threadIdx.x; u < p.n_units; u += kThreads) {
        const QUnit U = p.units[u];
        unsigned long long mass = 0, pairs = 0;
        for (int k = 0; k < U.g_count; k++) {
            const int g = p.u_group[U.g_first + k];
            mass += __ldcg(p.mf + par * kMaxGroups + g);
            pairs += c->fl_count[par][sh.gq[g]];
        }
        const bool pull = (double)mass * (double)p.alpha > (double)U.in_nnz + (double)U.in_rows &&
                          (long long)pairs >= p.min_pull;
        sh.upull[u] = pull ? 1 : 0;
    }
    __syncthreads();
    for (int g = threadIdx.x; g < p.n_groups; g += kThreads) {
        const QGroup G = p.groups[g];
        uint64_t tm = 0;
        for (int k = 0; k < G.t_count; k++) {
            const int u = p.t_unit[G.t_first + k];
            if (!sh.upull[u]) tm |= 1ull << p.t_state[G.t_first + k];
        }
        sh.tpush[g] = tm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int g = 0; g < p.n_groups; g++) {
            sh.gpref[g] = acc;
            if (sh.tpush[g]) acc += (long long)c->fl_count[par][sh.gq[g]];
        }
        sh.gpref[p.n_groups] = acc;
        long long ra = 0, npush = 0, npull = 0;
        for (int u = 0; u < p.n_units; u++) {
            sh.upref[u] = ra;
            if (sh.upull[u]) {
                ra += (p.units[u].in_rows + kThreads - 1) / kThreads * kThreads;
                npull++;
            } else {
                npush++;
            }
        }
        sh.upref[p.n_units] = ra;
        if (blockIdx.x == 0) {
            p.c->push_units += npush;
            p.c->pull_units += npull;
        }
    }
    __syncthreads();
    return true;
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
    // block sum
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(kFull, cnt, o);
    if (threadIdx.x == 0) *s_tmp = 0;
    __syncthreads();
    if (lane_id() == 0) atomicAdd((unsigned long long *)s_tmp, (unsigned long long)cnt);
    __syncthreads();
    if (threadIdx.x == 0) p.fin_sums[blockIdx.x] = *s_tmp;
}

__device__ void final_write(const KParams &p, long long *s_tmp) {
    const int64_t W = p.W;
    const int64_t per = (W + gridDim.x - 1) / gridDim.x;
    const int64_t w0 = (int64_t)min((long long)W, (long long)blockIdx.x * per);
    const int64_t w1 = (int64_t)min((long long)W, (long long)(w0 + per));
    __shared__ long long wsum[kWarps + 1];
    if (threadIdx.x == 0) {
        long long pre = 0, tot = 0;
        for (unsigned b = 0; b < gridDim.x; b++) {
            const long long s = *(volatile long long *)&p.fin_sums[b];
            if (b < blockIdx.x) pre += s;
            tot += s;
        }
        *s_tmp = pre;
        if (blockIdx.x == 0) p.c->answer_count = tot;
    }
    __syncthreads();
    long long run = *s_tmp;
    __syncthreads();
    if (!p.out_list) return;
    const unsigned lane = lane_id();
    for (int64_t base = w0; base < w1; base += kThreads) {
        const int64_t wi = base + threadIdx.x;
        uint64_t r = 0;
        if (wi < w1) {
            uint64_t fm = p.final_mask;
            while (fm) {
                const int q = __ffsll((long long)fm) - 1;
                fm &= fm - 1;
                r |= __ldcg(p.P + (size_t)q * W + wi);
            }
        }
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

__global__ void __launch_bounds__(kThreads) rpq_query_kernel(KParams p) {
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ unsigned long long s_cnt[kMaxStates], s_base[kMaxStates], s_acc[2];
    __shared__ unsigned long long s_mf[kMaxGroups];
    __shared__ long long s_claim;
    Shared sh = carve(p, smem);
    for (int g = threadIdx.x; g < p.n_groups; g += kThreads) {
        const QGroup G = p.groups[g];
        sh.gq[g] = G.q;
        sh.gd[g] = G.d;
        sh.gnbr[g] = p.adj[G.d].nbr;
        sh.tpush[g] = 0;
    }
    // prologue: clear P and the frontier bitsets; block 0 seeds level 0
    const size_t words = (size_t)p.S * p.W;
    for (size_t i = (size_t)blockIdx.x * kThreads + threadIdx.x; i < words;
         i += (size_t)gridDim.x * kThreads) {
        p.P[i] = 0;
        p.F0[i] = 0;
        p.F1[i] = 0;
    }
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < 2 * kMaxGroups; i += kThreads) p.mf[i] = 0;
        if (threadIdx.x == 0) {
            Counters *c = p.c;
            for (int k = 0; k < 3; k++) c->touched[k] = 0;
            for (int k = 0; k < 2; k++) {
                for (int q = 0; q < kMaxStates; q++) c->fl_count[k][q] = 0;
                c->lvl_bytes[k] = c->lvl_edges[k] = c->hub_packed[k] = 0;
                c->claim_hub[k] = c->claim_item[k] = c->claim_pull[k] = 0;
            }
            c->levels = c->visited = c->expanded = c->product_edges = c->push_bytes = 0;
            c->push_units = c->pull_units = c->answer_count = 0;
            // level 0 = Q_S x {v_s}: seed NX and the touched list TL_0
            const uint32_t wi = (uint32_t)p.source >> 6;
            const uint64_t bit = 1ull << (p.source & 63);
            unsigned long long n0 = 0;
            uint64_t sm = p.start_mask;
            while (sm) {
                const int q = __ffsll((long long)sm) - 1;
                sm &= sm - 1;
                p.NX[(size_t)q * p.W + wi] = bit;
                p.T0[n0++] = (uint32_t)q * (uint32_t)p.W + wi;
            }
            c->touched[0] = n0;
        }
    }
    if (!grid_barrier(p.c)) return;
    for (int j = 0;; j++) {
        commit_phase(p, j, sh, s_cnt, s_base, s_mf, s_acc);
        if (!grid_barrier(p.c)) return;
        if (!decide_phase(p, j, sh)) break;
        expand_phase(p, j, sh, &s_claim);
        if (!grid_barrier(p.c)) return;
    }
    final_phase(p, &s_claim);
    if (!grid_barrier(p.c)) return;
    final_write(p, &s_claim);
}

// ------------------------------------------------------------ host side --

struct QueryWorkspace : WorkspaceBase {
    int S_cap = 0;
    int64_t hub_cap = 0;
    int32_t n = 0, W = 0;
    DevBuf P, NX, F0, F1, T0, T1, T2, FL0, FL1, H0, H1, mf, fin, ctr, tables, out_list;
    void *staging = nullptr;  // pinned host: tables upload + counters download
    size_t staging_bytes = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    ~QueryWorkspace() override {
        if (staging) cudaFreeHost(staging);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
    }
};

constexpr size_t kTablesBytes = 256 * 1024;

// Grid of the persistent kernel: every SM holds the same number of CTAs
// (cooperative launch requires all of them resident).  Computed once per
// device for the largest automaton tables, so any query fits.
int g_grid[64];
std::mutex g_grid_mu;

rpq_status get_launch_shape(int device, int *grid) {
    if (device < 0 || device >= 64) return fail(RPQ_ERR_CUDA, "device id %d", device);
    std::lock_guard<std::mutex> lk(g_grid_mu);
    if (g_grid[device] > 0) {
        *grid = g_grid[device];
        return RPQ_OK;
    }
    int coop = 0, sms = 0;
    RPQ_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
    RPQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    if (!coop) return fail(RPQ_ERR_CUDA, "device lacks cooperative launch");
    const size_t smem = shared_bytes(kMaxGroups, kMaxUnits);
    RPQ_CUDA_TRY(cudaFuncSetAttribute(rpq_query_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    int per_sm = 0;
    RPQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rpq_query_kernel, kThreads,
                                                               smem));
    if (per_sm <= 0) return fail(RPQ_ERR_CUDA, "query kernel does not fit on an SM");
    const char *cap = getenv("RPQ_CTAS_PER_SM");
    per_sm = std::min(per_sm, cap ? std::max(1, atoi(cap)) : 4);
    g_grid[device] = sms * per_sm;
    *grid = g_grid[device];
    return RPQ_OK;
}

rpq_status ws_alloc(QueryWorkspace *ws, const rpq_graph *g, int S_cap, int64_t hub_cap) {
    const int64_t W = ((int64_t)g->n + 63) / 64;
    const size_t bits = sizeof(uint64_t) * (size_t)S_cap * W;
    const size_t tl = sizeof(uint32_t) * (size_t)S_cap * W;
    const size_t fl = sizeof(int32_t) * (size_t)S_cap * g->n;
    ws->S_cap = S_cap;
    ws->hub_cap = hub_cap;
    ws->n = g->n;
    ws->W = (int32_t)W;
    if (!ws->P.alloc(bits) || !ws->NX.alloc(bits) || !ws->F0.alloc(bits) || !ws->F1.alloc(bits) ||
        !ws->T0.alloc(tl) || !ws->T1.alloc(tl) || !ws->T2.alloc(tl) || !ws->FL0.alloc(fl) ||
        !ws->FL1.alloc(fl) || !ws->H0.alloc(sizeof(Hub) * hub_cap) ||
        !ws->H1.alloc(sizeof(Hub) * hub_cap) ||
        !ws->mf.alloc(sizeof(unsigned long long) * 2 * kMaxGroups) ||
        !ws->fin.alloc(sizeof(long long) * 152 * 64) || !ws->ctr.alloc(sizeof(Counters)) ||
        !ws->tables.alloc(kTablesBytes) || !ws->out_list.alloc(sizeof(int32_t) * (size_t)g->n))
        return fail(RPQ_ERR_OOM, "query workspace (%d states)", S_cap);
    RPQ_CUDA_TRY(cudaMemset(ws->NX.p, 0, bits));
    RPQ_CUDA_TRY(cudaMemset(ws->ctr.p, 0, sizeof(Counters)));
    ws->staging_bytes = kTablesBytes + sizeof(Counters) + 64;
    RPQ_CUDA_TRY(cudaMallocHost(&ws->staging, ws->staging_bytes));
    RPQ_CUDA_TRY(cudaEventCreate(&ws->ev0));
    RPQ_CUDA_TRY(cudaEventCreate(&ws->ev1));
    return RPQ_OK;
}

std::unique_ptr<QueryWorkspace> ws_acquire(rpq_graph *g, int S, int64_t hub_need, rpq_status *st) {
    {
        std::lock_guard<std::mutex> lk(g->ws_mu);
        for (size_t i = 0; i < g->ws_free.size(); i++) {
            auto *w = dynamic_cast<QueryWorkspace *>(g->ws_free[i].get());
            if (w && w->S_cap >= S && w->hub_cap >= hub_need) {
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
    int64_t hc = 1024;
    while (hc < hub_need) hc *= 2;
    *st = ws_alloc(w.get(), g, S_cap, hc);
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
    int64_t hub_need = 0;
};

rpq_status build_tables(const rpq_graph *g, const Automaton &a, Tables *t) {
    // group (q, d) -> targets; unit (d, q') -> sources
    std::map<std::pair<int, int>, uint64_t> gmap, umap;
    for (size_t i = 0; i < a.from.size(); i++) {
        const int s = a.sym[i];
        const int lab = s < a.L ? s : s - a.L;
        const bool inv = s >= a.L;
        if (lab >= g->L)
            return fail(RPQ_ERR_INVALID, "automaton label %d is not a label of the graph (L=%d)",
                        lab, g->L);
        const int d = inv ? g->L + lab : lab;
        gmap[{a.from[i], d}] |= 1ull << a.to[i];
        umap[{d, a.to[i]}] |= 1ull << a.from[i];
    }
    if ((int)gmap.size() > kMaxGroups || (int)umap.size() > kMaxUnits)
        return fail(RPQ_ERR_INVALID, "automaton has too many (state, label) pairs");
    std::map<std::pair<int, int>, int> uidx;
    for (auto &kv : umap) {
        QUnit u{};
        u.d = kv.first.first;
        u.q2 = kv.first.second;
        u.smask = kv.second;
        u.in_dir = g->inverse_dir(u.d);
        const DevAdj &A = g->adj[u.in_dir];
        u.in_rows = A.fmt == ADJ_EMPTY ? 0 : A.nrows;
        u.in_nnz = A.nnz;
        uidx[kv.first] = (int)t->units.size();
        t->units.push_back(u);
    }
    for (auto &kv : gmap) {
        QGroup G{};
        G.q = kv.first.first;
        G.d = kv.first.second;
        G.tmask = kv.second;
        G.t_first = (int32_t)t->t_unit.size();
        uint64_t m = G.tmask;
        while (m) {
            const int q2 = __builtin_ctzll(m);
            m &= m - 1;
            t->t_unit.push_back(uidx[{G.d, q2}]);
            t->t_state.push_back(q2);
        }
        G.t_count = (int32_t)t->t_unit.size() - G.t_first;
        t->groups.push_back(G);
        const DevAdj &A = g->adj[G.d];
        t->hub_need += A.nnz / kHubDeg + 1;
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

float env_float(const char *name, float dflt) {
    const char *v = getenv(name);
    return v ? (float)atof(v) : dflt;
}

}  // namespace

// Runs one query.  The answer goes to out_list_dev (device, `capacity`
// entries) or, when that is null, to out_host_list (host, copied when it
// fits in `capacity`); out_bits_dev receives the answer bitset if non-null.
rpq_status run_query(rpq_graph *g, const Automaton &a, int32_t source, int32_t max_levels,
                     int32_t *out_list_dev, int64_t capacity, uint64_t *out_bits_dev,
                     int32_t *out_host_list, rpq_stats *stats, int64_t *count, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (source < 0 || source >= g->n)
        return fail(RPQ_ERR_INVALID, "source %d outside [0, %d)", source, g->n);
    if (max_levels < 0) return fail(RPQ_ERR_INVALID, "max_levels must be >= 0");
    if (a.S <= 0 || a.S > kMaxStates) return fail(RPQ_ERR_INVALID, "automaton has %d states", a.S);
    Tables t;
    rpq_status s = build_tables(g, a, &t);
    if (s != RPQ_OK) return s;
    const size_t tbytes = sizeof(QGroup) * t.groups.size() + sizeof(QUnit) * t.units.size() +
                          sizeof(int32_t) * (t.t_unit.size() * 2 + t.u_group.size()) + 64;
    if (tbytes > kTablesBytes) return fail(RPQ_ERR_INVALID, "automaton tables too large");
    std::unique_ptr<QueryWorkspace> ws = ws_acquire(g, a.S, t.hub_need, &s);
    if (!ws) return s;
    // upload tables
    uint8_t *hs = static_cast<uint8_t *>(ws->staging);
    size_t off = 0;
    auto put = [&](const void *src, size_t bytes) {
        off = (off + 15) & ~size_t(15);
        size_t at = off;
        if (bytes) memcpy(hs + at, src, bytes);
        off += bytes;
        return at;
    };
    const size_t o_groups = put(t.groups.data(), sizeof(QGroup) * t.groups.size());
    const size_t o_units = put(t.units.data(), sizeof(QUnit) * t.units.size());
    const size_t o_tu = put(t.t_unit.data(), sizeof(int32_t) * t.t_unit.size());
    const size_t o_ts = put(t.t_state.data(), sizeof(int32_t) * t.t_state.size());
    const size_t o_ug = put(t.u_group.data(), sizeof(int32_t) * t.u_group.size());
    off = (off + 15) & ~size_t(15);
    RPQ_CUDA_TRY(cudaMemcpyAsync(ws->tables.p, hs, std::max<size_t>(off, 16), cudaMemcpyHostToDevice, st));
    uint8_t *dt = ws->tables.as<uint8_t>();

    KParams p{};
    p.adj = g->d_adj.as<DevAdj>();
    p.n = g->n;
    p.W = ws->W;
    p.S = a.S;
    p.n_groups = (int32_t)t.groups.size();
    p.n_units = (int32_t)t.units.size();
    p.n_targets = (int32_t)t.t_unit.size();
    p.source = source;
    p.max_levels = max_levels;
    p.start_mask = a.start_mask;
    p.final_mask = a.final_mask;
    p.alpha = env_float("RPQ_PULL_ALPHA", 4.0f);
    p.min_pull = (int32_t)env_float("RPQ_PULL_MIN", 256.0f);
    p.groups = reinterpret_cast<const QGroup *>(dt + o_groups);
    p.units = reinterpret_cast<const QUnit *>(dt + o_units);
    p.t_unit = reinterpret_cast<const int32_t *>(dt + o_tu);
    p.t_state = reinterpret_cast<const int32_t *>(dt + o_ts);
    p.u_group = reinterpret_cast<const int32_t *>(dt + o_ug);
    p.P = ws->P.as<uint64_t>();
    p.NX = ws->NX.as<uint64_t>();
    p.F0 = ws->F0.as<uint64_t>();
    p.F1 = ws->F1.as<uint64_t>();
    p.T0 = ws->T0.as<uint32_t>();
    p.T1 = ws->T1.as<uint32_t>();
    p.T2 = ws->T2.as<uint32_t>();
    p.FL0 = ws->FL0.as<int32_t>();
    p.FL1 = ws->FL1.as<int32_t>();
    p.H0 = ws->H0.as<Hub>();
    p.H1 = ws->H1.as<Hub>();
    p.hub_cap = ws->hub_cap;
    p.mf = ws->mf.as<unsigned long long>();
    p.fin_sums = ws->fin.as<long long>();
    p.c = ws->ctr.as<Counters>();
    p.out_bits = out_bits_dev;
    if (out_list_dev) {
        p.out_list = out_list_dev;
        p.capacity = capacity;
    } else if (out_host_list) {
        p.out_list = ws->out_list.as<int32_t>();
        p.capacity = g->n;
    } else {
        p.out_list = nullptr;
        p.capacity = 0;
    }
    const size_t smem = shared_bytes(kMaxGroups, kMaxUnits);
    int grid = 0;
    s = get_launch_shape(g->device, &grid);
    if (s != RPQ_OK) {
        ws_release(g, std::move(ws));
        return s;
    }
    if (grid > 152 * 64) grid = 152 * 64;
    RPQ_CUDA_TRY(cudaMemsetAsync(&p.c->status, 0, sizeof(int32_t), st));
    const bool timed = stats != nullptr;
    if (timed) RPQ_CUDA_TRY(cudaEventRecord(ws->ev0, st));
    void *args[] = {&p};
    RPQ_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)rpq_query_kernel, dim3(grid),
                                             dim3(kThreads), args, smem, st));
    if (timed) RPQ_CUDA_TRY(cudaEventRecord(ws->ev1, st));
    Counters *hc = reinterpret_cast<Counters *>(hs + kTablesBytes);
    RPQ_CUDA_TRY(cudaMemcpyAsync(hc, ws->ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (hc->status != 0) {
        // a failed traversal may leave NX dirty: restore the all-zero invariant
        cudaMemsetAsync(ws->NX.p, 0, ws->NX.bytes, st);
        cudaMemsetAsync(ws->ctr.p, 0, sizeof(Counters), st);
        cudaStreamSynchronize(st);
        const rpq_status e = (rpq_status)hc->status;
        ws_release(g, std::move(ws));
        return fail(e, "device traversal failed (status %d)", (int)e);
    }
    *count = hc->answer_count;
    const bool copy_list = out_host_list && !out_list_dev && *count <= capacity && *count > 0;
    if (stats) {
        stats->h2d_bytes = (int64_t)std::max<size_t>(off, 16);
        stats->d2h_bytes = (int64_t)sizeof(Counters) + (copy_list ? 4 * *count : 0);
        stats->levels = hc->levels;
        stats->visited_pairs = hc->visited;
        stats->expanded_pairs = hc->expanded;
        stats->product_edges = hc->product_edges;
        stats->push_bytes = hc->push_bytes;
        stats->answer_count = hc->answer_count;
        stats->push_unit_levels = hc->push_units;
        stats->pull_unit_levels = hc->pull_units;
        float ms = -1.0f;
        if (cudaEventElapsedTime(&ms, ws->ev0, ws->ev1) != cudaSuccess) ms = -1.0f;
        stats->device_ms = ms;
    }
    if (copy_list) {
        RPQ_CUDA_TRY(cudaMemcpyAsync(out_host_list, ws->out_list.p, sizeof(int32_t) * (*count),
                                     cudaMemcpyDeviceToHost, st));
        RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    }
    ws_release(g, std::move(ws));
    return RPQ_OK;
}

}  // namespace rpq
