// Lane-batched Algorithm 1 (section 4 of the paper; multi-source BFS is the
// extension its conclusion proposes): up to 256 single-source queries with
// different automata advance together.  Query i owns bit i of a 4-word lane
// vector; automaton state q of every query lives in "slot" q.  For every
// (vertex v, slot k) the frontier M, the visited set P and the next level NX
// hold one lane vector (layout [v][k][lane word]), so one pass over the rows
// of G^d serves every query whose automaton reads d.
//
// Per level:
//   expand  for every vertex v with a non-empty frontier vector and every
//           direction d:  X_{d,k2}[v] = OR_k M[v][k] & T[d][k][k2]  (the
//           aggregate-first order (N^a)^T x M, section 4), then for every
//           w in row v of G^d:  NX[w][k2] |= X & ~P[w][k2]  (atomicOr).
//           Rows longer than p.lane_hub edges are finished in chunks by
//           other warps.  When the frontier holds more than n / p.pull_div
//           vertices the level pulls instead: for every vertex w and unit
//           (d, k2), the lanes still missing (k2, w) OR the frontier lanes of
//           w's in-neighbours in direction d until none is missing.
//   commit  M_{j+1}[w] = NX[w], P[w] |= NX[w], NX[w] = 0 for every touched w;
//           the touched list becomes the next frontier list.
// The answer of lane i is {v : P[v][k] has bit i for a final slot k of i}.
#include <algorithm>
#include <array>
#include <atomic>
#include <string>
#include <thread>
#include <cstring>
#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <vector>

#include "lanes.h"

namespace rpq {

LaneWorkspace::~LaneWorkspace() {
    if (staging) cudaFreeHost(staging);
}

namespace {

constexpr int kLThreads = 256;
constexpr int kLWarps = kLThreads / 32;
constexpr int kLaneChunk = 128;   // edges per chunk of a longer row (one warp, 4 rounds)
constexpr uint64_t kLaneBarrierNs = 4000000000ull;

__device__ __forceinline__ int32_t *lane_list(const LParams &p, int idx) {
    return idx == 0 ? p.list0 : (idx == 1 ? p.list1 : p.list2);
}

__device__ bool lane_barrier(LaneCounters *c) {
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
                    if (*(volatile int32_t *)&c->status != 0) break;
                    if (global_timer_ns() - t0 > kLaneBarrierNs) {
                        atomicCAS(&c->status, 0, (int32_t)RPQ_ERR_TIMEOUT);
                        break;
                    }
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *(volatile int32_t *)&c->status == 0;
}

__device__ __forceinline__ void warp_append_i32(bool need, int32_t v, int32_t *list,
                                                unsigned long long *count) {
    const unsigned m = __ballot_sync(kFull, need);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(count, (unsigned long long)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (need) list[base + __popc(m & lanemask_lt())] = v;
}

// X_{d,k2}[v] for every unit of direction dir from the frontier row sm_M;
// returns whether any lane is set.  Whole warp.
__device__ bool lane_aggregate(const LParams &p, const LDir &dir, const uint64_t *sm_M,
                               uint64_t *sm_X) {
    bool any = false;
    for (int idx = lane_id(); idx < dir.unit_count * kLW; idx += 32) {
        const LUnit U = p.units[dir.unit_first + idx / kLW];
        const int lw = idx % kLW;
        uint64_t x = 0;
        for (int s = 0; s < U.src_count; s++) {
            const LSrc &S = p.srcs[U.src_first + s];
            x |= sm_M[S.k * kLW + lw] & S.mask[lw];
        }
        x &= p.dyn->active[lw];
        sm_X[idx] = x;
        any = any || x != 0;
    }
    __syncwarp();
    return __any_sync(kFull, any);
}

// Pushes the frontier lanes sm_X along edges [b, e) of direction dir.  Whole warp.
// Per edge and target slot, the 4 visited words (one 32-byte sector) are
// loaded as two 16-byte vectors; only lane words with new bits are OR-ed.
__device__ void lane_push(const LParams &p, const LDir &dir, const uint64_t *sm_X, int32_t b,
                          int32_t e, int32_t *TV, unsigned long long *tvc) {
    const int32_t *nbr = p.adj[dir.d].nbr;
    const unsigned lane = lane_id();
    for (int32_t base = b; base < e; base += 32) {
        const int32_t k = base + (int32_t)lane;
        const bool valid = k < e;
        const int32_t w = valid ? __ldg(nbr + k) : 0;
        bool first = false;
        for (int uu = 0; uu < dir.unit_count; uu++) {
            const uint64_t x0 = sm_X[uu * kLW + 0], x1 = sm_X[uu * kLW + 1];
            const uint64_t x2 = sm_X[uu * kLW + 2], x3 = sm_X[uu * kLW + 3];
            if (!(x0 | x1 | x2 | x3) || !valid) continue;
            const int k2 = p.units[dir.unit_first + uu].k2;
            const size_t row = ((size_t)w * p.K + k2) * kLW;
            const ulonglong2 pa = __ldcg(reinterpret_cast<const ulonglong2 *>(p.P + row));
            const ulonglong2 pb = __ldcg(reinterpret_cast<const ulonglong2 *>(p.P + row) + 1);
            const uint64_t y[kLW] = {x0 & ~pa.x, x1 & ~pa.y, x2 & ~pb.x, x3 & ~pb.y};
#pragma unroll
            for (int lw = 0; lw < kLW; lw++) {
                if (!y[lw]) continue;
                const unsigned long long old =
                    atomicOr((unsigned long long *)(p.NX + row + lw), (unsigned long long)y[lw]);
                if (old == 0ull) first = true;
            }
        }
        bool app = false;
        if (first) {
            const unsigned long long bit = 1ull << (w & 63);
            const unsigned long long old = atomicOr((unsigned long long *)(p.tv + (w >> 6)), bit);
            app = !(old & bit);
        }
        warp_append_i32(app, w, TV, tvc);
    }
}

__device__ void lane_load_row(const LParams &p, const uint64_t *M, int32_t v, uint64_t *sm_M) {
    const size_t base = (size_t)v * p.K * kLW;
    for (int idx = lane_id(); idx < p.K * kLW; idx += 32) sm_M[idx] = __ldcg(M + base + idx);
    __syncwarp();
}

// ------------------------------------------------------------ phases -----
__device__ void lane_expand_vertices(const LParams &p, int j, uint64_t *sm_M, uint64_t *sm_X) {
    const int cur = j % 3, nxt = (j + 1) % 3;
    const int32_t *A = lane_list(p, cur);
    const unsigned long long nA = *(volatile unsigned long long *)&p.c->list_count[cur];
    const uint64_t *M = (j & 1) ? p.M1 : p.M0;
    int32_t *TV = lane_list(p, nxt);
    unsigned long long *tvc = &p.c->list_count[nxt];
    const unsigned lane = lane_id();
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long i = (unsigned long long)gw; i < nA; i += (unsigned long long)nw) {
        const int32_t v = __ldcg(A + i);
        lane_load_row(p, M, v, sm_M);
        const int n_dirs = p.dyn->n_dirs;
        for (int D = 0; D < n_dirs; D++) {
            const LDir dir = p.dirs[D];
            if (!lane_aggregate(p, dir, sm_M, sm_X)) continue;
            int32_t b, e;
            adj_row(p.adj[dir.d], v, b, e);
            const int32_t e1 = min(e, b + p.lane_hub);
            if (e > e1 && lane == 0) {
                const unsigned long long nch =
                    (unsigned long long)((e - e1 + kLaneChunk - 1) / kLaneChunk);
                const unsigned long long old = atomicAdd(&p.c->hub_packed, (1ull << 40) | nch);
                const long long hi = (long long)(old >> 40);
                const long long cb = (long long)(old & ((1ull << 40) - 1));
                if (hi < p.hub_cap && cb + (long long)nch <= p.chunk_cap) {
                    LHub h;
                    h.v = v; h.dir = D; h.b = e1; h.e = e;
                    h.chunk_base = cb;
                    p.hubs[hi] = h;
                    for (unsigned long long k = 0; k < nch; k++) p.hub_cmap[cb + k] = (int32_t)hi;
                } else {
                    atomicCAS(&p.c->status, 0, (int32_t)RPQ_ERR_OOM);
                }
            }
            if (lane == 0) atomicAdd(&p.c->edges, (unsigned long long)(e - b));
            lane_push(p, dir, sm_X, b, e1, TV, tvc);
            __syncwarp();
        }
    }
}

__device__ void lane_expand_hubs(const LParams &p, int j, uint64_t *sm_M, uint64_t *sm_X) {
    const int nxt = (j + 1) % 3;
    const uint64_t *M = (j & 1) ? p.M1 : p.M0;
    int32_t *TV = lane_list(p, nxt);
    unsigned long long *tvc = &p.c->list_count[nxt];
    const unsigned long long packed = *(volatile unsigned long long *)&p.c->hub_packed;
    const long long nh = (long long)(packed >> 40);
    const long long nch = (long long)(packed & ((1ull << 40) - 1));
    const unsigned lane = lane_id();
    (void)nh;
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long c = gw; c < nch; c += nw) {
        const int hi = __ldcg(p.hub_cmap + c);
        const int32_t v = __ldcg(&p.hubs[hi].v);
        const int D = __ldcg(&p.hubs[hi].dir);
        const int32_t hb = __ldcg(&p.hubs[hi].b), he = __ldcg(&p.hubs[hi].e);
        const long long base = __ldcg(&p.hubs[hi].chunk_base);
        const int32_t b = hb + (int32_t)((c - base) * kLaneChunk);
        const int32_t e = min(he, b + kLaneChunk);
        lane_load_row(p, M, v, sm_M);
        const LDir dir = p.dirs[D];
        if (lane_aggregate(p, dir, sm_M, sm_X)) lane_push(p, dir, sm_X, b, e, TV, tvc);
        __syncwarp();
    }
    (void)lane;
}

// Pull level j (a warp per vertex w, grid-stride over all vertices): for each
// unit (d, k2), need = lanes that reached new pairs at level j, whose
// automaton can enter k2 by d, and that have not visited (k2, w); the warp
// ORs X_{d,k2}[u] = OR_s M[u][k_s] & mask_s over the in-neighbours u of w
// (rows of the inverse direction), 32 at a time, and stops when the OR
// covers need.  New lanes go to NX[w][k2]; w joins the touched list once.
__device__ void lane_pull(const LParams &p, int j) {
    const int cur = j % 3, nxt = (j + 1) % 3;
    const uint64_t *M = (j & 1) ? p.M1 : p.M0;
    int32_t *TV = lane_list(p, nxt);
    unsigned long long *tvc = &p.c->list_count[nxt];
    const unsigned lane = lane_id();
    uint64_t live[kLW];
#pragma unroll
    for (int lw = 0; lw < kLW; lw++)
        live[lw] = *(volatile unsigned long long *)&p.c->lane_new[cur][lw] & p.dyn->active[lw];
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const int n_dirs = p.dyn->n_dirs;
    for (long long w = gw; w < p.n; w += nw) {
        bool first = false;
        for (int D = 0; D < n_dirs; D++) {
            const LDir dir = p.dirs[D];
            const int dinv = dir.d < p.adj_half ? dir.d + p.adj_half : dir.d - p.adj_half;
            int32_t b, e;
            adj_row(p.adj[dinv], (int32_t)w, b, e);
            if (b >= e) continue;  // warp-uniform
            for (int uu = 0; uu < dir.unit_count; uu++) {
                const LUnit U = p.units[dir.unit_first + uu];
                const size_t row = ((size_t)w * p.K + U.k2) * kLW;
                uint64_t need[kLW];
                bool any = false;
#pragma unroll
                for (int lw = 0; lw < kLW; lw++) {
                    uint64_t reach = 0;
                    for (int sI = 0; sI < U.src_count; sI++) reach |= p.srcs[U.src_first + sI].mask[lw];
                    need[lw] = live[lw] & reach & ~__ldcg(p.P + row + lw);
                    any = any || need[lw];
                }
                if (!any) continue;  // warp-uniform (every lane computed the same)
                uint64_t acc[kLW] = {0, 0, 0, 0};
                int32_t scanned = 0;
                for (int32_t base = b; base < e; base += 32) {
                    scanned = min(e, base + 32) - b;
                    const int32_t k = base + (int32_t)lane;
                    uint64_t x[kLW] = {0, 0, 0, 0};
                    if (k < e) {
                        const int32_t u = __ldg(p.adj[dinv].nbr + k);
                        for (int sI = 0; sI < U.src_count; sI++) {
                            const LSrc &S = p.srcs[U.src_first + sI];
                            const size_t mr = ((size_t)u * p.K + S.k) * kLW;
#pragma unroll
                            for (int lw = 0; lw < kLW; lw++) x[lw] |= __ldcg(M + mr + lw) & S.mask[lw];
                        }
                    }
                    bool done = true;
#pragma unroll
                    for (int lw = 0; lw < kLW; lw++) {
                        const uint32_t lo = __reduce_or_sync(kFull, (uint32_t)(x[lw] & need[lw]));
                        const uint32_t hi = __reduce_or_sync(kFull, (uint32_t)((x[lw] & need[lw]) >> 32));
                        acc[lw] |= ((uint64_t)hi << 32) | lo;
                        done = done && (acc[lw] == need[lw]);
                    }
                    if (done) break;  // warp-uniform
                }
                if (lane == 0) atomicAdd(&p.c->edges, (unsigned long long)scanned);
                if ((int)lane < kLW && acc[lane]) {
                    const unsigned long long old =
                        atomicOr((unsigned long long *)(p.NX + row + lane), (unsigned long long)acc[lane]);
                    if (old == 0ull) first = true;
                }
            }
        }
        // w joins the touched list once (its touched bit decides)
        bool app = false;
        const bool fw = __any_sync(kFull, first);
        if (fw && lane == 0) {
            const unsigned long long bit = 1ull << (w & 63);
            const unsigned long long old = atomicOr((unsigned long long *)(p.tv + (w >> 6)), bit);
            app = !(old & bit);
        }
        warp_append_i32(app, (int32_t)w, TV, tvc);
    }
}

// Commit of level j -> j+1 (grid-stride, a warp per list entry).
__device__ void lane_commit(const LParams &p, int j) {
    const int cur = j % 3, nxt = (j + 1) % 3;
    const int32_t *A = lane_list(p, cur);
    const int32_t *TV = lane_list(p, nxt);
    const unsigned long long nA = *(volatile unsigned long long *)&p.c->list_count[cur];
    const unsigned long long nT = *(volatile unsigned long long *)&p.c->list_count[nxt];
    uint64_t *Mc = (j & 1) ? p.M1 : p.M0;
    uint64_t *Mn = (j & 1) ? p.M0 : p.M1;
    const int words = p.K * kLW;
    const unsigned lane = lane_id();
    const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    // (a) level j's frontier rows are done: clear them
    for (long long i = gwarp; i < (long long)nA; i += nwarps) {
        const size_t base = (size_t)__ldcg(A + i) * words;
        for (int idx = lane; idx < words; idx += 32) Mc[base + idx] = 0;
    }
    // (b) move NX -> M_{j+1}, P |= NX
    uint64_t orr[kLW] = {0, 0, 0, 0};
    for (long long i = gwarp; i < (long long)nT; i += nwarps) {
        const int32_t w = __ldcg(TV + i);
        const size_t base = (size_t)w * words;
        for (int idx = lane; idx < words; idx += 32) {
            const uint64_t nx = __ldcg(p.NX + base + idx);
            if (nx) {
                p.NX[base + idx] = 0;
                p.P[base + idx] = __ldcg(p.P + base + idx) | nx;
                Mn[base + idx] = nx;
                orr[idx % kLW] |= nx;
            }
        }
        if (lane == 0) p.tv[w >> 6] = 0;
    }
#pragma unroll
    for (int lw = 0; lw < kLW; lw++) {
        const uint32_t lo = __reduce_or_sync(kFull, (uint32_t)orr[lw]);
        const uint32_t hi = __reduce_or_sync(kFull, (uint32_t)(orr[lw] >> 32));
        const uint64_t v = ((uint64_t)hi << 32) | lo;
        if (lane == 0 && v) atomicOr(&p.c->lane_new[nxt][lw], (unsigned long long)v);
    }
}

// Counters for the next level; run by one thread after the commit barrier
// of level j (nothing reads them until the next expansion).
__device__ void lane_reset_for_next(const LParams &p, int j) {
    LaneCounters *c = p.c;
    c->list_count[(j + 2) % 3] = 0;
    for (int lw = 0; lw < kLW; lw++) c->lane_new[(j + 2) % 3][lw] = 0;
    c->claim_v = 0;
    c->claim_h = 0;
    c->hub_packed = 0;
}

__global__ void __launch_bounds__(kLThreads) lane_batch_kernel(LParams p, int32_t max_levels,
                                                               int32_t *lane_last) {
    extern __shared__ __align__(16) uint64_t lsm[];
    const int warp = threadIdx.x >> 5;
    uint64_t *sm_M = lsm + (size_t)warp * 2 * p.K * kLW;
    uint64_t *sm_X = sm_M + p.K * kLW;
    for (int j = 0;; j++) {
        const unsigned long long nA = *(volatile unsigned long long *)&p.c->list_count[j % 3];
        if (p.pull_div > 0 && nA * (unsigned long long)p.pull_div > (unsigned long long)p.n) {
            lane_pull(p, j);
            if (!lane_barrier(p.c)) return;
        } else {
            lane_expand_vertices(p, j, sm_M, sm_X);
            if (!lane_barrier(p.c)) return;
            lane_expand_hubs(p, j, sm_M, sm_X);
            if (!lane_barrier(p.c)) return;
        }
        lane_commit(p, j);
        if (!lane_barrier(p.c)) return;
        const unsigned long long nT =
            *(volatile unsigned long long *)&p.c->list_count[(j + 1) % 3];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            for (int lw = 0; lw < kLW; lw++) {
                uint64_t m = *(volatile unsigned long long *)&p.c->lane_new[(j + 1) % 3][lw];
                while (m) {
                    const int b = __ffsll((long long)m) - 1;
                    m &= m - 1;
                    lane_last[lw * 64 + b] = j + 1;
                }
            }
            lane_reset_for_next(p, j);
            p.c->step = j + 1;
        }
        if (nT == 0 || (max_levels > 0 && j + 1 >= max_levels)) break;
        if (!lane_barrier(p.c)) return;
    }
}

// -------------------------------------------------------- extraction -----
// A32[lane][v / 32] = bits of vertices v..v+31 answering lane `lane`.
// For 32 vertices per warp: R[v] = OR_k P[v][k] & fmask[k] per lane word,
// then one ballot per set lane gives A32[row(lane)][v / 32].  Lanes with
// row(lane) < 0 are not extracted.  When `clear` is set, the bits of the
// extracted lanes are also removed from P and from the frontier rows M
// (their slots are being recycled).
__global__ void lane_extract_kernel(uint64_t *__restrict__ P, uint64_t *__restrict__ M, int32_t n,
                                    int32_t K, const uint64_t *__restrict__ fmask,
                                    const int32_t *__restrict__ lane_row, uint32_t *__restrict__ A32,
                                    int64_t words32, int clear) {
    __shared__ int32_t srow[kLanes];
    __shared__ uint64_t smask[kLW];
    for (int i = threadIdx.x; i < kLanes; i += blockDim.x) srow[i] = lane_row[i];
    __syncthreads();
    if (threadIdx.x < kLW) {
        uint64_t m = 0;
        for (int b = 0; b < 64; b++)
            if (srow[threadIdx.x * 64 + b] >= 0) m |= 1ull << b;
        smask[threadIdx.x] = m;
    }
    __syncthreads();
    const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    const unsigned lane = lane_id();
    for (long long chunk = gw; chunk < words32; chunk += nw) {
        const int32_t v = (int32_t)(chunk * 32 + lane);
        uint64_t r[kLW] = {0, 0, 0, 0};
        if (v < n) {
            const size_t base = (size_t)v * K * kLW;
            for (int k = 0; k < K; k++)
#pragma unroll
                for (int lw = 0; lw < kLW; lw++) {
                    const size_t idx = base + (size_t)k * kLW + lw;
                    const uint64_t pv = P[idx];
                    r[lw] |= pv & __ldg(fmask + k * kLW + lw);
                    if (clear && (pv & smask[lw])) P[idx] = pv & ~smask[lw];
                    if (clear) {
                        const uint64_t mv = M[idx];
                        if (mv & smask[lw]) M[idx] = mv & ~smask[lw];
                    }
                }
        }
#pragma unroll
        for (int lw = 0; lw < kLW; lw++) {
            r[lw] &= smask[lw];
            const uint32_t lo = __reduce_or_sync(kFull, (uint32_t)r[lw]);
            const uint32_t hi = __reduce_or_sync(kFull, (uint32_t)(r[lw] >> 32));
            uint64_t any = ((uint64_t)hi << 32) | lo;
            while (any) {
                const int b = __ffsll((long long)any) - 1;
                any &= any - 1;
                const unsigned bits = __ballot_sync(kFull, (r[lw] >> b) & 1ull);
                const int row = srow[lw * 64 + b];
                if (lane == 0) A32[(size_t)row * words32 + chunk] = bits;
            }
        }
    }
}

constexpr int kCountChunk = 1024;  // 32-bit words per counting chunk

__global__ void lane_count_kernel(const uint32_t *__restrict__ A32, int64_t words32, int n_lanes,
                                  int64_t chunks, int64_t *__restrict__ cnt) {
    // one block per (lane, chunk)
    const long long id = blockIdx.x;
    if (id >= (long long)n_lanes * chunks) return;
    const int ln = (int)(id / chunks);
    const long long ch = id % chunks;
    const long long w0 = ch * kCountChunk, w1 = (long long)min((long long)words32, (long long)(w0 + kCountChunk));
    long long c = 0;
    for (long long w = w0 + threadIdx.x; w < w1; w += blockDim.x)
        c += __popc(A32[(size_t)ln * words32 + w]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFull, c, o);
    __shared__ long long s[32];
    if (lane_id() == 0) s[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += s[i];
        cnt[id] = t;
    }
}

__global__ void lane_write_kernel(const uint32_t *__restrict__ A32, int64_t words32, int n_lanes,
                                  int64_t chunks, const int64_t *__restrict__ pos,
                                  int32_t *__restrict__ out, int64_t capacity) {
    const long long id = blockIdx.x;
    if (id >= (long long)n_lanes * chunks) return;
    const int ln = (int)(id / chunks);
    const long long ch = id % chunks;
    const long long w0 = ch * kCountChunk, w1 = (long long)min((long long)words32, (long long)(w0 + kCountChunk));
    __shared__ long long wsum[33];
    long long run = pos[id];
    const unsigned lane = lane_id();
    for (long long base = w0; base < w1; base += blockDim.x) {
        const long long w = base + threadIdx.x;
        uint32_t bits = w < w1 ? A32[(size_t)ln * words32 + w] : 0u;
        const int c = __popc(bits);
        int incl = c;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(kFull, incl, o);
            if ((int)lane >= o) incl += y;
        }
        if (lane == 31) wsum[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long acc = 0;
            for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
                const long long s = wsum[i];
                wsum[i] = acc;
                acc += s;
            }
            wsum[32] = acc;
        }
        __syncthreads();
        long long p = run + wsum[threadIdx.x >> 5] + incl - c;
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1;
            if (p < capacity) out[p] = (int32_t)(w * 32 + b);
            p++;
        }
        run += wsum[32];
        __syncthreads();
    }
}

// ---- one level step as separate kernels (server: captured in a graph) ----
__global__ void __launch_bounds__(kLThreads) lane_step_vertices_kernel(LParams p) {
    extern __shared__ __align__(16) uint64_t lsm[];
    const int warp = threadIdx.x >> 5;
    uint64_t *sm_M = lsm + (size_t)warp * 2 * p.K * kLW;
    uint64_t *sm_X = sm_M + p.K * kLW;
    const int j = *(volatile int32_t *)&p.c->step;
    lane_expand_vertices(p, j, sm_M, sm_X);
}

__global__ void __launch_bounds__(kLThreads) lane_step_hubs_kernel(LParams p) {
    extern __shared__ __align__(16) uint64_t lsm[];
    const int warp = threadIdx.x >> 5;
    uint64_t *sm_M = lsm + (size_t)warp * 2 * p.K * kLW;
    uint64_t *sm_X = sm_M + p.K * kLW;
    const int j = *(volatile int32_t *)&p.c->step;
    lane_expand_hubs(p, j, sm_M, sm_X);
}

__global__ void __launch_bounds__(kLThreads) lane_step_commit_kernel(LParams p) {
    const int j = *(volatile int32_t *)&p.c->step;
    lane_commit(p, j);
}

__global__ void lane_step_finish_kernel(LParams p, LaneStepOut *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int j = p.c->step;
    out->next_count = p.c->list_count[(j + 1) % 3];
    for (int lw = 0; lw < kLW; lw++) out->lane_new[lw] = p.c->lane_new[(j + 1) % 3][lw];
    out->status = p.c->status;
    lane_reset_for_next(p, j);
    p.c->step = j + 1;
    out->step = j + 1;
}

// Seeds (v, k, lane word, mask lo, mask hi) into frontier M_step and P, and
// appends vertices to the frontier list of the current step.
__global__ void lane_seed_step_kernel(LParams p, const int32_t *__restrict__ seeds, int n_seeds,
                                      const int32_t *__restrict__ verts, int n_verts, int step) {
    uint64_t *M = (step & 1) ? p.M1 : p.M0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_seeds; i += gridDim.x * blockDim.x) {
        const int32_t *s = seeds + 5 * i;
        const uint64_t m = (uint64_t)(uint32_t)s[3] | ((uint64_t)(uint32_t)s[4] << 32);
        const size_t idx = ((size_t)s[0] * p.K + s[1]) * kLW + s[2];
        atomicOr((unsigned long long *)(M + idx), (unsigned long long)m);
        atomicOr((unsigned long long *)(p.P + idx), (unsigned long long)m);
        // the seeded lanes have a frontier at this level (a pull reads it)
        atomicOr(&p.c->lane_new[step % 3][s[2]], (unsigned long long)m);
    }
    int32_t *A = lane_list(p, step % 3);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_verts; i += gridDim.x * blockDim.x) {
        const unsigned long long pos = atomicAdd(&p.c->list_count[step % 3], 1ull);
        A[pos] = verts[i];
    }
}

int g_lane_grid[64];
std::mutex g_lane_grid_mu;

rpq_status lane_grid(int device, size_t smem, int *grid) {
    std::lock_guard<std::mutex> lk(g_lane_grid_mu);
    if (device < 0 || device >= 64) return fail(RPQ_ERR_CUDA, "device id %d", device);
    if (g_lane_grid[device] > 0) {
        *grid = g_lane_grid[device];
        return RPQ_OK;
    }
    const size_t max_smem = (size_t)kLWarps * 2 * kLaneMaxSlots * kLW * sizeof(uint64_t);
    RPQ_CUDA_TRY(cudaFuncSetAttribute(lane_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)max_smem));
    int per_sm = 0, sms = 0;
    RPQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    RPQ_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lane_batch_kernel,
                                                               kLThreads, max_smem));
    if (per_sm <= 0) return fail(RPQ_ERR_CUDA, "lane kernel does not fit on an SM");
    per_sm = std::min(per_sm, 4);
    g_lane_grid[device] = sms * per_sm;
    (void)smem;
    *grid = g_lane_grid[device];
    return RPQ_OK;
}

}  // namespace

// ------------------------------------------------------- host helpers ----

// Builds the lane tables for queries (automata) placed in lanes 0..count-1.
rpq_status lane_build_tables(const rpq_graph *g, const Automaton *const *autos, int count,
                             int K, std::vector<LDir> *dirs, std::vector<LUnit> *units,
                             std::vector<LSrc> *srcs, std::vector<uint64_t> *fmask,
                             std::vector<uint64_t> *smask) {
    // (d, k2) -> (k -> mask)
    std::map<std::pair<int, int>, std::map<int, std::array<uint64_t, kLW>>> T;
    fmask->assign((size_t)K * kLW, 0);
    smask->assign((size_t)K * kLW, 0);
    for (int i = 0; i < count; i++) {
        const Automaton *a = autos[i];
        if (!a) continue;
        const int lw = i / 64;
        const uint64_t bit = 1ull << (i % 64);
        for (int q = 0; q < a->S; q++) {
            if ((a->final_mask >> q) & 1) (*fmask)[q * kLW + lw] |= bit;
            if ((a->start_mask >> q) & 1) (*smask)[q * kLW + lw] |= bit;
        }
        for (size_t t = 0; t < a->from.size(); t++) {
            const int s = a->sym[t];
            const int lab = s < a->L ? s : s - a->L;
            if (lab >= g->L)
                return fail(RPQ_ERR_INVALID, "query %d: label %d is not a label of the graph", i, lab);
            const int d = s < a->L ? lab : g->L + lab;
            auto &m = T[{d, a->to[t]}][a->from[t]];
            m[lw] |= bit;
        }
    }
    dirs->clear();
    units->clear();
    srcs->clear();
    int last_d = -1;
    for (auto &kv : T) {
        const int d = kv.first.first;
        if (d != last_d) {
            dirs->push_back(LDir{d, (int32_t)units->size(), 0, 0});
            last_d = d;
        }
        LUnit u{d, kv.first.second, (int32_t)srcs->size(), 0};
        for (auto &km : kv.second) {
            LSrc s{};
            s.k = km.first;
            for (int lw = 0; lw < kLW; lw++) s.mask[lw] = km.second[lw];
            srcs->push_back(s);
        }
        u.src_count = (int32_t)srcs->size() - u.src_first;
        units->push_back(u);
        dirs->back().unit_count++;
    }
    return RPQ_OK;
}

rpq_status lane_ws_alloc(LaneWorkspace *ws, const rpq_graph *g, int K) {
    const size_t words = (size_t)g->n * K * kLW;
    const size_t tvw = ((size_t)g->n + 63) / 64;
    const int64_t words32 = ((int64_t)g->n + 31) / 32;
    const size_t list_cap = (size_t)g->n + 2 * kLanes;  // distinct vertices + seeds of one step
    long long hub_cap = 1024, chunk_cap = 1024;
    for (int d = 0; d < 2 * g->L; d++) {
        hub_cap += g->adj[d].nnz / kLaneHubMin + 1;
        chunk_cap += g->adj[d].nnz / kLaneChunk + 1;
    }
    ws->n = g->n;
    ws->K = K;
    ws->hub_cap = hub_cap;
    ws->chunk_cap = chunk_cap;
    const int64_t chunks = (words32 + kCountChunk - 1) / kCountChunk;
    if (!ws->M0.alloc(words * 8) || !ws->M1.alloc(words * 8) || !ws->P.alloc(words * 8) ||
        !ws->NX.alloc(words * 8) || !ws->tv.alloc(tvw * 8) || !ws->l0.alloc(4 * list_cap) ||
        !ws->l1.alloc(4 * list_cap) || !ws->l2.alloc(4 * list_cap) ||
        !ws->hubs.alloc(sizeof(LHub) * hub_cap) ||
        !ws->hub_cmap.alloc(sizeof(int32_t) * chunk_cap) || !ws->ctr.alloc(sizeof(LaneCounters)) ||
        !ws->tables.alloc(1 << 20) || !ws->A32.alloc((size_t)kLanes * words32 * 4) ||
        !ws->cnt.alloc(sizeof(int64_t) * (kLanes * chunks + 1)) ||
        !ws->pos.alloc(sizeof(int64_t) * (kLanes * chunks + 1)))
        return fail(RPQ_ERR_OOM, "lane workspace (%d slots)", K);
    // cleared before any stream uses the workspace: a plain cudaMemset is
    // ordered only on the legacy default stream, which non-blocking streams
    // (the server's) do not wait for
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->NX.p, 0, words * 8, 0));
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->M0.p, 0, words * 8, 0));
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->M1.p, 0, words * 8, 0));
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->P.p, 0, words * 8, 0));
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->tv.p, 0, tvw * 8, 0));
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->ctr.p, 0, sizeof(LaneCounters), 0));
    RPQ_CUDA_TRY(cudaStreamSynchronize(0));
    ws->staging_bytes = (1 << 20) + 4096;
    RPQ_CUDA_TRY(cudaMallocHost(&ws->staging, ws->staging_bytes));
    return RPQ_OK;
}

std::unique_ptr<LaneWorkspace> lane_ws_acquire(rpq_graph *g, int K, rpq_status *st) {
    {
        std::lock_guard<std::mutex> lk(g->ws_mu);
        for (size_t i = 0; i < g->ws_free.size(); i++) {
            auto *w = dynamic_cast<LaneWorkspace *>(g->ws_free[i].get());
            if (w && w->K >= K) {
                std::unique_ptr<LaneWorkspace> r(static_cast<LaneWorkspace *>(g->ws_free[i].release()));
                g->ws_free.erase(g->ws_free.begin() + i);
                *st = RPQ_OK;
                return r;
            }
        }
    }
    std::unique_ptr<LaneWorkspace> w(new LaneWorkspace());
    int Kc = 4;
    while (Kc < K) Kc *= 2;
    *st = lane_ws_alloc(w.get(), g, Kc);
    if (*st != RPQ_OK) return nullptr;
    return w;
}

void lane_ws_release(rpq_graph *g, std::unique_ptr<LaneWorkspace> w) {
    std::lock_guard<std::mutex> lk(g->ws_mu);
    g->ws_free.emplace_back(std::move(w));
}

rpq_status lane_ws_acquire_fixed(rpq_graph *g, int K, std::unique_ptr<LaneWorkspace> *out) {
    rpq_status st = RPQ_OK;
    *out = lane_ws_acquire(g, K, &st);
    return *out ? RPQ_OK : st;
}

void lane_ws_return(rpq_graph *g, std::unique_ptr<LaneWorkspace> w) {
    lane_ws_release(g, std::move(w));
}

LParams lane_params(rpq_graph *g, LaneWorkspace *ws, size_t o_dyn, size_t o_dirs, size_t o_units,
                    size_t o_srcs) {
    uint8_t *dt = ws->tables.as<uint8_t>();
    LParams p{};
    p.adj = g->d_adj.as<DevAdj>();
    p.n = g->n;
    p.K = ws->K;
    p.dyn = reinterpret_cast<const LaneDyn *>(dt + o_dyn);
    p.dirs = reinterpret_cast<const LDir *>(dt + o_dirs);
    p.units = reinterpret_cast<const LUnit *>(dt + o_units);
    p.srcs = reinterpret_cast<const LSrc *>(dt + o_srcs);
    p.M0 = ws->M0.as<uint64_t>();
    p.M1 = ws->M1.as<uint64_t>();
    p.P = ws->P.as<uint64_t>();
    p.NX = ws->NX.as<uint64_t>();
    p.tv = ws->tv.as<uint64_t>();
    p.list0 = ws->l0.as<int32_t>();
    p.list1 = ws->l1.as<int32_t>();
    p.list2 = ws->l2.as<int32_t>();
    p.hubs = ws->hubs.as<LHub>();
    p.hub_cmap = ws->hub_cmap.as<int32_t>();
    p.hub_cap = ws->hub_cap;
    p.chunk_cap = ws->chunk_cap;
    p.c = ws->ctr.as<LaneCounters>();
    p.adj_half = g->L;
    // the graph's tuning; RPQ_LANE_HUB and RPQ_LANE_PULL_DIV override
    const char *h = getenv("RPQ_LANE_HUB");
    const char *pd = getenv("RPQ_LANE_PULL_DIV");
    p.lane_hub = std::max(kLaneHubMin, h ? atoi(h) : g->lane_hub);
    p.pull_div = std::max(0, pd ? atoi(pd) : g->lane_pull_div);
    return p;
}

size_t lane_smem(int K) { return (size_t)kLWarps * 2 * K * kLW * sizeof(uint64_t); }

rpq_status lane_set_smem_limits() {
    static std::once_flag once;
    static rpq_status st = RPQ_OK;
    std::call_once(once, [] {
        const int mx = (int)lane_smem(kLaneMaxSlots);
        if (cudaFuncSetAttribute(lane_step_vertices_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
            cudaFuncSetAttribute(lane_step_hubs_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess)
            st = fail(RPQ_ERR_CUDA, "lane step kernels: %s", cudaGetErrorString(cudaGetLastError()));
    });
    return st;
}

rpq_status lane_capture_step(const LParams &p, LaneStepOut *out_dev, cudaStream_t st,
                             cudaGraphExec_t *exec) {
    rpq_status s = lane_set_smem_limits();
    if (s != RPQ_OK) return s;
    int sms = 0;
    RPQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0));
    const size_t smem = lane_smem(p.K);
    cudaGraph_t graph;
    RPQ_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    // captured, not launched: each replay of the graph launches these
    // kLaneStepKernels
    lane_step_vertices_kernel<<<sms * 4, kLThreads, smem, st>>>(p);
    lane_step_hubs_kernel<<<sms * 4, kLThreads, smem, st>>>(p);
    lane_step_commit_kernel<<<sms * 8, kLThreads, 0, st>>>(p);
    lane_step_finish_kernel<<<1, 32, 0, st>>>(p, out_dev);
    RPQ_CUDA_TRY(cudaStreamEndCapture(st, &graph));
    cudaError_t e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(RPQ_ERR_CUDA, "step graph: %s", cudaGetErrorString(e));
    return RPQ_OK;
}

rpq_status lane_seed(const LParams &p, const int32_t *seeds_dev, int n_seeds,
                     const int32_t *verts_dev, int n_verts, int step, cudaStream_t st) {
    if (n_seeds == 0 && n_verts == 0) return RPQ_OK;
    lane_seed_step_kernel<<<1, 256, 0, st>>>(p, seeds_dev, n_seeds, verts_dev, n_verts, step);
    note_launch();
    RPQ_CUDA_TRY(cudaGetLastError());
    return RPQ_OK;
}

// Answers of `count` lanes: lane_ids_host[i] gets row i of the extraction.
// Extraction, counting, scan and ordered write; `clear` also recycles the
// lanes' bits.  Offsets (count + 1) and answers come back to the host, or
// the answers go to out_dev (capacity entries) when it is given.
rpq_status lane_harvest_impl(rpq_graph *g, LaneWorkspace *ws, const LParams &p,
                             const uint64_t *fmask_dev, const int32_t *lane_row_dev,
                             int count, bool clear, int cur_step,
                             std::vector<int64_t> *offsets_host,
                             std::vector<int32_t> *answers_host, int32_t *out_dev,
                             int64_t capacity, cudaStream_t st) {
    const int64_t words32 = ((int64_t)g->n + 31) / 32;
    const int64_t chunks = (words32 + kCountChunk - 1) / kCountChunk;
    if (count > 0) RPQ_CUDA_TRY(cudaMemsetAsync(ws->A32.p, 0, (size_t)count * words32 * 4, st));
    uint64_t *Mcur = (cur_step & 1) ? p.M1 : p.M0;
    lane_extract_kernel<<<152 * 8, 256, 0, st>>>(p.P, Mcur, g->n, p.K, fmask_dev, lane_row_dev,
                                                 ws->A32.as<uint32_t>(), words32, clear ? 1 : 0);
    note_launch();
    RPQ_CUDA_TRY(cudaGetLastError());
    offsets_host->assign((size_t)count + 1, 0);
    if (count == 0) return RPQ_OK;
    const long long nblk = (long long)count * chunks;
    lane_count_kernel<<<(unsigned)nblk, 256, 0, st>>>(ws->A32.as<uint32_t>(), words32, count,
                                                     chunks, ws->cnt.as<int64_t>());
    note_launch();
    RPQ_CUDA_TRY(cudaGetLastError());
    rpq_status s = device_exclusive_scan<int64_t>(ws->cnt.as<int64_t>(), ws->pos.as<int64_t>(),
                                                  nblk, ws->pos.as<int64_t>() + nblk, st);
    if (s != RPQ_OK) return s;
    std::vector<int64_t> hpos((size_t)nblk + 1);
    RPQ_CUDA_TRY(cudaMemcpyAsync(hpos.data(), ws->pos.p, sizeof(int64_t) * (nblk + 1),
                                 cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < count; i++) (*offsets_host)[i] = hpos[(size_t)i * chunks];
    (*offsets_host)[count] = hpos[nblk];
    const int64_t total = hpos[nblk];
    if (total == 0) return RPQ_OK;
    if (out_dev) {
        if (total <= capacity) {
            lane_write_kernel<<<(unsigned)nblk, 256, 0, st>>>(ws->A32.as<uint32_t>(), words32, count,
                                                               chunks, ws->pos.as<int64_t>(), out_dev,
                                                               capacity);
            note_launch();
            RPQ_CUDA_TRY(cudaGetLastError());
        }
        return RPQ_OK;
    }
    DevBuf tmp;
    if (!tmp.alloc(sizeof(int32_t) * total)) return fail(RPQ_ERR_OOM, "answer staging");
    lane_write_kernel<<<(unsigned)nblk, 256, 0, st>>>(ws->A32.as<uint32_t>(), words32, count, chunks,
                                                       ws->pos.as<int64_t>(), tmp.as<int32_t>(),
                                                       total);
    note_launch();
    RPQ_CUDA_TRY(cudaGetLastError());
    answers_host->resize((size_t)total);
    RPQ_CUDA_TRY(cudaMemcpyAsync(answers_host->data(), tmp.p, sizeof(int32_t) * total,
                                 cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    return RPQ_OK;
}

rpq_status lane_harvest(rpq_graph *g, LaneWorkspace *ws, const LParams &p,
                        const uint64_t *fmask_dev, const int32_t *lane_ids_host, int count,
                        std::vector<int64_t> *offsets_host, std::vector<int32_t> *answers_host,
                        cudaStream_t st) {
    // lane -> row map in the staging tail, uploaded to the end of the tables buffer
    std::vector<int32_t> row(kLanes, -1);
    for (int i = 0; i < count; i++) row[lane_ids_host[i]] = i;
    int32_t *hrow = reinterpret_cast<int32_t *>(static_cast<uint8_t *>(ws->staging) +
                                                ws->staging_bytes - 4096 + 2048);
    memcpy(hrow, row.data(), sizeof(int32_t) * kLanes);
    int32_t *drow = reinterpret_cast<int32_t *>(ws->tables.as<uint8_t>() + (1 << 20) - 2048);
    RPQ_CUDA_TRY(cudaMemcpyAsync(drow, hrow, sizeof(int32_t) * kLanes, cudaMemcpyHostToDevice, st));
    int cur = 0;
    LaneCounters hc;
    RPQ_CUDA_TRY(cudaMemcpyAsync(&hc, ws->ctr.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    cur = hc.step;
    return lane_harvest_impl(g, ws, p, fmask_dev, drow, count, true, cur, offsets_host,
                             answers_host, nullptr, 0, st);
}

// Runs one lane group (<= 256 queries) to completion and writes the answers.
// out (host or device per out_is_dev), capacity entries; offsets[i]
// (group-relative) for i in [0, count].
bool same_automaton(const Automaton &a, const Automaton &b);

rpq_status lane_run_group(rpq_graph *g, const Automaton *const *autos, const int32_t *sources,
                          int count, int32_t max_levels, int32_t *out, bool out_is_dev,
                          int64_t capacity, int64_t *offsets, int32_t *lane_levels, float *ms,
                          cudaStream_t st, int64_t *edges_out = nullptr) {
    int K = 1;
    for (int i = 0; i < count; i++) K = std::max(K, autos[i]->S);
    if (K > kLaneMaxSlots) return fail(RPQ_ERR_INVALID, "automaton with more than 64 states");
    for (int i = 0; i < count; i++)
        if (sources[i] < 0 || sources[i] >= g->n)
            return fail(RPQ_ERR_INVALID, "query %d: source %d outside [0, %d)", i, sources[i], g->n);
    std::vector<LDir> dirs;
    std::vector<LUnit> units;
    std::vector<LSrc> srcs;
    std::vector<uint64_t> fmask, smask;
    rpq_status s = lane_build_tables(g, autos, count, K, &dirs, &units, &srcs, &fmask, &smask);
    if (s != RPQ_OK) return s;
    rpq_status as = RPQ_OK;
    std::unique_ptr<LaneWorkspace> ws = lane_ws_acquire(g, K, &as);
    if (!ws) return as;
    K = ws->K;  // slots beyond the automata's states stay empty
    fmask.resize((size_t)K * kLW, 0);
    std::map<std::tuple<int, int, int>, uint64_t> seedm;
    for (int i = 0; i < count; i++) {
        const uint64_t sm = autos[i]->start_mask;
        for (int q = 0; q < autos[i]->S; q++)
            if ((sm >> q) & 1) seedm[std::make_tuple(sources[i], q, i / 64)] |= 1ull << (i % 64);
    }
    std::vector<int32_t> seeds, frontier;
    for (auto &kv : seedm) {
        seeds.push_back(std::get<0>(kv.first));
        seeds.push_back(std::get<1>(kv.first));
        seeds.push_back(std::get<2>(kv.first));
        seeds.push_back((int32_t)(uint32_t)kv.second);
        seeds.push_back((int32_t)(uint32_t)(kv.second >> 32));
        frontier.push_back(std::get<0>(kv.first));
    }
    std::sort(frontier.begin(), frontier.end());
    frontier.erase(std::unique(frontier.begin(), frontier.end()), frontier.end());
    LaneDyn dyn{};
    dyn.n_dirs = (int32_t)dirs.size();
    for (int lw = 0; lw < kLW; lw++) {
        const int lo = lw * 64, hi = std::min(count, lo + 64);
        dyn.active[lw] = hi <= lo ? 0ull : (hi - lo == 64 ? ~0ull : ((1ull << (hi - lo)) - 1));
    }
    uint8_t *hs = static_cast<uint8_t *>(ws->staging);
    size_t off = 0;
    const size_t limit = (1 << 20) - 4096;
    auto put = [&](const void *p, size_t bytes) {
        off = (off + 15) & ~size_t(15);
        const size_t at = off;
        if (bytes && at + bytes <= limit) {
            if (p) memcpy(hs + at, p, bytes);
            else memset(hs + at, 0, bytes);
        }
        off += bytes;
        return at;
    };
    const size_t o_dyn = put(&dyn, sizeof(dyn));
    const size_t o_dirs = put(dirs.data(), sizeof(LDir) * dirs.size());
    const size_t o_units = put(units.data(), sizeof(LUnit) * units.size());
    const size_t o_srcs = put(srcs.data(), sizeof(LSrc) * srcs.size());
    const size_t o_fm = put(fmask.data(), sizeof(uint64_t) * fmask.size());
    const size_t o_seed = put(seeds.data(), sizeof(int32_t) * seeds.size());
    const size_t o_front = put(frontier.data(), sizeof(int32_t) * frontier.size());
    const size_t o_last = put(nullptr, sizeof(int32_t) * kLanes);
    std::vector<int32_t> row(kLanes, -1);
    for (int i = 0; i < count; i++) row[i] = i;
    const size_t o_row = put(row.data(), sizeof(int32_t) * kLanes);
    off = (off + 15) & ~size_t(15);
    if (off > limit) {
        lane_ws_release(g, std::move(ws));
        return fail(RPQ_ERR_INVALID, "lane tables too large");
    }
    uint8_t *dt = ws->tables.as<uint8_t>();
    RPQ_CUDA_TRY(cudaMemcpyAsync(dt, hs, off, cudaMemcpyHostToDevice, st));
    const size_t words = (size_t)g->n * K * kLW;
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->P.p, 0, words * 8, st));
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->ctr.p, 0, sizeof(LaneCounters), st));
    LParams p = lane_params(g, ws.get(), o_dyn, o_dirs, o_units, o_srcs);
    // pulling pays only when the lanes share one automaton: lanes of
    // different automata are rarely all covered early, so a pulled scan
    // rarely stops early (the mixed rmat20 batch: 1,083 q/s pulling at
    // divisor 2 against 3,567 pushing).  RPQ_LANE_PULL_DIV still overrides.
    if (!getenv("RPQ_LANE_PULL_DIV")) {
        bool shared = true;
        for (int i = 1; i < count && shared; i++)
            shared = autos[i] == autos[0] || same_automaton(*autos[0], *autos[i]);
        if (!shared) p.pull_div = 0;
    }
    s = lane_seed(p, reinterpret_cast<const int32_t *>(dt + o_seed), (int)(seeds.size() / 5),
                  reinterpret_cast<const int32_t *>(dt + o_front), (int)frontier.size(), 0, st);
    if (s != RPQ_OK) return s;
    int32_t *lane_last = reinterpret_cast<int32_t *>(dt + o_last);
    int grid = 0;
    const size_t smem = lane_smem(K);
    s = lane_grid(g->device, smem, &grid);
    if (s != RPQ_OK) {
        lane_ws_release(g, std::move(ws));
        return s;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    int32_t ml = max_levels;
    void *args[] = {&p, &ml, &lane_last};
    cudaError_t le = cudaLaunchCooperativeKernel((const void *)lane_batch_kernel, dim3(grid),
                                                 dim3(kLThreads), args, smem, st);
    if (le != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return fail(RPQ_ERR_CUDA, "lane kernel launch: %s", cudaGetErrorString(le));
    }
    note_launch();
    cudaEventRecord(e1, st);
    LaneCounters hc;
    RPQ_CUDA_TRY(cudaMemcpyAsync(&hc, ws->ctr.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
    std::vector<int32_t> hl(kLanes);
    RPQ_CUDA_TRY(cudaMemcpyAsync(hl.data(), lane_last, sizeof(int32_t) * kLanes,
                                 cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    float kms = 0;
    cudaEventElapsedTime(&kms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (hc.status != 0) {
        cudaMemsetAsync(ws->NX.p, 0, words * 8, st);
        cudaMemsetAsync(ws->M0.p, 0, words * 8, st);
        cudaMemsetAsync(ws->M1.p, 0, words * 8, st);
        cudaMemsetAsync(ws->tv.p, 0, ((size_t)g->n + 63) / 64 * 8, st);
        cudaMemsetAsync(ws->ctr.p, 0, sizeof(LaneCounters), st);
        cudaStreamSynchronize(st);
        lane_ws_release(g, std::move(ws));
        return fail((rpq_status)hc.status, "lane traversal failed (status %d)", hc.status);
    }
    // answers; the frontier buffers are zeroed for the next group (the last
    // level's frontier rows are not cleared by a commit)
    std::vector<int64_t> offs;
    std::vector<int32_t> host_ans;
    s = lane_harvest_impl(g, ws.get(), p, reinterpret_cast<const uint64_t *>(dt + o_fm),
                          reinterpret_cast<const int32_t *>(dt + o_row), count, false, hc.step,
                          &offs, &host_ans, out_is_dev ? out : nullptr, out_is_dev ? capacity : 0,
                          st);
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->M0.p, 0, words * 8, st));
    RPQ_CUDA_TRY(cudaMemsetAsync(ws->M1.p, 0, words * 8, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    if (s != RPQ_OK) {
        lane_ws_release(g, std::move(ws));
        return s;
    }
    for (int i = 0; i <= count; i++) offsets[i] = offs[i];
    for (int i = 0; i < count; i++) lane_levels[i] = hl[i];
    if (ms) *ms = kms;
    if (edges_out) *edges_out = (int64_t)hc.edges;
    const int64_t total = offs[count];
    if (!out_is_dev && total <= capacity && total > 0) memcpy(out, host_ans.data(), 4 * total);
    lane_ws_release(g, std::move(ws));
    return RPQ_OK;
}

rpq_status bitsets_to_lists(const uint32_t *bits, int64_t words32, int count, int32_t *out,
                            bool out_is_dev, int64_t capacity, int64_t *offsets, void *stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    offsets[0] = 0;
    if (count == 0) return RPQ_OK;
    const int64_t chunks = (words32 + kCountChunk - 1) / kCountChunk;
    const long long nblk = (long long)count * chunks;
    DevBuf cnt, pos;
    if (!cnt.alloc(sizeof(int64_t) * (nblk + 1)) || !pos.alloc(sizeof(int64_t) * (nblk + 1)))
        return fail(RPQ_ERR_OOM, "answer compaction buffers");
    lane_count_kernel<<<(unsigned)nblk, 256, 0, st>>>(bits, words32, count, chunks,
                                                     cnt.as<int64_t>());
    note_launch();
    RPQ_CUDA_TRY(cudaGetLastError());
    rpq_status s = device_exclusive_scan<int64_t>(cnt.as<int64_t>(), pos.as<int64_t>(), nblk,
                                                  pos.as<int64_t>() + nblk, st);
    if (s != RPQ_OK) return s;
    std::vector<int64_t> hpos((size_t)nblk + 1);
    RPQ_CUDA_TRY(cudaMemcpyAsync(hpos.data(), pos.p, sizeof(int64_t) * (nblk + 1),
                                 cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < count; i++) offsets[i] = hpos[(size_t)i * chunks];
    offsets[count] = hpos[nblk];
    const int64_t total = hpos[nblk];
    if (total == 0 || total > capacity) return RPQ_OK;
    if (out_is_dev) {
        lane_write_kernel<<<(unsigned)nblk, 256, 0, st>>>(bits, words32, count, chunks,
                                                           pos.as<int64_t>(), out, capacity);
        note_launch();
        RPQ_CUDA_TRY(cudaGetLastError());
        RPQ_CUDA_TRY(cudaStreamSynchronize(st));
        return RPQ_OK;
    }
    DevBuf tmp;
    if (!tmp.alloc(sizeof(int32_t) * total)) return fail(RPQ_ERR_OOM, "answer staging");
    lane_write_kernel<<<(unsigned)nblk, 256, 0, st>>>(bits, words32, count, chunks,
                                                       pos.as<int64_t>(), tmp.as<int32_t>(), total);
    note_launch();
    RPQ_CUDA_TRY(cudaGetLastError());
    RPQ_CUDA_TRY(cudaMemcpyAsync(out, tmp.p, sizeof(int32_t) * total, cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    return RPQ_OK;
}

// Batch by query slots: `slots` concurrent persistent query kernels, each on
// 1/slots of the grid and its own stream, take the queries in turn; every
// answer lands as a bitset row, and the rows become sorted lists at the end.
rpq_status slot_batch(rpq_graph *g, const Automaton *const *autos, const int32_t *sources,
                      int n, int32_t max_levels, int slots, int32_t *out, bool out_is_dev,
                      int64_t capacity, int64_t *offsets, rpq_stats *stats, cudaStream_t st) {
    const int64_t W = ((int64_t)g->n + 63) / 64;
    DevBuf bits;
    if (!bits.alloc(sizeof(uint64_t) * (size_t)W * std::max(n, 1)))
        return fail(RPQ_ERR_OOM, "answer bitsets of %d queries", n);
    // callers' earlier work on `st` must be visible to the slot streams
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    std::atomic<int> next{0};
    std::atomic<int> first_err{(int)RPQ_OK};
    std::mutex msg_mu;
    std::string msg;
    auto worker = [&]() {
        cudaSetDevice(g->device);
        cudaStream_t s2 = nullptr;
        const cudaError_t ce = cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking);
        if (ce != cudaSuccess) {
            std::lock_guard<std::mutex> lk(msg_mu);
            if (msg.empty())
                msg = std::string("cudaStreamCreateWithFlags (slot stream): ") + cudaGetErrorString(ce);
            first_err = (int)RPQ_ERR_CUDA;
            return;
        }
        for (;;) {
            const int i = next.fetch_add(1);
            if (i >= n || first_err.load() != (int)RPQ_OK) break;
            int64_t cnt = 0;
            rpq_stats local{};
            const rpq_status r = run_query_slot(g, *autos[i], sources[i], max_levels, nullptr, 0,
                                                bits.as<uint64_t>() + (size_t)i * W, nullptr,
                                                stats ? &local : nullptr, &cnt, s2, slots);
            if (r != RPQ_OK) {
                int expect = (int)RPQ_OK;
                if (first_err.compare_exchange_strong(expect, (int)r)) {
                    std::lock_guard<std::mutex> lk(msg_mu);
                    msg = rpq_last_error_str();
                }
                break;
            }
            if (stats) stats[i] = local;
        }
        cudaStreamSynchronize(s2);
        cudaStreamDestroy(s2);
    };
    std::vector<std::thread> th;
    for (int k = 0; k < slots; k++) th.emplace_back(worker);
    for (auto &t : th) t.join();
    if (first_err.load() != (int)RPQ_OK)
        return fail((rpq_status)first_err.load(), "%s", msg.c_str());
    return bitsets_to_lists(reinterpret_cast<const uint32_t *>(bits.p), 2 * W, n, out, out_is_dev,
                            capacity, offsets, st);
}

bool same_automaton(const Automaton &a, const Automaton &b) {
    if (a.S != b.S || a.L != b.L || a.start_mask != b.start_mask || a.final_mask != b.final_mask ||
        a.from.size() != b.from.size())
        return false;
    std::vector<std::tuple<int, int, int>> x, y;
    for (size_t t = 0; t < a.from.size(); t++) {
        x.emplace_back(a.from[t], a.sym[t], a.to[t]);
        y.emplace_back(b.from[t], b.sym[t], b.to[t]);
    }
    std::sort(x.begin(), x.end());
    std::sort(y.begin(), y.end());
    return x == y;
}

}  // namespace rpq

using namespace rpq;

extern "C" rpq_status rpq_query_batch(const rpq_graph *g, int32_t n, const rpq_nfa *const *nfas,
                                      const int32_t *sources, int32_t max_levels,
                                      int64_t *out_offsets, int32_t *out_vertices, int64_t capacity,
                                      rpq_stats *stats, void *stream) {
    clear_error();
    if (!g || n < 0 || (n > 0 && (!nfas || !sources)) || !out_offsets)
        return fail(RPQ_ERR_INVALID, "null argument");
    if (capacity < 0 || (capacity > 0 && !out_vertices)) return fail(RPQ_ERR_INVALID, "bad output");
    if (max_levels < 0) return fail(RPQ_ERR_INVALID, "max_levels must be >= 0");
    for (int i = 0; i < n; i++)
        if (!nfas[i]) return fail(RPQ_ERR_INVALID, "automaton %d is null", i);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rpq_graph *gm = const_cast<rpq_graph *>(g);
    const bool dev = out_vertices && is_device_pointer(out_vertices);
    out_offsets[0] = 0;
    int64_t total = 0;
    bool overflow = false;
    std::vector<const Automaton *> autos(n);
    for (int i = 0; i < n; i++) autos[i] = &nfas[i]->a;
    // engine: bit lanes pay off when the queries share their automaton (their
    // frontiers then overlap level by level: multi-source BFS); otherwise
    // concurrent query slots use the GPU better
    bool shared = n >= 16;
    for (int i = 1; i < n && shared; i++) shared = same_automaton(*autos[0], *autos[i]);
    const char *eng = getenv("RPQ_BATCH_ENGINE");
    const bool use_lanes = eng ? strcmp(eng, "lanes") == 0 : shared;
    if (!use_lanes) {
        const char *sl = getenv("RPQ_SLOTS");
        const int slots = std::max(1, std::min(64, sl ? atoi(sl) : kDefaultSlots));
        for (int i = 0; i < n; i++)
            if (sources[i] < 0 || sources[i] >= gm->n)
                return fail(RPQ_ERR_INVALID, "query %d: source %d outside [0, %d)", i, sources[i],
                            gm->n);
        rpq_status s = slot_batch(gm, autos.data(), sources, n, max_levels, std::min(slots, std::max(n, 1)),
                                  out_vertices, dev, capacity, out_offsets, stats, st);
        if (s != RPQ_OK) return s;
        total = out_offsets[n];
        overflow = total > capacity;
    }
    for (int g0 = 0; use_lanes && g0 < n; g0 += kLanes) {
        const int cnt = std::min(kLanes, n - g0);
        std::vector<int64_t> offs(cnt + 1);
        std::vector<int32_t> lv(cnt);
        float ms = 0;
        int64_t lane_edges = 0;
        const int64_t room = overflow ? 0 : std::max<int64_t>(0, capacity - total);
        rpq_status s = lane_run_group(gm, autos.data() + g0, sources + g0, cnt, max_levels,
                                      out_vertices ? out_vertices + total : nullptr, dev, room,
                                      offs.data(), lv.data(), &ms, st, &lane_edges);
        if (s != RPQ_OK) return s;
        for (int i = 0; i < cnt; i++) out_offsets[g0 + i + 1] = total + offs[i + 1];
        if (stats) {
            for (int i = 0; i < cnt; i++) {
                rpq_stats &x = stats[g0 + i];
                x.levels = lv[i];
                x.visited_pairs = -1;
                x.expanded_pairs = -1;
                // the group's shared pass: the same count for every query of it
                x.product_edges = lane_edges;
                x.push_bytes = -1;
                x.answer_count = offs[i + 1] - offs[i];
                x.push_unit_levels = -1;
                x.pull_unit_levels = -1;
                x.h2d_bytes = -1;
                x.d2h_bytes = -1;
                x.device_ms = ms;
            }
        }
        if (total + offs[cnt] > capacity) overflow = true;
        total += offs[cnt];
    }
    if (overflow)
        return fail(RPQ_ERR_CAPACITY, "batch answers hold %lld vertices, capacity %lld",
                    (long long)total, (long long)capacity);
    return RPQ_OK;
}

// ------------------------------------------------------ batch autotune --
namespace rpq {
namespace {
// Lane engine tuning: times the sample batch (lane groups of up to 256) on
// the lane kernel under every (inline row length, pull divisor) pair and
// keeps the fastest by device time.
rpq_status autotune_batch(rpq_graph *g, int n, const rpq_nfa *const *nfas, const int32_t *sources,
                          int32_t *hub_out, int32_t *pull_out, cudaStream_t st) {
    static const int32_t kHubs[] = {32, 64, 128, 256};
    static const int32_t kPulls[] = {0, 2, 4, 8, 16};
    std::vector<const Automaton *> autos(n);
    for (int i = 0; i < n; i++) autos[i] = &nfas[i]->a;
    const int32_t keep_h = g->lane_hub, keep_p = g->lane_pull_div;
    double best = -1;
    int32_t best_h = keep_h, best_p = keep_p;
    std::vector<int64_t> offs((size_t)kLanes + 1);
    std::vector<int32_t> lv(kLanes);
    for (int32_t h : kHubs) {
        for (int32_t pd : kPulls) {
            g->lane_hub = h;
            g->lane_pull_div = pd;
            double total = 0;
            for (int rep = 0; rep < 2; rep++) {  // the first pass warms the workspace
                total = 0;
                for (int g0 = 0; g0 < n; g0 += kLanes) {
                    const int cnt = std::min(kLanes, n - g0);
                    float ms = 0;
                    rpq_status s = lane_run_group(g, autos.data() + g0, sources + g0, cnt, 0,
                                                  nullptr, false, 0, offs.data(), lv.data(), &ms, st);
                    if (s != RPQ_OK) {
                        g->lane_hub = keep_h;
                        g->lane_pull_div = keep_p;
                        return s;
                    }
                    total += ms;
                }
            }
            if (best < 0 || total < best) {
                best = total;
                best_h = h;
                best_p = pd;
            }
        }
    }
    g->lane_hub = best_h;
    g->lane_pull_div = best_p;
    if (hub_out) *hub_out = best_h;
    if (pull_out) *pull_out = best_p;
    return RPQ_OK;
}
}  // namespace
}  // namespace rpq

extern "C" rpq_status rpq_graph_autotune_batch(rpq_graph *g, int32_t n, const rpq_nfa *const *nfas,
                                               const int32_t *sources, int32_t *lane_hub_out,
                                               int32_t *pull_div_out, void *stream) {
    clear_error();
    if (!g || n <= 0 || !nfas || !sources) return fail(RPQ_ERR_INVALID, "bad argument");
    for (int32_t i = 0; i < n; i++) {
        if (!nfas[i]) return fail(RPQ_ERR_INVALID, "automaton %d is null", i);
        if (sources[i] < 0 || sources[i] >= g->n)
            return fail(RPQ_ERR_INVALID, "source %d outside [0, %d)", sources[i], g->n);
    }
    return autotune_batch(g, n, nfas, sources, lane_hub_out, pull_div_out,
                          static_cast<cudaStream_t>(stream));
}
