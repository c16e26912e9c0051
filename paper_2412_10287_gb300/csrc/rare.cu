// Rare labels first: an evaluation order for single-source queries whose
// every accepted word must read some rare label.  The paper finds its BFS
// slowest where it "does not exploit" rare labels or evaluation order
// (sections 5.4-5.5) and names rare-label use as future work (section 6).
//
// Plan, for an automaton N, a source v_s and a label direction d (a label
// or an inverse label) that every accepting path of N reads:
//   1. U = the vertices with an edge in direction d (few: d is rare).
//   2. Backward: the pairs (q, v) from which a pair (q_d, u), q_d a state
//      with a d-transition and u in U, is reachable without reading d --
//      the single-source search of the reversed automaton (section 4,
//      SSR of N^-) restricted to N's transitions other than d, from the
//      source set U with start states {q_d}.  Every pair outside this set,
//      before the first d, can never lead to an accepted word.
//   3. Forward: Algorithm 1 on the two-copy automaton N2 (copy 0: before
//      reading d, copy 1: after; d-transitions lead from copy 0 to copy 1;
//      starts in copy 0, finals in copy 1; the same language, since every
//      accepted word reads d), with the copy-0 pairs outside the backward
//      set marked visited before the launch, so the traversal never enters
//      them.
// The answer is exactly the query's answer; only the work changes.
#include <algorithm>
#include <cstdlib>
#include <vector>

#include "graph.h"

namespace rpq {
namespace {

// Vertices with a non-empty row in A (order irrelevant: a source set).
__global__ void nonempty_rows_kernel(DevAdj A, int32_t n, int32_t *out,
                                     unsigned long long *count) {
    const int32_t rows = A.fmt == ADJ_DENSE ? n : A.fmt == ADJ_HYPER ? A.nrows : 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) {
        int32_t v;
        bool keep;
        if (A.fmt == ADJ_DENSE) {
            v = i;
            keep = __ldg(A.off + i + 1) > __ldg(A.off + i);
        } else {
            v = __ldg(A.rows + i);
            keep = __ldg(A.off + i + 1) > __ldg(A.off + i);
        }
        if (keep) out[atomicAdd(count, 1ull)] = v;
    }
}

int direction_of(const rpq_graph *g, const Automaton &a, int sym) {
    return sym < a.L ? sym : g->L + (sym - a.L);
}

// Whether some final state is reachable from a start state without a
// transition of direction d (then d is not read by every accepted word).
bool reaches_final_without(const rpq_graph *g, const Automaton &a, int d) {
    uint64_t seen = a.start_mask, frontier = a.start_mask;
    while (frontier) {
        uint64_t next = 0;
        for (size_t t = 0; t < a.from.size(); t++)
            if (((frontier >> a.from[t]) & 1ull) && direction_of(g, a, a.sym[t]) != d)
                next |= 1ull << a.to[t];
        frontier = next & ~seen;
        seen |= next;
    }
    return (seen & a.final_mask) != 0;
}

}  // namespace

rpq_status run_query_rare(rpq_graph *g, const Automaton &a, int32_t source, int32_t max_levels,
                          int32_t *out_list_dev, int64_t capacity, int32_t *out_host_list,
                          rpq_stats *stats, int64_t *count, void *stream, bool host_list,
                          bool *applied) {
    *applied = false;
    const char *env = getenv("RPQ_RARE_MAX");
    const int64_t rare_max = env ? (int64_t)atoll(env) : g->rare_max;
    if (rare_max <= 0 || a.S > kMaxStates / 2 || a.start_mask == 0) return RPQ_OK;
    // the rarest direction that every accepted word reads, among those read
    // somewhere past the start: a direction whose transitions all leave
    // start states bounds nothing (the forward search reads those edges
    // first anyway)
    int best = -1;
    int64_t best_edges = 0;
    for (size_t t = 0; t < a.sym.size(); t++) {
        const int d = direction_of(g, a, a.sym[t]);
        if (d < 0 || d >= 2 * g->L) return RPQ_OK;  // left to the plain query's checks
        const int64_t e = g->adj[d].nnz;
        if (e > rare_max || (best >= 0 && e >= best_edges)) continue;
        bool past_start = false;
        for (size_t u = 0; u < a.sym.size(); u++)
            if (direction_of(g, a, a.sym[u]) == d && !((a.start_mask >> a.from[u]) & 1ull))
                past_start = true;
        if (!past_start || reaches_final_without(g, a, d)) continue;
        best = d;
        best_edges = e;
    }
    if (best < 0) return RPQ_OK;
    *applied = true;
    const int d = best, S = a.S, L = a.L;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (source < 0 || source >= g->n)
        return fail(RPQ_ERR_INVALID, "source %d outside [0, %d)", source, g->n);

    // 1. U: vertices with an edge in direction d
    DevBuf ubuf, ucnt;
    const int64_t umax = std::max<int64_t>(1, std::min<int64_t>(g->adj[d].nnz, g->n));
    if (!ubuf.alloc(sizeof(int32_t) * umax) || !ucnt.alloc(sizeof(unsigned long long)))
        return fail(RPQ_ERR_OOM, "rare-label seeds");
    RPQ_CUDA_TRY(cudaMemsetAsync(ucnt.p, 0, sizeof(unsigned long long), st));
    int sms = 0;
    RPQ_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device));
    nonempty_rows_kernel<<<sms * 4, 256, 0, st>>>(g->adj[d], g->n, ubuf.as<int32_t>(),
                                                  ucnt.as<unsigned long long>());
    RPQ_CUDA_TRY(cudaGetLastError());
    note_launch();
    unsigned long long nu = 0;
    RPQ_CUDA_TRY(cudaMemcpyAsync(&nu, ucnt.p, sizeof(nu), cudaMemcpyDeviceToHost, st));
    RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int32_t> U((size_t)nu);
    if (nu) {
        RPQ_CUDA_TRY(cudaMemcpyAsync(U.data(), ubuf.p, sizeof(int32_t) * nu, cudaMemcpyDeviceToHost, st));
        RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    }

    // 2. backward: N's transitions other than d, reversed, from {q_d} x U
    Automaton R;
    R.S = S;
    R.L = L;
    R.final_mask = S == 64 ? ~0ull : ((1ull << S) - 1);
    for (size_t t = 0; t < a.from.size(); t++) {
        const int s = a.sym[t];
        if (direction_of(g, a, s) == d) {
            R.start_mask |= 1ull << a.from[t];
        } else {
            R.from.push_back(a.to[t]);
            R.to.push_back(a.from[t]);
            R.sym.push_back(s < L ? s + L : s - L);
        }
    }
    const int64_t W = ((int64_t)g->n + 63) / 64;
    DevBuf allowed;
    if (!allowed.alloc(sizeof(uint64_t) * (size_t)S * W))
        return fail(RPQ_ERR_OOM, "backward pair set (%d states)", S);
    if (nu == 0) {
        RPQ_CUDA_TRY(cudaMemsetAsync(allowed.p, 0, sizeof(uint64_t) * (size_t)S * W, st));
    } else {
        QueryExtras bx;
        bx.sources = U.data();
        bx.n_sources = (int32_t)nu;
        bx.reach_bits_out = allowed.as<uint64_t>();
        int64_t bcount = 0;
        rpq_status s = run_query_ex(g, R, &bx, 0, 0, nullptr, 0, nullptr, nullptr, nullptr, &bcount,
                                    stream, 1, false);
        if (s != RPQ_OK) return s;
    }

    // 3. forward on the two-copy automaton, copy 0 pruned to the backward set
    Automaton N2;
    N2.S = 2 * S;
    N2.L = L;
    N2.start_mask = a.start_mask;
    N2.final_mask = a.final_mask << S;
    for (size_t t = 0; t < a.from.size(); t++) {
        const bool cross = direction_of(g, a, a.sym[t]) == d;
        N2.from.push_back(a.from[t]);
        N2.to.push_back(cross ? a.to[t] + S : a.to[t]);
        N2.sym.push_back(a.sym[t]);
        N2.from.push_back(a.from[t] + S);
        N2.to.push_back(a.to[t] + S);
        N2.sym.push_back(a.sym[t]);
    }
    QueryExtras fx;
    fx.premask_bits = allowed.as<uint64_t>();
    fx.premask_states = S;
    return run_query_ex(g, N2, &fx, source, max_levels, out_list_dev, capacity, nullptr,
                        out_host_list, stats, count, stream, 1, host_list);
}

}  // namespace rpq

using namespace rpq;

extern "C" rpq_status rpq_graph_set_rare_plan(rpq_graph *g, int64_t max_edges) {
    clear_error();
    if (!g || max_edges < 0) return fail(RPQ_ERR_INVALID, "bad argument");
    g->rare_max = max_edges;
    return RPQ_OK;
}
