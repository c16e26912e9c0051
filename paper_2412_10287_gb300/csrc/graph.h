// The device-resident graph: per-label Boolean decomposition {G^a} (section 3
// of the paper) stored as CSR (rows = sources) and CSC (rows = destinations).
#pragma once

#include <memory>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace rpq {

// Query workspaces are cached on the graph so repeated queries do not
// allocate; each concrete workspace type derives from this.
struct WorkspaceBase {
    virtual ~WorkspaceBase() = default;
};

}  // namespace rpq

struct rpq_graph {
    int32_t n = 0;           // vertices
    int32_t L = 0;           // labels
    int64_t m_input = 0;     // COO entries given
    int64_t m_unique = 0;    // distinct (src, dst, label) triples
    int device = 0;
    // adjacency of label direction d in [0, 2L): d < L -> CSR of G^d (out-rows);
    // d >= L -> CSC of G^{d-L} (in-rows), i.e. the out-rows of G^{(d-L)^-}.
    std::vector<rpq::DevAdj> adj;
    std::vector<int64_t> nnz;  // distinct edges per label
    // per direction d: rows with at least kLongRow edges, and the sum over
    // them of ceil(deg / kLongChunk) (sizes of the query kernel's row lists)
    std::vector<int64_t> long_rows, long_chunks;
    // ... and its non-empty rows of fewer than kLongRow edges
    std::vector<int64_t> short_rows;
    static constexpr int kLongRow = 32;
    static constexpr int kLongChunk = 128;
    rpq::DevBuf d_adj;         // device copy of adj
    rpq::DevBuf csr_nbr, csc_nbr;  // distinct neighbour ids, label-major
    std::vector<std::unique_ptr<rpq::DevBuf>> owned;  // offsets / hypersparse rows

    // push/pull threshold used by single queries (set by rpq_graph_autotune)
    float pull_alpha = 2.0f;
    int32_t pull_min = 256;
    // a level runs on one CTA, with no grid barrier, while its push edge mass
    // and frontier items stay within these (solo_mass < 0: never)
    int32_t solo_mass = 2048;
    int32_t solo_items = 256;
    // Algorithm 2 while the visited set is smaller than this (0: never)
    int64_t alg2_until = 0;
    // single queries whose accepted words all read a label direction with at
    // most this many edges run rare label first (rare.cu; 0: never)
    int64_t rare_max = 0;
    // lane engine tuning (rpq_graph_autotune_batch)
    int32_t lane_hub = 128;
    int32_t lane_pull_div = 0;

    std::mutex ws_mu;
    std::vector<std::unique_ptr<rpq::WorkspaceBase>> ws_free;

    // direction whose rows are the in-rows of direction d (for pull)
    int32_t inverse_dir(int32_t d) const { return d < L ? d + L : d - L; }
};
