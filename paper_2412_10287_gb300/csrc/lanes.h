// Lane-batched traversal: up to 256 single-source queries advance together,
// one query per bit of a 4 x 64-bit lane vector.  Shared by the batch entry
// point (one persistent launch per batch) and the server (one CUDA-graph
// replay per level step).
#pragma once

#include <memory>
#include <vector>

#include "graph.h"

namespace rpq {

constexpr int kLW = 4;               // lane words per (vertex, state slot)
constexpr int kLanes = 64 * kLW;     // queries per lane group
constexpr int kLaneMaxSlots = 64;    // state slots (max automaton states in a group)

// (direction d, target slot k2): the lanes whose automaton has k -d-> k2,
// per source slot k, are LSrc entries [src_first, src_first + src_count).
struct LUnit {
    int32_t d, k2, src_first, src_count;
};
struct LSrc {
    int32_t k, pad;
    uint64_t mask[kLW];
};
// A direction with at least one lane transition; its units are
// [unit_first, unit_first + unit_count).
struct LDir {
    int32_t d, unit_first, unit_count, pad;
};

struct LHub {
    int32_t v, dir, b, e;
    long long chunk_base;
};

struct LaneCounters {
    unsigned bar_count, bar_gen;
    int32_t status, step;                    // step: level steps done (selects buffers)
    unsigned long long list_count[3];        // vertex lists, rotating by level
    unsigned long long hub_packed;           // (entries << 40) | chunks for this level
    unsigned long long claim_v, claim_h, claim_z, claim_c;
    unsigned long long lane_new[3][kLW];     // lanes that reached new pairs, by level
    unsigned long long edges;                // edges traversed (all levels)
};

// Per-step values read by the kernels from device memory (so a captured
// step graph stays valid when lanes join or leave).
struct LaneDyn {
    int32_t n_dirs, pad;
    uint64_t active[kLW];  // lanes allowed to expand
};

// What the host reads after each level step.
struct LaneStepOut {
    unsigned long long next_count;     // vertices in the next frontier list
    unsigned long long lane_new[kLW];  // lanes that reached new pairs this step
    int32_t status, step;
};

struct LParams {
    const DevAdj *adj;
    int32_t n, K;            // vertices, state slots
    const LaneDyn *dyn;
    const LDir *dirs;
    const LUnit *units;
    const LSrc *srcs;
    uint64_t *M0, *M1, *P, *NX;  // [n][K][kLW]
    uint64_t *tv;                // touched-vertex bitset, ceil(n/64) words
    int32_t *list0, *list1, *list2;
    LHub *hubs;
    int32_t *hub_cmap;           // chunk -> hub entry
    long long hub_cap, chunk_cap;
    LaneCounters *c;
    // tuning (rpq_graph_autotune_batch): edges of a (vertex, direction) row
    // pushed inline before the rest goes to chunks (>= kLaneHubMin); pull
    // instead of push when the frontier holds more than n / pull_div
    // vertices (0: never pull)
    int32_t lane_hub, pull_div;
    int32_t adj_half;  // L: direction d and d +- L are inverse to each other
};

constexpr int kLaneHubMin = 32;  // smallest inline row length (sizes the hub lists)

// Device workspace of one lane group (sized for n vertices and K slots).
struct LaneWorkspace : WorkspaceBase {
    int32_t n = 0, K = 0;
    long long hub_cap = 0, chunk_cap = 0;
    DevBuf M0, M1, P, NX, tv, l0, l1, l2, hubs, hub_cmap, ctr, tables, A32, cnt, pos;
    void *staging = nullptr;
    size_t staging_bytes = 0;
    ~LaneWorkspace() override;
};

// Concurrent query slots of the slots engine by default: 12 kernels of
// 1/12 of the grid each (measured best of 4-16 on the mixed rmat20 batch).
constexpr int kDefaultSlots = 12;

// Kernels in one captured lane level step (one replay launches them all).
constexpr int kLaneStepKernels = 4;

// ---- lane engine entry points used by the server (lanes.cu) ----
rpq_status lane_ws_acquire_fixed(rpq_graph *g, int K, std::unique_ptr<LaneWorkspace> *out);
void lane_ws_return(rpq_graph *g, std::unique_ptr<LaneWorkspace> w);
rpq_status lane_build_tables(const rpq_graph *g, const Automaton *const *autos, int count, int K,
                             std::vector<LDir> *dirs, std::vector<LUnit> *units,
                             std::vector<LSrc> *srcs, std::vector<uint64_t> *fmask,
                             std::vector<uint64_t> *smask);
// Parameters of the lane kernels over workspace ws with its tables buffer
// laid out as [LaneDyn | LDir[] | LUnit[] | LSrc[]] at the given offsets.
LParams lane_params(rpq_graph *g, LaneWorkspace *ws, size_t o_dyn, size_t o_dirs, size_t o_units,
                    size_t o_srcs);
// Captures one level step (expand, hub chunks, commit, finish) as a graph.
rpq_status lane_capture_step(const LParams &p, LaneStepOut *out_dev, cudaStream_t st,
                             cudaGraphExec_t *exec);
// Seeds: records (v, k, lane word, mask lo, mask hi) into the current frontier
// and the visited set, and appends the vertices to the current frontier list.
rpq_status lane_seed(const LParams &p, const int32_t *seeds_dev, int n_seeds,
                     const int32_t *verts_dev, int n_verts, int step, cudaStream_t st);
// Answers of the lanes in lane_ids (count of them) into out_dev (sorted per
// lane); offsets_host gets count + 1 entries.  Clears the lanes' bits.
rpq_status lane_harvest(rpq_graph *g, LaneWorkspace *ws, const LParams &p,
                        const uint64_t *fmask_dev, const int32_t *lane_ids_host, int count,
                        std::vector<int64_t> *offsets_host, std::vector<int32_t> *answers_host,
                        cudaStream_t st);

}  // namespace rpq
