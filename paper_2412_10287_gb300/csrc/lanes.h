// Lane-batched traversal: up to 256 single-source queries advance together,
// one query per bit of a 4 x 64-bit lane vector.  Shared by the batch entry
// point (one persistent launch per batch) and the server (one CUDA-graph
// replay per level step).
#pragma once

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

struct LaneTables {
    int32_t n_dirs, n_units, n_srcs, pad;
};

struct LParams {
    const DevAdj *adj;
    int32_t n, K;            // vertices, state slots
    int32_t n_dirs;
    const LDir *dirs;
    const LUnit *units;
    const LSrc *srcs;
    uint64_t *M0, *M1, *P, *NX;  // [n][K][kLW]
    uint64_t *tv;                // touched-vertex bitset, ceil(n/64) words
    int32_t *list0, *list1, *list2;
    LHub *hubs;
    long long hub_cap;
    LaneCounters *c;
    uint64_t active[kLW];        // lanes allowed to expand this step
};

// Device workspace of one lane group (sized for n vertices and K slots).
struct LaneWorkspace : WorkspaceBase {
    int32_t n = 0, K = 0;
    long long hub_cap = 0;
    DevBuf M0, M1, P, NX, tv, l0, l1, l2, hubs, ctr, tables, A32, cnt, pos;
    void *staging = nullptr;
    size_t staging_bytes = 0;
    ~LaneWorkspace() override;
};

}  // namespace rpq
