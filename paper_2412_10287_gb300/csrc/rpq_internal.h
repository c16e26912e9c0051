// Internal declarations shared by the translation units of librpq.so.
#pragma once

#include <cstdarg>
#include <cstddef>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "rpq.h"

namespace rpq {

// Kernels this library has launched in this process (every thread and
// device), read by rpq_kernel_launches.
extern std::atomic<unsigned long long> g_kernel_launches;
inline void note_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }

// ----------------------------------------------------------------- errors --
// Records a message for rpq_last_error() on this thread and returns `st`.
rpq_status fail(rpq_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
void clear_error();
const char *rpq_last_error_str();  // this thread's last message

// ------------------------------------------------------------- allocator --
// The device allocator (rpq_set_allocator): a pair of callbacks and their
// context, or all null for cudaMalloc / cudaFree.
struct Allocator {
    void *(*alloc)(size_t, void *) = nullptr;
    void (*free_fn)(void *, void *) = nullptr;
    void *ctx = nullptr;
};
// Allocates with the current allocator and reports which one it was, so
// that the memory goes back to that allocator even after a change.
void *dev_alloc(size_t bytes, Allocator *used);  // nullptr on failure
void dev_free(void *p, const Allocator &used);

// RAII device buffer from the library allocator.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    Allocator by;  // the allocator that made p
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { reset(); }
    bool alloc(size_t b) {
        reset();
        if (b == 0) b = 16;
        p = dev_alloc(b, &by);
        bytes = p ? b : 0;
        return p != nullptr;
    }
    void reset() {
        if (p) dev_free(p, by);
        p = nullptr;
        bytes = 0;
    }
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// ---------------------------------------------------------- host automaton --
constexpr int kMaxStates = 64;

struct Automaton {
    int32_t S = 0;  // number of states (<= 64)
    int32_t L = 0;  // number of graph labels; symbols are in [0, 2L)
    std::vector<int32_t> from, to, sym;
    uint64_t start_mask = 0, final_mask = 0;
};

// Regex -> minimised DFA; returns RPQ_OK or an error (message recorded).
rpq_status compile_regex(const char *text, int32_t n_labels, Automaton *out);
bool automaton_accepts(const Automaton &a, const int32_t *word, int32_t len);
Automaton automaton_reverse(const Automaton &a);

bool is_device_pointer(const void *p);

// Exclusive scan of n values into out (int64); the sum goes to *total_dev
// (device pointer).  Synchronises the stream before returning.
template <class T>
rpq_status device_exclusive_scan(const T *in, int64_t *out, int64_t n, int64_t *total_dev,
                                 cudaStream_t st);

// Single query (query.cu).  See run_query there for the output contract.
rpq_status run_query(rpq_graph *g, const Automaton &a, int32_t source, int32_t max_levels,
                     int32_t *out_list_dev, int64_t capacity, uint64_t *out_bits_dev,
                     int32_t *out_host_list, rpq_stats *stats, int64_t *count, void *stream,
                     bool host_list = false);
rpq_status run_query_slot(rpq_graph *g, const Automaton &a, int32_t source, int32_t max_levels,
                          int32_t *out_list_dev, int64_t capacity, uint64_t *out_bits_dev,
                          int32_t *out_host_list, rpq_stats *stats, int64_t *count, void *stream,
                          int grid_div, bool host_list = false);
// Optional parts of a query beyond the single-source answer (query.cu).
struct QueryExtras {
    // the source set V_s (host memory, n_sources >= 1 entries; repeats
    // allowed); null for the single source of the call
    const int32_t *sources = nullptr;
    int32_t n_sources = 0;
    // level of first reach of each answer vertex (device memory, one per
    // answer entry); the answer itself must then go to device memory
    int32_t *out_levels_dev = nullptr;
    // a shortest witness of `target`: path_len + 1 vertices and path_len
    // symbols into host memory of path_cap entries each; path_len = -1 when
    // the target is not in the answer
    bool witness = false;
    int32_t target = 0;
    int32_t *path_v = nullptr, *path_s = nullptr;
    int32_t path_cap = 0;
    int32_t path_len = -1;
    // device [S][ceil(n/64)] words: after the query, bit v of row q is set
    // iff the pair (q, v) was visited
    uint64_t *reach_bits_out = nullptr;
    // device [premask_states][ceil(n/64)] words: before the query, the pairs
    // (q, v), q < premask_states, whose bit is clear are marked visited, so
    // the traversal never enters them (pruning); their P rows are cleared
    // densely at the end
    const uint64_t *premask_bits = nullptr;
    int32_t premask_states = 0;
};
rpq_status run_query_ex(rpq_graph *g, const Automaton &a, QueryExtras *x, int32_t source,
                        int32_t max_levels, int32_t *out_list_dev, int64_t capacity,
                        uint64_t *out_bits_dev, int32_t *out_host_list, rpq_stats *stats,
                        int64_t *count, void *stream, int grid_div, bool host_list = false);
// Rare label first (rare.cu): when every accepted word of `a` reads a label
// direction with few edges, the query runs as a backward search from that
// label's edges and a forward search pruned to what it found; *applied
// tells whether it did (else nothing ran and the caller runs the plain
// query).  Same output contract as run_query.
rpq_status run_query_rare(rpq_graph *g, const Automaton &a, int32_t source, int32_t max_levels,
                          int32_t *out_list_dev, int64_t capacity, int32_t *out_host_list,
                          rpq_stats *stats, int64_t *count, void *stream, bool host_list,
                          bool *applied);
// The calling thread's last host answer (run_query with a host list).
rpq_status last_host_answer(const int32_t **answer, int64_t *count);

// Sorted vertex lists of `count` answer bitsets (row i at bits + i * words32
// uint32 words) into out (host or device, capacity entries); offsets
// (count + 1) on the host.  lanes.cu.
rpq_status bitsets_to_lists(const uint32_t *bits, int64_t words32, int count, int32_t *out,
                            bool out_is_dev, int64_t capacity, int64_t *offsets, void *stream);

}  // namespace rpq

struct rpq_nfa {
    rpq::Automaton a;
};
