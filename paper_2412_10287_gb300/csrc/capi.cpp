// C ABI entry points of librpq.so (declared in include/rpq.h): argument
// checks, error reporting, the pluggable allocator, automaton handles and
// the host/device output routing around the query kernels.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>

#include "graph.h"
#include "rpq_internal.h"

namespace rpq {

namespace {
thread_local std::string t_error;

std::mutex g_alloc_mu;
Allocator g_alloc;
std::atomic<int64_t> g_live_objects{0};
}  // namespace

rpq_status fail(rpq_status st, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_error = buf;
    return st;
}

void clear_error() { t_error.clear(); }

const char *rpq_last_error_str() { return t_error.c_str(); }

void *dev_alloc(size_t bytes, Allocator *used) {
    Allocator a;
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        a = g_alloc;
    }
    *used = a;
    if (a.alloc) return a.alloc(bytes, a.ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p, const Allocator &used) {
    if (!p) return;
    if (used.free_fn) used.free_fn(p, used.ctx);
    else cudaFree(p);
}

bool is_device_pointer(const void *p) {
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

void count_object(int delta) { g_live_objects += delta; }

std::atomic<unsigned long long> g_kernel_launches{0};

}  // namespace rpq

using namespace rpq;

extern "C" const char *rpq_last_error(void) { return t_error.c_str(); }

extern "C" const char *rpq_version(void) { return "0.1.0"; }

extern "C" uint64_t rpq_kernel_launches(void) {
    return (uint64_t)g_kernel_launches.load(std::memory_order_relaxed);
}

extern "C" rpq_status rpq_set_allocator(void *(*alloc)(size_t, void *), void (*free_fn)(void *, void *),
                                        void *ctx) {
    clear_error();
    if ((alloc == nullptr) != (free_fn == nullptr))
        return fail(RPQ_ERR_INVALID, "alloc and free must both be set or both be null");
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc.alloc = alloc;
    g_alloc.free_fn = free_fn;
    g_alloc.ctx = ctx;
    return RPQ_OK;
}

// ------------------------------------------------------------ automata --

namespace {
// Compiled automata of recent expressions, by (text, label count): a query
// stream repeats its templates, and a copy of a small automaton is far
// cheaper than Glushkov + subset construction + minimisation again.
std::mutex g_compiled_mu;
std::map<std::pair<std::string, int32_t>, Automaton> g_compiled;
constexpr size_t kCompiledMax = 4096;
}  // namespace

extern "C" rpq_status rpq_nfa_compile(const char *regex, int32_t n_labels, rpq_nfa **out) {
    clear_error();
    if (!out) return fail(RPQ_ERR_INVALID, "out is null");
    *out = nullptr;
    std::unique_ptr<rpq_nfa> h(new rpq_nfa());
    if (regex) {
        std::lock_guard<std::mutex> lk(g_compiled_mu);
        auto it = g_compiled.find({std::string(regex), n_labels});
        if (it != g_compiled.end()) {
            h->a = it->second;
            *out = h.release();
            return RPQ_OK;
        }
    }
    rpq_status s = compile_regex(regex, n_labels, &h->a);
    if (s != RPQ_OK) return s;
    {
        std::lock_guard<std::mutex> lk(g_compiled_mu);
        if (g_compiled.size() >= kCompiledMax) g_compiled.clear();
        g_compiled.emplace(std::make_pair(std::string(regex), n_labels), h->a);
    }
    *out = h.release();
    return RPQ_OK;
}

extern "C" rpq_status rpq_nfa_from_transitions(int32_t n_states, int32_t n_labels, int32_t n_trans,
                                               const int32_t *from, const int32_t *to,
                                               const int32_t *label, int32_t n_start,
                                               const int32_t *starts, int32_t n_final,
                                               const int32_t *finals, rpq_nfa **out) {
    clear_error();
    if (!out) return fail(RPQ_ERR_INVALID, "out is null");
    *out = nullptr;
    if (n_states <= 0 || n_states > kMaxStates)
        return fail(RPQ_ERR_INVALID, "n_states must be in [1, %d]", kMaxStates);
    if (n_labels <= 0) return fail(RPQ_ERR_INVALID, "n_labels must be positive");
    if (n_trans < 0 || n_start < 0 || n_final < 0) return fail(RPQ_ERR_INVALID, "negative count");
    if ((n_trans && (!from || !to || !label)) || (n_start && !starts) || (n_final && !finals))
        return fail(RPQ_ERR_INVALID, "null array");
    std::unique_ptr<rpq_nfa> h(new rpq_nfa());
    Automaton &a = h->a;
    a.S = n_states;
    a.L = n_labels;
    for (int32_t i = 0; i < n_trans; i++) {
        if (from[i] < 0 || from[i] >= n_states || to[i] < 0 || to[i] >= n_states)
            return fail(RPQ_ERR_INVALID, "transition %d: state out of range", i);
        if (label[i] < 0 || label[i] >= 2 * n_labels)
            return fail(RPQ_ERR_INVALID, "transition %d: label %d outside [0, %d)", i, label[i],
                        2 * n_labels);
        a.from.push_back(from[i]);
        a.to.push_back(to[i]);
        a.sym.push_back(label[i]);
    }
    for (int32_t i = 0; i < n_start; i++) {
        if (starts[i] < 0 || starts[i] >= n_states) return fail(RPQ_ERR_INVALID, "start state out of range");
        a.start_mask |= 1ull << starts[i];
    }
    for (int32_t i = 0; i < n_final; i++) {
        if (finals[i] < 0 || finals[i] >= n_states) return fail(RPQ_ERR_INVALID, "final state out of range");
        a.final_mask |= 1ull << finals[i];
    }
    *out = h.release();
    return RPQ_OK;
}

extern "C" void rpq_nfa_free(rpq_nfa *nfa) { delete nfa; }

extern "C" rpq_status rpq_nfa_info(const rpq_nfa *nfa, int32_t *n_states, int32_t *n_trans,
                                   int32_t *n_labels) {
    clear_error();
    if (!nfa) return fail(RPQ_ERR_INVALID, "nfa is null");
    if (n_states) *n_states = nfa->a.S;
    if (n_trans) *n_trans = (int32_t)nfa->a.from.size();
    if (n_labels) *n_labels = nfa->a.L;
    return RPQ_OK;
}

extern "C" rpq_status rpq_nfa_export(const rpq_nfa *nfa, int32_t *from, int32_t *to, int32_t *label,
                                     int32_t capacity, uint64_t *start_mask, uint64_t *final_mask) {
    clear_error();
    if (!nfa) return fail(RPQ_ERR_INVALID, "nfa is null");
    const int32_t T = (int32_t)nfa->a.from.size();
    if (start_mask) *start_mask = nfa->a.start_mask;
    if (final_mask) *final_mask = nfa->a.final_mask;
    if (capacity < T) return fail(RPQ_ERR_CAPACITY, "need %d transitions", T);
    for (int32_t i = 0; i < T; i++) {
        if (from) from[i] = nfa->a.from[i];
        if (to) to[i] = nfa->a.to[i];
        if (label) label[i] = nfa->a.sym[i];
    }
    return RPQ_OK;
}

extern "C" rpq_status rpq_nfa_accepts(const rpq_nfa *nfa, const int32_t *word, int32_t length,
                                      int32_t *accepted) {
    clear_error();
    if (!nfa || !accepted || (length > 0 && !word)) return fail(RPQ_ERR_INVALID, "null argument");
    if (length < 0) return fail(RPQ_ERR_INVALID, "negative length");
    *accepted = automaton_accepts(nfa->a, word, length) ? 1 : 0;
    return RPQ_OK;
}

extern "C" rpq_status rpq_nfa_reverse(const rpq_nfa *nfa, rpq_nfa **out) {
    clear_error();
    if (!nfa || !out) return fail(RPQ_ERR_INVALID, "null argument");
    std::unique_ptr<rpq_nfa> h(new rpq_nfa());
    h->a = automaton_reverse(nfa->a);
    *out = h.release();
    return RPQ_OK;
}

// --------------------------------------------------------------- query --

extern "C" rpq_status rpq_query(const rpq_graph *g, const rpq_nfa *nfa, int32_t source,
                                int32_t max_levels, int32_t *out_vertices, int64_t capacity,
                                int64_t *out_count, rpq_stats *stats, void *stream) {
    clear_error();
    if (!g || !nfa || !out_count) return fail(RPQ_ERR_INVALID, "null argument");
    if (capacity < 0 || (capacity > 0 && !out_vertices))
        return fail(RPQ_ERR_INVALID, "bad output buffer");
    *out_count = 0;
    rpq_graph *gm = const_cast<rpq_graph *>(g);
    const bool dev = out_vertices && is_device_pointer(out_vertices);
    int64_t count = 0;
    // a host answer (or none asked for) goes through the thread's pinned
    // buffer, where rpq_last_answer finds it
    bool rare = false;
    rpq_status s = run_query_rare(gm, nfa->a, source, max_levels, dev ? out_vertices : nullptr,
                                  capacity, dev ? nullptr : out_vertices, stats, &count, stream,
                                  !dev, &rare);
    if (!rare && s == RPQ_OK)
        s = run_query(gm, nfa->a, source, max_levels, dev ? out_vertices : nullptr, capacity,
                      nullptr, dev ? nullptr : out_vertices, stats, &count, stream, !dev);
    if (s != RPQ_OK) return s;
    *out_count = count;
    if (count > capacity)
        return fail(RPQ_ERR_CAPACITY, "answer has %lld vertices, capacity %lld", (long long)count,
                    (long long)capacity);
    return RPQ_OK;
}

extern "C" rpq_status rpq_query_multi(const rpq_graph *g, const rpq_nfa *nfa, int32_t n_sources,
                                      const int32_t *sources, int32_t max_levels,
                                      int32_t *out_vertices, int64_t capacity, int64_t *out_count,
                                      rpq_stats *stats, void *stream) {
    clear_error();
    if (!g || !nfa || !out_count || n_sources < 0 || (n_sources > 0 && !sources))
        return fail(RPQ_ERR_INVALID, "null argument");
    if (capacity < 0 || (capacity > 0 && !out_vertices))
        return fail(RPQ_ERR_INVALID, "bad output buffer");
    if (max_levels < 0) return fail(RPQ_ERR_INVALID, "max_levels must be >= 0");
    *out_count = 0;
    if (stats) *stats = rpq_stats{};
    if (n_sources == 0) return RPQ_OK;  // V_s empty: no pair at level 0, empty answer
    if (is_device_pointer(sources)) return fail(RPQ_ERR_INVALID, "sources must be host memory");
    rpq_graph *gm = const_cast<rpq_graph *>(g);
    const bool dev = out_vertices && is_device_pointer(out_vertices);
    QueryExtras x;
    x.sources = sources;
    x.n_sources = n_sources;
    int64_t count = 0;
    rpq_status s = run_query_ex(gm, nfa->a, &x, 0, max_levels, dev ? out_vertices : nullptr,
                                capacity, nullptr, dev ? nullptr : out_vertices, stats, &count,
                                stream, 1, !dev);
    if (s != RPQ_OK) return s;
    *out_count = count;
    if (count > capacity)
        return fail(RPQ_ERR_CAPACITY, "answer has %lld vertices, capacity %lld", (long long)count,
                    (long long)capacity);
    return RPQ_OK;
}

extern "C" rpq_status rpq_query_sdr(const rpq_graph *g, const rpq_nfa *nfa, int32_t target,
                                    int32_t max_levels, int32_t *out_vertices, int64_t capacity,
                                    int64_t *out_count, rpq_stats *stats, void *stream) {
    clear_error();
    if (!g || !nfa || !out_count) return fail(RPQ_ERR_INVALID, "null argument");
    if (capacity < 0 || (capacity > 0 && !out_vertices))
        return fail(RPQ_ERR_INVALID, "bad output buffer");
    *out_count = 0;
    // section 4: SDR of N for v_f is SSR of the reversed automaton N^- from v_f
    const Automaton rev = automaton_reverse(nfa->a);
    rpq_graph *gm = const_cast<rpq_graph *>(g);
    const bool dev = out_vertices && is_device_pointer(out_vertices);
    int64_t count = 0;
    rpq_status s = run_query(gm, rev, target, max_levels, dev ? out_vertices : nullptr, capacity,
                             nullptr, dev ? nullptr : out_vertices, stats, &count, stream, !dev);
    if (s != RPQ_OK) return s;
    *out_count = count;
    if (count > capacity)
        return fail(RPQ_ERR_CAPACITY, "answer has %lld vertices, capacity %lld", (long long)count,
                    (long long)capacity);
    return RPQ_OK;
}

extern "C" rpq_status rpq_query_levels(const rpq_graph *g, const rpq_nfa *nfa, int32_t n_sources,
                                       const int32_t *sources, int32_t max_levels,
                                       int32_t *out_vertices, int32_t *out_levels, int64_t capacity,
                                       int64_t *out_count, void *stream) {
    clear_error();
    if (!g || !nfa || !out_count || n_sources < 0 || (n_sources > 0 && !sources))
        return fail(RPQ_ERR_INVALID, "null argument");
    if (capacity < 0 || (capacity > 0 && (!out_vertices || !out_levels)))
        return fail(RPQ_ERR_INVALID, "bad output buffers");
    if (max_levels < 0) return fail(RPQ_ERR_INVALID, "max_levels must be >= 0");
    *out_count = 0;
    if (n_sources == 0) return RPQ_OK;
    if (is_device_pointer(sources)) return fail(RPQ_ERR_INVALID, "sources must be host memory");
    const bool dv = out_vertices && is_device_pointer(out_vertices);
    const bool dl = out_levels && is_device_pointer(out_levels);
    if (capacity > 0 && dv != dl)
        return fail(RPQ_ERR_INVALID, "out_vertices and out_levels must both be device or host memory");
    rpq_graph *gm = const_cast<rpq_graph *>(g);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the answer and its levels are computed in device memory: the caller's
    // or temporary buffers of n entries (an answer holds at most n vertices)
    DevBuf tv, tl;
    int32_t *v_dev = out_vertices, *l_dev = out_levels;
    int64_t cap_dev = capacity;
    if (!dv) {
        if (!tv.alloc(sizeof(int32_t) * (size_t)g->n) || !tl.alloc(sizeof(int32_t) * (size_t)g->n))
            return fail(RPQ_ERR_OOM, "answer buffers (%d entries)", g->n);
        v_dev = tv.as<int32_t>();
        l_dev = tl.as<int32_t>();
        cap_dev = g->n;
    }
    QueryExtras x;
    x.sources = sources;
    x.n_sources = n_sources;
    x.out_levels_dev = l_dev;
    int64_t count = 0;
    rpq_status s = run_query_ex(gm, nfa->a, &x, 0, max_levels, v_dev, cap_dev, nullptr, nullptr,
                                nullptr, &count, stream, 1, false);
    if (s != RPQ_OK) return s;
    *out_count = count;
    if (count > capacity)
        return fail(RPQ_ERR_CAPACITY, "answer has %lld vertices, capacity %lld", (long long)count,
                    (long long)capacity);
    if (!dv && count > 0) {
        RPQ_CUDA_TRY(cudaMemcpyAsync(out_vertices, v_dev, sizeof(int32_t) * (size_t)count,
                                     cudaMemcpyDeviceToHost, st));
        RPQ_CUDA_TRY(cudaMemcpyAsync(out_levels, l_dev, sizeof(int32_t) * (size_t)count,
                                     cudaMemcpyDeviceToHost, st));
        RPQ_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return RPQ_OK;
}

extern "C" rpq_status rpq_query_witness(const rpq_graph *g, const rpq_nfa *nfa, int32_t n_sources,
                                        const int32_t *sources, int32_t target, int32_t max_levels,
                                        int32_t *path_vertices, int32_t *path_symbols,
                                        int32_t capacity, int32_t *out_length, void *stream) {
    clear_error();
    if (!g || !nfa || !out_length || n_sources <= 0 || !sources)
        return fail(RPQ_ERR_INVALID, "null argument or empty source set");
    if (capacity < 0 || (capacity > 0 && (!path_vertices || !path_symbols)))
        return fail(RPQ_ERR_INVALID, "bad output buffers");
    if (target < 0 || target >= g->n)
        return fail(RPQ_ERR_INVALID, "target %d outside [0, %d)", target, g->n);
    if (max_levels < 0) return fail(RPQ_ERR_INVALID, "max_levels must be >= 0");
    if (is_device_pointer(sources) || (capacity > 0 && (is_device_pointer(path_vertices) ||
                                                        is_device_pointer(path_symbols))))
        return fail(RPQ_ERR_INVALID, "sources and path buffers must be host memory");
    *out_length = -1;
    rpq_graph *gm = const_cast<rpq_graph *>(g);
    QueryExtras x;
    x.sources = sources;
    x.n_sources = n_sources;
    x.witness = true;
    x.target = target;
    x.path_v = path_vertices;
    x.path_s = path_symbols;
    x.path_cap = capacity;
    int64_t count = 0;
    rpq_status s = run_query_ex(gm, nfa->a, &x, 0, max_levels, nullptr, 0, nullptr, nullptr,
                                nullptr, &count, stream, 1, false);
    if (s != RPQ_OK) return s;
    *out_length = x.path_len;
    if (x.path_len >= 0 && x.path_len + 1 > capacity)
        return fail(RPQ_ERR_CAPACITY, "witness has %d vertices, capacity %d", x.path_len + 1,
                    capacity);
    return RPQ_OK;
}

extern "C" rpq_status rpq_last_answer(const int32_t **answer, int64_t *count) {
    clear_error();
    return last_host_answer(answer, count);
}

extern "C" rpq_status rpq_query_bitset(const rpq_graph *g, const rpq_nfa *nfa, int32_t source,
                                       int32_t max_levels, uint64_t *out_bits, int64_t *out_count,
                                       rpq_stats *stats, void *stream) {
    clear_error();
    if (!g || !nfa || !out_bits || !out_count) return fail(RPQ_ERR_INVALID, "null argument");
    rpq_graph *gm = const_cast<rpq_graph *>(g);
    int32_t n = 0;
    rpq_status s = rpq_graph_info(g, -1, &n, nullptr, nullptr);
    if (s != RPQ_OK) return s;
    const size_t words = ((size_t)n + 63) / 64;
    int64_t count = 0;
    if (is_device_pointer(out_bits)) {
        s = run_query(gm, nfa->a, source, max_levels, nullptr, 0, out_bits, nullptr, stats, &count,
                      stream);
    } else {
        DevBuf tmp;
        if (!tmp.alloc(words * sizeof(uint64_t))) return fail(RPQ_ERR_OOM, "bitset buffer");
        s = run_query(gm, nfa->a, source, max_levels, nullptr, 0, tmp.as<uint64_t>(), nullptr,
                      stats, &count, stream);
        if (s == RPQ_OK) {
            cudaStream_t st = static_cast<cudaStream_t>(stream);
            if (cudaMemcpyAsync(out_bits, tmp.p, words * sizeof(uint64_t), cudaMemcpyDeviceToHost,
                                st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return fail(RPQ_ERR_CUDA, "bitset copy: %s", cudaGetErrorString(cudaGetLastError()));
        }
    }
    if (s != RPQ_OK) return s;
    *out_count = count;
    return RPQ_OK;
}

